// knn.cu - the adaptive support radius of Sec. 2.2.
//
//   d_n(a)   distance to the n-th nearest node (eq. adaptive_support_radius),
//            at every point of a Fibonacci auxiliary grid;
//   d~_n(q)  its degree-zero MLS (Shepard) approximation with a constant
//            support radius rho_aux, at every quadrature node q;
//   delta(q) = (1 + eps) d~_n(q);  n(q) = #X(q) (eq. number_of_local_nodes);
//   guard    if n(q) < m, delta(q) = (1 + eps) d_n(q) computed exactly at q.
//
// All searches are warp-per-query over the band/cell structure. Membership is
// decided on exact FP64 squared chords ((dx*dx + dy*dy) + dz*dz, no FMA); FP32
// copies of the points only pre-filter candidates with a proven error margin,
// so the node sets and the n-th smallest chord are bit-exact.
#include "common.cuh"
#include "kernels.h"

namespace hamls {

constexpr int KNN_WARPS = 4;

// error bound of the FP32 squared chord relative to the exact one (points and
// query rounded to FP32): |c2f - c2| <= 4.2e-7 sqrt(c2) + 2e-7 c2 + 5e-14
__device__ __forceinline__ double c2_margin(double c2) { return 1e-6 * sqrt(c2) + 1e-6 * c2 + 1e-13; }

// ---------------------------------------------------------------- k-NN
// n-th smallest exact squared chord from q to the points of g (+inf when the
// set has fewer than n points), keeping exact FP64 chords throughout. `list`
// is this warp's shared scratch (n doubles). Slow path of knn_nth.
__device__ double knn_nth_exact(const Cells& g, double qx, double qy, double qz, int n, double* list, double r0,
                                bool* failed) {
  const int lane = threadIdx.x & 31;
  const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
  const double PI = 3.14159265358979323846;
  // phase 1: find a radius whose enumeration holds a few times n candidates
  double r = fmin(fmax(r0, 1e-7), PI), rlo = 0.0, rhi = PI;
  bool have_lo = false, have_hi = false;
  const uint32_t lowT = (uint32_t)n + (uint32_t)n / 4 + 4u, highT = 16u * (uint32_t)n + 64u;
  for (int it = 0; it < 80; ++it) {
    Cap c = make_cap(qx, qy, qz, r);
    uint32_t bc = cap_box_count(g, c);
    if (bc < lowT) {
      if (r >= PI) break;
      rlo = r;
      have_lo = true;
    } else if (bc > highT) {
      rhi = r;
      have_hi = true;
    } else {
      break;
    }
    if (have_lo && have_hi) {
      if (rhi < rlo * 1.002) {
        r = rhi;
        break;
      }
      r = sqrt(rlo * rhi);
    } else if (have_lo) {
      r = fmin(2.0 * r, PI);
    } else {
      if (r < 1e-6) break;
      r = 0.5 * r;
    }
  }
  // phase 2: scan, keep the n smallest exact squared chords; valid once the
  // n-th smallest lies inside the scanned cap
  for (int it = 0; it < 64; ++it) {
    for (int i = lane; i < n; i += 32) list[i] = __longlong_as_double(0x7ff0000000000000ll);
    __syncwarp();
    double thr = __longlong_as_double(0x7ff0000000000000ll);
    float thr_f = __int_as_float(0x7f800000);
    Cap c = make_cap(qx, qy, qz, r);
    for_cap_candidates(g, c, [&](bool valid, uint32_t idx) {
      double c2 = 0.0;
      bool want = false;
      if (valid) {
        float4 p = g.pf[idx];
        float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
        float c2f = dx * dx + dy * dy + dz * dz;
        if (c2f <= thr_f) {
          c2 = chord2_exact(g.px[idx], g.py[idx], g.pz[idx], qx, qy, qz);
          want = c2 < thr;
        }
      }
      unsigned ball = __ballot_sync(FULL, want);
      while (ball) {
        const int src = __ffs(ball) - 1;
        ball &= ball - 1;
        const double v = __shfl_sync(FULL, c2, src);
        if (v < list[n - 1]) {
          int pos = 0;
          for (int k0 = 0; k0 < n; k0 += 32) {
            int i = k0 + lane;
            pos += __popc(__ballot_sync(FULL, i < n && list[i] < v));
          }
          double prev[KNN_MAX / 32];
#pragma unroll
          for (int kk = 0; kk < KNN_MAX / 32; ++kk) {
            int i = kk * 32 + lane;
            prev[kk] = (i >= 1 && i < n) ? list[i - 1] : 0.0;
          }
          __syncwarp();
#pragma unroll
          for (int kk = 0; kk < KNN_MAX / 32; ++kk) {
            int i = kk * 32 + lane;
            if (i > pos && i < n) list[i] = prev[kk];
          }
          if (lane == (pos & 31)) list[pos] = v;
          __syncwarp();
        }
      }
      thr = list[n - 1];
      if (thr < 1e300) {
        double t = thr + c2_margin(thr);
        thr_f = __double2float_ru(t);
      }
    });
    const double nth = list[n - 1];
    __syncwarp();
    const double sr = sin(0.5 * r);
    const double rho2 = 4.0 * sr * sr;
    if (nth < rho2 || r >= PI) return nth;
    if (nth < 1e300) {
      // n candidates lie within the chord sqrt(nth): the cap through the
      // n-th of them holds at least n nodes, so the next scan is valid
      r = fmin(PI, fmax(1.25 * r, geodesic_from_chord2(nth) * (1.0 + 1e-7) + 1e-12));
    } else {
      r = fmin(PI, fmax(2.0 * r, 0.25 * r0));
    }
  }
  *failed = true;
  return __longlong_as_double(0x7ff0000000000000ll);
}

// FP32 error bound of a squared chord computed from FP32-rounded points and
// query (see c2_margin), evaluated in FP32 with slack.
__device__ __forceinline__ float c2_margin_f(float c2) { return 1.05e-6f * sqrtf(c2) + 1.05e-6f * c2 + 1e-13f; }

constexpr int KNN_EXTRA = 8;                       // FP32 keys kept beyond the n-th
constexpr int KNN_LIST = KNN_MAX + KNN_EXTRA;      // warp list capacity
constexpr int KNN_SCRATCH = KNN_LIST * 8;          // bytes of warp scratch knn_nth needs

// n-th smallest exact squared chord from q to the points of g, found in FP32:
// the scan keeps the H = n + 8 smallest FP32 chords (with indices) in a sorted
// warp list; then only the few candidates whose FP32 chord lies within twice
// the FP32 error bound m of the n-th FP32 value T are measured exactly. With
// A = #{FP32 chord < T - 2m}, those A are certainly among the n nearest and
// the answer is the (n - A)-th smallest exact chord of the uncertain ones.
// It needs every uncertain candidate in the list (its last key > T + 2m, or
// fewer than H candidates): otherwise, or with more than 32 uncertain ones,
// the exact FP64 search runs instead.
__device__ double knn_nth(const Cells& g, double qx, double qy, double qz, int n, unsigned char* scratch,
                          double r0, bool* failed, unsigned long long* exact_fb = nullptr) {
  const int lane = threadIdx.x & 31;
  const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
  const float INF_F = __int_as_float(0x7f800000);
  const int H = n + KNN_EXTRA;
  float* lkey = reinterpret_cast<float*>(scratch);
  uint32_t* lidx = reinterpret_cast<uint32_t*>(lkey + KNN_LIST);
  const float PI_F = 3.14159265f;
  // phase 1: a radius whose enumeration holds a few times n candidates
  float r = fminf(fmaxf((float)r0, 1e-7f), PI_F), rlo = 0.f, rhi = PI_F;
  bool have_lo = false, have_hi = false;
  const uint32_t lowT = (uint32_t)n + (uint32_t)n / 4 + 4u, highT = 16u * (uint32_t)n + 64u;
  for (int it = 0; it < 80; ++it) {
    Cap c = make_cap_f(qxf, qyf, qzf, r);
    uint32_t bc = cap_box_count(g, c);
    if (bc < lowT) {
      if (r >= PI_F) break;
      rlo = r;
      have_lo = true;
    } else if (bc > highT) {
      rhi = r;
      have_hi = true;
    } else {
      break;
    }
    if (have_lo && have_hi) {
      if (rhi < rlo * 1.002f) {
        r = rhi;
        break;
      }
      r = sqrtf(rlo * rhi);
    } else if (have_lo) {
      r = fminf(2.f * r, PI_F);
    } else {
      if (r < 1e-6f) break;
      r = 0.5f * r;
    }
  }
  // phase 2
  for (int it = 0; it < 64; ++it) {
    for (int i = lane; i < H; i += 32) {
      lkey[i] = INF_F;
      lidx[i] = 0xFFFFFFFFu;
    }
    __syncwarp();
    float thr = INF_F;
    Cap c = make_cap_f(qxf, qyf, qzf, r);
    for_cap_candidates(g, c, [&](bool valid, uint32_t idx) {
      float c2f = INF_F;
      if (valid) {
        const float4 p = g.pf[idx];
        const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
        c2f = dx * dx + dy * dy + dz * dz;
      }
      unsigned ball = __ballot_sync(FULL, valid && c2f < thr);
      while (ball) {
        const int src = __ffs(ball) - 1;
        ball &= ball - 1;
        const float v = __shfl_sync(FULL, c2f, src);
        const uint32_t vi = __shfl_sync(FULL, idx, src);
        if (v < lkey[H - 1]) {
          int pos = 0;
          for (int k0 = 0; k0 < H; k0 += 32) {
            const int i = k0 + lane;
            pos += __popc(__ballot_sync(FULL, i < H && lkey[i] <= v));
          }
          float pk[(KNN_LIST + 31) / 32];
          uint32_t pi[(KNN_LIST + 31) / 32];
#pragma unroll
          for (int kk = 0; kk < (KNN_LIST + 31) / 32; ++kk) {
            const int i = kk * 32 + lane;
            pk[kk] = (i >= 1 && i < H) ? lkey[i - 1] : 0.f;
            pi[kk] = (i >= 1 && i < H) ? lidx[i - 1] : 0u;
          }
          __syncwarp();
#pragma unroll
          for (int kk = 0; kk < (KNN_LIST + 31) / 32; ++kk) {
            const int i = kk * 32 + lane;
            if (i > pos && i < H) {
              lkey[i] = pk[kk];
              lidx[i] = pi[kk];
            }
          }
          if (lane == (pos & 31) && pos < H) {
            lkey[pos] = v;
            lidx[pos] = vi;
          }
          __syncwarp();
        }
      }
      thr = lkey[H - 1];
    });
    __syncwarp();
    const float T = lkey[n - 1];
    if (!(T < INF_F)) {                               // fewer than n candidates so far
      if (r >= PI_F) {
        *failed = true;
        return __longlong_as_double(0x7ff0000000000000ll);
      }
      r = fminf(PI_F, fmaxf(2.f * r, 0.25f * (float)r0));
      continue;
    }
    const float m = c2_margin_f(T);
    const float last = lkey[H - 1];
    int A = 0, u0 = H, u1 = 0;
    for (int k0 = 0; k0 < H; k0 += 32) {
      const int i = k0 + lane;
      const float kv = i < H ? lkey[i] : INF_F;
      A += __popc(__ballot_sync(FULL, i < H && kv < T - 2.f * m));
      const unsigned inu = __ballot_sync(FULL, i < H && kv >= T - 2.f * m && kv <= T + 2.f * m);
      if (inu) {
        u0 = min(u0, k0 + __ffs(inu) - 1);
        u1 = max(u1, k0 + 32 - __clz(inu));
      }
    }
    const int nu = u1 - u0;
    double nth;
    if (!(last > T + 2.f * m || last == INF_F) || nu > 32 || nu < n - A || n - A < 1) {
      if (exact_fb && lane == 0) atomicAdd(exact_fb, 1ull);
      return knn_nth_exact(g, qx, qy, qz, n, reinterpret_cast<double*>(scratch), r0, failed);
    }
    {
      double e = __longlong_as_double(0x7ff0000000000000ll);
      if (lane < nu) {
        const uint32_t id = lidx[u0 + lane];
        e = chord2_exact(g.px[id], g.py[id], g.pz[id], qx, qy, qz);
      }
      // rank of this lane's exact chord among the uncertain ones (ties by lane)
      int rank = 0;
      for (int s2 = 0; s2 < nu; ++s2) {
        const double o = __shfl_sync(FULL, e, s2);
        rank += (o < e || (o == e && s2 < lane)) ? 1 : 0;
      }
      const unsigned hit = __ballot_sync(FULL, lane < nu && rank == n - A - 1);
      nth = __shfl_sync(FULL, e, __ffs(hit) - 1);
    }
    const double sr = sin(0.5 * (double)r);
    const double rho2 = 4.0 * sr * sr;
    if (nth < rho2 || r >= PI_F) return nth;
    r = fminf(PI_F, fmaxf(1.25f * r, 2.f * asinf(fminf(1.f, 0.5f * sqrtf((float)nth))) * (1.f + 1e-5f) + 1e-6f));
  }
  *failed = true;
  return __longlong_as_double(0x7ff0000000000000ll);
}

// d_n at the auxiliary points, a tile of 32 neighbouring points per warp (32
// consecutive points of an ordering by latitude bands about as tall as the
// tile is wide, then longitude). The exact d_n of the representative r (the
// tile point nearest the tile's centroid) bounds every other: d_n(a) <=
// d_n(r) + d(a, r) (d_n is 1-Lipschitz), so all n nearest nodes of every tile
// point lie within R = d_n(r) + 2 max_a d(a, r) of r. The warp streams the
// candidates of that cap once through shared memory; each lane keeps a
// max-heap of the H = n + 8 smallest FP32 chords from its own point. Heap
// updates are buffered per lane and applied once per 32 staged candidates, so
// the warp does not diverge on every insertion. The exact n-th chord then
// follows as in knn_nth, with FP64 only for the uncertain few.
constexpr int TK_WARPS = 2;
constexpr int TK_PEND = 16;

__host__ __device__ __forceinline__ size_t tile_warp_bytes(int n) {
  // heap keys + indices, pending keys + indices, knn_nth scratch, staged candidates
  return (size_t)(n + KNN_EXTRA) * 32 * 8 + (size_t)TK_PEND * 32 * 8 + KNN_SCRATCH + 32 * 16 + 32 * 4;
}

__device__ __forceinline__ void heap_replace_root(float* hkey, uint32_t* hidx, int size, int lane, float v,
                                                  uint32_t id) {
  int k = 0;
  for (;;) {
    const int l = 2 * k + 1;
    if (l >= size) break;
    int mc = l;
    float hm = hkey[l * 32 + lane];
    if (l + 1 < size) {
      const float hr = hkey[(l + 1) * 32 + lane];
      if (hr > hm) {
        mc = l + 1;
        hm = hr;
      }
    }
    if (!(hm > v)) break;
    hkey[k * 32 + lane] = hm;
    hidx[k * 32 + lane] = hidx[mc * 32 + lane];
    k = mc;
  }
  hkey[k * 32 + lane] = v;
  hidx[k * 32 + lane] = id;
}

__global__ void __launch_bounds__(TK_WARPS * 32) aux_knn_tile_kernel(Cells nodes, Cells aux,
                                                                     const uint32_t* __restrict__ tile_order,
                                                                     int n, double r0, double* __restrict__ dn_sorted,
                                                                     float* __restrict__ dn_f, DevStatus* st,
                                                                     unsigned long long* ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int H = n + KNN_EXTRA;
  unsigned char* base = smem_raw + warp * tile_warp_bytes(n);
  float* hkey = reinterpret_cast<float*>(base);                      // [H][32]
  uint32_t* hidx = reinterpret_cast<uint32_t*>(hkey + H * 32);       // [H][32]
  float* pkey = reinterpret_cast<float*>(hidx + H * 32);             // [TK_PEND][32]
  uint32_t* pidx = reinterpret_cast<uint32_t*>(pkey + TK_PEND * 32);  // [TK_PEND][32]
  unsigned char* kscr = reinterpret_cast<unsigned char*>(pidx + TK_PEND * 32);
  float4* sf = reinterpret_cast<float4*>(kscr + KNN_SCRATCH);        // [32]
  uint32_t* si = reinterpret_cast<uint32_t*>(sf + 32);                // [32]
  const float INF_F = __int_as_float(0x7f800000);
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1ull);
    t = __shfl_sync(FULL, t, 0);
    const long long first = (long long)t * 32;
    if (first >= aux.n) break;
    const int cnt = (int)min(32ll, (long long)aux.n - first);
    const bool act = lane < cnt;
    const uint32_t fi = tile_order[first + (act ? lane : 0)];
    const double ax = aux.px[fi], ay = aux.py[fi], az = aux.pz[fi];
    const float axf = (float)ax, ayf = (float)ay, azf = (float)az;
    // representative: the tile point nearest the centroid
    const float cx = warp_sum(act ? axf : 0.f), cy = warp_sum(act ? ayf : 0.f), cz = warp_sum(act ? azf : 0.f);
    float dc = act ? (axf - cx / cnt) * (axf - cx / cnt) + (ayf - cy / cnt) * (ayf - cy / cnt) +
                         (azf - cz / cnt) * (azf - cz / cnt)
                   : INF_F;
    int rl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(FULL, dc, o);
      const int ol = __shfl_xor_sync(FULL, rl, o);
      if (od < dc || (od == dc && ol < rl)) {
        dc = od;
        rl = ol;
      }
    }
    const double rx = __shfl_sync(FULL, ax, rl), ry = __shfl_sync(FULL, ay, rl), rz = __shfl_sync(FULL, az, rl);
    const float rxf = (float)rx, ryf = (float)ry, rzf = (float)rz;
    // spread: an upper bound of max_a d(a, r) in FP32
    float sp = 0.f;
    if (act) {
      const float dx = axf - rxf, dy = ayf - ryf, dz = azf - rzf;
      sp = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(dx * dx + dy * dy + dz * dz)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sp = fmaxf(sp, __shfl_xor_sync(FULL, sp, o));
    bool failed = false;
    const double c2r = knn_nth(nodes, rx, ry, rz, n, kscr, r0, &failed, &st->cnt[C_KNN_EXACT_FB]);
    const float dr = 2.f * asinf(fminf(1.f, 0.5f * sqrtf((float)c2r)));
    const float R = fminf((dr + 2.f * sp) * (1.f + 1e-5f) + 1e-6f, 3.14159265f);
    for (int k = 0; k < H; ++k) {
      hkey[k * 32 + lane] = INF_F;
      hidx[k * 32 + lane] = 0xFFFFFFFFu;
    }
    float root = INF_F;
    int pc = 0;
    unsigned long long ncand = 0, nins = 0;
    __syncwarp();
    Cap c = make_cap_f(rxf, ryf, rzf, R);
    for_cap_candidates<true>(nodes, c, [&](bool valid, uint32_t idx) {
      if (valid) {
        sf[lane] = nodes.pf[idx];
        si[lane] = idx;
      }
      const int nv = __popc(__ballot_sync(FULL, valid));
      ncand += nv;
      __syncwarp();
      for (int cc = 0; cc < nv; ++cc) {
        const float4 p = sf[cc];
        const float dx = p.x - axf, dy = p.y - ayf, dz = p.z - azf;
        const float c2f = dx * dx + dy * dy + dz * dz;
        if (act && c2f < root) {
          ++nins;
          if (pc < TK_PEND) {
            pkey[pc * 32 + lane] = c2f;
            pidx[pc * 32 + lane] = si[cc];
            ++pc;
          } else {
            heap_replace_root(hkey, hidx, H, lane, c2f, si[cc]);
            root = hkey[lane];
          }
        }
      }
      __syncwarp();
      // apply the buffered insertions
      while (__any_sync(FULL, pc > 0)) {
        if (pc > 0) {
          --pc;
          const float v = pkey[pc * 32 + lane];
          if (v < root) {
            heap_replace_root(hkey, hidx, H, lane, v, pidx[pc * 32 + lane]);
            root = hkey[lane];
          }
        }
      }
    });
    // exact n-th: pop the KNN_EXTRA largest (heap sort tail), then resolve the
    // entries within 2m of the n-th FP32 value T with FP64 chords
    const float rootH = root;
    int size = H;
    for (int pp = 0; pp < KNN_EXTRA; ++pp) {
      const float top = hkey[lane];
      const uint32_t tid = hidx[lane];
      --size;
      const float lv = hkey[size * 32 + lane];
      const uint32_t li = hidx[size * 32 + lane];
      heap_replace_root(hkey, hidx, size, lane, lv, li);
      hkey[size * 32 + lane] = top;
      hidx[size * 32 + lane] = tid;
    }
    const float T = hkey[lane];                       // n-th smallest FP32 chord
    const float m = c2_margin_f(T);
    int A = 0, nu = 0;
    double ue[8];
#pragma unroll
    for (int s2 = 0; s2 < 8; ++s2) ue[s2] = 0.0;
    bool ok = act && T < INF_F && (rootH > T + 2.f * m || rootH == INF_F);
    if (ok) {
      for (int k = 0; k < H; ++k) {
        const float kv = hkey[k * 32 + lane];
        if (kv < T - 2.f * m) {
          ++A;
        } else if (kv <= T + 2.f * m) {
          if (nu >= 8) {
            ok = false;
            break;
          }
          const uint32_t id = hidx[k * 32 + lane];
          double x = chord2_exact(nodes.px[id], nodes.py[id], nodes.pz[id], ax, ay, az);
#pragma unroll
          for (int s2 = 0; s2 < 8; ++s2) {
            if (s2 < nu) {
              if (ue[s2] > x) {
                const double tt = ue[s2];
                ue[s2] = x;
                x = tt;
              }
            } else if (s2 == nu) {
              ue[s2] = x;
            }
          }
          ++nu;
        }
      }
    }
    double res = __longlong_as_double(0x7ff0000000000000ll);
    const int want = n - A - 1;
    if (ok && want >= 0 && want < nu) {
#pragma unroll
      for (int s2 = 0; s2 < 8; ++s2)
        if (s2 == want) res = ue[s2];
    } else {
      ok = false;
    }
    // lanes that could not conclude: exact warp search, one by one
    unsigned redo = __ballot_sync(FULL, act && !ok);
    nins = warp_sum(nins);
    if (lane == 0) {
      atomicAdd(&st->cnt[C_KNN_CAND], ncand);
      atomicAdd(&st->cnt[C_KNN_INS], nins);
      if (redo) atomicAdd(&st->cnt[C_KNN_LANE_FB], (unsigned long long)__popc(redo));
    }
    while (redo) {
      const int src = __ffs(redo) - 1;
      redo &= redo - 1;
      const double qx = __shfl_sync(FULL, ax, src), qy = __shfl_sync(FULL, ay, src), qz = __shfl_sync(FULL, az, src);
      bool f2 = false;
      const double v = knn_nth(nodes, qx, qy, qz, n, kscr, r0, &f2, &st->cnt[C_KNN_EXACT_FB]);
      if (lane == src) {
        res = v;
        failed = failed || f2;
      }
    }
    if (act) {
      if (failed || !(res < 1e300)) set_flag(st, ST_KNN);
      const double dn = geodesic_from_chord2(res);
      dn_sorted[fi] = dn;
      dn_f[fi] = (float)dn;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(KNN_WARPS * 32) knn_query_kernel(Cells nodes, const double* __restrict__ q,
                                                                   int64_t nq, int n, double r0,
                                                                   double* __restrict__ out, DevStatus* st) {
  __shared__ __align__(16) unsigned char lists[KNN_WARPS][KNN_SCRATCH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * KNN_WARPS;
  for (int64_t i = (int64_t)blockIdx.x * KNN_WARPS + warp; i < nq; i += nw) {
    bool failed = false;
    double c2 = knn_nth(nodes, q[3 * i], q[3 * i + 1], q[3 * i + 2], n, lists[warp], r0, &failed);
    if (lane == 0) {
      if (failed) set_flag(st, ST_KNN);
      out[i] = c2;
    }
  }
}

// --------------------------------------------------------- Shepard / delta
template <bool F64>
__global__ void __launch_bounds__(128) shepard_kernel(SupportArgs a, double rho_aux2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int L = 2 * a.N + 2, MQ = (a.N + 1) * L;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const float rho_f = (float)a.rho_aux, r2_f = (float)rho_aux2, irho_f = 1.f / rho_f;
  for (int j = warp; j < MQ; j += nw) {
    const int k = j / L, jj = j - k * L;
    const float qxf = a.sf[k] * a.cpf[jj], qyf = a.sf[k] * a.spf[jj], qzf = a.tf[k];
    Cap c = make_cap_f(qxf, qyf, qzf, rho_f);
    if (F64) {
      // FP64 form: exact membership and FP64 weights (FP32 only pre-filters)
      const double qx = a.ring_s[k] * a.cphi[jj], qy = a.ring_s[k] * a.sphi[jj], qz = a.ring_t[k];
      const float hi_f = (float)(rho_aux2 + c2_margin(rho_aux2));
      double sw = 0.0, swd = 0.0;
      for_cap_candidates(a.aux, c, [&](bool valid, uint32_t idx) {
        if (!valid) return;
        const float4 p = a.aux.pf[idx];
        const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
        if (dx * dx + dy * dy + dz * dz > hi_f) return;
        const double c2 = chord2_exact(a.aux.px[idx], a.aux.py[idx], a.aux.pz[idx], qx, qy, qz);
        if (!(c2 < rho_aux2)) return;
        const double w = wendland(geodesic_from_chord2(c2) / a.rho_aux);
        sw += w;
        swd += w * a.dn_aux_sorted[idx];
      });
      sw = warp_sum(sw);
      swd = warp_sum(swd);
      if (lane == 0) {
        const double PI = 3.14159265358979323846;
        double delta = (1.0 + a.eps) * (swd / sw);
        if (!(sw > 0.0) || !(delta < 0.5 * PI)) {
          set_flag(a.st, ST_SUPPORT);
          delta = fmin(delta, 0.5 * PI);
          if (!(delta > 0.0)) delta = 0.5 * PI;
        }
        const double sr = sin(0.5 * delta);
        const double rho2 = 4.0 * sr * sr;
        a.delta[j] = delta;
        a.rho2[j] = rho2;
        a.deltaf[j] = (float)delta;
        a.rho2f[j] = (float)rho2;
        a.guarded[j] = 0;
      }
    } else {
      // MIXED: the support radius in FP32 throughout
      float sw = 0.f, swd = 0.f;
      for_cap_candidates(a.aux, c, [&](bool valid, uint32_t idx) {
        if (!valid) return;
        const float4 p = a.aux.pf[idx];
        const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
        const float c2f = dx * dx + dy * dy + dz * dz;
        if (!(c2f < r2_f)) return;
        const float w = wendland(geodesic_from_chord2(c2f) * irho_f);
        sw += w;
        swd += w * a.dn_aux_f[idx];
      });
      sw = warp_sum(sw);
      swd = warp_sum(swd);
      if (lane == 0) {
        const float HPI = 1.57079632f;
        float delta = (1.f + (float)a.eps) * (swd / sw);
        if (!(sw > 0.f) || !(delta < HPI)) {
          set_flag(a.st, ST_SUPPORT);
          delta = fminf(delta, HPI);
          if (!(delta > 0.f)) delta = HPI;
        }
        const float sr = sinf(0.5f * delta);
        const float rho2 = 4.f * sr * sr;
        a.deltaf[j] = delta;
        a.rho2f[j] = rho2;
        a.delta[j] = (double)delta;
        a.rho2[j] = (double)rho2;
        a.guarded[j] = 0;
      }
    }
  }
}

// ------------------------------------------------------ neighbour counts
// exact #{i : |x_i - q|^2 < rho2} (FP32 certain-in / certain-out, FP64 only
// for the few candidates within the FP32 error bound of the boundary). The
// FP32 query and radius come from FP32 tables: no FP64 work per candidate.
__device__ __forceinline__ uint32_t ball_count(const Cells& g, float qxf, float qyf, float qzf, double qx, double qy,
                                               double qz, float deltaf, double rho2) {
  const float r2f = (float)rho2;
  // q here is a product of FP32 table entries (error up to ~2e-7 per coordinate)
  const float mg = 2e-6f * sqrtf(r2f) + 2e-6f * r2f + 1e-13f;
  const float lo = r2f - mg, hi = r2f + mg;
  uint32_t cnt = 0;
  Cap c = make_cap_f(qxf, qyf, qzf, deltaf);
  for_cap_candidates(g, c, [&](bool valid, uint32_t idx) {
    if (!valid) return;
    const float4 p = g.pf[idx];
    const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
    const float c2f = dx * dx + dy * dy + dz * dz;
    if (c2f < lo) {
      ++cnt;
    } else if (c2f <= hi) {
      if (chord2_exact(g.px[idx], g.py[idx], g.pz[idx], qx, qy, qz) < rho2) ++cnt;
    }
  });
  return warp_sum(cnt);
}

__global__ void __launch_bounds__(128) count_kernel(SupportArgs a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int L = 2 * a.N + 2, MQ = (a.N + 1) * L;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < MQ; j += nw) {
    const int k = j / L, jj = j - k * L;
    const double qx = a.ring_s[k] * a.cphi[jj], qy = a.ring_s[k] * a.sphi[jj], qz = a.ring_t[k];
    const float qxf = a.sf[k] * a.cpf[jj], qyf = a.sf[k] * a.spf[jj], qzf = a.tf[k];
    uint32_t cnt = ball_count(a.nodes, qxf, qyf, qzf, qx, qy, qz, a.deltaf[j], a.rho2[j]);
    if (lane == 0) {
      a.count[j] = (int32_t)cnt;
      if ((int)cnt < a.m) {
        unsigned long long pos = atomicAdd(&a.st->cnt[C_GUARD_LIST], 1ull);
        a.guard_list[pos] = (uint32_t)j;
      }
    }
  }
}

// guard: delta = (1 + eps) d_n(q) computed exactly at q (Sec. 2.2 notes that
// the smoothed radius holds at least n nodes only for a fine enough auxiliary
// grid; this restores #X(q) >= m where it does not)
__global__ void __launch_bounds__(KNN_WARPS * 32) guard_kernel(SupportArgs a, double r0) {
  __shared__ __align__(16) unsigned char lists[KNN_WARPS][KNN_SCRATCH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = 2 * a.N + 2;
  const int nw = gridDim.x * KNN_WARPS;
  const int total = (int)a.st->cnt[C_GUARD_LIST];
  for (int e = blockIdx.x * KNN_WARPS + warp; e < total; e += nw) {
    const int j = (int)a.guard_list[e];
    const int k = j / L, jj = j - k * L;
    const double qx = a.ring_s[k] * a.cphi[jj], qy = a.ring_s[k] * a.sphi[jj], qz = a.ring_t[k];
    bool failed = false;
    double c2 = knn_nth(a.nodes, qx, qy, qz, a.n_target, lists[warp], r0, &failed);
    double delta = (1.0 + a.eps) * geodesic_from_chord2(c2);
    const double PI = 3.14159265358979323846;
    bool bad = failed || !(delta < 0.5 * PI);
    if (bad) delta = 0.5 * PI;
    const double sr = sin(0.5 * delta);
    const double rho2 = 4.0 * sr * sr;
    uint32_t cnt = ball_count(a.nodes, (float)qx, (float)qy, (float)qz, qx, qy, qz, (float)delta, rho2);
    if (lane == 0) {
      if (bad) set_flag(a.st, ST_SUPPORT);
      if ((int)cnt < a.m) set_flag(a.st, ST_UNDERDET);
      a.delta[j] = delta;
      a.rho2[j] = rho2;
      a.deltaf[j] = (float)delta;
      a.rho2f[j] = (float)rho2;
      a.count[j] = (int32_t)cnt;
      a.guarded[j] = 1;
    }
  }
}

// cost keys for the MLS work order (heaviest first) and n(q) statistics
__global__ void order_keys_kernel(SupportArgs a, int MQ) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long c = 0, mn = ~0ull, mx = 0, g = 0;
  if (j < MQ) {
    int cnt = a.count[j];
    c = (unsigned long long)cnt;
    mn = mx = c;
    g = a.guarded[j];
    a.order_keys[j] = 0xFFFFFu - (uint32_t)min(cnt, 0xFFFFF);
    a.order_vals[j] = (uint32_t)j;
  }
  c = warp_sum(c);
  g = warp_sum(g);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(FULL, mn, o));
    mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&a.st->cnt[C_SUM_N], c);
    atomicAdd(&a.st->cnt[C_GUARD], g);
    atomicMin(&a.st->cnt[C_MIN_N], mn);
    atomicMax(&a.st->cnt[C_MAX_N], mx);
  }
}

static int grid_for(int work_warps, int warps_per_block, int cap_blocks) {
  int b = (work_warps + warps_per_block - 1) / warps_per_block;
  return b < 1 ? 1 : (b > cap_blocks ? cap_blocks : b);
}

static double initial_radius(int n, int M) { return 2.0 * sqrt((double)n / (double)(M > 0 ? M : 1)); }

void run_aux_knn(const SupportArgs& a, cudaStream_t s, int64_t* launches) {
  const size_t smem = tile_warp_bytes(a.n_target) * TK_WARPS;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(aux_knn_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aux_knn_tile_kernel, TK_WARPS * 32, smem);
  if (per_sm < 1) per_sm = 1;
  aux_knn_tile_kernel<<<per_sm * a.num_sms, TK_WARPS * 32, smem, s>>>(
      a.nodes, a.aux, a.tile_order, a.n_target, initial_radius(a.n_target, a.nodes.n), a.dn_aux_sorted, a.dn_aux_f,
      a.st, &a.st->cnt[C_TILE]);
  ++*launches;
}

void run_shepard(const SupportArgs& a, cudaStream_t s, int64_t* launches) {
  const int MQ = (a.N + 1) * (2 * a.N + 2);
  const double sr = sin(0.5 * a.rho_aux);
  const double rho_aux2 = 4.0 * sr * sr;
  const int blocks = grid_for(MQ, 4, 148 * 16);
  if (a.fp64)
    shepard_kernel<true><<<blocks, 128, 0, s>>>(a, rho_aux2);
  else
    shepard_kernel<false><<<blocks, 128, 0, s>>>(a, rho_aux2);
  ++*launches;
}

void run_counts(const SupportArgs& a, cudaStream_t s, int64_t* launches) {
  const int MQ = (a.N + 1) * (2 * a.N + 2);
  count_kernel<<<grid_for(MQ, 4, 148 * 16), 128, 0, s>>>(a);
  guard_kernel<<<148 * 2, KNN_WARPS * 32, 0, s>>>(a, initial_radius(a.n_target, a.nodes.n));
  order_keys_kernel<<<(MQ + 255) / 256, 256, 0, s>>>(a, MQ);
  *launches += 3;
}

void run_knn_queries(const Cells& nodes, const double* q, int64_t nq, int n, double* c2_out, DevStatus* st,
                     cudaStream_t s, int64_t* launches) {
  if (nq <= 0) return;
  knn_query_kernel<<<grid_for((int)nq, KNN_WARPS, 148 * 16), KNN_WARPS * 32, 0, s>>>(
      nodes, q, nq, n, initial_radius(n, nodes.n), c2_out, st);
  ++*launches;
}

__global__ void __launch_bounds__(128) ball_query_kernel(Cells g, const double* __restrict__ q,
                                                         const double* __restrict__ rho2, int64_t nq,
                                                         int64_t* __restrict__ count, int64_t* __restrict__ idsum,
                                                         uint64_t* __restrict__ idhash) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < nq; j += nw) {
    const double qx = q[3 * j], qy = q[3 * j + 1], qz = q[3 * j + 2], r2 = rho2[j];
    const double delta = 2.0 * asin(fmin(1.0, 0.5 * sqrt(r2)));
    const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
    const double mg = c2_margin(r2);
    const float lo = (float)(r2 - mg), hi = (float)(r2 + mg);
    unsigned long long cnt = 0, sum = 0, hx = 0;
    Cap c = make_cap(qx, qy, qz, delta);
    for_cap_candidates(g, c, [&](bool valid, uint32_t idx) {
      if (!valid) return;
      float4 p = g.pf[idx];
      float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
      float c2f = dx * dx + dy * dy + dz * dz;
      bool in = false;
      if (c2f < lo) in = true;
      else if (c2f <= hi) in = chord2_exact(g.px[idx], g.py[idx], g.pz[idx], qx, qy, qz) < r2;
      if (in) {
        uint32_t o = g.perm[idx];
        ++cnt;
        sum += o;
        hx ^= splitmix64(o);
      }
    });
    cnt = warp_sum(cnt);
    sum = warp_sum(sum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hx ^= __shfl_xor_sync(FULL, hx, o);
    if (lane == 0) {
      count[j] = (int64_t)cnt;
      idsum[j] = (int64_t)sum;
      idhash[j] = hx;
    }
  }
}

void run_ball_queries(const Cells& nodes, const double* q, const double* rho2, int64_t nq, int64_t* count,
                      int64_t* idsum, uint64_t* idhash, cudaStream_t s, int64_t* launches) {
  if (nq <= 0) return;
  ball_query_kernel<<<grid_for((int)nq, 4, 148 * 16), 128, 0, s>>>(nodes, q, rho2, nq, count, idsum, idhash);
  ++*launches;
}

}  // namespace hamls
