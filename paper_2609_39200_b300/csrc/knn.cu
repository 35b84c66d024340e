// knn.cu - the adaptive support radius of Sec. 2.2.
//
//   d_n(a)   distance to the n-th nearest node (eq. adaptive_support_radius),
//            at every point of a Fibonacci auxiliary grid (aux_knn_kernel);
//   d~_n(q)  its degree-zero MLS (Shepard) approximation with a constant
//            support radius rho_aux, at every quadrature node q: the members
//            and weights depend on the plan only and are stored once as a
//            sparse operator (shepard_rows_kernel), applied per replan
//            (shepard_apply_kernel);
//   delta(q) = (1 + eps) d~_n(q); n(q) = #X(q) (eq. number_of_local_nodes) is
//            counted by the MLS gather;
//   guard    if n(q) < m, delta(q) = (1 + eps) d_n(q) computed exactly at q
//            (guard_kernel, inside the fit, for the positions the gather lists).
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
__device__ __noinline__ double knn_nth_exact(const Cells& g, double qx, double qy, double qz, int n, double* list, double r0,
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

constexpr int KL_MAX = 16;                             // FP32 chords a lane keeps (n > 48)
constexpr int KNN_SCRATCH = KNN_MAX * 8 + 32 * 4;      // warp scratch: exact-path list, uncertain ids

// Phase 1 of a search without a known radius: a radius whose candidate
// enumeration (counted from the run table alone) holds a few times n points.
__device__ __noinline__ float knn_initial_radius(const Cells& g, float qxf, float qyf, float qzf, int n, float r0) {
  const float PI_F = 3.14159265f;
  float r = fminf(fmaxf(r0, 1e-7f), PI_F), rlo = 0.f, rhi = PI_F;
  bool have_lo = false, have_hi = false;
  const uint32_t lowT = (uint32_t)n + (uint32_t)n / 4 + 4u, highT = 16u * (uint32_t)n + 64u;
  for (int it = 0; it < 80; ++it) {
    Cap c = make_cap_f(qxf, qyf, qzf, r);
    const uint32_t bc = cap_box_count(g, c);
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
  return r;
}

// FP32 geodesic distance of a squared chord for the search radii and their
// bounds (each used with a relative margin of 1e-5 or more): the arcsin
// series below a half-chord of 1/4, asinf (clamped to 1) above
__device__ __forceinline__ float geodesic_f(float c2) {
  const float s = 0.5f * sqrtf(c2);
  return s > 0.25f ? 2.f * asinf(fminf(1.f, s)) : geodesic_series_f(c2);
}

// A radius beyond r for a cap that held fewer than n points: the enumeration
// at the new radius (counted from the run table alone) holds about 2 to 8
// times as many points as at r, so the scans of a search grow geometrically
// in work even where the radius must cross an empty region (a hole in the
// node set) and a fixed radius factor would add a huge annulus.
__device__ __noinline__ float knn_grow_radius(const Cells& g, float qxf, float qyf, float qzf, float r, int n) {
  const float PI_F = 3.14159265f;
  const uint32_t bc0 = cap_box_count(g, make_cap_f(qxf, qyf, qzf, r));
  const uint32_t lowT = max(2u * bc0, (uint32_t)n + (uint32_t)n / 4 + 4u), highT = 4u * lowT + 64u;
  float rlo = r, rhi = PI_F, d = 0.125f;
  bool have_hi = false;
  for (int it = 0; it < 60; ++it) {
    const float r1 = have_hi ? sqrtf(rlo * rhi) : fminf(rlo * (1.f + d) + 1e-6f, PI_F);
    const uint32_t bc = cap_box_count(g, make_cap_f(qxf, qyf, qzf, r1));
    if (bc < lowT) {
      if (r1 >= PI_F) return PI_F;
      rlo = r1;
      d *= 2.f;
    } else if (bc > highT) {
      rhi = r1;
      have_hi = true;
    } else {
      return r1;
    }
    if (have_hi && rhi < rlo * 1.002f) return rhi;
  }
  return have_hi ? rhi : PI_F;
}

// One scan of the cap of radius r. Every lane keeps, in registers, the KL
// smallest FP32 squared chords among the candidates it is dealt (sorted,
// with indices) - no warp-serialised list. The n-th smallest key T over the
// warp is bracketed, tl < T <= th, by a search on values that stops once
// th - tl is within the FP32 error bound m or (tl, th] holds at most 8 keys. Then
// keys < tl - 2m are certainly among the n nearest (A of them), keys above
// th + 2m certainly not, and the answer is the (n - A)-th smallest exact FP64
// chord among the keys in [tl - 2m, th + 2m].
// Returns 0 with the exact n-th chord in nth, 1 when the cap was too small
// (r_next to retry), 2 when a lane's list may have dropped a needed key or
// too many keys are uncertain (the caller runs the exact search).
// Per-lane tallies of a search (summed over the warp when reported).
struct KnnTally {
  uint32_t cand = 0, scans = 0;
};

template <int KL>
__device__ int knn_select(const Cells& g, double qx, double qy, double qz, float r, int n, uint32_t* ustage,
                          double& nth, float& r_next, KnnTally& tally) {
  const int lane = threadIdx.x & 31;
  const float PI_F = 3.14159265f;
  const float INF_F = __int_as_float(0x7f800000);
  const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
  float key[KL];
  uint32_t kid[KL];
#pragma unroll
  for (int s2 = 0; s2 < KL; ++s2) {
    key[s2] = INF_F;
    kid[s2] = 0xFFFFFFFFu;
  }
  Cap c = make_cap_f(qxf, qyf, qzf, r);
  ++tally.scans;
  // only points of the cap can be among the n nearest when it holds n of
  // them; the bound is the widened radius's squared chord plus the FP32 error
  const float rc2 = 4.f * c.rs * c.rs;                // squared chord of the widened radius
  const float rcap2 = rc2 * (1.f + 1e-6f) + c2_margin_f(rc2) + 1e-12f;
  for_cap_candidates<true>(g, c, [&](bool valid, uint32_t idx) {
    if (!valid) return;
    ++tally.cand;
    const float4 p = g.pf[idx];
    const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
    const float x = dx * dx + dy * dy + dz * dz;
    if (x < key[KL - 1] && x <= rcap2) {
      // insert after equal keys: every slot decides from the old list at once
      bool gt[KL];
#pragma unroll
      for (int s2 = 0; s2 < KL; ++s2) gt[s2] = key[s2] > x;
#pragma unroll
      for (int s2 = KL - 1; s2 > 0; --s2) {
        key[s2] = gt[s2] ? (gt[s2 - 1] ? key[s2 - 1] : x) : key[s2];
        kid[s2] = gt[s2] ? (gt[s2 - 1] ? kid[s2 - 1] : idx) : kid[s2];
      }
      key[0] = gt[0] ? x : key[0];
      kid[0] = gt[0] ? idx : kid[0];
    }
  });
  int fin = 0;
#pragma unroll
  for (int s2 = 0; s2 < KL; ++s2) fin += key[s2] < INF_F ? 1 : 0;
  const int fin_total = warp_sum(fin);
  if (fin_total < n) {                          // fewer than n points in the cap
    if (__any_sync(FULL, key[KL - 1] < INF_F)) return 2;  // unless a lane list overflowed
    r_next = knn_grow_radius(g, qxf, qyf, qzf, r, n);
    return 1;
  }
  // Isolate the n-th smallest key T in a window (tl, th] with cl = count(<= tl)
  // < n <= ch = count(<= th): interpolation on the counts (the keys are
  // roughly uniform in squared chord, i.e. in area), safeguarded to cut at
  // least an eighth of the window, until the window holds at most 8 keys or is
  // narrower than the FP32 error bound.
  float th = 0.f;
#pragma unroll
  for (int s2 = 0; s2 < KL; ++s2)
    if (key[s2] < INF_F) th = fmaxf(th, key[s2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) th = fmaxf(th, __shfl_xor_sync(FULL, th, o));
  // (at most 8 keys: the exact step below ranks up to 32 in parallel, and
  // narrowing further costs a count per step, many where the keys of a node
  // track crowd together)
  float tl = -1e-30f;
  int cl = 0, ch = fin_total;
  for (int it = 0; it < 48 && ch - cl > 8; ++it) {
    const float w = th - tl;
    if (w <= c2_margin_f(th)) break;
    float f = __fdividef((float)(n - cl) - 0.5f, (float)(ch - cl));
    f = fminf(fmaxf(f, 0.125f), 0.875f);
    const float mid = tl + w * f;
    int cnt = 0;
#pragma unroll
    for (int s2 = 0; s2 < KL; ++s2) cnt += key[s2] <= mid ? 1 : 0;
    const int c = warp_sum(cnt);
    if (c >= n) {
      th = mid;
      ch = c;
    } else {
      tl = mid;
      cl = c;
    }
  }
  const float m = c2_margin_f(th);
  const float tlo = tl - 2.f * m, thi = th + 2.f * m;
  // a full lane list dropped keys >= its last one: they must lie above thi
  if (__any_sync(FULL, key[KL - 1] <= thi)) return 2;
  int A = 0, mine = 0;
#pragma unroll
  for (int s2 = 0; s2 < KL; ++s2) {
    A += key[s2] < tlo ? 1 : 0;
    mine += (key[s2] >= tlo && key[s2] <= thi) ? 1 : 0;
  }
  A = warp_sum(A);
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const int nu = __shfl_sync(FULL, incl, 31);
  if (nu > 32 || n - A < 1 || nu < n - A) return 2;
  int off = incl - mine;
#pragma unroll
  for (int s2 = 0; s2 < KL; ++s2)
    if (key[s2] >= tlo && key[s2] <= thi) ustage[off++] = kid[s2];
  __syncwarp();
  double e = __longlong_as_double(0x7ff0000000000000ll);
  if (lane < nu) {
    const uint32_t id = ustage[lane];
    e = chord2_exact(g.px[id], g.py[id], g.pz[id], qx, qy, qz);
  }
  // ranks on the bit patterns (non-negative doubles and +inf order as
  // integers), off the FP64 pipe
  const long long eb = __double_as_longlong(e);
  int rank = 0;
  for (int s2 = 0; s2 < nu; ++s2) {
    const long long o = __shfl_sync(FULL, eb, s2);
    rank += (o < eb || (o == eb && s2 < lane)) ? 1 : 0;
  }
  const unsigned hit = __ballot_sync(FULL, lane < nu && rank == n - A - 1);
  nth = __longlong_as_double(__shfl_sync(FULL, eb, __ffs(hit) - 1));
  __syncwarp();
  // every point within geodesic r of q was enumerated; is the n-th inside?
  const float gn = geodesic_f((float)nth);
  if (gn * (1.f + 2e-6f) <= r || r >= PI_F) return 0;
  // the cap through the n-th candidate holds n points: the next scan is final
  r_next = fminf(PI_F, gn * (1.f + 1e-5f) + 1e-6f);
  return 1;
}

// n-th smallest exact squared chord from q to the points of g (+inf and
// *failed when there are fewer than n points). r_hint > 0: a radius known to
// hold at least n points (then one scan suffices); otherwise phase 1 finds one.
// KL: length of the per-lane lists (8, 12 or 16 for the auxiliary grid by n, 16 elsewhere).
template <int KL>
__device__ double knn_nth(const Cells& g, double qx, double qy, double qz, int n, unsigned char* scratch,
                          double r0, bool* failed, KnnTally& tally,
                          unsigned long long* exact_fb = nullptr, float r_hint = -1.f) {
  const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
  float r = r_hint > 0.f ? fminf(r_hint, 3.14159265f) : knn_initial_radius(g, qxf, qyf, qzf, n, (float)r0);
  uint32_t* ustage = reinterpret_cast<uint32_t*>(scratch + KNN_MAX * 8);
  for (int it = 0; it < 64; ++it) {
    double nth;
    float rn = r;
    const int rc = knn_select<KL>(g, qx, qy, qz, r, n, ustage, nth, rn, tally);
    if (rc == 0) return nth;
    if (rc == 2) {
      if (exact_fb && (threadIdx.x & 31) == 0) atomicAdd(exact_fb, 1ull);
      return knn_nth_exact(g, qx, qy, qz, n, reinterpret_cast<double*>(scratch), r0, failed);
    }
    if (r >= 3.14159265f) break;
    r = rn;
  }
  *failed = true;
  return __longlong_as_double(0x7ff0000000000000ll);
}

// d_n at the auxiliary points. A warp walks chunks of AK_CHUNK consecutive
// points of a spatially coherent order (thin latitude bands, then longitude;
// chunks handed out dynamically). Each search starts from the previous
// point's exact d_n plus the distance between the two points: d_n is
// 1-Lipschitz, so that cap holds at least n nodes and one scan suffices. The
// exact chords of a chunk become geodesic distances together, 32 per FP64
// asin instruction.
constexpr int AK_WARPS = 4;
constexpr int AK_CHUNK = 32;

template <int KL>
__global__ void __launch_bounds__(AK_WARPS * 32) aux_knn_kernel(Cells nodes, Cells aux,
                                                                const uint32_t* __restrict__ order, int n, double r0,
                                                                double* __restrict__ dn_sorted,
                                                                float* __restrict__ dn_f, DevStatus* st,
                                                                unsigned long long* ctr) {
  __shared__ __align__(16) unsigned char scr[AK_WARPS][KNN_SCRATCH];
  __shared__ double res[AK_WARPS][AK_CHUNK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  KnnTally tally;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1ull);
    t = __shfl_sync(FULL, t, 0);
    const long long first = (long long)t * AK_CHUNK;
    if (first >= aux.n) break;
    const int cnt = (int)min((long long)AK_CHUNK, (long long)aux.n - first);
    float prev = -1.f, pxf = 0.f, pyf = 0.f, pzf = 0.f;
    bool failed = false;
    for (int k = 0; k < cnt; ++k) {
      const uint32_t fi = order[first + k];
      const double ax = aux.px[fi], ay = aux.py[fi], az = aux.pz[fi];
      const float axf = (float)ax, ayf = (float)ay, azf = (float)az;
      float hint = -1.f;
      if (prev >= 0.f) {
        const float dx = axf - pxf, dy = ayf - pyf, dz = azf - pzf;
        hint = (prev + geodesic_f(dx * dx + dy * dy + dz * dz)) * (1.f + 1e-5f) + 2e-6f;
      }
      const double c2 = knn_nth<KL>(nodes, ax, ay, az, n, scr[warp], r0, &failed, tally, &st->cnt[C_KNN_EXACT_FB],
                                    hint);
      prev = (c2 < 1e300) ? geodesic_f((float)c2) : -1.f;
      pxf = axf;
      pyf = ayf;
      pzf = azf;
      if (lane == 0) res[warp][k] = c2;
    }
    __syncwarp();
    if (failed && lane == 0) set_flag(st, ST_KNN);
    for (int k = lane; k < cnt; k += 32) {
      const double c2 = res[warp][k];
      if (!(c2 < 1e300)) set_flag(st, ST_KNN);
      const uint32_t fi = order[first + k];
      const double dn = geodesic_from_chord2(c2);
      dn_sorted[fi] = dn;
      dn_f[fi] = (float)dn;
    }
    __syncwarp();
  }
  const unsigned long long cand = warp_sum((unsigned long long)tally.cand);
  if (lane == 0) {
    atomicAdd(&st->cnt[C_KNN_CAND], cand);
    atomicAdd(&st->cnt[C_KNN_SCAN], (unsigned long long)tally.scans);
  }
}

template <int KL>
__global__ void __launch_bounds__(KNN_WARPS * 32) knn_query_kernel(Cells nodes, const double* __restrict__ q,
                                                                   int64_t nq, int n, double r0,
                                                                   double* __restrict__ out, DevStatus* st) {
  __shared__ __align__(16) unsigned char lists[KNN_WARPS][KNN_SCRATCH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * KNN_WARPS;
  for (int64_t i = (int64_t)blockIdx.x * KNN_WARPS + warp; i < nq; i += nw) {
    bool failed = false;
    KnnTally tally;
    double c2 = knn_nth<KL>(nodes, q[3 * i], q[3 * i + 1], q[3 * i + 2], n, lists[warp], r0, &failed, tally);
    if (lane == 0) {
      if (failed) set_flag(st, ST_KNN);
      out[i] = c2;
    }
  }
}

// --------------------------------------------------------- Shepard / delta
// Work-order key of a grid node, heaviest first: the support radius, in
// octaves of the uniform-density radius d_typ = 2 sqrt(n/M), stands in for
// the node's cost (large radii sit in holes of the node set, where a cap
// collects its nodes from a long rim). Within a class the stable sort keeps
// the grid order, so consecutive work shares cached nodes.
__device__ __forceinline__ uint32_t order_key(float delta, float dtyp) {
  const float c = fminf(fmaxf(log2f(fmaxf(delta, 1e-30f) / dtyp), 0.f), 7.f);
  return 7u - (uint32_t)c;
}

// The Shepard operator. The auxiliary grid, the quadrature grid and rho_aux
// depend on the plan only, so the members of every grid node's Shepard cap
// and their Wendland weights phi(d(q, a)/rho_aux) are found once, at plan
// time, and each replan applies them to the new d_n:
//   d~_n(q) = sum_a w_qa d_n(a) / sum_a w_qa.
// FP64 form: exact membership and FP64 weights (FP32 only pre-filters);
// MIXED: FP32 throughout. Members are stored in enumeration order.
template <bool F64, bool FILL>
__global__ void __launch_bounds__(128) shepard_rows_kernel(SupportArgs a, double rho_aux2, uint32_t* rows,
                                                           uint32_t* col, void* wv, void* swv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int L = 2 * a.N + 2, MQ = (a.N + 1) * L;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const float rho_f = (float)a.rho_aux, r2_f = (float)rho_aux2, irho_f = 1.f / rho_f;
  const float hi_f = (float)(rho_aux2 + c2_margin(rho_aux2));
  for (int j = warp; j < MQ; j += nw) {
    const int k = j / L, jj = j - k * L;
    const float qxf = a.sf[k] * a.cpf[jj], qyf = a.sf[k] * a.spf[jj], qzf = a.tf[k];
    const double qx = a.ring_s[k] * a.cphi[jj], qy = a.ring_s[k] * a.sphi[jj], qz = a.ring_t[k];
    const Cap c = make_cap_f(qxf, qyf, qzf, rho_f);
    uint32_t pos = FILL ? rows[j] : 0u;
    double sw = 0.0;
    float swf = 0.f;
    for_cap_candidates(a.aux, c, [&](bool valid, uint32_t idx) {
      bool in = false;
      double w = 0.0;
      float wf = 0.f;
      if (valid) {
        const float4 p = a.aux.pf[idx];
        const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
        const float c2f = dx * dx + dy * dy + dz * dz;
        if (F64) {
          if (c2f <= hi_f) {
            const double c2 = chord2_exact(a.aux.px[idx], a.aux.py[idx], a.aux.pz[idx], qx, qy, qz);
            in = c2 < rho_aux2;
            if (in && FILL) w = weight_phi(a.weight_fn, geodesic_from_chord2(c2) / a.rho_aux);
          }
        } else {
          in = c2f < r2_f;
          if (in && FILL) wf = weight_phi(a.weight_fn, geodesic_from_chord2(c2f) * irho_f);
        }
      }
      const unsigned b = __ballot_sync(FULL, in);
      if (FILL && in) {
        const uint32_t e = pos + __popc(b & ((1u << lane) - 1u));
        col[e] = idx;
        if (F64) {
          reinterpret_cast<double*>(wv)[e] = w;
          sw += w;
        } else {
          reinterpret_cast<float*>(wv)[e] = wf;
          swf += wf;
        }
      }
      pos += __popc(b);
    });
    if (FILL) {
      if (F64) {
        sw = warp_sum(sw);
        if (lane == 0) reinterpret_cast<double*>(swv)[j] = sw;
      } else {
        swf = warp_sum(swf);
        if (lane == 0) reinterpret_cast<float*>(swv)[j] = swf;
      }
    } else if (lane == 0) {
      rows[j] = pos;
    }
  }
}

// delta(q) = (1 + eps) d~_n(q) with the Shepard operator; one thread per grid
// node (about 28 members each), summing its members in stored order. Also
// resets the guard flag and writes the work-order key.
template <bool F64>
__global__ void __launch_bounds__(256) shepard_apply_kernel(SupportArgs a) {
  using T = typename std::conditional<F64, double, float>::type;
  const int MQ = (a.N + 1) * (2 * a.N + 2);
  const T* w = reinterpret_cast<const T*>(a.shep_w);
  const T* sws = reinterpret_cast<const T*>(a.shep_sw);
  const T* dn = F64 ? reinterpret_cast<const T*>(a.dn_aux_sorted) : reinterpret_cast<const T*>(a.dn_aux_f);
  const float dtyp = 2.f * sqrtf((float)a.n_target / (float)a.nodes.n);
  // four lanes per row (a row holds about a dozen members): interleaved,
  // coalesced reads of the row, then two shuffles
  constexpr int G = 4;
  const int lane = threadIdx.x & 31, g = lane & (G - 1);
  const int rows_per_pass = gridDim.x * (blockDim.x / G);
  for (int jw = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / G; jw < MQ; jw += rows_per_pass) {
    const int j = jw + lane / G;
    T swd = T(0);
    if (j < MQ) {
      const uint32_t e0 = a.shep_start[j], e1 = a.shep_start[j + 1];
      for (uint32_t e = e0 + g; e < e1; e += G) swd += w[e] * dn[a.shep_col[e]];
    }
    swd += __shfl_xor_sync(FULL, swd, 1);
    swd += __shfl_xor_sync(FULL, swd, 2);
    if (j >= MQ || g != 0) continue;
    const T sw = sws[j];
    if (F64) {
      const double PI = 3.14159265358979323846;
      double delta = (1.0 + a.eps) * ((double)swd / (double)sw);
      if (!(sw > 0) || !(delta < 0.5 * PI)) {
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
      a.order_keys[j] = order_key((float)delta, dtyp);
    } else {
      const float HPI = 1.57079632f;
      float delta = (1.f + (float)a.eps) * ((float)swd / (float)sw);
      if (!(sw > 0) || !(delta < HPI)) {
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
      a.order_keys[j] = order_key(delta, dtyp);
    }
    a.guarded[j] = 0;
    a.order_vals[j] = (uint32_t)j;
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
    const int j = (int)a.order[a.guard_list[e]];
    const int k = j / L, jj = j - k * L;
    const double qx = a.ring_s[k] * a.cphi[jj], qy = a.ring_s[k] * a.sphi[jj], qz = a.ring_t[k];
    bool failed = false;
    KnnTally tally;
    double c2 = knn_nth<KL_MAX>(a.nodes, qx, qy, qz, a.n_target, lists[warp], r0, &failed, tally);
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
      atomicAdd(&a.st->cnt[C_SUM_N], (unsigned long long)cnt);
      atomicAdd(&a.st->cnt[C_GUARD], 1ull);
      atomicMin(&a.st->cnt[C_MIN_N], (unsigned long long)cnt);
      atomicMax(&a.st->cnt[C_MAX_N], (unsigned long long)cnt);
    }
  }
}

static int grid_for(int work_warps, int warps_per_block, int cap_blocks) {
  int b = (work_warps + warps_per_block - 1) / warps_per_block;
  return b < 1 ? 1 : (b > cap_blocks ? cap_blocks : b);
}

static double initial_radius(int n, int M) { return 2.0 * sqrt((double)n / (double)(M > 0 ? M : 1)); }

template <int KL>
static void launch_aux_knn(const SupportArgs& a, cudaStream_t s) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aux_knn_kernel<KL>, AK_WARPS * 32, 0);
  if (per_sm < 1) per_sm = 1;
  aux_knn_kernel<KL><<<per_sm * a.num_sms, AK_WARPS * 32, 0, s>>>(a.nodes, a.aux, a.tile_order, a.n_target,
                                                                  initial_radius(a.n_target, a.nodes.n),
                                                                  a.dn_aux_sorted, a.dn_aux_f, a.st,
                                                                  &a.st->cnt[C_TILE]);
}

// Lane lists of 8, 12 or 16 keys: a lane holds about n/32 of the keys up to
// the n-th, and a list that fills up to the bracket sends the point to the
// exact search, so the length keeps that rare (n = 40: 1.25 per lane, a
// lane with 8 of them about 3e-5) while each candidate costs a fixed
// compare-and-select network of the list's length.
void run_aux_knn(const SupportArgs& a, cudaStream_t s, int64_t* launches) {
  if (a.n_target <= 40)
    launch_aux_knn<8>(a, s);
  else if (a.n_target <= 48)
    launch_aux_knn<12>(a, s);
  else
    launch_aux_knn<KL_MAX>(a, s);
  ++*launches;
}

static double aux_radius2(const SupportArgs& a) {
  const double sr = sin(0.5 * a.rho_aux);
  return 4.0 * sr * sr;
}

void shepard_rows(const SupportArgs& a, uint32_t* rows, uint32_t* col, void* w, void* sw, bool fill,
                  cudaStream_t s, int64_t* launches) {
  const int MQ = (a.N + 1) * (2 * a.N + 2);
  const int blocks = grid_for(MQ, 4, a.num_sms * 16);
  const double r2 = aux_radius2(a);
  if (a.fp64) {
    if (fill)
      shepard_rows_kernel<true, true><<<blocks, 128, 0, s>>>(a, r2, rows, col, w, sw);
    else
      shepard_rows_kernel<true, false><<<blocks, 128, 0, s>>>(a, r2, rows, col, w, sw);
  } else {
    if (fill)
      shepard_rows_kernel<false, true><<<blocks, 128, 0, s>>>(a, r2, rows, col, w, sw);
    else
      shepard_rows_kernel<false, false><<<blocks, 128, 0, s>>>(a, r2, rows, col, w, sw);
  }
  ++*launches;
}

void run_shepard(const SupportArgs& a, cudaStream_t s, int64_t* launches) {
  const int MQ = (a.N + 1) * (2 * a.N + 2);
  const int blocks = (4 * MQ + 255) / 256;   // four lanes per row
  if (a.fp64)
    shepard_apply_kernel<true><<<blocks, 256, 0, s>>>(a);
  else
    shepard_apply_kernel<false><<<blocks, 256, 0, s>>>(a);
  ++*launches;
}

void run_guard(const SupportArgs& a, cudaStream_t s, int64_t* launches) {
  guard_kernel<<<a.num_sms * 2, KNN_WARPS * 32, 0, s>>>(a, initial_radius(a.n_target, a.nodes.n));
  ++*launches;
}

void run_knn_queries(const Cells& nodes, const double* q, int64_t nq, int n, double* c2_out, DevStatus* st,
                     cudaStream_t s, int64_t* launches) {
  if (nq <= 0) return;
  const int blocks = grid_for((int)nq, KNN_WARPS, current_sm_count() * 16);
  if (n <= 48)
    knn_query_kernel<12><<<blocks, KNN_WARPS * 32, 0, s>>>(nodes, q, nq, n, initial_radius(n, nodes.n), c2_out, st);
  else
    knn_query_kernel<KL_MAX><<<blocks, KNN_WARPS * 32, 0, s>>>(nodes, q, nq, n, initial_radius(n, nodes.n), c2_out,
                                                               st);
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
  ball_query_kernel<<<grid_for((int)nq, 4, current_sm_count() * 16), 128, 0, s>>>(nodes, q, rho2, nq, count, idsum, idhash);
  ++*launches;
}

}  // namespace hamls
