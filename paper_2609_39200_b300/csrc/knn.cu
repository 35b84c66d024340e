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
// set has fewer than n points). `list` is this warp's shared scratch (n slots).
__device__ double knn_nth(const Cells& g, double qx, double qy, double qz, int n, double* list, double r0,
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

__global__ void __launch_bounds__(KNN_WARPS * 32) aux_knn_kernel(Cells nodes, Cells aux, int n, double r0,
                                                                 double* __restrict__ dn_sorted, DevStatus* st) {
  __shared__ double lists[KNN_WARPS][KNN_MAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = gridDim.x * KNN_WARPS;
  for (int i = blockIdx.x * KNN_WARPS + warp; i < aux.n; i += nw) {
    bool failed = false;
    double c2 = knn_nth(nodes, aux.px[i], aux.py[i], aux.pz[i], n, lists[warp], r0, &failed);
    if (lane == 0) {
      if (failed || !(c2 < 1e300)) set_flag(st, ST_KNN);
      dn_sorted[i] = geodesic_from_chord2(c2);
    }
  }
}

__global__ void __launch_bounds__(KNN_WARPS * 32) knn_query_kernel(Cells nodes, const double* __restrict__ q,
                                                                   int64_t nq, int n, double r0,
                                                                   double* __restrict__ out, DevStatus* st) {
  __shared__ double lists[KNN_WARPS][KNN_MAX];
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
  const double PI = 3.14159265358979323846;
  for (int j = warp; j < MQ; j += nw) {
    const int k = j / L, jj = j - k * L;
    const double qx = a.ring_s[k] * a.cphi[jj], qy = a.ring_s[k] * a.sphi[jj], qz = a.ring_t[k];
    const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
    Cap c = make_cap(qx, qy, qz, a.rho_aux);
    double sw = 0.0, swd = 0.0;
    const double hi_f = rho_aux2 + c2_margin(rho_aux2);
    for_cap_candidates(a.aux, c, [&](bool valid, uint32_t idx) {
      if (!valid) return;
      float4 p = a.aux.pf[idx];
      float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
      float c2f = dx * dx + dy * dy + dz * dz;
      if (F64) {
        if ((double)c2f > hi_f) return;
        double c2 = chord2_exact(a.aux.px[idx], a.aux.py[idx], a.aux.pz[idx], qx, qy, qz);
        if (!(c2 < rho_aux2)) return;
        double w = wendland(geodesic_from_chord2(c2) / a.rho_aux);
        sw += w;
        swd += w * a.dn_aux_sorted[idx];
      } else {
        if (!(c2f < (float)rho_aux2)) return;
        float w = wendland(geodesic_from_chord2(c2f) / (float)a.rho_aux);
        sw += w;
        swd += (double)(w * (float)a.dn_aux_sorted[idx]);
      }
    });
    sw = warp_sum(sw);
    swd = warp_sum(swd);
    if (lane == 0) {
      double delta = (1.0 + a.eps) * (swd / sw);
      if (!(sw > 0.0) || !(delta < 0.5 * PI)) {
        set_flag(a.st, ST_SUPPORT);
        delta = fmin(delta, 0.5 * PI);
        if (!(delta > 0.0)) delta = 0.5 * PI;
      }
      a.delta[j] = delta;
      const double sr = sin(0.5 * delta);
      a.rho2[j] = 4.0 * sr * sr;
      a.guarded[j] = 0;
    }
  }
}

// ------------------------------------------------------ neighbour counts
// exact #{i : |x_i - q|^2 < rho2} (FP32 certain-in / certain-out, FP64 otherwise)
__device__ __forceinline__ uint32_t ball_count(const Cells& g, double qx, double qy, double qz, double delta,
                                               double rho2) {
  const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
  const double mg = c2_margin(rho2);
  const float lo = (float)(rho2 - mg), hi = (float)(rho2 + mg);
  uint32_t cnt = 0;
  Cap c = make_cap(qx, qy, qz, delta);
  for_cap_candidates(g, c, [&](bool valid, uint32_t idx) {
    if (!valid) return;
    float4 p = g.pf[idx];
    float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
    float c2f = dx * dx + dy * dy + dz * dz;
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
    uint32_t cnt = ball_count(a.nodes, qx, qy, qz, a.delta[j], a.rho2[j]);
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
  __shared__ double lists[KNN_WARPS][KNN_MAX];
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
    uint32_t cnt = ball_count(a.nodes, qx, qy, qz, delta, rho2);
    if (lane == 0) {
      if (bad) set_flag(a.st, ST_SUPPORT);
      if ((int)cnt < a.m) set_flag(a.st, ST_UNDERDET);
      a.delta[j] = delta;
      a.rho2[j] = rho2;
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
  aux_knn_kernel<<<grid_for(a.aux.n, KNN_WARPS, 148 * 16), KNN_WARPS * 32, 0, s>>>(
      a.nodes, a.aux, a.n_target, initial_radius(a.n_target, a.nodes.n), a.dn_aux_sorted, a.st);
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
