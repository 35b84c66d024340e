// mls.cu - Algorithm 1 step 2: the regularised MLS value at every quadrature
// node (Sec. 2.2, 2.3).
//
// Per grid node q with support radius delta and local nodes X(q) (open
// geodesic ball, eq. mls_local_node_set):
//   weights   w_i = v_i phi(d(q, x_i)/delta), Wendland phi (eq. weight_function_radial);
//   basis     monomials u^a v^b, a + b <= K, of the tangent coordinates of the
//             orthogonal projection onto T_q S^2 (Pi_K^tan), ascending degree;
//   Gram      H = B^T B of eq. (mls local vectors) with unit-norm columns. It is
//             assembled from the weighted moments sum_i w_i u^a v^b (a+b <= 2K)
//             and sum_i w_i y_i u^a v^b (a+b <= K): every Gram entry is one
//             moment, scaled by the column norms and the weight sum;
//   solve     C = L L^T (eq. mls local Cholesky factor), d = L^{-1} b,
//             e = L^{-1} z, r_0 = |d|^2, chi = 1/(1 - r_0) (eq. chi via
//             coupling); if chi > chi_T, tau by bisection on
//             r_tau = sum_j d_j^2 / (1 + tau mu_j) = 1 - 1/chi_T (eq.
//             regularized MLS amplification); tau~ = S(t) tau with the C^3
//             smoothstep S and t = (chi - chi_T)/(chi_full - chi_T);
//   value     c_1 = (beta - sum_j d_j e_j/(1 + tau~ mu_j)) / (1 - sum_j d_j^2/(1 + tau~ mu_j)),
//             the first coefficient of the regularised problem (eq. regularized
//             MLS problem) in closed form (Schur complement of its normal equations).
//
// Execution: the gather kernel gives each grid node (heaviest first) to one
// warp: the 32 lanes stream its candidates (coalesced runs of the sorted
// points), test the ball, count n(q), accumulate the moments and
// reduce-scatter them into a moment buffer. The solve kernel then runs one
// local problem per thread.
//
// Values-only refits (end of this file): for fixed nodes c_1 is linear in the
// value moments, so the fit is stored as a sparse operator of the values.
//
// Precision forms: FP64 (everything in double) and MIXED (FP32 gather and
// moments on centred, delta-scaled coordinates, FP32 solve; nodes whose FP32
// Cholesky meets a tiny pivot are re-solved in FP64 from the same moments).
#include <type_traits>
#include "common.cuh"
#include "kernels.h"

namespace hamls {

__host__ __device__ constexpr int dim_tan(int K) { return (K + 1) * (K + 2) / 2; }
__host__ __device__ constexpr int deg_of(int j) {
  int k = 0;
  while ((k + 1) * (k + 2) / 2 <= j) ++k;
  return k;
}
__host__ __device__ constexpr int ea_of(int j) { return deg_of(j) - (j - deg_of(j) * (deg_of(j) + 1) / 2); }
__host__ __device__ constexpr int eb_of(int j) { return j - deg_of(j) * (deg_of(j) + 1) / 2; }
__host__ __device__ constexpr int midx(int a, int b, int D) { return b * (D + 1) - b * (b - 1) / 2 + a; }
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <int K>
struct Shape {
  static constexpr int m = dim_tan(K);
  static constexpr int mm = m - 1;
  static constexpr int NM = dim_tan(2 * K);   // weighted moments, degree <= 2K
  static constexpr int NY = dim_tan(K);       // value moments, degree <= K
  static constexpr int NV = NM + NY;
};

struct SolveParams {
  double chiT, chiF, floor_;
  double mu[KMAX + 1];
};

template <typename S>
__device__ __forceinline__ S smoothstep3(S t) {
  S t2 = t * t;
  return t2 * t2 * (S(35) + t * (S(-84) + t * (S(70) - S(20) * t)));
}

template <typename S>
__device__ __forceinline__ S rsqrt_t(S x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

// The local problem from its moments. mw: NM weighted moments, my: NY value
// moments (unnormalised weights). Returns c1; also chi, tau~, the smallest
// squared pivot and the number of dropped directions. With defer given, a
// problem with chi > chi_T stops before the bisection for tau and sets
// *defer (the caller solves it again, without defer, in a pass of its own).
// BT: arithmetic of the bisection for tau (FP32 is enough when S = double
// only serves to make the Cholesky of an ill-conditioned FP32 Gram reliable).
template <typename S, int K, typename BT = S>
__device__ __forceinline__ S solve_local(const S* mw, const S* my, const SolveParams& P, S& chi_out, S& tau_out,
                                         S& minpiv, int& ndrop, int* defer = nullptr) {
  constexpr int m = Shape<K>::m, mm = m - 1, D2 = 2 * K, D1 = K;
  const S W = mw[0];
  S is[m];
#pragma unroll
  for (int j = 1; j < m; ++j) {
    const S g = mw[midx(2 * ea_of(j), 2 * eb_of(j), D2)];
    is[j] = g > S(0) ? rsqrt_t<S>(g) : S(0);
  }
  const S isW = rsqrt_t<S>(W);
  S L[mm * (mm + 1) / 2];
#pragma unroll
  for (int i = 0; i < mm; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      L[tri(i, j)] = mw[midx(ea_of(i + 1) + ea_of(j + 1), eb_of(i + 1) + eb_of(j + 1), D2)] * is[i + 1] * is[j + 1];
  S bv[mm], zv[mm];
#pragma unroll
  for (int j = 0; j < mm; ++j) {
    bv[j] = mw[midx(ea_of(j + 1), eb_of(j + 1), D2)] * is[j + 1] * isW;
    zv[j] = my[midx(ea_of(j + 1), eb_of(j + 1), D1)] * is[j + 1] * isW;
  }
  const S beta = my[0] / W;
  // Cholesky with the pivot floor. In FP64 (slow square roots and
  // divisions on this pipe) 1/l_jj is one reciprocal square root, l_jj
  // = s_jj / sqrt(s_jj) one product, and the substitutions reuse 1/l_jj.
  bool drop[mm];
  S invd[mm];
  minpiv = S(1);
  ndrop = 0;
#pragma unroll
  for (int j = 0; j < mm; ++j) {
    S sjj = L[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) sjj -= L[tri(j, k)] * L[tri(j, k)];
    drop[j] = !(sjj > S(P.floor_));
    ndrop += drop[j] ? 1 : 0;
    minpiv = sjj < minpiv ? sjj : minpiv;
    S ljj, inv;
    if (sizeof(S) == 8) {
      inv = drop[j] ? S(0) : rsqrt_t<S>(sjj);
      ljj = drop[j] ? S(0) : sjj * inv;
    } else {
      ljj = drop[j] ? S(0) : sqrt(sjj);
      inv = drop[j] ? S(0) : S(1) / ljj;
    }
    invd[j] = inv;
    L[tri(j, j)] = ljj;
#pragma unroll
    for (int i = j + 1; i < mm; ++i) {
      S v = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[tri(i, k)] * L[tri(j, k)];
      L[tri(i, j)] = v * inv;
    }
  }
  // d = L^{-1} b, e = L^{-1} z, grouped by degree
  S d[mm], e[mm];
  S Dl[K + 1], Sl[K + 1];
#pragma unroll
  for (int l = 0; l <= K; ++l) Dl[l] = Sl[l] = S(0);
#pragma unroll
  for (int j = 0; j < mm; ++j) {
    S vb = bv[j], vz = zv[j];
#pragma unroll
    for (int k = 0; k < j; ++k) {
      vb -= L[tri(j, k)] * d[k];
      vz -= L[tri(j, k)] * e[k];
    }
    const S inv = (sizeof(S) == 8) ? invd[j] : (drop[j] ? S(0) : S(1) / L[tri(j, j)]);
    d[j] = vb * inv;
    e[j] = vz * inv;
    Dl[deg_of(j + 1)] += d[j] * d[j];
    Sl[deg_of(j + 1)] += d[j] * e[j];
  }
  S r0 = S(0);
#pragma unroll
  for (int l = 1; l <= K; ++l) r0 += Dl[l];
  const S inf = S(1) / S(0);
  const S chi = r0 < S(1) ? S(1) / (S(1) - r0) : inf;
  S tt = S(0);
  const S chiT = S(P.chiT);
  if (defer && chi > chiT) {
    *defer = 1;
    chi_out = chi;
    tau_out = S(0);
    return S(0);
  }
  if (chi > chiT) {
    BT Db[K + 1];
#pragma unroll
    for (int l = 1; l <= K; ++l) Db[l] = BT(Dl[l]);
    const BT rstar = BT(1) - BT(1) / BT(P.chiT);
    BT lo = BT(0), hi = BT(r0) / (BT(P.mu[1]) * rstar);
    const BT tol = sizeof(BT) == 8 ? BT(1e-16) : BT(1e-7);
    for (int it = 0; it < 200; ++it) {
      const BT mid = BT(0.5) * (lo + hi);
      BT r = BT(0);
#pragma unroll
      for (int l = 1; l <= K; ++l) r += Db[l] / (BT(1) + mid * BT(P.mu[l]));
      if (r > rstar) lo = mid;
      else hi = mid;
      if (hi - lo <= tol * hi) break;
    }
    const S tau = S(BT(0.5) * (lo + hi));
    S t = (chi == inf) ? S(1) : (chi - chiT) / (S(P.chiF) - chiT);
    t = t < S(1) ? t : S(1);
    tt = smoothstep3(t) * tau;
  }
  S num = beta, den = S(1);
#pragma unroll
  for (int l = 1; l <= K; ++l) {
    const S f = S(1) / (S(1) + tt * S(P.mu[l]));
    num -= Sl[l] * f;
    den -= Dl[l] * f;
  }
  chi_out = chi;
  tau_out = tt;
  return num / den;
}

template <typename T, int K>
__device__ __forceinline__ void accumulate(T (&acc)[Shape<K>::NV], T w, T u, T v, T y) {
  // w u^a and v^b once, then one fused multiply-add per moment
  constexpr int D2 = 2 * K, D1 = K, NM = Shape<K>::NM;
  T wu[D2 + 1], vp[D2 + 1];
  wu[0] = w;
  vp[0] = T(1);
  vp[1] = v;
#pragma unroll
  for (int e = 1; e <= D2; ++e) wu[e] = wu[e - 1] * u;
#pragma unroll
  for (int e = 2; e <= D2; ++e) vp[e] = vp[e - 1] * v;
#pragma unroll
  for (int a = 0; a <= D2; ++a) acc[midx(a, 0, D2)] += wu[a];
#pragma unroll
  for (int b = 1; b <= D2; ++b)
#pragma unroll
    for (int a = 0; a <= D2 - b; ++a) acc[midx(a, b, D2)] = fma(wu[a], vp[b], acc[midx(a, b, D2)]);
  T wyu[D1 + 1];
  wyu[0] = w * y;
#pragma unroll
  for (int e = 1; e <= D1; ++e) wyu[e] = wyu[e - 1] * u;
#pragma unroll
  for (int a = 0; a <= D1; ++a) acc[NM + midx(a, 0, D1)] += wyu[a];
#pragma unroll
  for (int b = 1; b <= D1; ++b)
#pragma unroll
    for (int a = 0; a <= D1 - b; ++a) acc[NM + midx(a, b, D1)] = fma(wyu[a], vp[b], acc[NM + midx(a, b, D1)]);
}

// The value weights of the local problem. For fixed nodes the Gram moments,
// chi and tau~ are fixed, and c1 is linear in the value moments my (Sec. 2.3:
// beta and e = L^{-1} z carry the data, nothing else does):
//   c1 = sum_k gamma_k my_k,
//   gamma_0 = 1 / (W den),
//   gamma_(a,b) = -h_j is_j isW / den for the basis direction j = (a, b),
// with h = L^{-T} g, g_j = d_j / (1 + tau~ mu_deg(j)) (the adjoint of the
// forward substitution, dropped directions contribute nothing). Same steps as
// solve_local up to tau~; FP64 throughout.
template <int K>
__device__ void solve_gamma(const double* mw, const SolveParams& P, double* gamma) {
  using S = double;
  constexpr int m = Shape<K>::m, mm = m - 1, D2 = 2 * K, D1 = K;
  const S W = mw[0];
  S is[m];
#pragma unroll
  for (int j = 1; j < m; ++j) {
    const S g = mw[midx(2 * ea_of(j), 2 * eb_of(j), D2)];
    is[j] = g > S(0) ? rsqrt_t<S>(g) : S(0);
  }
  const S isW = rsqrt_t<S>(W);
  S L[mm * (mm + 1) / 2];
#pragma unroll
  for (int i = 0; i < mm; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      L[tri(i, j)] = mw[midx(ea_of(i + 1) + ea_of(j + 1), eb_of(i + 1) + eb_of(j + 1), D2)] * is[i + 1] * is[j + 1];
  S bv[mm];
#pragma unroll
  for (int j = 0; j < mm; ++j) bv[j] = mw[midx(ea_of(j + 1), eb_of(j + 1), D2)] * is[j + 1] * isW;
  bool drop[mm];
  S inv[mm];
#pragma unroll
  for (int j = 0; j < mm; ++j) {
    S sjj = L[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) sjj -= L[tri(j, k)] * L[tri(j, k)];
    drop[j] = !(sjj > S(P.floor_));
    // as solve_local's FP64 form: 1/l_jj by one reciprocal square root
    inv[j] = drop[j] ? S(0) : rsqrt_t<S>(sjj);
    L[tri(j, j)] = drop[j] ? S(0) : sjj * inv[j];
#pragma unroll
    for (int i = j + 1; i < mm; ++i) {
      S v = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[tri(i, k)] * L[tri(j, k)];
      L[tri(i, j)] = v * inv[j];
    }
  }
  S d[mm];
  S Dl[K + 1];
#pragma unroll
  for (int l = 0; l <= K; ++l) Dl[l] = S(0);
#pragma unroll
  for (int j = 0; j < mm; ++j) {
    S vb = bv[j];
#pragma unroll
    for (int k = 0; k < j; ++k) vb -= L[tri(j, k)] * d[k];
    d[j] = vb * inv[j];
    Dl[deg_of(j + 1)] += d[j] * d[j];
  }
  S r0 = S(0);
#pragma unroll
  for (int l = 1; l <= K; ++l) r0 += Dl[l];
  const S infv = S(1) / S(0);
  const S chi = r0 < S(1) ? S(1) / (S(1) - r0) : infv;
  S tt = S(0);
  const S chiT = S(P.chiT);
  if (chi > chiT) {
    const S rstar = S(1) - S(1) / chiT;
    S lo = S(0), hi = r0 / (S(P.mu[1]) * rstar);
    for (int it = 0; it < 200; ++it) {
      const S mid = S(0.5) * (lo + hi);
      S r = S(0);
#pragma unroll
      for (int l = 1; l <= K; ++l) r += Dl[l] / (S(1) + mid * S(P.mu[l]));
      if (r > rstar) lo = mid;
      else hi = mid;
      if (hi - lo <= S(1e-16) * hi) break;
    }
    const S tau = S(0.5) * (lo + hi);
    S t = (chi == infv) ? S(1) : (chi - chiT) / (S(P.chiF) - chiT);
    t = t < S(1) ? t : S(1);
    tt = smoothstep3(t) * tau;
  }
  S f[K + 1], den = S(1);
  f[0] = S(0);
#pragma unroll
  for (int l = 1; l <= K; ++l) {
    f[l] = S(1) / (S(1) + tt * S(P.mu[l]));
    den -= Dl[l] * f[l];
  }
  S h[mm];
#pragma unroll
  for (int j = mm - 1; j >= 0; --j) {
    S v = f[deg_of(j + 1)] * d[j];
#pragma unroll
    for (int k = j + 1; k < mm; ++k) v -= L[tri(k, j)] * h[k];
    h[j] = v * inv[j];
  }
  gamma[0] = S(1) / (W * den);
#pragma unroll
  for (int j = 0; j < mm; ++j) gamma[midx(ea_of(j + 1), eb_of(j + 1), D1)] = -h[j] * is[j + 1] * isW / den;
}

constexpr int MLS_WARPS = 4;

// Warp reduce-scatter of NV <= 64 per-lane partial sums: five exchange steps
// (partner lane ^ 16, 8, 4, 2, 1), each halving, rounded up, the set a lane
// carries: a lane with the step's bit keeps the upper half and sends the
// lower one, the other the reverse, one shuffle per kept entry (38 -> 19 ->
// 10 -> 5 -> 3 -> 2 at K = 3: 39 shuffles). Afterwards each lane holds the
// totals of at most two entries; idx gives their original indices (-1 for a
// padding slot).
template <typename T, int S, int O, int H = (S + 1) / 2>
__device__ __forceinline__ void rs_step(const T (&in)[S], T (&out)[H], int lane) {
  const bool b = lane & O;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const T lo = in[i];
    const T hi = (H + i < S) ? in[(H + i < S) ? H + i : 0] : T(0);
    out[i] = (b ? hi : lo) + __shfl_xor_sync(FULL, b ? lo : hi, O);
  }
}

template <int S, int O>
__device__ __forceinline__ void rs_index(int lane, int& j, bool& valid) {
  constexpr int H = (S + 1) / 2;
  j = (lane & O) ? H + j : j;
  valid = valid && j < S;
}

template <typename T, int NV>
__device__ __forceinline__ void reduce_scatter(const T (&acc)[NV], T (&out)[2], int (&idx)[2]) {
  static_assert(NV <= 64, "at most 64 moments");
  constexpr int S1 = NV, S2 = (S1 + 1) / 2, S3 = (S2 + 1) / 2, S4 = (S3 + 1) / 2, S5 = (S4 + 1) / 2;
  constexpr int S6 = (S5 + 1) / 2;
  const int lane = threadIdx.x & 31;
  T v2[S2], v3[S3], v4[S4], v5[S5], v6[S6];
  rs_step<T, S1, 16>(acc, v2, lane);
  rs_step<T, S2, 8>(v2, v3, lane);
  rs_step<T, S3, 4>(v3, v4, lane);
  rs_step<T, S4, 2>(v4, v5, lane);
  rs_step<T, S5, 1>(v5, v6, lane);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    int j = i;
    bool valid = i < S6;
    rs_index<S5, 1>(lane, j, valid);
    rs_index<S4, 2>(lane, j, valid);
    rs_index<S3, 4>(lane, j, valid);
    rs_index<S2, 8>(lane, j, valid);
    rs_index<S1, 16>(lane, j, valid);
    out[i] = i < S6 ? v6[i < S6 ? i : 0] : T(0);
    idx[i] = valid ? j : -1;
  }
}

// Gather: one warp per grid node (heaviest first; the `heavy` first nodes of
// the work order are handed out one at a time, the rest in chunks of 16). The
// warp streams the node's candidates, accumulates the moments and writes them
// to mom[position * NVP + i] for the solve kernel.
//
// The gather also counts n(q) = #X(q) (eq. number_of_local_nodes) and lists
// the positions with n(q) < m for the guard. LIST = true gathers only the
// listed positions again, after the guard has widened their supports.
// WF: the weight function (0 phi_{3,2}, 1 phi_{3,1}) as a constant of the
// instance, so a member's weight is one polynomial with no selection.
template <int K, bool MIXED, bool LIST, int WF>
// 7 blocks of 4 warps per SM (at most 72 registers): more warps hide the
// gather's L2 latency better than the registers they cost
__global__ void __launch_bounds__(MLS_WARPS * 32, 7) mls_gather_kernel(MlsArgs a, unsigned long long* ctr,
                                                                    long long heavy) {
  using T = typename std::conditional<MIXED, float, double>::type;
  constexpr int NV = Shape<K>::NV, NVP = (NV + 1) & ~1;
  const int lane = threadIdx.x & 31;
  const int L = 2 * a.N + 2;
  T* mom = reinterpret_cast<T*>(a.mom);
  const long long items = LIST ? (long long)a.st->cnt[C_GUARD_LIST] : (long long)a.MQ;
  unsigned long long s_n = 0, s_min = ~0ull, s_max = 0, s_guarded = 0;   // lane 0's tallies
  for (;;) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(ctr, 1ull);
    c = __shfl_sync(FULL, c, 0);
    long long p0, p1;
    if (LIST || (long long)c < heavy) {
      p0 = (long long)c;
      p1 = p0 + 1;
    } else {
      p0 = heavy + ((long long)c - heavy) * 16;
      p1 = p0 + 16;
    }
    if (p0 >= items) break;
    if (p1 > items) p1 = items;
    for (long long it = p0; it < p1; ++it) {
      const long long pos = LIST ? (long long)a.guard_list[it] : it;
      const int j = (int)a.order[pos];
      uint32_t nin = 0;
      const int k = j / L, jj = j - k * L;
      T acc[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = T(0);
      if (MIXED) {
        // FP32 throughout: grid tables, support radius and frame in FP32
        const float st = a.sf[k], ct = a.tf[k], cp = a.cpf[jj], sp = a.spf[jj];
        const float qxf = st * cp, qyf = st * sp, qzf = ct;
        const float df = a.deltaf[j], r2f = a.rho2f[j], idf = 1.f / df;
        const float e1x = ct * cp * idf, e1y = ct * sp * idf, e1z = -st * idf;
        const float e2x = -sp * idf, e2y = cp * idf;
        Cap cap = make_cap_f(qxf, qyf, qzf, df);
        for_cap_candidates(a.nodes, cap, [&](bool valid, uint32_t idx) {
          if (!valid) return;
          const float4 p = a.nodes.pf[idx];
          const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
          const float c2 = dx * dx + dy * dy + dz * dz;
          if (!(c2 < r2f)) return;
          ++nin;
          float w = weight_phi(WF, geodesic_series_f(c2) * idf);
          if (a.swf) w *= a.swf[idx];
          const float u = e1x * dx + e1y * dy + e1z * dz;
          const float v = e2x * dx + e2y * dy;
          accumulate<T, K>(acc, (T)w, (T)u, (T)v, (T)p.w);
        });
      } else {
        const double st = a.ring_s[k], ct = a.ring_t[k], cp = a.cphi[jj], sp = a.sphi[jj];
        const double qx = st * cp, qy = st * sp, qz = ct;
        const double delta = a.delta[j], rho2 = a.rho2[j];
        // tangent frame scaled by 1/delta: e1 = d/dtheta, e2 = d/dphi
        const double id = 1.0 / delta;
        const double e1x = ct * cp * id, e1y = ct * sp * id, e1z = -st * id;
        const double e2x = -sp * id, e2y = cp * id;
        const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
        const float hi_f = (float)(rho2 + 1e-6 * sqrt(rho2) + 1e-6 * rho2 + 1e-13);
        Cap cap = make_cap_f(qxf, qyf, qzf, a.deltaf[j]);
        for_cap_candidates(a.nodes, cap, [&](bool valid, uint32_t idx) {
          if (!valid) return;
          const float4 p = a.nodes.pf[idx];
          const float fx = p.x - qxf, fy = p.y - qyf, fz = p.z - qzf;
          if (fx * fx + fy * fy + fz * fz > hi_f) return;
          const double X = a.nodes.px[idx], Y = a.nodes.py[idx], Z = a.nodes.pz[idx];
          const double c2 = chord2_exact(X, Y, Z, qx, qy, qz);
          if (!(c2 < rho2)) return;
          ++nin;
          const double dx = X - qx, dy = Y - qy, dz = Z - qz;
          double w = weight_phi(WF, geodesic_from_chord2(c2) * id);
          if (a.sw) w *= a.sw[idx];
          const double u = e1x * dx + e1y * dy + e1z * dz;
          const double v = e2x * dx + e2y * dy;
          accumulate<T, K>(acc, (T)w, (T)u, (T)v, (T)a.sy[idx]);
        });
      }
      T o[2];
      int oi[2];
      reduce_scatter<T, NV>(acc, o, oi);
      T* dst = mom + pos * NVP;
      if (oi[0] >= 0) dst[oi[0]] = o[0];
      if (oi[1] >= 0) dst[oi[1]] = o[1];
      if (!LIST) {
        nin = warp_sum(nin);
        if (lane == 0) {
          a.count[j] = (int32_t)nin;
          if ((int)nin < a.m) {
            const unsigned long long e = atomicAdd(&a.st->cnt[C_GUARD_LIST], 1ull);
            a.guard_list[e] = (uint32_t)pos;
          } else {
            s_n += nin;
            s_min = min(s_min, (unsigned long long)nin);
            s_max = max(s_max, (unsigned long long)nin);
            s_guarded += a.guarded[j];
          }
        }
      }
    }
  }
  if (!LIST && lane == 0) {
    atomicAdd(&a.st->cnt[C_SUM_N], s_n);
    atomicAdd(&a.st->cnt[C_GUARD], s_guarded);
    atomicMin(&a.st->cnt[C_MIN_N], s_min);
    atomicMax(&a.st->cnt[C_MAX_N], s_max);
  }
}

// Solve: one thread per grid node. MIXED solves in FP32; a node whose FP32
// Cholesky meets a tiny pivot is appended to a list and re-solved in FP64 by
// redo_kernel, so the FP64 work runs on full warps instead of diverging here.
// Likewise a node with chi > chi_T (about one in seven, so nearly every warp
// holds one) is listed for reg_kernel, which runs the bisection for tau on
// full warps; the others finish here.
template <int K, bool MIXED>
__global__ void __launch_bounds__(128) mls_solve_kernel(MlsArgs a, SolveParams P) {
  using T = typename std::conditional<MIXED, float, double>::type;
  constexpr int NV = Shape<K>::NV, NM = Shape<K>::NM, NVP = (NV + 1) & ~1;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = pos < a.MQ;
  const T* src = reinterpret_cast<const T*>(a.mom) + (act ? pos : 0) * NVP;
  T mom[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) mom[i] = act ? src[i] : (i == 0 ? T(1) : T(0));
  T chi, tau, minpiv;
  int ndrop, defer = 0;
  const T c1 = solve_local<T, K>(mom, mom + NM, P, chi, tau, minpiv, ndrop, &defer);
  const bool redo = MIXED && act && (ndrop > 0 || !(minpiv >= T(a.fp64_pivot)) || (!defer && !isfinite(c1)));
  const bool reg = act && !redo && defer;
  if (act && !redo && !reg) {
    const int j = (int)a.order[pos];
    a.fgrid[j] = (double)c1;
    a.chi[j] = (double)chi;
    a.tau[j] = (double)tau;
  }
  const unsigned rb = __ballot_sync(FULL, redo);
  if (rb) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.st->cnt[C_REDO_LIST], (unsigned long long)__popc(rb));
    base = __shfl_sync(FULL, base, 0);
    if (redo) a.redo_list[base + __popc(rb & ((1u << lane) - 1u))] = (uint32_t)pos;
  }
  const unsigned gb = __ballot_sync(FULL, reg);
  if (gb) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&a.st->cnt[C_REG_LIST], (unsigned long long)__popc(gb));
    base = __shfl_sync(FULL, base, 0);
    if (reg) a.reg_list[base + __popc(gb & ((1u << lane) - 1u))] = (uint32_t)pos;
  }
  const bool done = act && !redo && !reg;
  const unsigned long long nd = warp_sum((unsigned long long)(done ? ndrop : 0));
  if (lane == 0 && nd) atomicAdd(&a.st->cnt[C_DROP], nd);
}

// The listed nodes with chi > chi_T, solved again in full (bisection for
// tau included; the same arithmetic as a solve that never deferred). MIXED:
// a value that is not finite sends the node on to the FP64 re-solve.
template <int K, bool MIXED>
__global__ void __launch_bounds__(128) reg_kernel(MlsArgs a, SolveParams P) {
  using T = typename std::conditional<MIXED, float, double>::type;
  constexpr int NV = Shape<K>::NV, NM = Shape<K>::NM, NVP = (NV + 1) & ~1;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.st->cnt[C_REG_LIST];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < total; e0 += stride) {
    const long long e = e0 + lane;
    const bool act = e < total;
    const long long pos = act ? (long long)a.reg_list[e] : 0;
    const T* src = reinterpret_cast<const T*>(a.mom) + pos * NVP;
    T mom[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) mom[i] = act ? src[i] : (i == 0 ? T(1) : T(0));
    T chi, tau, minpiv;
    int ndrop;
    const T c1 = solve_local<T, K>(mom, mom + NM, P, chi, tau, minpiv, ndrop);
    const bool redo = MIXED && act && !isfinite(c1);
    if (act && !redo) {
      const int j = (int)a.order[pos];
      a.fgrid[j] = (double)c1;
      a.chi[j] = (double)chi;
      a.tau[j] = (double)tau;
    }
    const unsigned rb = __ballot_sync(FULL, redo);
    if (rb) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&a.st->cnt[C_REDO_LIST], (unsigned long long)__popc(rb));
      base = __shfl_sync(FULL, base, 0);
      if (redo) a.redo_list[base + __popc(rb & ((1u << lane) - 1u))] = (uint32_t)pos;
    }
    const unsigned long long nreg = __popc(__ballot_sync(FULL, act && !redo && tau > T(0)));
    const unsigned long long nd = warp_sum((unsigned long long)((act && !redo) ? ndrop : 0));
    if (lane == 0) {
      if (nreg) atomicAdd(&a.st->cnt[C_REG], nreg);
      if (nd) atomicAdd(&a.st->cnt[C_DROP], nd);
    }
  }
}

// MIXED: FP64 local solves of the listed nodes from their FP32 moments.
template <int K>
__global__ void __launch_bounds__(128) redo_kernel(MlsArgs a, SolveParams P) {
  constexpr int NV = Shape<K>::NV, NM = Shape<K>::NM, NVP = (NV + 1) & ~1;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.st->cnt[C_REDO_LIST];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < total; e0 += stride) {
    const long long e = e0 + lane;
    const bool act = e < total;
    const long long pos = act ? (long long)a.redo_list[e] : 0;
    const float* src = reinterpret_cast<const float*>(a.mom) + pos * NVP;
    double mom[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) mom[i] = act ? (double)src[i] : (i == 0 ? 1.0 : 0.0);
    double chi, tau, minpiv;
    int ndrop;
    const double c1 = solve_local<double, K, float>(mom, mom + NM, P, chi, tau, minpiv, ndrop);
    if (act) {
      const int j = (int)a.order[pos];
      a.fgrid[j] = c1;
      a.chi[j] = chi;
      a.tau[j] = tau;
    }
    const unsigned long long nreg = __popc(__ballot_sync(FULL, act && tau > 0.0));
    const unsigned long long nd = warp_sum((unsigned long long)(act ? ndrop : 0));
    const unsigned long long nr = __popc(__ballot_sync(FULL, act));
    if (lane == 0) {
      atomicAdd(&a.st->cnt[C_REG], nreg);
      atomicAdd(&a.st->cnt[C_DROP], nd);
      atomicAdd(&a.st->cnt[C_REDO], nr);
    }
  }
}

template <int K, bool MIXED, int WF>
static void launch_gather(const MlsArgs& a, unsigned long long* ctr, cudaStream_t s, int part) {
  if (part == 1) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mls_gather_kernel<K, MIXED, false, WF>, MLS_WARPS * 32,
                                                  0);
    if (per_sm < 1) per_sm = 1;
    const long long heavy = a.MQ < 4096 ? a.MQ : (a.MQ / 8 > 4096 ? a.MQ / 8 : 4096);
    mls_gather_kernel<K, MIXED, false, WF><<<per_sm * a.num_sms, MLS_WARPS * 32, 0, s>>>(a, ctr, heavy);
  } else {
    // the listed positions (usually none) gathered again with their guarded radii
    mls_gather_kernel<K, MIXED, true, WF><<<a.num_sms, MLS_WARPS * 32, 0, s>>>(a, &a.st->cnt[C_LIST_BATCH], 0);
  }
}

template <int K, bool MIXED>
static void launch_mls(const MlsArgs& a, const SolveParams& P, unsigned long long* ctr, cudaStream_t s,
                       int64_t* launches, int part) {
  if (a.weight_fn == 1)
    launch_gather<K, MIXED, 1>(a, ctr, s, part);
  else
    launch_gather<K, MIXED, 0>(a, ctr, s, part);
  if (part == 1) {
    ++*launches;
    return;
  }
  mls_solve_kernel<K, MIXED><<<(a.MQ + 127) / 128, 128, 0, s>>>(a, P);
  reg_kernel<K, MIXED><<<a.num_sms * 8, 128, 0, s>>>(a, P);
  *launches += 3;
  if (MIXED) {
    redo_kernel<K><<<a.num_sms * 8, 128, 0, s>>>(a, P);
    ++*launches;
  }
}

void run_mls(const MlsArgs& a, bool mixed, cudaStream_t s, int64_t* launches, int part) {
  SolveParams P;
  P.chiT = a.chiT;
  P.chiF = a.chiF;
  P.floor_ = a.floor_;
  for (int l = 0; l <= KMAX; ++l) P.mu[l] = a.mu[l];
  unsigned long long* ctr = &a.st->cnt[C_BATCH];
  switch (a.K * 2 + (mixed ? 1 : 0)) {
    case 2: launch_mls<1, false>(a, P, ctr, s, launches, part); break;
    case 3: launch_mls<1, true>(a, P, ctr, s, launches, part); break;
    case 4: launch_mls<2, false>(a, P, ctr, s, launches, part); break;
    case 5: launch_mls<2, true>(a, P, ctr, s, launches, part); break;
    case 6: launch_mls<3, false>(a, P, ctr, s, launches, part); break;
    case 7: launch_mls<3, true>(a, P, ctr, s, launches, part); break;
    case 8: launch_mls<4, false>(a, P, ctr, s, launches, part); break;
    case 9: launch_mls<4, true>(a, P, ctr, s, launches, part); break;
    default: break;
  }
}

// ------------------------------------------------ values-only refits
// The fit as a linear operator of the values for fixed nodes:
//   f(q_j) = sum_{i in X(q_j)} A_ji y_i,  A_ji = w_i sum_k gamma_jk u_i^a_k v_i^b_k,
// with gamma_j from solve_gamma on grid node j's Gram moments and (w_i, u_i,
// v_i) the weight and tangent coordinates of the gather.

// gamma per grid node (indexed by node, from the moments of its work position)
template <int K, bool MIXED>
__global__ void __launch_bounds__(128) gamma_kernel(MlsArgs a, SolveParams P, double* __restrict__ gamma) {
  using T = typename std::conditional<MIXED, float, double>::type;
  constexpr int NV = Shape<K>::NV, NM = Shape<K>::NM, NY = Shape<K>::NY, NVP = (NV + 1) & ~1;
  const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= a.MQ) return;
  const T* src = reinterpret_cast<const T*>(a.mom) + pos * NVP;
  double mw[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mw[i] = (double)src[i];
  double g[NY];
  solve_gamma<K>(mw, P, g);
  const int j = (int)a.order[pos];
#pragma unroll
  for (int i = 0; i < NY; ++i) gamma[(size_t)j * NY + i] = g[i];
}

// One warp per grid node: the members of its ball in the gather's order and
// test, counted (FILL = false: rows[j], and the total) or written
// (FILL = true: rows = CSR start; col = the node's position in the plan's
// cell order, val = A_ji). Columns in cell order keep the value reads of
// neighbouring rows close together.
template <int K, bool MIXED, bool FILL>
__global__ void __launch_bounds__(128) op_rows_kernel(MlsArgs a, const double* __restrict__ gamma, uint32_t* rows,
                                                      uint32_t* __restrict__ col, void* valv,
                                                      unsigned long long* total) {
  constexpr int NY = Shape<K>::NY, D1 = K;
  const int lane = threadIdx.x & 31;
  const int L = 2 * a.N + 2;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned below = (1u << lane) - 1u;
  unsigned long long tot = 0;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < a.MQ; j += nw) {
    const int k = j / L, jj = j - k * L;
    double gm[NY];
#pragma unroll
    for (int i = 0; i < NY; ++i) gm[i] = FILL ? gamma[(size_t)j * NY + i] : 0.0;
    uint32_t pos = FILL ? rows[j] : 0u;
    // A_ji from (w, u, v) in FP64
    auto entry = [&](double w, double u, double v) {
      double s = 0.0, vb = 1.0;
#pragma unroll
      for (int b = 0; b <= D1; ++b) {
        double t = vb;
#pragma unroll
        for (int aa = 0; aa <= D1 - b; ++aa) {
          s += gm[midx(aa, b, D1)] * t;
          if (aa < D1 - b) t *= u;
        }
        if (b < D1) vb *= v;
      }
      return w * s;
    };
    if (MIXED) {
      const float st = a.sf[k], ct = a.tf[k], cp = a.cpf[jj], sp = a.spf[jj];
      const float qxf = st * cp, qyf = st * sp, qzf = ct;
      const float df = a.deltaf[j], r2f = a.rho2f[j], idf = 1.f / df;
      const float e1x = ct * cp * idf, e1y = ct * sp * idf, e1z = -st * idf;
      const float e2x = -sp * idf, e2y = cp * idf;
      const Cap cap = make_cap_f(qxf, qyf, qzf, df);
      for_cap_candidates(a.nodes, cap, [&](bool valid, uint32_t idx) {
        bool in = false;
        float w = 0.f, u = 0.f, v = 0.f;
        if (valid) {
          const float4 p = a.nodes.pf[idx];
          const float dx = p.x - qxf, dy = p.y - qyf, dz = p.z - qzf;
          const float c2 = dx * dx + dy * dy + dz * dz;
          in = c2 < r2f;
          if (in && FILL) {
            w = weight_phi(a.weight_fn, geodesic_series_f(c2) * idf);
            if (a.swf) w *= a.swf[idx];
            u = e1x * dx + e1y * dy + e1z * dz;
            v = e2x * dx + e2y * dy;
          }
        }
        const unsigned bal = __ballot_sync(FULL, in);
        if (FILL && in) {
          const uint32_t e = pos + __popc(bal & below);
          col[e] = idx;
          reinterpret_cast<float*>(valv)[e] = (float)entry((double)w, (double)u, (double)v);
        }
        pos += __popc(bal);
      });
    } else {
      const double st = a.ring_s[k], ct = a.ring_t[k], cp = a.cphi[jj], sp = a.sphi[jj];
      const double qx = st * cp, qy = st * sp, qz = ct;
      const double delta = a.delta[j], rho2 = a.rho2[j];
      const double id = 1.0 / delta;
      const double e1x = ct * cp * id, e1y = ct * sp * id, e1z = -st * id;
      const double e2x = -sp * id, e2y = cp * id;
      const float qxf = (float)qx, qyf = (float)qy, qzf = (float)qz;
      const float hi_f = (float)(rho2 + 1e-6 * sqrt(rho2) + 1e-6 * rho2 + 1e-13);
      const Cap cap = make_cap_f(qxf, qyf, qzf, a.deltaf[j]);
      for_cap_candidates(a.nodes, cap, [&](bool valid, uint32_t idx) {
        bool in = false;
        double w = 0.0, u = 0.0, v = 0.0;
        if (valid) {
          const float4 p = a.nodes.pf[idx];
          const float fx = p.x - qxf, fy = p.y - qyf, fz = p.z - qzf;
          if (fx * fx + fy * fy + fz * fz <= hi_f) {
            const double X = a.nodes.px[idx], Y = a.nodes.py[idx], Z = a.nodes.pz[idx];
            const double c2 = chord2_exact(X, Y, Z, qx, qy, qz);
            in = c2 < rho2;
            if (in && FILL) {
              const double dx = X - qx, dy = Y - qy, dz = Z - qz;
              w = weight_phi(a.weight_fn, geodesic_from_chord2(c2) * id);
              if (a.sw) w *= a.sw[idx];
              u = e1x * dx + e1y * dy + e1z * dz;
              v = e2x * dx + e2y * dy;
            }
          }
        }
        const unsigned bal = __ballot_sync(FULL, in);
        if (FILL && in) {
          const uint32_t e = pos + __popc(bal & below);
          col[e] = idx;
          reinterpret_cast<double*>(valv)[e] = entry(w, u, v);
        }
        pos += __popc(bal);
      });
    }
    if (!FILL && lane == 0) {
      rows[j] = pos;
      tot += pos;
    }
  }
  if (!FILL && lane == 0 && tot) atomicAdd(total, tot);
}

// f(q_j) = sum A_ji y_i; one warp per grid node (rows run from ~30 to tens of
// thousands of entries), lane partial sums reduced in a tree. V = double:
// FP64 throughout; V = float: FP32 entries times FP32 values, the rounding
// level of the MIXED form's FP32 moments.
template <typename V>
__global__ void __launch_bounds__(256) op_apply_kernel(int MQ, const uint32_t* __restrict__ rows,
                                                       const uint32_t* __restrict__ col, const V* __restrict__ val,
                                                       const V* __restrict__ y, double* __restrict__ f,
                                                       DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < MQ; j += nw) {
    const uint32_t e0 = rows[j], e1 = rows[j + 1];
    V s = V(0);
    for (uint32_t e = e0 + lane; e < e1; e += 32) s += val[e] * y[col[e]];
    s = warp_sum(s);
    if (lane == 0) {
      if (!isfinite(s)) set_flag(st, ST_NONFINITE);
      f[j] = (double)s;
    }
  }
}

// the values in the plan's cell order: ys[s] = y[perm[s]] (FP64) or
// yf[s] = (float) y[perm[s]]
__global__ void gather_values_kernel(const double* __restrict__ y, const uint32_t* __restrict__ perm, int n,
                                     float* __restrict__ yf, double* __restrict__ ys) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = y[perm[i]];
  if (yf) yf[i] = (float)v;
  if (ys) ys[i] = v;
}

template <int K, bool MIXED>
static void launch_op(const MlsArgs& a, const SolveParams& P, int part, double* gamma, uint32_t* rows, uint32_t* col,
                      void* val, unsigned long long* total, cudaStream_t s, int64_t* launches) {
  const int wblocks = (a.MQ + 3) / 4 < a.num_sms * 64 ? (a.MQ + 3) / 4 : a.num_sms * 64;
  if (part == 0) {
    op_rows_kernel<K, MIXED, false><<<wblocks, 128, 0, s>>>(a, gamma, rows, col, val, total);
    ++*launches;
  } else {
    gamma_kernel<K, MIXED><<<(a.MQ + 127) / 128, 128, 0, s>>>(a, P, gamma);
    op_rows_kernel<K, MIXED, true><<<wblocks, 128, 0, s>>>(a, gamma, rows, col, val, total);
    *launches += 2;
  }
}

void run_refit_operator(const MlsArgs& a, bool mixed, int part, double* gamma, uint32_t* rows, uint32_t* col,
                        void* val, unsigned long long* total, cudaStream_t s, int64_t* launches) {
  SolveParams P;
  P.chiT = a.chiT;
  P.chiF = a.chiF;
  P.floor_ = a.floor_;
  for (int l = 0; l <= KMAX; ++l) P.mu[l] = a.mu[l];
  switch (a.K * 2 + (mixed ? 1 : 0)) {
    case 2: launch_op<1, false>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 3: launch_op<1, true>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 4: launch_op<2, false>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 5: launch_op<2, true>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 6: launch_op<3, false>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 7: launch_op<3, true>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 8: launch_op<4, false>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    case 9: launch_op<4, true>(a, P, part, gamma, rows, col, val, total, s, launches); break;
    default: break;
  }
}

void run_refit_apply(int MQ, bool mixed, const uint32_t* rows, const uint32_t* col, const void* val,
                     const double* y, const uint32_t* perm, int M, float* yf, double* ys, double* f, DevStatus* st,
                     cudaStream_t s, int64_t* launches) {
  const int cap = current_sm_count() * 64;
  const int blocks = (MQ + 7) / 8 < cap ? (MQ + 7) / 8 : cap;
  if (mixed) {
    gather_values_kernel<<<(M + 255) / 256, 256, 0, s>>>(y, perm, M, yf, nullptr);
    op_apply_kernel<float><<<blocks, 256, 0, s>>>(MQ, rows, col, reinterpret_cast<const float*>(val), yf, f, st);
  } else {
    gather_values_kernel<<<(M + 255) / 256, 256, 0, s>>>(y, perm, M, nullptr, ys);
    op_apply_kernel<double><<<blocks, 256, 0, s>>>(MQ, rows, col, reinterpret_cast<const double*>(val), ys, f, st);
  }
  *launches += 2;
}

// ---------------------------------------------- refits of many value sets
// The same operator applied to B value sets: y (B x M doubles, set b at b M)
// is transposed to M x B floats (the B values of one node contiguous) and its
// rows gathered into the plan's cell order (yT; the operator's columns),
// one warp per grid node walks its row once and every lane accumulates the
// sets b = lane, lane + 32, ... (each entry's B values are one coalesced
// read), giving fT (M_Q x B floats), transposed again to the B grids the
// batched step 3 takes (B x M_Q doubles).
__global__ void __launch_bounds__(256) to_float_t_kernel(const double* __restrict__ y, int B, int M,
                                                         float* __restrict__ yT) {
  __shared__ float t[32][33];
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, i = i0 + tx;
    t[r][tx] = (b < B && i < M) ? (float)y[(size_t)b * M + i] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, b = b0 + tx;
    if (i < M && b < B) yT[(size_t)i * B + b] = t[tx][r];
  }
}

// rows of B floats gathered into the plan's cell order: yT[s] = yo[perm[s]]
// (blocks of 32 sets x 8 rows)
__global__ void __launch_bounds__(256) gather_rows_kernel(const float* __restrict__ yo, const uint32_t* __restrict__ perm,
                                                          int M, int B, float* __restrict__ yT) {
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int b = blockIdx.y * 32 + (threadIdx.x & 31);
  if (r >= M || b >= B) return;
  yT[(size_t)r * B + b] = yo[(size_t)perm[r] * B + b];
}

// Rows of more than OP_LONG entries (grid nodes at the centre of a hole of
// the node set collect tens of thousands) are taken by whole blocks
// (op_apply_batch_long_kernel); the others by one warp each.
constexpr uint32_t OP_LONG = 256;

// the entries [e0, e1) of one row for the sets b = lane + 32 q
template <int BL>
__device__ __forceinline__ void op_row_part(const uint32_t* __restrict__ col, const float* __restrict__ val,
                                            const float* __restrict__ yT, int B, uint32_t e0, uint32_t e1,
                                            uint32_t step, float (&acc)[BL]) {
  const int lane = threadIdx.x & 31;
  for (uint32_t base = e0; base < e1; base += step) {
    const uint32_t e = base + lane;
    const uint32_t cl = e < e1 ? col[e] : 0u;
    const float vl = e < e1 ? val[e] : 0.f;
    const int cnt = (int)min(32u, e1 - base);
    for (int i = 0; i < cnt; i += 8) {
      float yv[8][BL];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t c = __shfl_sync(FULL, cl, (i + u) & 31);
        const float* yr = yT + (size_t)c * B;
#pragma unroll
        for (int q = 0; q < BL; ++q) {
          const int b = lane + 32 * q;
          yv[u][q] = (i + u < cnt && b < B) ? yr[b] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float v = __shfl_sync(FULL, vl, (i + u) & 31);
#pragma unroll
        for (int q = 0; q < BL; ++q) acc[q] = fmaf(v, yv[u][q], acc[q]);
      }
    }
  }
}

template <int BL>
__global__ void __launch_bounds__(256) op_apply_batch_long_kernel(const uint32_t* __restrict__ list,
                                                                  const uint32_t* __restrict__ nlist,
                                                                  const uint32_t* __restrict__ rows,
                                                                  const uint32_t* __restrict__ col,
                                                                  const float* __restrict__ val,
                                                                  const float* __restrict__ yT, int B,
                                                                  float* __restrict__ fT, DevStatus* st) {
  __shared__ float part[8][BL * 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t n = *nlist;
  for (uint32_t t = blockIdx.x; t < n; t += gridDim.x) {
    const uint32_t j = list[t];
    const uint32_t e0 = rows[j], e1 = rows[j + 1];
    float acc[BL];
#pragma unroll
    for (int q = 0; q < BL; ++q) acc[q] = 0.f;
    // warp w takes the 32-entry chunks w, w + 8, ... of the row
    op_row_part<BL>(col, val, yT, B, e0 + 32 * warp, e1, 256, acc);
#pragma unroll
    for (int q = 0; q < BL; ++q) part[warp][lane + 32 * q] = acc[q];
    __syncthreads();
    // the eight partial sums of every set, added in warp order
    if (warp == 0) {
      bool bad = false;
#pragma unroll
      for (int q = 0; q < BL; ++q) {
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += part[w][lane + 32 * q];
        const int b = lane + 32 * q;
        if (b < B) {
          if (!isfinite(sum)) bad = true;
          fT[(size_t)j * B + b] = sum;
        }
      }
      if (__any_sync(FULL, bad) && lane == 0) set_flag(st, ST_NONFINITE);
    }
    __syncthreads();
  }
}

// the rows of more than OP_LONG entries, listed (their count in *nlist)
__global__ void op_long_rows_kernel(int MQ, const uint32_t* __restrict__ rows, uint32_t* __restrict__ list,
                                    uint32_t* nlist) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < MQ && rows[j + 1] - rows[j] > OP_LONG) list[atomicAdd(nlist, 1u)] = (uint32_t)j;
}

template <int BL>
__global__ void __launch_bounds__(256) op_apply_batch_kernel(int MQ, const uint32_t* __restrict__ rows,
                                                             const uint32_t* __restrict__ col,
                                                             const float* __restrict__ val,
                                                             const float* __restrict__ yT, int B,
                                                             float* __restrict__ fT, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < MQ; j += nw) {
    const uint32_t e0 = rows[j], e1 = rows[j + 1];
    if (e1 - e0 > OP_LONG) continue;          // a block takes it
    float acc[BL];
#pragma unroll
    for (int q = 0; q < BL; ++q) acc[q] = 0.f;
    // 32 entries at a time (one coalesced load of columns and entries), then
    // their value rows eight at a time, all eight gathers in flight at once
    op_row_part<BL>(col, val, yT, B, e0, e1, 32, acc);
#pragma unroll
    for (int q = 0; q < BL; ++q) {
      const int b = lane + 32 * q;
      if (b < B) {
        if (!isfinite(acc[q])) bad = true;
        fT[(size_t)j * B + b] = acc[q];
      }
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) set_flag(st, ST_NONFINITE);
}

__global__ void __launch_bounds__(256) from_float_t_kernel(const float* __restrict__ fT, int MQ, int B,
                                                           double* __restrict__ f) {
  __shared__ float t[32][33];
  const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, b = b0 + tx;
    t[r][tx] = (j < MQ && b < B) ? fT[(size_t)j * B + b] : 0.f;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int b = b0 + r, j = j0 + tx;
    if (b < B && j < MQ) f[(size_t)b * MQ + j] = (double)t[tx][r];
  }
}

void list_long_rows(int MQ, const uint32_t* rows, uint32_t* list, uint32_t* nlist, cudaStream_t s,
                    int64_t* launches) {
  cudaMemsetAsync(nlist, 0, sizeof(uint32_t), s);
  op_long_rows_kernel<<<(MQ + 255) / 256, 256, 0, s>>>(MQ, rows, list, nlist);
  ++*launches;
}

void run_refit_apply_batch(int MQ, const uint32_t* rows, const uint32_t* col, const float* val, const double* y,
                           const uint32_t* perm, int M, int B, float* yo, float* yT, float* fT, double* f,
                           const uint32_t* long_list, const uint32_t* nlong, DevStatus* st, cudaStream_t s,
                           int64_t* launches) {
  to_float_t_kernel<<<dim3((M + 31) / 32, (B + 31) / 32), 256, 0, s>>>(y, B, M, yo);
  gather_rows_kernel<<<dim3((M + 7) / 8, (B + 31) / 32), 256, 0, s>>>(yo, perm, M, B, yT);
  const int cap = current_sm_count() * 64;
  const int blocks = (MQ + 7) / 8 < cap ? (MQ + 7) / 8 : cap;
  const int lblocks = current_sm_count() * 4;
#define HAMLS_OP_BATCH(BLV)                                                                               \
  op_apply_batch_kernel<BLV><<<blocks, 256, 0, s>>>(MQ, rows, col, val, yT, B, fT, st);                     \
  op_apply_batch_long_kernel<BLV><<<lblocks, 256, 0, s>>>(long_list, nlong, rows, col, val, yT, B, fT, st)
  if (B <= 32) {
    HAMLS_OP_BATCH(1);
  } else if (B <= 64) {
    HAMLS_OP_BATCH(2);
  } else if (B <= 128) {
    HAMLS_OP_BATCH(4);
  } else {
    HAMLS_OP_BATCH(8);
  }
#undef HAMLS_OP_BATCH
  ++*launches;
  from_float_t_kernel<<<dim3((MQ + 31) / 32, (B + 31) / 32), 256, 0, s>>>(fT, MQ, B, f);
  *launches += 4;
}

int value_moment_count(int K) { return (K + 1) * (K + 2) / 2; }

int mls_moment_slots(int K) {
  const int nv = dim_tan(2 * K) + dim_tan(K);
  return (nv + 1) & ~1;
}

}  // namespace hamls
