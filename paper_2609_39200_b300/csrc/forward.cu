// forward.cu - the forward transform of the problem statement (Sec. 1, the
// sampling matrix F of eq. LSQR-Problem_Regularized): values at points x of
// the real field with coefficients fhat (packed m >= 0, l = m..N; fully
// normalised spherical harmonics with the Condon-Shortley phase, the
// convention of the fit's coefficients),
//   f(x) = sum_l fhat_l^0 Pbar_l^0(t) + 2 Re sum_{m>=1} e^{i m phi} sum_{l>=m} fhat_l^m Pbar_l^m(t),
// t = cos theta. A thread takes four points; every thread of a warp walks the
// same (m, l) sequence, so coefficients and recurrence factors are uniform
// loads, each serving four recurrences.
//
// Everything in T (float for mixed plans, double for FP64 plans): per order m
// the seed Pbar_m^m = Pbar_{m-1}^{m-1} * (-sqrt((2m+1)/(2m)) sin theta) and
// e^{i m phi} by one rotation with e^{i phi} = (x + i y) / sin theta; per
// degree the three-term recurrence Pbar_l^m = a_lm (t Pbar_{l-1}^m - b_lm Pbar_{l-2}^m)
// (the plan's recurrence factors). In FP32 a term of order m and degree l
// carries a relative error of about (m + (l - m)) 2^-24 <= N 2^-24 from the
// seed chain, the rotation and the recurrence, inside the FP32 error bound of
// the whole sum, 2 (N + 3) 2^-24 sum |terms|. Near the poles the seed falls far below
// the FP32 range (sin theta = 0.1, m = 51: 1e-51) while Pbar_l^m climbs back
// to O(1) by l = 512, so the value carries a binary exponent e: the true
// value is p 2^e; the seed is rescaled by 2^60 whenever it falls below 2^-60,
// and the recurrence values, together with the order's sums kept in the same
// frame, are rescaled by 2^-60 (checked every eight degrees) whenever they
// pass 2^60 while e < 0. An order's sum enters f times 2^e (zero when
// e <= -120: then every term is below 2^-60 |fhat|).
#include "common.cuh"
#include "kernels.h"

namespace hamls {

namespace {

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using t = float2;
};
template <>
struct Vec2<double> {
  using t = double2;
};

// 2^e for the exponent frames (e = 0, -60, -120, ...), zero at and below
// 2^-120; built from the bit pattern (no FP64 operation)
template <typename T>
__device__ __forceinline__ T scale_of(int e);
template <>
__device__ __forceinline__ float scale_of<float>(int e) {
  return e <= -120 ? 0.f : __int_as_float((e + 127) << 23);
}
template <>
__device__ __forceinline__ double scale_of<double>(int e) {
  return e <= -120 ? 0.0 : __longlong_as_double((long long)(e + 1023) << 52);
}

}  // namespace

// packed complex coefficients (doubles, re/im interleaved) -> T2
template <typename T2>
__global__ void fwd_coeffs_kernel(const double* __restrict__ c, int64_t n, T2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    out[i].x = c[2 * i];
    out[i].y = c[2 * i + 1];
  }
}

// the recurrence factors (a_lm, b_lm) as T2, packed like the coefficients
template <typename T2>
__global__ void fwd_ab_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              T2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    out[i].x = a[i];
    out[i].y = b[i];
  }
}

// Points i = 0..P-1 at (px[i s], py[i s], pz[i s]); out[perm ? perm[i] : i].
// A thread takes FWD_PPT consecutive points (neighbours when they are the
// plan's sorted nodes), so that each coefficient and recurrence factor it
// loads serves FWD_PPT independent recurrences.
constexpr int FWD_PPT = 4;

template <typename T>
__global__ void __launch_bounds__(256) forward_kernel(int N, const typename Vec2<T>::t* __restrict__ cf,
                                                      const typename Vec2<T>::t* __restrict__ ab,
                                                      const double* __restrict__ px, const double* __restrict__ py,
                                                      const double* __restrict__ pz, int64_t stride, int64_t P,
                                                      const uint32_t* __restrict__ perm, double* __restrict__ out) {
  using T2 = typename Vec2<T>::t;
  constexpr int Q = FWD_PPT;
  extern __shared__ double fwd_smem[];
  T* fm = reinterpret_cast<T*>(fwd_smem);          // -sqrt((2m+1)/(2m)), m = 1..N
  T* g1 = reinterpret_cast<T*>(fwd_smem + N + 1);   // sqrt(2m+3): Pbar_{m+1}^m = g1 t Pbar_m^m
  float* kb = reinterpret_cast<float*>(fwd_smem + 2 * (N + 1));   // the order bound's constant
  for (int m = threadIdx.x; m <= N; m += blockDim.x) {
    fm[m] = (T)(m > 0 ? -sqrt((2.0 * m + 1.0) / (2.0 * m)) : 0.0);
    g1[m] = (T)sqrt(2.0 * m + 3.0);
    // |Pbar_l^m(t)| <= sqrt((2l+1)/(4 pi)) s^m sqrt((l+m)!/(l-m)!) / (2^m m!)
    // (|d^m P_l / dt^m| is largest at t = 1, where it is (l+m)!/(2^m m! (l-m)!)),
    // increasing in l: log2 of the bound at l = N, less m log2 s, plus
    // log2(N + 1) for the order's number of terms
    const double LN2 = 0.69314718055994530942;
    kb[m] = (float)(0.5 * log2((2.0 * N + 1.0) / (4.0 * 3.14159265358979323846)) +
                    (0.5 * (lgamma(N + m + 1.0) - lgamma(N - m + 1.0)) - lgamma(m + 1.0)) / LN2 - m +
                    log2(N + 1.0));
  }
  __syncthreads();
  const T HI = (T)1.152921504606846976e18;         // 2^60
  const T LO = (T)8.673617379884035472e-19;        // 2^-60
  const int64_t groups = (P + Q - 1) / Q;
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < groups;
       gi += (int64_t)gridDim.x * blockDim.x) {
    T s[Q], cph[Q], sph[Q], pmm[Q], cr[Q], sr[Q], f[Q], t[Q];
    float ls[Q];                                    // log2 sin theta (-inf at the poles)
    int em[Q];
    bool on[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int64_t i = gi * Q + q;
      on[q] = i < P;
      const int64_t ii = on[q] ? i : gi * Q;
      const double x = px[ii * stride], y = py[ii * stride], z = pz[ii * stride];
      const double sd = sqrt(x * x + y * y);
      s[q] = (T)sd;
      ls[q] = on[q] ? log2f((float)sd) : -__int_as_float(0x7f800000);
      cph[q] = sd > 0.0 ? (T)(x / sd) : T(1);
      sph[q] = sd > 0.0 ? (T)(y / sd) : T(0);
      t[q] = (T)z;
      pmm[q] = (T)0.28209479177387814347;           // Pbar_0^0 = 1 / sqrt(4 pi)
      em[q] = 0;                                    // Pbar_m^m = pmm 2^em
      cr[q] = T(1);                                 // e^{i m phi}
      sr[q] = T(0);
      f[q] = T(0);
    }
    for (int m = 0; m <= N; ++m) {
      const size_t row0 = (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
      // values and the order's sums in the frame 2^e of the point's seed
      T p1[Q], p2[Q], accr[Q], acci[Q];
      int e[Q];
      const T2 c0 = cf[row0];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (m > 0) {
          pmm[q] *= fm[m] * s[q];
          if (pmm[q] != T(0) && fabs(pmm[q]) < LO) {
            pmm[q] *= HI;
            em[q] -= 60;
          }
          const T c2 = cr[q] * cph[q] - sr[q] * sph[q];
          sr[q] = sr[q] * cph[q] + cr[q] * sph[q];
          cr[q] = c2;
        }
        e[q] = em[q];
        p2[q] = T(0);
        p1[q] = pmm[q];
        accr[q] = c0.x * p1[q];
        acci[q] = c0.y * p1[q];
      }
      // an order whose bound stays below 2^-80 for all of the thread's points
      // contributes less than 2^-80 max |fhat| to each of them: skipped
      bool need = m == 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) need |= (float)m * ls[q] + kb[m] >= -80.f;
      if (!need) continue;
      if (m < N) {
        const T2 c1 = cf[row0 + 1];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const T p = g1[m] * t[q] * p1[q];
          p2[q] = p1[q];
          p1[q] = p;
          accr[q] += c1.x * p;
          acci[q] += c1.y * p;
        }
      }
      // eight degrees per step, two at a time so that the recurrence
      // alternates between the two registers; a value (and the sums) leaving
      // [.., 2^60) while its frame is below 1 is rescaled once per step (the
      // growth over eight degrees is below 2^38, far inside the FP32 range)
      int l = m + 2;
      for (; l + 7 <= N; l += 8) {
        const size_t o = row0 + (size_t)(l - m);
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
          const T2 fa = ab[o + k], fb = ab[o + k + 1];
          const T2 ca = cf[o + k], cb = cf[o + k + 1];
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            p2[q] = fa.x * (t[q] * p1[q] - fa.y * p2[q]);
            accr[q] += ca.x * p2[q];
            acci[q] += ca.y * p2[q];
            p1[q] = fb.x * (t[q] * p2[q] - fb.y * p1[q]);
            accr[q] += cb.x * p1[q];
            acci[q] += cb.y * p1[q];
          }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (e[q] < 0 && fabs(p1[q]) > HI) {
            p1[q] *= LO;
            p2[q] *= LO;
            accr[q] *= LO;
            acci[q] *= LO;
            e[q] += 60;
          }
        }
      }
      for (; l <= N; ++l) {
        const size_t o = row0 + (size_t)(l - m);
        const T2 f2 = ab[o];
        const T2 c = cf[o];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const T p = f2.x * (t[q] * p1[q] - f2.y * p2[q]);
          p2[q] = p1[q];
          p1[q] = p;
          accr[q] += c.x * p;
          acci[q] += c.y * p;
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const T sc = scale_of<T>(e[q]);
        f[q] += sc * (m == 0 ? accr[q] : T(2) * (accr[q] * cr[q] - acci[q] * sr[q]));
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int64_t i = gi * Q + q;
      if (on[q]) out[perm ? (int64_t)perm[i] : i] = (double)f[q];
    }
  }
}

void run_forward(const ForwardArgs& a, cudaStream_t s, int64_t* launches) {
  const int64_t ncoef = (int64_t)(a.N + 1) * (a.N + 2) / 2;
  const int cb = (int)((ncoef + 255) / 256);
  const size_t smem = (size_t)(a.N + 1) * (sizeof(double) + sizeof(double) + sizeof(float));
  const int64_t want = ((a.P + FWD_PPT - 1) / FWD_PPT + 255) / 256;
  const int blocks = (int)(want < (int64_t)a.num_sms * 8 ? (want < 1 ? 1 : want) : (int64_t)a.num_sms * 8);
  if (a.mixed) {
    float2* cf = reinterpret_cast<float2*>(a.cws);
    float2* ab = reinterpret_cast<float2*>(a.abws);
    fwd_coeffs_kernel<float2><<<cb, 256, 0, s>>>(a.coeffs, ncoef, cf);
    fwd_ab_kernel<float2><<<cb, 256, 0, s>>>(a.a_rec, a.b_rec, ncoef, ab);
    forward_kernel<float><<<blocks, 256, smem, s>>>(a.N, cf, ab, a.px, a.py, a.pz, a.stride, a.P, a.perm, a.out);
  } else {
    double2* cf = reinterpret_cast<double2*>(a.cws);
    double2* ab = reinterpret_cast<double2*>(a.abws);
    fwd_coeffs_kernel<double2><<<cb, 256, 0, s>>>(a.coeffs, ncoef, cf);
    fwd_ab_kernel<double2><<<cb, 256, 0, s>>>(a.a_rec, a.b_rec, ncoef, ab);
    forward_kernel<double><<<blocks, 256, smem, s>>>(a.N, cf, ab, a.px, a.py, a.pz, a.stride, a.P, a.perm, a.out);
  }
  *launches += 3;
}

}  // namespace hamls
