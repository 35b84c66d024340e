// quad.cu - Algorithm 1 step 3: fhat = F^H W f on the product grid.
//
// Ring DFT. F_k(m) = sum_j f_{kj} e^{-i m phi_j}, m = 0..N, for every ring k.
// Two real rings are packed into one complex sequence z = f_a + i f_b of
// length L = 2N+2 and transformed by a self-sorting (Stockham) mixed-radix
// FFT in shared memory; the spectra separate by conjugate symmetry:
// F_a(m) = (Z(m) + conj Z(L-m))/2, F_b(m) = (Z(m) - conj Z(L-m))/(2i).
// L = 2(N+1) has arbitrary prime factors (N = 256 gives 2 * 257), so every
// radix stage is a generic radix-R pass: output (j, r) of the stage with
// current sub-transform size Ns is
//   sum_q in[j + q L/R] * w_L^{q ((j mod Ns) L/(Ns R) + r L/R)},
// written to position (j / Ns) Ns R + (j mod Ns) + r Ns.
//
// Legendre quadrature. fhat_l^m = sum_k A^m[l, k] F_k(m) with the folded
// matrix of grid.cu: for the northern columns c < hc the pair (c, N - c)
// contributes A^m[l, c] (F_c + (-1)^{l+m} F_{N-c}). A single fit is a
// matrix-vector product bound by HBM bandwidth on the matrix.
#include <string.h>
#include "common.cuh"
#include "kernels.h"

namespace hamls {

template <typename T>
struct C2;
template <>
struct C2<float> { using t = float2; };
template <>
struct C2<double> { using t = double2; };

template <typename T>
__global__ void __launch_bounds__(256) ring_fft_kernel(const double* __restrict__ f, int N, QuadArgs qa,
                                                       const typename C2<T>::t* __restrict__ W,
                                                       typename C2<T>::t* __restrict__ F) {
  using cT = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 2 * N + 2;
  cT* buf0 = reinterpret_cast<cT*>(smem_raw);
  cT* buf1 = buf0 + L;
  cT* sW = buf1 + L;                        // the twiddles, read many times per stage
  const int ra = 2 * blockIdx.x, rb = ra + 1;
  const bool hasb = rb <= N;
  // value set blockIdx.y of a batch: grids M_Q apart, spectra (N+1)^2 apart
  f += (size_t)blockIdx.y * (size_t)(N + 1) * L;
  F += (size_t)blockIdx.y * (size_t)(N + 1) * (N + 1);
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    sW[j] = W[j];
    T x = (T)f[(size_t)ra * L + j];
    T y = hasb ? (T)f[(size_t)rb * L + j] : T(0);
    buf0[j].x = x;
    buf0[j].y = y;
  }
  __syncthreads();
  cT* in = buf0;
  cT* out = buf1;
  int Ns = 1;
  for (int st = 0; st < qa.nrad; ++st) {
    const int R = qa.radices[st];
    const int T_ = L / R;
    const int NsR = Ns * R;
    const int strideA = L / NsR, strideB = L / R;
    if (R <= 32 && T_ >= (int)blockDim.x) {
      // one butterfly per thread (while there are at least as many
      // butterflies as threads): group g = (hi, jl) reads in[j + q T_] for
      // q < R and writes out[hi Ns R + jl + r Ns] for r < R (one division per
      // group); twiddle exponents q (jl strideA + r strideB) advance by
      // additions mod L. A large radix with few butterflies (19 for
      // L = 1026: 54 of them) takes the one-output-per-thread form below.
      for (int g = threadIdx.x; g < T_; g += blockDim.x) {
        const int hi = g / Ns, jl = g - hi * Ns;
        const int j = hi * Ns + jl;
        const int base = hi * NsR + jl;
        int step = jl * strideA;             // exponent step of output r, mod L
        for (int r = 0; r < R; ++r) {
          int e = 0;
          T ax = 0, ay = 0;
          for (int q = 0; q < R; ++q) {
            const cT v = in[j + q * T_];
            const cT w = sW[e];
            ax += v.x * w.x - v.y * w.y;
            ay += v.x * w.y + v.y * w.x;
            e += step;
            if (e >= L) e -= L;
          }
          out[base + r * Ns].x = ax;
          out[base + r * Ns].y = ay;
          step += strideB;
          if (step >= L) step -= L;
        }
      }
      __syncthreads();
      cT* t = in;
      in = out;
      out = t;
      Ns *= R;
      continue;
    }
    for (int o = threadIdx.x; o < L; o += blockDim.x) {
      const int hi = o / NsR, rem = o - hi * NsR;
      const int r = rem / Ns, jl = rem - r * Ns;
      const int j = hi * Ns + jl;
      int step = jl * strideA + r * strideB;
      step %= L;
      int e = 0;
      T ax = 0, ay = 0;
      for (int q = 0; q < R; ++q) {
        const cT v = in[j + q * T_];
        const cT w = sW[e];
        ax += v.x * w.x - v.y * w.y;
        ay += v.x * w.y + v.y * w.x;
        e += step;
        if (e >= L) e -= L;
      }
      out[o].x = ax;
      out[o].y = ay;
    }
    __syncthreads();
    cT* t = in;
    in = out;
    out = t;
    Ns *= R;
  }
  for (int m = threadIdx.x; m <= N; m += blockDim.x) {
    const cT zm = in[m];
    const cT zc = in[(L - m) % L];            // Z(L - m), to be conjugated
    cT fa, fb;
    fa.x = T(0.5) * (zm.x + zc.x);
    fa.y = T(0.5) * (zm.y - zc.y);
    // (Z(m) - conj Z(L-m)) / (2i)
    const T dx = zm.x - zc.x, dy = zm.y + zc.y;
    fb.x = T(0.5) * dy;
    fb.y = T(-0.5) * dx;
    F[(size_t)ra * (N + 1) + m] = fa;
    if (hasb) F[(size_t)rb * (N + 1) + m] = fb;
  }
}

// One block per (order m, 32 consecutive degrees l): the even/odd folded
// vectors of order m go to shared memory, and each warp streams four matrix
// rows at once (coalesced, four loads in flight), reducing with shuffles.
constexpr int LEG_ROWS = 32;

// The matrix rows: degree order with hc columns (FP64), or the parity-grouped
// FP32 layout (l32_row) with rows of ld columns.
template <typename T>
__global__ void __launch_bounds__(256) legendre_kernel(int N, int hc, int ld, bool grouped, const T* __restrict__ A,
                                                       const typename C2<T>::t* __restrict__ F,
                                                       double* __restrict__ coeffs) {
  using cT = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.x;
  const int l0 = m + blockIdx.y * LEG_ROWS;
  if (l0 > N) return;
  cT* E = reinterpret_cast<cT*>(smem_raw);
  cT* O = E + hc;
  for (int c = threadIdx.x; c < hc; c += blockDim.x) {
    const cT a = F[(size_t)c * (N + 1) + m];
    const int cs = N - c;
    if (cs != c) {
      const cT b = F[(size_t)cs * (N + 1) + m];
      E[c].x = a.x + b.x;
      E[c].y = a.y + b.y;
      O[c].x = a.x - b.x;
      O[c].y = a.y - b.y;
    } else {
      E[c] = a;
      O[c] = a;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t row0 = (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
  const int lw = l0 + warp * 4;                     // this warp's first degree
  T sr[4], si[4];
  const T* row[4];
  bool on[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    sr[r] = si[r] = T(0);
    on[r] = lw + r <= N;
    const int l = on[r] ? lw + r : m;
    row[r] = A + (row0 + (grouped ? l32_row(N, m, l) : l - m)) * ld;
  }
  for (int c = lane; c < hc; c += 32) {
    T av[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) av[r] = on[r] ? row[r][c] : T(0);
    const cT e = E[c], o = O[c];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const cT g = ((lw + r + m) & 1) ? o : e;
      sr[r] += av[r] * g.x;
      si[r] += av[r] * g.y;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const T xr = warp_sum(sr[r]), xi = warp_sum(si[r]);
    if (lane == 0 && on[r]) {
      const size_t o = row0 + (size_t)(lw + r - m);
      coeffs[2 * o] = (double)xr;
      coeffs[2 * o + 1] = (double)xi;
    }
  }
}

template <typename T>
static void launch_quad(const QuadArgs& a, const typename C2<T>::t* W, const T* A, cudaStream_t s,
                        int64_t* launches, int part) {
  using cT = typename C2<T>::t;
  const int N = a.g->N, L = 2 * N + 2, hc = a.g->hc;
  const size_t smem_fft = 3 * (size_t)L * sizeof(cT);
  const size_t smem_leg = 2 * (size_t)hc * sizeof(cT);
  static unsigned done_fft = 0, done_leg = 0;   // per device
  set_smem_attr_once((const void*)ring_fft_kernel<T>, 200 * 1024, &done_fft);
  set_smem_attr_once((const void*)legendre_kernel<T>, 200 * 1024, &done_leg);
  if (part & 1) {
    ring_fft_kernel<T><<<(N + 2) / 2, 256, smem_fft, s>>>(a.fgrid, N, a, W, reinterpret_cast<cT*>(a.F));
    ++*launches;
  }
  if (part & 2) {
    const dim3 grid(N + 1, (N + 1 + LEG_ROWS - 1) / LEG_ROWS);
    const bool grouped = sizeof(T) == 4;
    legendre_kernel<T><<<grid, 256, smem_leg, s>>>(N, hc, grouped ? a.g->hcp : hc, grouped, A,
                                                   reinterpret_cast<const cT*>(a.F), a.coeffs);
    ++*launches;
  }
}

// The folded spectra of a batch, the A operand of the tensor-core Legendre
// contraction: for value set b, order m and column c < hc,
//   E = F_c(m) + F_{N-c}(m),  O = F_c(m) - F_{N-c}(m)   (E = O = F_c(m) if c = N - c),
// stored as G[(2m + p) * 2B + 2b + {0: re, 1: im}][c], p = 0 for E, 1 for O
// (FP32; the tensor-core kernel splits it for 3xTF32 as it reads it).
// A 32 x 32 tile of (c, m) per block: reads along m, writes along c.
__global__ void __launch_bounds__(256) fold_spectra_kernel(const float2* __restrict__ F, int N, int hc, int hcp,
                                                           int B, float* __restrict__ G) {
  __shared__ float2 E[32][33], O[32][33];
  const int b = blockIdx.z, m0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const float2* Fb = F + (size_t)b * (N + 1) * (N + 1);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r, m = m0 + tx;
    float2 e = make_float2(0.f, 0.f), o = e;
    if (c < hc && m <= N) {
      const float2 a = Fb[(size_t)c * (N + 1) + m];
      if (N - c != c) {
        const float2 z = Fb[(size_t)(N - c) * (N + 1) + m];
        e = make_float2(a.x + z.x, a.y + z.y);
        o = make_float2(a.x - z.x, a.y - z.y);
      } else {
        e = a;
        o = a;
      }
    }
    E[tx][r] = e;
    O[tx][r] = o;
  }
  __syncthreads();
  const size_t rs = (size_t)hcp, ps = (size_t)2 * B * hcp;
  for (int r = ty; r < 32; r += 8) {
    const int m = m0 + r, c = c0 + tx;
    if (m > N || c >= hc) continue;
    const size_t o = (size_t)(2 * m) * ps + (size_t)(2 * b) * rs + c;
    G[o] = E[r][tx].x;
    G[o + rs] = E[r][tx].y;
    G[o + ps] = O[r][tx].x;
    G[o + ps + rs] = O[r][tx].y;
  }
}

cudaError_t run_spectra_batch(const GridTables& g, const int* radices, int nrad, const double* fgrid, int B,
                              float2* F, float* G, cudaStream_t s, int64_t* launches) {
  const int N = g.N, L = 2 * N + 2;
  QuadArgs qa;
  memset(&qa, 0, sizeof(qa));
  qa.g = &g;
  for (int i = 0; i < nrad; ++i) qa.radices[i] = radices[i];
  qa.nrad = nrad;
  static unsigned done_fft = 0;
  set_smem_attr_once((const void*)ring_fft_kernel<float>, 200 * 1024, &done_fft);
  ring_fft_kernel<float><<<dim3((N + 2) / 2, B), 256, 3 * (size_t)L * sizeof(float2), s>>>(fgrid, N, qa, g.W32, F);
  fold_spectra_kernel<<<dim3((N + 1 + 31) / 32, (g.hc + 31) / 32, B), 256, 0, s>>>(F, N, g.hc, g.hcp, B, G);
  *launches += 2;
  return cudaGetLastError();
}

void run_quadrature(const QuadArgs& a, bool mixed, cudaStream_t s, int64_t* launches, int part) {
  if (mixed)
    launch_quad<float>(a, a.g->W32, a.g->A32, s, launches, part);
  else
    launch_quad<double>(a, a.g->W64, a.g->A64, s, launches, part);
}

}  // namespace hamls
