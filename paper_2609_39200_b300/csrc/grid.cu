// grid.cu - Algorithm 1 step 1 and the plan-time tables of step 3.
//
// The S^2 product rule of Sec. 2.1: Gauss-Legendre nodes t_k in cos(theta)
// (N+1 nodes, descending), phi_j = 2 pi j / (2N+2). Gauss-Legendre nodes come
// from Newton's method on P_{N+1} in the colatitude, weights from
// w = 2 / ((1 - t^2) P'_{N+1}(t)^2).
//
// Step 3 on this grid is fhat_l^m = (2 pi/(2N+2)) sum_k w_k Pbar_l^m(t_k) F_k(m)
// (eq. quadrature_based_approximation with the product weights). The matrix
// A^m[l, k] = (2 pi/(2N+2)) w_k Pbar_l^m(t_k) is generated once per plan by
// the normalised three-term recurrence in FP64 and folded over the equator:
// t_{N-k} = -t_k and Pbar_l^m(-t) = (-1)^{l+m} Pbar_l^m(t), so only the
// hc = floor(N/2) + 1 northern columns are stored.
#include "common.cuh"
#include "kernels.h"

namespace hamls {

int current_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  return n;
}

// done_mask: one bit per device (devices 0..31; others set the attribute on
// every call). Setting it twice is harmless, so a race only repeats the call.
void set_smem_attr_once(const void* func, int bytes, unsigned* done_mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = dev < 32 ? 1u << dev : 0u;
  if (bit && (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit)) return;
  cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (bit) __atomic_fetch_or(done_mask, bit, __ATOMIC_ACQ_REL);
}

// P_n and D_n = P_n - P_{n-1} at t = cos(theta) = 1 - u, u = 2 sin^2(theta/2),
// by the three-term recurrence rewritten on differences:
//   D_{k+1} = (k D_k - (2k+1) u P_k) / (k+1),  P_{k+1} = P_k + D_{k+1},
// which has no cancellation near t = 1 (the poles).
__device__ void legendre_pd(int n, double u, double& P, double& D) {
  double p = 1.0 - u, d = -u;
  for (int k = 1; k < n; ++k) {
    d = (k * d - (2 * k + 1) * u * p) / (k + 1);
    p += d;
  }
  P = p;
  D = d;
}

// Gauss-Legendre nodes by Newton's method on P_{N+1}(cos theta) in the
// colatitude theta (northern half; the southern half is the exact mirror
// t_{N-k} = -t_k, w_{N-k} = w_k). dP/dtheta = n (D_n - u P_n) / sin(theta) and
// w = 2 / ((1 - t^2) P'(t)^2) = 2 sin^2(theta) / (n (D_n - u P_n))^2.
__global__ void gl_kernel(int N, double* t_out, double* w_out, double* s_out, float* tf, float* sf) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = N + 1;
  if (k >= (n + 1) / 2) return;
  const bool middle = (n & 1) && k == (n - 1) / 2;
  double th = middle ? 0.5 * 3.14159265358979323846 : 3.14159265358979323846 * (k + 0.75) / (n + 0.5);
  double P, D, u, sh;
  for (int it = 0; it < 100 && !middle; ++it) {
    sh = sin(0.5 * th);
    u = 2.0 * sh * sh;
    legendre_pd(n, u, P, D);
    const double dth = P * sin(th) / (n * (D - u * P));
    th -= dth;
    // Newton converges quadratically: after a correction of 1e-14 the
    // error is far below FP64 resolution (a threshold under the resolution
    // itself would never be met and run every iteration)
    if (fabs(dth) <= 1e-14 * th) break;
  }
  sh = sin(0.5 * th);
  u = middle ? 1.0 : 2.0 * sh * sh;
  legendre_pd(n, u, P, D);
  double st, ct;
  sincos(th, &st, &ct);
  if (middle) {
    st = 1.0;
    ct = 0.0;
  }
  const double g = n * (D - u * P);
  const double w = 2.0 * st * st / (g * g);
  t_out[k] = ct;
  w_out[k] = w;
  s_out[k] = st;
  tf[k] = (float)ct;
  sf[k] = (float)st;
  if (!middle) {
    t_out[N - k] = -ct;
    w_out[N - k] = w;
    s_out[N - k] = st;
    tf[N - k] = -(float)ct;
    sf[N - k] = (float)st;
  }
}

__global__ void phi_kernel(int L, double* cphi, double* sphi, double2* W64, float2* W32, float* cpf, float* spf) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= L) return;
  double s, c;
  sincospi(2.0 * j / L, &s, &c);     // angle 2 pi j / L, argument exact
  cphi[j] = c;
  sphi[j] = s;
  W64[j] = make_double2(c, -s);      // exp(-2 pi i j / L)
  if (W32) W32[j] = make_float2((float)c, (float)-s);
  cpf[j] = (float)c;
  spf[j] = (float)s;
}

// a_lm = sqrt((4l^2 - 1)/(l^2 - m^2)), b_lm = sqrt(((l-1)^2 - m^2)/(4(l-1)^2 - 1)),
// packed m-major like the coefficients.
__global__ void rec_kernel(int N, double* a_rec, double* b_rec) {
  int m = blockIdx.x;
  for (int l = m + threadIdx.x; l <= N; l += blockDim.x) {
    size_t o = (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2 + (l - m);
    double a = 0.0, b = 0.0;
    if (l >= m + 2) {
      double ll = l, mm = m;
      a = sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm));
      b = sqrt(((ll - 1.0) * (ll - 1.0) - mm * mm) / (4.0 * (ll - 1.0) * (ll - 1.0) - 1.0));
    }
    a_rec[o] = a;
    b_rec[o] = b;
  }
}

// one thread per (m, folded column c): Pbar_l^m(t_c) for l = m..N. The FP64
// matrix has rows in degree order and hc columns; the FP32 matrix has, within
// each order m, the rows of even l - m first, then the odd ones (each parity
// group contiguous, the operand of the batched tensor-core contraction), and
// rows of hcp >= hc columns whose padding is zero.
__global__ void legendre_gen_kernel(int N, int hc, int hcp, const double* __restrict__ t,
                                    const double* __restrict__ w, const double* __restrict__ s,
                                    const double* __restrict__ a_rec, const double* __restrict__ b_rec,
                                    double* __restrict__ A64, float* __restrict__ A32) {
  const int m = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t row0 = (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
  if (c >= hc) {
    if (A32 && c < hcp)
      for (int l = m; l <= N; ++l) A32[(row0 + l32_row(N, m, l)) * hcp + c] = 0.f;
    return;
  }
  const double tc = t[c], sc = s[c];
  const double h = 2.0 * 3.14159265358979323846 / (2.0 * N + 2.0) * w[c];
  double pmm = 0.28209479177387814347;   // 1/sqrt(4 pi)
  for (int k = 1; k <= m; ++k) pmm *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * sc;
  double pm2 = 0.0, pm1 = 0.0;          // Pbar_{l-2}^m, Pbar_{l-1}^m
  for (int l = m; l <= N; ++l) {
    double p;
    if (l == m) {
      p = pmm;
    } else if (l == m + 1) {
      p = sqrt(2.0 * m + 3.0) * tc * pmm;
    } else {
      const size_t o = row0 + (l - m);
      p = a_rec[o] * (tc * pm1 - b_rec[o] * pm2);
    }
    pm2 = pm1;
    pm1 = p;
    const double v = h * p;
    if (A64) A64[(row0 + (l - m)) * hc + c] = v;
    if (A32) A32[(row0 + l32_row(N, m, l)) * hcp + c] = (float)v;
  }
}

void build_grid_tables(GridTables& g, bool want32, bool want64, cudaStream_t s, int64_t* launches) {
  const int N = g.N, L = 2 * N + 2;
  gl_kernel<<<(N + 2) / 2 / 128 + 1, 128, 0, s>>>(N, g.t, g.w, g.s, g.tf, g.sf);
  phi_kernel<<<(L + 255) / 256, 256, 0, s>>>(L, g.cphi, g.sphi, g.W64, want32 ? g.W32 : nullptr, g.cpf, g.spf);
  rec_kernel<<<N + 1, 256, 0, s>>>(N, g.a_rec, g.b_rec);
  dim3 grid((g.hcp + 63) / 64, N + 1);
  legendre_gen_kernel<<<grid, 64, 0, s>>>(N, g.hc, g.hcp, g.t, g.w, g.s, g.a_rec, g.b_rec,
                                          want64 ? g.A64 : nullptr, want32 ? g.A32 : nullptr);
  *launches += 4;
}

// Fibonacci grid: z_i = 1 - (2i+1)/n, phi_i = 2 pi {i (1 - 1/Phi)} with the
// fractional part taken exactly in 0.64 fixed point and truncated to 53 bits.
__global__ void fibonacci_kernel(double* x, double* y, double* z, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long G = 0x61C8864680B583EAull;
  unsigned long long f = ((unsigned long long)i * G) >> 11;
  double frac = (double)f * 0x1p-53;
  double zz = 1.0 - (2.0 * i + 1.0) / (double)n;
  double sn, cs;
  sincospi(2.0 * frac, &sn, &cs);
  double r = sqrt((1.0 - zz) * (1.0 + zz));
  x[i] = r * cs;
  y[i] = r * sn;
  z[i] = zz;
}

void fibonacci_points(double* x, double* y, double* z, int n, cudaStream_t s, int64_t* launches) {
  fibonacci_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, y, z, n);
  ++*launches;
}

}  // namespace hamls
