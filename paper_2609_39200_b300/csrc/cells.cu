// cells.cu - neighbour structure over a point set on S^2: integer cell keys,
// a stable LSD radix sort of (key, index), the CSR run table and the sorted
// FP64/FP32 copies of the points. Everything is bit-exact integer work or
// exact copies; see common.cuh for the key definition.
#include "common.cuh"
#include "kernels.h"

namespace hamls {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

int radix_blocks(int n) { return (n + SORT_TILE - 1) / SORT_TILE; }

// ------------------------------------------------------------- cell keys
__global__ void keys_kernel(const double* __restrict__ xyz, int n, int B, int P, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ idx, DevStatus* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = xyz[3 * (size_t)i], y = xyz[3 * (size_t)i + 1], z = xyz[3 * (size_t)i + 2];
  // unit-vector check in FP32 where it is certain (the FP32 |x|^2 is within
  // 4e-7 of the exact one), in FP64 otherwise
  const float xf = (float)x, yf = (float)y, zf = (float)z;
  const float r2f = xf * xf + yf * yf + zf * zf;
  bool ok = isfinite(r2f) && fabsf(r2f - 1.f) < 5e-7f;
  if (!ok) {
    const double r2 = x * x + y * y + z * z;
    ok = isfinite(x) && isfinite(y) && isfinite(z) && fabs(r2 - 1.0) < 1e-6;
  }
  uint32_t key;
  if (!ok) {
    set_flag(st, ST_BADNODE);
    key = cell_key64(0.0, 0.0, 1.0, B, P);
  } else if (!cell_key_fast(xf, yf, zf, (float)__dsub_rn(1.0, fabs(z)), B, P, key)) {
    key = cell_key64(x, y, z, B, P);
  }
  keys[i] = key;
  idx[i] = (uint32_t)i;
}

// points generated on the device (auxiliary grid) are already valid
__global__ void keys_kernel_soa(const double* __restrict__ px, const double* __restrict__ py,
                                const double* __restrict__ pz, int n, int B, int P,
                                uint32_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = cell_key64(px[i], py[i], pz[i], B, P);
  idx[i] = (uint32_t)i;
}

// ------------------------------------------------------------ radix sort
__global__ void __launch_bounds__(SORT_THREADS) radix_hist(const uint32_t* __restrict__ kin, int n, int shift,
                                                           uint32_t mask, uint32_t* __restrict__ counts,
                                                           int nblocks) {
  __shared__ uint32_t h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const int tile0 = blockIdx.x * SORT_TILE;
#pragma unroll 4
  for (int r = 0; r < SORT_ITEMS; ++r) {
    int i = tile0 + r * SORT_THREADS + tid;
    if (i < n) atomicAdd(&h[(kin[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  counts[(size_t)tid * nblocks + blockIdx.x] = h[tid];
}

// Exclusive scan of `len` counts in place: block sums of 1024-entry tiles,
// one block scans the sums, then every tile scans itself from its offset.
constexpr int SCAN_TILE = 1024;

int scan_partials(int n) { return (256 * radix_blocks(n) + SCAN_TILE - 1) / SCAN_TILE + 1; }

__device__ __forceinline__ uint32_t block_scan_256(uint32_t v, uint32_t* sh, uint32_t& total) {
  // inclusive scan over 256 threads (8 warps)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < 8 ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      uint32_t t = __shfl_up_sync(FULL, w, o);
      if (lane >= o) w += t;
    }
    if (lane < 8) sh[8 + lane] = w;
  }
  __syncthreads();
  total = sh[15];
  const uint32_t r = x + (warp > 0 ? sh[8 + warp - 1] : 0u);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) scan_tile_sums(const uint32_t* __restrict__ a, int len,
                                                      uint32_t* __restrict__ part) {
  __shared__ uint32_t sh[16];
  const int base = blockIdx.x * SCAN_TILE;
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < SCAN_TILE / 256; ++r) {
    const int i = base + r * 256 + threadIdx.x;
    if (i < len) s += a[i];
  }
  uint32_t total;
  block_scan_256(s, sh, total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) scan_sums(uint32_t* __restrict__ part, int np) {
  __shared__ uint32_t sh[16];
  uint32_t carry = 0;
  for (int b0 = 0; b0 < np; b0 += 256) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < np ? part[i] : 0u;
    uint32_t total;
    const uint32_t incl = block_scan_256(v, sh, total);
    if (i < np) part[i] = carry + incl - v;
    carry += total;
  }
}

__global__ void __launch_bounds__(256) scan_tiles(uint32_t* __restrict__ a, int len,
                                                  const uint32_t* __restrict__ part) {
  __shared__ uint32_t sh[16];
  const int base = blockIdx.x * SCAN_TILE;
  uint32_t carry = part[blockIdx.x];
#pragma unroll
  for (int r = 0; r < SCAN_TILE / 256; ++r) {
    const int i = base + r * 256 + threadIdx.x;
    const uint32_t v = i < len ? a[i] : 0u;
    uint32_t total;
    const uint32_t incl = block_scan_256(v, sh, total);
    if (i < len) a[i] = carry + incl - v;
    carry += total;
  }
}

__global__ void __launch_bounds__(SORT_THREADS) radix_scatter(const uint32_t* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin,
                                                              uint32_t* __restrict__ kout,
                                                              uint32_t* __restrict__ vout,
                                                              const uint32_t* __restrict__ offsets, int n,
                                                              int shift, uint32_t mask, int nblocks) {
  __shared__ uint32_t warp_cnt[SORT_THREADS / 32][256];
  __shared__ uint32_t digit_base[256];
  __shared__ uint32_t blk_off[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  blk_off[tid] = offsets[(size_t)tid * nblocks + blockIdx.x];
  digit_base[tid] = 0;
  const int tile0 = blockIdx.x * SORT_TILE;
  for (int r = 0; r < SORT_ITEMS; ++r) {
#pragma unroll
    for (int w = 0; w < SORT_THREADS / 32; ++w) warp_cnt[w][tid] = 0;
    __syncthreads();
    const int i = tile0 + r * SORT_THREADS + tid;
    const bool ok = i < n;
    const uint32_t k = ok ? kin[i] : 0u, v = ok ? vin[i] : 0u;
    const uint32_t d = ok ? ((k >> shift) & mask) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(FULL, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && lane == __ffs(peers) - 1) warp_cnt[warp][d] = __popc(peers);
    __syncthreads();
    uint32_t run = digit_base[tid];
#pragma unroll
    for (int w = 0; w < SORT_THREADS / 32; ++w) {
      uint32_t c = warp_cnt[w][tid];
      warp_cnt[w][tid] = run;
      run += c;
    }
    digit_base[tid] = run;
    __syncthreads();
    if (ok) {
      uint32_t pos = blk_off[d] + warp_cnt[warp][d] + (uint32_t)rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
  }
}

// Half angles and z of every band edge (see Cells::edge).
__global__ void edge_table_kernel(int B, float4* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > B) return;
  // 2/B exactly (B a power of two)
  const float zstep = (B & (B - 1)) == 0 ? __int_as_float((128 - (__ffs(B) - 1)) << 23) : 2.f / (float)B;
  float a, b;
  edge_half_angles(-1.f + (float)e * zstep, a, b);
  out[e] = make_float4(a, b, (b - a) * (b + a), 0.f);
}

void build_edge_table(int B, float4* out, cudaStream_t s, int64_t* launches) {
  edge_table_kernel<<<(B + 1 + 255) / 256, 256, 0, s>>>(B, out);
  ++*launches;
}

void exclusive_scan_u32(uint32_t* a, int len, uint32_t* part, cudaStream_t s, int64_t* launches) {
  const int nt = (len + SCAN_TILE - 1) / SCAN_TILE;
  scan_tile_sums<<<nt, 256, 0, s>>>(a, len, part);
  scan_sums<<<1, 256, 0, s>>>(part, nt);
  scan_tiles<<<nt, 256, 0, s>>>(a, len, part);
  *launches += 3;
}

// Stable sort of (keys, vals) by the low `bits` key bits. Returns true when the
// result ended in the *_alt buffers.
bool radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int n, int bits,
                      uint32_t* counts, cudaStream_t s, int64_t* launches) {
  if (n <= 0) return false;
  const int nb = radix_blocks(n);
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    const int w = min(8, bits - shift);
    const uint32_t mask = (1u << w) - 1u;
    const int len = 256 * nb, nt = (len + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* part = counts + len;
    radix_hist<<<nb, SORT_THREADS, 0, s>>>(ki, n, shift, mask, counts, nb);
    scan_tile_sums<<<nt, 256, 0, s>>>(counts, len, part);
    scan_sums<<<1, 256, 0, s>>>(part, nt);
    scan_tiles<<<nt, 256, 0, s>>>(counts, len, part);
    radix_scatter<<<nb, SORT_THREADS, 0, s>>>(ki, vi, ko, vo, counts, n, shift, mask, nb);
    *launches += 5;
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    alt = !alt;
  }
  return alt;
}

// ---------------------------------------------------------------- CSR runs
// start[c] = first sorted position whose key is >= c, c = 0..ncells.
__global__ void csr_kernel(const uint32_t* __restrict__ sk, int n, int ncells, uint32_t* __restrict__ start) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  int prev = (i == 0) ? -1 : (int)sk[i - 1];
  int cur = (i == n) ? ncells : (int)sk[i];
  for (int c = prev + 1; c <= cur; ++c) start[c] = (uint32_t)i;
}

// --------------------------------------------------------------- staging
__global__ void stage_points_kernel(const double* __restrict__ xyz, const uint32_t* __restrict__ perm, int n,
                                    double* __restrict__ px, double* __restrict__ py, double* __restrict__ pz,
                                    float4* __restrict__ pf, const double* __restrict__ wts,
                                    double* __restrict__ sw, float* __restrict__ swf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  size_t o = perm[i];
  double x = xyz[3 * o], y = xyz[3 * o + 1], z = xyz[3 * o + 2];
  px[i] = x;
  py[i] = y;
  pz[i] = z;
  pf[i] = make_float4((float)x, (float)y, (float)z, 0.f);
  if (wts) {
    double w = wts[o];
    sw[i] = w;
    swf[i] = (float)w;
  }
}

__global__ void stage_soa_kernel(const double* __restrict__ ax, const double* __restrict__ ay,
                                 const double* __restrict__ az, const uint32_t* __restrict__ perm, int n,
                                 double* __restrict__ px, double* __restrict__ py, double* __restrict__ pz,
                                 float4* __restrict__ pf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t o = perm[i];
  double x = ax[o], y = ay[o], z = az[o];
  px[i] = x;
  py[i] = y;
  pz[i] = z;
  pf[i] = make_float4((float)x, (float)y, (float)z, 0.f);
}

// per fit: values into sorted order (FP64 and the FP32 slot of pf)
__global__ void stage_values_kernel(const double* __restrict__ y, const uint32_t* __restrict__ perm, int n,
                                    double* __restrict__ sy, float4* __restrict__ pf, int write64, DevStatus* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = y[perm[i]];
  if (!isfinite(v)) {
    set_flag(st, ST_NONFINITE);
    v = 0.0;
  }
  if (write64) sy[i] = v;
  pf[i].w = (float)v;
}

void build_cells(const CellBuild& cb, cudaStream_t s, int64_t* launches) {
  const int n = cb.n;
  const int T = 256;
  const int gb = (n + T - 1) / T;
  if (cb.xyz_aos)
    keys_kernel<<<gb, T, 0, s>>>(cb.xyz_aos, n, cb.B, cb.P, cb.keys, cb.vals, cb.st);
  else
    keys_kernel_soa<<<gb, T, 0, s>>>(cb.ax, cb.ay, cb.az, n, cb.B, cb.P, cb.keys, cb.vals);
  ++*launches;
  int bits = 0;
  while ((1u << bits) < (uint32_t)(cb.B * cb.P)) ++bits;
  bool alt = radix_sort_pairs(cb.keys, cb.vals, cb.keys_alt, cb.vals_alt, n, bits, cb.counts, s, launches);
  const uint32_t* sk = alt ? cb.keys_alt : cb.keys;
  const uint32_t* perm = alt ? cb.vals_alt : cb.vals;
  csr_kernel<<<(n + 1 + T - 1) / T, T, 0, s>>>(sk, n, cb.B * cb.P, cb.start);
  ++*launches;
  if (cb.xyz_aos)
    stage_points_kernel<<<gb, T, 0, s>>>(cb.xyz_aos, perm, n, cb.px, cb.py, cb.pz, cb.pf, cb.wts, cb.sw, cb.swf);
  else
    stage_soa_kernel<<<gb, T, 0, s>>>(cb.ax, cb.ay, cb.az, perm, n, cb.px, cb.py, cb.pz, cb.pf);
  ++*launches;
  *cb.perm_out = perm;
  *cb.keys_out = sk;
}

// A second ordering of already sorted points by a coarser band structure:
// 32 consecutive points of it form a compact tile.
void build_tile_order(const double* px, const double* py, const double* pz, int n, int B, int P, uint32_t* keys,
                      uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* counts,
                      const uint32_t** order_out, cudaStream_t s, int64_t* launches) {
  keys_kernel_soa<<<(n + 255) / 256, 256, 0, s>>>(px, py, pz, n, B, P, keys, vals);
  ++*launches;
  int bits = 0;
  while ((1ull << bits) < (unsigned long long)B * P) ++bits;
  bool alt = radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, bits, counts, s, launches);
  *order_out = alt ? vals_alt : vals;
}

void launch_cell_keys(const double* xyz, int n, int B, int P, uint32_t* keys, uint32_t* vals, DevStatus* st,
                      cudaStream_t s) {
  keys_kernel<<<(n + 255) / 256, 256, 0, s>>>(xyz, n, B, P, keys, vals, st);
}

void launch_csr(const uint32_t* sk, int n, int ncells, uint32_t* start, cudaStream_t s) {
  csr_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(sk, n, ncells, start);
}

void stage_values(const double* y, const uint32_t* perm, int n, double* sy, float4* pf, bool write64,
                  DevStatus* st, cudaStream_t s, int64_t* launches) {
  const int T = 256;
  stage_values_kernel<<<(n + T - 1) / T, T, 0, s>>>(y, perm, n, sy, pf, write64 ? 1 : 0, st);
  ++*launches;
}

}  // namespace hamls
