// cells.cu - neighbour structure over a point set on S^2: integer cell keys,
// a stable LSD radix sort of (key, index), the CSR run table and the sorted
// FP64/FP32 copies of the points. Everything is bit-exact integer work or
// exact copies; see common.cuh for the key definition.
#include <algorithm>

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

// ------------------------------------------------- counting sort by cell
// A cell holds a few points, so the points are sorted by counting: each
// takes an arrival rank in its cell (an atomic on the cell's count), the
// counts are scanned into the CSR start table, each point scatters to
// start + rank, and a last pass orders every cell's points by input index
// (the order a stable sort gives, whatever order the atomics ran in) while
// writing the sorted FP64/FP32 copies.
//
// The key of a point comes from FP32 arithmetic where that is provably the
// FP64 key (cell_key_fast); the rest (about one point in a hundred) are
// listed and keyed in FP64 by a second kernel, so no warp of the first
// waits on the slow FP64 pipe for one lane.
__device__ __forceinline__ void load_point(const double* __restrict__ xyz, const double* __restrict__ ax,
                                           const double* __restrict__ ay, const double* __restrict__ az, size_t i,
                                           double& x, double& y, double& z) {
  if (xyz) {
    x = xyz[3 * i];
    y = xyz[3 * i + 1];
    z = xyz[3 * i + 2];
  } else {
    x = ax[i];
    y = ay[i];
    z = az[i];
  }
}

__global__ void cell_count_kernel(const double* __restrict__ xyz, const double* __restrict__ ax,
                                  const double* __restrict__ ay, const double* __restrict__ az, int n, int B, int P,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ rank,
                                  uint32_t* __restrict__ count, uint32_t* __restrict__ slow,
                                  uint32_t* __restrict__ nslow, DevStatus* st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool act = i < n;
  bool fast = true;
  if (act) {
    double x, y, z;
    load_point(xyz, ax, ay, az, (size_t)i, x, y, z);
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    bool ok = true;
    if (xyz) {
      // unit-vector check in FP32 where it is certain (the FP32 |x|^2 is
      // within 4e-7 of the exact one), in FP64 otherwise
      const float r2f = xf * xf + yf * yf + zf * zf;
      ok = isfinite(r2f) && fabsf(r2f - 1.f) < 5e-7f;
      if (!ok) {
        const double r2 = x * x + y * y + z * z;
        ok = isfinite(x) && isfinite(y) && isfinite(z) && fabs(r2 - 1.0) < 1e-6;
      }
    }
    uint32_t key = 0;
    if (!ok) {
      set_flag(st, ST_BADNODE);
      key = cell_key64(0.0, 0.0, 1.0, B, P);
    } else {
      fast = cell_key_fast(xf, yf, zf, (float)__dsub_rn(1.0, fabs(z)), B, P, key);
    }
    if (fast) {
      keys[i] = key;
      rank[i] = atomicAdd(&count[key], 1u);
    }
  }
  const unsigned bal = __ballot_sync(FULL, act && !fast);
  if (bal) {
    const int leader = __ffs(bal) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(nslow, (uint32_t)__popc(bal));
    base = __shfl_sync(FULL, base, leader);
    if (act && !fast) slow[base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

__global__ void cell_count_slow_kernel(const double* __restrict__ xyz, const double* __restrict__ ax,
                                       const double* __restrict__ ay, const double* __restrict__ az, int B, int P,
                                       const uint32_t* __restrict__ slow, const uint32_t* __restrict__ nslow,
                                       uint32_t* __restrict__ keys, uint32_t* __restrict__ rank,
                                       uint32_t* __restrict__ count) {
  const uint32_t ns = *nslow;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += gridDim.x * blockDim.x) {
    const uint32_t i = slow[t];
    double x, y, z;
    load_point(xyz, ax, ay, az, i, x, y, z);
    const uint32_t key = cell_key64(x, y, z, B, P);
    keys[i] = key;
    rank[i] = atomicAdd(&count[key], 1u);
  }
}

__global__ void cell_scatter_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ rank,
                                    const uint32_t* __restrict__ start, int n, uint32_t* __restrict__ tmp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  tmp[start[keys[i]] + rank[i]] = (uint32_t)i;
}

// tmp holds every cell's points in arrival order; a point's place in its
// cell is the number of the cell's points with a smaller input index
__global__ void cell_order_kernel(const uint32_t* __restrict__ tmp, const uint32_t* __restrict__ keys,
                                  const uint32_t* __restrict__ start, int n, const double* __restrict__ xyz,
                                  const double* __restrict__ ax, const double* __restrict__ ay,
                                  const double* __restrict__ az, const double* __restrict__ wts,
                                  uint32_t* __restrict__ perm, uint32_t* __restrict__ skeys, double* __restrict__ px,
                                  double* __restrict__ py, double* __restrict__ pz, float4* __restrict__ pf,
                                  double* __restrict__ sw, float* __restrict__ swf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t i = tmp[j];
  const uint32_t key = keys[i];
  const uint32_t c0 = start[key], c1 = start[key + 1];
  uint32_t r = 0;
  for (uint32_t m = c0; m < c1; ++m) r += tmp[m] < i ? 1u : 0u;
  const uint32_t p = c0 + r;
  perm[p] = i;
  skeys[p] = key;
  double x, y, z;
  load_point(xyz, ax, ay, az, i, x, y, z);
  px[p] = x;
  py[p] = y;
  pz[p] = z;
  pf[p] = make_float4((float)x, (float)y, (float)z, 0.f);
  if (wts) {
    const double w = wts[i];
    sw[p] = w;
    swf[p] = (float)w;
  }
}

void build_cells(const CellBuild& cb, cudaStream_t s, int64_t* launches) {
  const int n = cb.n;
  const int T = 256;
  const int gb = (n + T - 1) / T;
  const int ncells = cb.B * cb.P;
  uint32_t* nslow = cb.counts;               // one word
  uint32_t* part = cb.counts + 4;            // scan scratch
  const double* xyz = cb.xyz_aos;
  cudaMemsetAsync(cb.start, 0, ((size_t)ncells + 1) * sizeof(uint32_t), s);
  cudaMemsetAsync(nslow, 0, sizeof(uint32_t), s);
  if (n > 0) {
    cell_count_kernel<<<gb, T, 0, s>>>(xyz, cb.ax, cb.ay, cb.az, n, cb.B, cb.P, cb.keys, cb.vals, cb.start,
                                       cb.keys_alt, nslow, cb.st);
    cell_count_slow_kernel<<<std::min(gb, 128), T, 0, s>>>(xyz, cb.ax, cb.ay, cb.az, cb.B, cb.P, cb.keys_alt,
                                                           nslow, cb.keys, cb.vals, cb.start);
    *launches += 2;
  }
  exclusive_scan_u32(cb.start, ncells + 1, part, s, launches);
  if (n > 0) {
    // the arrival ranks (vals) and the slow list (keys_alt) are spent: the
    // scatter reuses keys_alt, the sorted keys go to vals
    cell_scatter_kernel<<<gb, T, 0, s>>>(cb.keys, cb.vals, cb.start, n, cb.keys_alt);
    cell_order_kernel<<<gb, T, 0, s>>>(cb.keys_alt, cb.keys, cb.start, n, xyz, cb.ax, cb.ay, cb.az,
                                       xyz ? cb.wts : nullptr, cb.vals_alt, cb.vals, cb.px, cb.py, cb.pz, cb.pf,
                                       cb.sw, cb.swf);
    *launches += 2;
  }
  *cb.perm_out = cb.vals_alt;
  *cb.keys_out = cb.vals;
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
