// tcgemm.cu - FP32-accurate matrix products on the 5th-generation tensor
// cores (tcgen05, sm_103a): D = A B^T with A (rows x K) and B (cols x K) both
// K-major FP32, computed as 3xTF32,
//   A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T,
// x_hi = x with its 13 low mantissa bits cleared (exact in TF32), x_lo =
// x - x_hi (exact in FP32, < 2^-10 |x|); the dropped A_lo B_lo term and the
// TF32 rounding of the lo parts are ~2^-20 relative per product, accumulated
// in FP32 in tensor memory. This is the Legendre contraction of step 3 for
// many value sets at once (eq. quadrature_based_approximation): for a fixed
// order m and parity, the coefficients of all value sets are one product of
// the spectra (value sets x latitudes) with the rows of the quadrature
// matrix (degrees x latitudes).
//
// One CTA (4 warps) computes a 128 x NT tile of D (NT <= 256 columns of
// tensor memory). Both operands are held in global memory as FP32 and cross
// HBM once: per K step of 32 (one 128-byte row of a swizzled tile) one thread
// has TMA bring the two FP32 tiles (boxes of 32 rows x 32 FP32, 128-byte
// swizzle) into one of two shared-memory stages, all threads split them into
// hi (in place) and lo tiles, and the thread issues the 4 x 3 tcgen05.mma of
// the step; tcgen05.commit frees the stage for the TMA two steps ahead. The
// epilogue reads D from tensor memory (warp w owns lanes 32w..32w+31) and
// hands 16 columns at a time to the caller's epilogue.
//
// Every wait on an mbarrier is bounded (about two seconds of clock); a wait
// that gives up sets an error flag, the CTA skips its remaining work, waits
// (bounded again) for the copies and products it has in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <mutex>
#include "../../include/hamls.h"
#include "../../include/hamls_debug.h"
#include "common.cuh"
#include "kernels.h"
#include "mbarrier.cuh"

namespace hamls {

constexpr int TC_THREADS = 320;           // warp 0 TMA, warp 1 MMA, warps 2-5 split, warps 6-9 epilogue
constexpr int TC_BK = 32;                 // K per stage: one 128-byte swizzled row of FP32
constexpr int TC_BOX = 32;                // rows per TMA box
constexpr int TC_MAXN = 256;              // columns of D per CTA (tensor-memory columns)
constexpr int TC_TILE_A = 128 * TC_BK * 4;              // 16 KB
constexpr int TC_TILE_B = TC_MAXN * TC_BK * 4;          // 32 KB
constexpr int TC_STAGE = TC_TILE_A + TC_TILE_B;         // the FP32 tiles of one K step: 48 KB
constexpr int TC_NST = 3;                               // stages in the ring
constexpr int TC_SMEM = (TC_NST + 1) * TC_STAGE + 1024 + 256;   // ring, lo tiles, alignment, barriers
constexpr int TC_TMEM_COLS = 2 * TC_MAXN;               // two accumulators

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;      // stride byte offset
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// M = 128, N columns
__device__ __forceinline__ uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ the kernel
// Persistent: one CTA per SM walks the tiles t = block, block + grid, ...
// with its warps in four roles, each counting the uses of the two stages and
// the two tensor-memory accumulators the same way:
//   warp 0 (one thread)  TMA: waits until a stage's products are done, then
//                        loads the stage's two FP32 tiles (full[s]); three
//                        stages in the ring;
//   warps 2-5            split: wait for full[s] and for the lo tiles to be
//                        free (lofree: the previous step's products are done),
//                        split their share of the stage into hi (in place) and
//                        lo (the one pair of lo tiles), fence the writes for
//                        the tensor core, arrive on ready;
//   warp 1 (one thread)  MMA: waits for an accumulator the epilogue has
//                        emptied (tempty[a]), then per K step for ready: 4 x 3
//                        products, commit to empty[s] and to lofree; after a
//                        tile's last step, commit to tfull[a];
//   warps 6-9            epilogue: wait for tfull[a], read the accumulator
//                        (warp w owns tensor-memory lanes 32 (w mod 4) ...),
//                        store through the caller's epilogue, arrive on
//                        tempty[a].
// So a tile's epilogue runs under the next tile's loads and products. A
// fresh barrier counts its "previous" phase as complete, so a role waits for
// parity (use & 1) ^ 1 before reusing what a use freed. Every wait is bounded:
// a role that gives up raises the CTA's abort flag, which the others read
// before each step; at the end the TMA thread waits (bounded) for the loads it
// issued and the MMA thread for its products, then tensor memory is freed.
__device__ __forceinline__ void tf32_split4(float4* hi, float4* lo) {
  float4 v = *hi, h;
  h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
  h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
  h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
  h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
  *hi = h;
  *lo = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool aborted(const volatile int* f) { return *f != 0; }

template <class Epi>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                 const __grid_constant__ CUtensorMap mapB,
                                                                 const TcJob* __restrict__ jobs, int ntiles,
                                                                 int mtiles, int K, Epi epi, unsigned* err) {
  extern __shared__ unsigned char tc_raw[];
  // stages on a 1024-byte boundary (the 128-byte swizzle repeats every 1024)
  const uint32_t base = smem_addr(tc_raw);
  unsigned char* sm = tc_raw + ((1024u - (base & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + (TC_NST + 1) * TC_STAGE);
  uint64_t* empty = full + TC_NST;
  uint64_t* ready = empty + TC_NST;
  uint64_t* lofree = ready + 1;
  uint64_t* tfull = lofree + 1;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(done + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KT = (K + TC_BK - 1) / TC_BK;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TC_NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(ready, 128);
    mbar_init(lofree, 1);
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    prefetch_map(&mapA);
    prefetch_map(&mapB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // stage s: A | B (FP32 as loaded, hi in place after the split); the lo
  // tiles of the step being multiplied after the ring: A lo | B lo
  auto tileA = [&](int s) { return sm + s * TC_STAGE; };
  auto tileB = [&](int s) { return sm + s * TC_STAGE + TC_TILE_A; };
  unsigned char* loA = sm + TC_NST * TC_STAGE;
  unsigned char* loB = loA + TC_TILE_A;
  auto fail = [&]() {
    *abort = 1;
    atomicOr(err, 1u);
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      int it = 0, issued[TC_NST] = {0, 0, 0};
      for (int t = blockIdx.x; t < ntiles && !aborted(abort); t += gridDim.x) {
        TcJob job = jobs[t / mtiles];
        const int a_y = job.a_y + 128 * (t % mtiles);
        const int nb = job.nt / TC_BOX;
        const uint32_t bytes = (uint32_t)(128 / TC_BOX + nb) * TC_BOX * TC_BK * 4;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = it % TC_NST, n = it / TC_NST;
          if (!mbar_wait_bounded(&empty[s], (uint32_t)(n & 1) ^ 1u) || aborted(abort)) {
            fail();
            break;
          }
          mbar_expect_tx(&full[s], bytes);
          for (int r = 0; r < 128 / TC_BOX; ++r)
            tma_load_3d(tileA(s) + r * TC_BOX * TC_BK * 4, &mapA, kt * TC_BK, a_y + r * TC_BOX, job.a_z, &full[s]);
          for (int r = 0; r < nb; ++r)
            tma_load_3d(tileB(s) + r * TC_BOX * TC_BK * 4, &mapB, kt * TC_BK, job.b_y + r * TC_BOX, 0, &full[s]);
          ++issued[s];
        }
      }
      if (aborted(abort)) {
        // every load issued must land before the CTA may exit
        for (int s = 0; s < TC_NST; ++s)
          if (issued[s] > 0) (void)mbar_wait_bounded(&full[s], (uint32_t)((issued[s] - 1) & 1));
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      int it = 0, tc = 0;
      for (int t = blockIdx.x; t < ntiles && !aborted(abort); t += gridDim.x, ++tc) {
        TcJob job = jobs[t / mtiles];
        const uint32_t idesc = tf32_idesc(job.nt);
        const int a = tc & 1, u = tc >> 1;
        if (!mbar_wait_bounded(&tempty[a], (uint32_t)(u & 1) ^ 1u)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(a * TC_MAXN);
        bool ok = true;
        for (int kt = 0; kt < KT; ++kt, ++it) {
          const int s = it % TC_NST;
          if (!mbar_wait_bounded(ready, (uint32_t)(it & 1)) || aborted(abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = smem_addr(tileA(s)), a_lo = smem_addr(loA);
          const uint32_t b_hi = smem_addr(tileB(s)), b_lo = smem_addr(loB);
#pragma unroll
          for (int k = 0; k < TC_BK / 8; ++k) {
            // K = 8 TF32 per product: 32 bytes further along the swizzled row
            const uint32_t off = (uint32_t)k * 32u;
            const uint32_t acc0 = (kt > 0 || k > 0) ? 1u : 0u;
            mma_tf32(acc, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc, acc0);
            mma_tf32(acc, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
            mma_tf32(acc, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
          }
          mma_commit(&empty[s]);
          mma_commit(lofree);
        }
        if (!ok) {
          fail();
          break;
        }
        mma_commit(&tfull[a]);
      }
      // every product issued is complete before tensor memory is freed
      mma_commit(done);
      if (!mbar_wait_bounded(done, 0)) fail();
    }
  } else if (warp < 6) {
    // -------------------------------------------------------------- split
    const int st = tid - 64;                        // 0..127
    int it = 0;
    for (int t = blockIdx.x; t < ntiles && !aborted(abort); t += gridDim.x) {
      const int nt = jobs[t / mtiles].nt;
      bool ok = true;
      for (int kt = 0; kt < KT; ++kt, ++it) {
        const int s = it % TC_NST, n = it / TC_NST;
        // the stage has landed, and the previous step's products no longer read the lo tiles
        if (!mbar_wait_bounded(&full[s], (uint32_t)(n & 1)) ||
            !mbar_wait_bounded(lofree, (uint32_t)(it & 1) ^ 1u) || aborted(abort)) {
          ok = false;
          break;
        }
        float4* ah = reinterpret_cast<float4*>(tileA(s));
        float4* al = reinterpret_cast<float4*>(loA);
#pragma unroll 4
        for (int i = st; i < 128 * TC_BK / 4; i += 128) tf32_split4(ah + i, al + i);
        float4* bh = reinterpret_cast<float4*>(tileB(s));
        float4* bl = reinterpret_cast<float4*>(loB);
#pragma unroll 4
        for (int i = st; i < nt * TC_BK / 4; i += 128) tf32_split4(bh + i, bl + i);
        fence_async_smem();
        mbar_arrive(ready);
      }
      if (!ok) {
        fail();
        break;
      }
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int lg = warp & 3;                        // tensor-memory lane group
    const int row = lg * 32 + lane;                 // row of the 128-row tile
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles && !aborted(abort); t += gridDim.x, ++tc) {
      TcJob job = jobs[t / mtiles];
      job.a_y += 128 * (t % mtiles);
      const int a = tc & 1, u = tc >> 1;
      if (!mbar_wait_bounded(&tfull[a], (uint32_t)(u & 1))) {
        fail();
        break;
      }
      tc_fence_after();
      for (int c0 = 0; c0 < job.nt; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(a * TC_MAXN + c0), v);
        epi.store16(job, row, c0, v, lane);
      }
      tc_fence_before();
      mbar_arrive(&tempty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------ host helpers
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// FP32 tensor of shape (d0 inner, d1, d2) with row stride s1 and plane stride
// s2 (bytes, multiples of 16), boxes of 32 x 32 x 1, 128-byte swizzle, zero fill
bool tc_make_map(CUtensorMap* map, const float* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
                 uint64_t s2) {
  EncodeTiled fn = encoder();
  if (!fn || (s1 % 16) || (s2 % 16) || (reinterpret_cast<uintptr_t>(base) % 16)) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {s1, s2};
  cuuint32_t box[3] = {TC_BK, TC_BOX, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class Epi>
static cudaError_t tc_launch(const CUtensorMap* maps, const TcJob* jobs, int njobs, int mtiles, int K, const Epi& epi,
                             unsigned* err, cudaStream_t s) {
  static unsigned done = 0;
  set_smem_attr_once((const void*)tc_gemm_kernel<Epi>, TC_SMEM, &done);
  const int ntiles = njobs * mtiles;
  const int sms = current_sm_count();
  const int grid = ntiles < sms ? ntiles : sms;
  tc_gemm_kernel<Epi><<<grid, TC_THREADS, TC_SMEM, s>>>(maps[0], maps[1], jobs, ntiles, mtiles, K, epi, err);
  return cudaGetLastError();
}

// ------------------------------------------------------ Legendre epilogue
// Tile of order m (e0), parity p (e1): rows j0 + c (e2 = j0) of the parity
// group, which holds e3 degrees l = m + p + 2 j; D row r of the tile is the
// real (r even) or imaginary part of value set r / 2.
struct EpiLegendre {
  double* coeffs;
  int N, rows;            // rows of D that exist: 2 B
  size_t ncoef;
  // row: the thread's row of the tile (tensor-memory lane), with the
  // imaginary part of its set in the neighbouring lane (row + 1); the even
  // lane writes the 16 complex coefficients of its set for columns c0 ...
  __device__ void store16(const TcJob& j, int row, int c0, const float* v, int lane) const {
    float w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
    const int r = j.a_y + row;
    if ((lane & 1) || r >= rows) return;
    const int m = j.e0;
    const size_t row0 = (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
    double2* out = reinterpret_cast<double2*>(coeffs) + (size_t)(r >> 1) * ncoef + row0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int jj = j.e2 + c0 + i;
      if (c0 + i < j.nt && jj < j.e3) {
        const int l = m + j.e1 + 2 * jj;
        out[l - m] = make_double2((double)v[i], (double)w[i]);
      }
    }
  }
};

int tc_legendre_jobs(int N, TcJob* out) {
  int n = 0;
  for (int m = 0; m <= N; ++m) {
    const size_t row0 = (size_t)m * (N + 1) - (size_t)m * (m - 1) / 2;
    const int ne = (N - m) / 2 + 1, no = (N - m + 1) / 2;
    for (int p = 0; p < 2; ++p) {
      const int rows = p ? no : ne;
      const int start = (int)row0 + (p ? ne : 0);
      for (int j0 = 0; j0 < rows; j0 += TC_MAXN) {
        const int cnt = rows - j0 < TC_MAXN ? rows - j0 : TC_MAXN;
        if (out) {
          TcJob& j = out[n];
          j.a_y = 0;
          j.a_z = 2 * m + p;
          j.b_y = start + j0;
          j.nt = (cnt + 31) / 32 * 32;
          j.e0 = m;
          j.e1 = p;
          j.e2 = j0;
          j.e3 = rows;
        }
        ++n;
      }
    }
  }
  return n;
}

cudaError_t tc_legendre(const GridTables& g, const float* G, int B, const TcJob* jobs, int njobs, double* coeffs,
                        unsigned* err, cudaStream_t s, int64_t* launches) {
  const int N = g.N;
  const uint64_t ncoef = (uint64_t)(N + 1) * (N + 2) / 2;
  CUtensorMap maps[2];
  memset(maps, 0, sizeof(maps));
  const uint64_t ld = (uint64_t)g.hcp * 4;
  const uint64_t zs = (uint64_t)2 * (N + 1);
  if (!tc_make_map(&maps[0], G, (uint64_t)g.hc, (uint64_t)(2 * B), zs, ld, ld * 2 * B) ||
      !tc_make_map(&maps[1], g.A32, (uint64_t)g.hc, ncoef, 1, ld, ld * ncoef))
    return cudaErrorInvalidValue;
  EpiLegendre epi{coeffs, N, 2 * B, (size_t)ncoef};
  ++*launches;
  return tc_launch(maps, jobs, njobs, (2 * B + 127) / 128, g.hc, epi, err, s);
}

// ------------------------------------------------------------ debug GEMM
// C (M x N, row stride ldc) = A (M x K) B (N x K)^T
struct EpiDense {
  float* C;
  int M, N, ldc;
  __device__ void store16(const TcJob& j, int row, int c0, const float* v, int) const {
    const int r = j.a_y + row;
    if (r >= M) return;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int cc = j.b_y + c0 + i;
      if (cc < N) C[(size_t)r * ldc + cc] = v[i];
    }
  }
};

}  // namespace hamls

using namespace hamls;

extern "C" hamls_status hamls_debug_tc_gemm(const float* A, const float* B, float* C, int M, int N, int K,
                                            cudaStream_t stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (K % 4)) return HAMLS_ERR_INVALID_ARG;
  // jobs: 128-row tiles of A times 256-column tiles of B (the last ones
  // rounded up to 32 columns)
  const int mt = (M + 127) / 128;
  const int ntl = (N + TC_MAXN - 1) / TC_MAXN;
  const int njobs = mt * ntl;
  TcJob* hj = new TcJob[njobs];
  for (int i = 0; i < mt; ++i)
    for (int jn = 0; jn < ntl; ++jn) {
      TcJob& j = hj[i * ntl + jn];
      memset(&j, 0, sizeof(j));
      j.a_y = i * 128;
      j.a_z = 0;
      j.b_y = jn * TC_MAXN;
      const int cols = N - j.b_y < TC_MAXN ? N - j.b_y : TC_MAXN;
      j.nt = (cols + 31) / 32 * 32;
    }
  // scratch for this call: the job table and an error word (the kernel
  // splits the FP32 operands into hi and lo as it reads them)
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t bj = up(sizeof(TcJob) * njobs + 16);
  char* mem = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&mem, bj, stream);
  TcJob* dj = reinterpret_cast<TcJob*>(mem);
  unsigned* derr = reinterpret_cast<unsigned*>(mem + sizeof(TcJob) * njobs);
  CUtensorMap maps[2];
  memset(maps, 0, sizeof(maps));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dj, hj, sizeof(TcJob) * njobs, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, 4, stream);
  if (e == cudaSuccess) {
    const uint64_t ld = (uint64_t)K * 4;
    if (!tc_make_map(&maps[0], A, (uint64_t)K, (uint64_t)M, 1, ld, ld * M) ||
        !tc_make_map(&maps[1], B, (uint64_t)K, (uint64_t)N, 1, ld, ld * N))
      e = cudaErrorInvalidValue;
  }
  EpiDense epi{C, M, N, N};
  if (e == cudaSuccess) e = tc_launch(maps, dj, njobs, 1, K, epi, derr, stream);
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (mem) cudaFreeAsync(mem, stream);
  delete[] hj;
  if (e == cudaErrorInvalidValue) return HAMLS_ERR_INVALID_ARG;
  if (e != cudaSuccess) return HAMLS_ERR_CUDA;
  return herr ? HAMLS_ERR_TIMEOUT : HAMLS_OK;
}
