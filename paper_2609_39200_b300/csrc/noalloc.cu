// noalloc.cu - the cell-list build without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another component
// owns all device memory (a fixed pool handed out by an embedding runtime),
// real-time loops that must never enter the allocator, or hosts whose policy
// forbids allocations after start-up. hamls_cells_noalloc serves them: the
// caller passes the nodes and the three output arrays; the sort's scratch
// (the second key/index pair, the digit histograms and the scan partials)
// lives in one file-scope static __device__ array of fixed size, reserved on
// every GPU that loads the library until the process exits.
#include <cuda_runtime.h>
#include <mutex>
#include "../../include/hamls.h"
#include "common.cuh"
#include "kernels.h"

using namespace hamls;

namespace {

constexpr int64_t NOALLOC_MAX_M = (int64_t)1 << 20;       // nodes per call
constexpr int64_t NOALLOC_SORT_BLOCKS = (NOALLOC_MAX_M + 4095) / 4096;
constexpr int64_t NOALLOC_COUNT_WORDS = 256 * NOALLOC_SORT_BLOCKS + 256;   // histograms + scan partials
constexpr int64_t NOALLOC_STATUS_WORDS = (sizeof(DevStatus) + 3) / 4;
constexpr int64_t NOALLOC_WORDS = 2 * NOALLOC_MAX_M + NOALLOC_COUNT_WORDS + NOALLOC_STATUS_WORDS;

// 2 x 4 MiB of key/index ping-pong plus ~257 KiB of histograms: about 8.3 MiB.
static __device__ __align__(256) uint32_t g_cells_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[MAX_DEVICES] = {nullptr};

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" hamls_status hamls_cells_noalloc(const double* nodes_xyz, int64_t M, int bands, int cells,
                                            uint32_t* keys_sorted, uint32_t* perm, uint32_t* cell_start,
                                            cudaStream_t stream) {
  if (!nodes_xyz || !keys_sorted || !perm || !cell_start) return HAMLS_ERR_INVALID_ARG;
  if (M < 1 || bands < 2 || (bands & 1) || bands > 4096 || cells < 4 || (cells & 3) || cells > 8192)
    return HAMLS_ERR_INVALID_ARG;
  if (M > NOALLOC_MAX_M) return HAMLS_ERR_CAPACITY;
  if (!device_ptr(nodes_xyz) || !device_ptr(keys_sorted) || !device_ptr(perm) || !device_ptr(cell_start))
    return HAMLS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HAMLS_ERR_CUDA;
  uint32_t* scratch;
  {
    // once per device, with that device current: the device address of the
    // static array (its host-side name is only a stand-in)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_cells_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return HAMLS_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<uint32_t*>(ptr);
    }
    scratch = g_scratch_ptr[dev];
  }
  const int n = (int)M;
  if ((int64_t)256 * radix_blocks(n) + scan_partials(n) > NOALLOC_COUNT_WORDS) return HAMLS_ERR_CAPACITY;
  // the scratch belongs to the current device: the stream must too
  int sdev = -1;
  if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess) {
    cudaGetLastError();
    return HAMLS_ERR_INVALID_ARG;
  }
  if (sdev != dev) return HAMLS_ERR_INVALID_ARG;
  // an error the caller left pending is the caller's: report it without
  // clearing it and launch nothing, so that the checks below see only this
  // call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return HAMLS_ERR_CUDA;
  uint32_t* keys_alt = scratch;
  uint32_t* vals_alt = scratch + NOALLOC_MAX_M;
  uint32_t* counts = scratch + 2 * NOALLOC_MAX_M;
  DevStatus* st = reinterpret_cast<DevStatus*>(scratch + 2 * NOALLOC_MAX_M + NOALLOC_COUNT_WORDS);
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), stream) != cudaSuccess) return HAMLS_ERR_CUDA;
  int bits = 0;
  while ((1ull << bits) < (unsigned long long)bands * cells) ++bits;
  const int passes = (bits + 7) / 8;
  // start where the ping-pong passes end in the caller's arrays (an odd
  // count starts in the scratch, an even one in the caller's arrays)
  uint32_t *k0 = keys_sorted, *v0 = perm, *k1 = keys_alt, *v1 = vals_alt;
  if (passes & 1) {
    k0 = keys_alt;
    v0 = vals_alt;
    k1 = keys_sorted;
    v1 = perm;
  }
  int64_t launches = 0;
  launch_cell_keys(nodes_xyz, n, bands, cells, k0, v0, st, stream);
  if (cudaGetLastError() != cudaSuccess) return HAMLS_ERR_CUDA;
  radix_sort_pairs(k0, v0, k1, v1, n, bits, counts, stream, &launches);
  if (cudaGetLastError() != cudaSuccess) return HAMLS_ERR_CUDA;
  launch_csr(keys_sorted, n, bands * cells, cell_start, stream);
  return cudaGetLastError() == cudaSuccess ? HAMLS_OK : HAMLS_ERR_CUDA;
}
