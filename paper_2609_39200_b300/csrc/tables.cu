// tables.cu - the per-bandwidth tables of steps 1 and 3, shared by plans.
//
// The quadrature grid of Sec. 2.1 (Gauss-Legendre nodes and weights, the
// longitudes), the FFT twiddles and the folded quadrature matrix of eq.
// quadrature_based_approximation depend on the bandwidth N alone (and, for the
// matrix, on the precision form). Plans of the same device, N and form share
// one copy, reference-counted: the first plan builds it on its stream and
// records an event; later plans make their streams wait for that event. At
// N = 1024 the FP64 matrix alone is about 2.2 GB, which a pool of plans could
// not afford per plan.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>
#include <mutex>
#include <new>
#include <vector>
#include "common.cuh"
#include "kernels.h"

namespace hamls {

namespace {

std::mutex g_tables_mutex;
std::vector<SharedTables*> g_tables;

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// lay the tables out in one block (base == nullptr: measure only)
size_t carve_tables(GridTables& g, char* base, bool mixed, int njobs, TcJob** jobs) {
  const int N = g.N, L = 2 * N + 2;
  const size_t ncoef = (size_t)(N + 1) * (N + 2) / 2;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += up256(bytes ? bytes : 1);
    return p;
  };
  g.t = reinterpret_cast<double*>(take(sizeof(double) * (N + 1)));
  g.w = reinterpret_cast<double*>(take(sizeof(double) * (N + 1)));
  g.s = reinterpret_cast<double*>(take(sizeof(double) * (N + 1)));
  g.cphi = reinterpret_cast<double*>(take(sizeof(double) * L));
  g.sphi = reinterpret_cast<double*>(take(sizeof(double) * L));
  g.a_rec = reinterpret_cast<double*>(take(sizeof(double) * ncoef));
  g.b_rec = reinterpret_cast<double*>(take(sizeof(double) * ncoef));
  g.A64 = mixed ? nullptr : reinterpret_cast<double*>(take(sizeof(double) * ncoef * g.hc));
  g.A32 = mixed ? reinterpret_cast<float*>(take(sizeof(float) * ncoef * g.hcp)) : nullptr;
  g.W64 = reinterpret_cast<double2*>(take(sizeof(double2) * L));
  g.W32 = reinterpret_cast<float2*>(take(sizeof(float2) * L));
  g.tf = reinterpret_cast<float*>(take(sizeof(float) * (N + 1)));
  g.sf = reinterpret_cast<float*>(take(sizeof(float) * (N + 1)));
  g.cpf = reinterpret_cast<float*>(take(sizeof(float) * L));
  g.spf = reinterpret_cast<float*>(take(sizeof(float) * L));
  *jobs = reinterpret_cast<TcJob*>(take(sizeof(TcJob) * (size_t)njobs));
  return off;
}

void shape_tables(GridTables& g, int N) {
  memset(&g, 0, sizeof(g));
  g.N = N;
  g.hc = N / 2 + 1;
  g.hcp = (g.hc + 7) / 8 * 8;
}

}  // namespace

size_t tables_bytes(int N, bool mixed) {
  GridTables g;
  shape_tables(g, N);
  TcJob* j = nullptr;
  return carve_tables(g, nullptr, mixed, mixed ? tc_legendre_jobs(N, nullptr) : 0, &j);
}

SharedTables* tables_acquire(int N, bool mixed, cudaStream_t s, int64_t* launches, cudaError_t* err) {
  *err = cudaSuccess;
  int dev = 0;
  if ((*err = cudaGetDevice(&dev)) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_tables_mutex);
  for (SharedTables* t : g_tables)
    if (t->device == dev && t->N == N && t->mixed == mixed) {
      if ((*err = cudaStreamWaitEvent(s, t->ready, 0)) != cudaSuccess) return nullptr;
      ++t->refs;
      return t;
    }
  SharedTables* t = new (std::nothrow) SharedTables();
  if (!t) {
    *err = cudaErrorMemoryAllocation;
    return nullptr;
  }
  t->device = dev;
  t->N = N;
  t->mixed = mixed;
  t->refs = 1;
  shape_tables(t->g, N);
  t->njobs = mixed ? tc_legendre_jobs(N, nullptr) : 0;
  const size_t bytes = carve_tables(t->g, nullptr, mixed, t->njobs, &t->jobs);
  if ((*err = cudaMalloc(&t->mem, bytes)) != cudaSuccess) {
    delete t;
    return nullptr;
  }
  carve_tables(t->g, reinterpret_cast<char*>(t->mem), mixed, t->njobs, &t->jobs);
  if ((*err = cudaEventCreateWithFlags(&t->ready, cudaEventDisableTiming)) != cudaSuccess) {
    cudaFree(t->mem);
    delete t;
    return nullptr;
  }
  build_grid_tables(t->g, mixed, !mixed, s, launches);
  if (t->njobs > 0) {
    std::vector<TcJob> hj((size_t)t->njobs);
    tc_legendre_jobs(N, hj.data());
    // pageable source: the copy is complete when cudaMemcpyAsync returns
    *err = cudaMemcpyAsync(t->jobs, hj.data(), sizeof(TcJob) * hj.size(), cudaMemcpyHostToDevice, s);
  }
  if (*err == cudaSuccess) *err = cudaEventRecord(t->ready, s);
  if (*err == cudaSuccess) *err = cudaGetLastError();
  if (*err != cudaSuccess) {
    cudaStreamSynchronize(s);
    cudaEventDestroy(t->ready);
    cudaFree(t->mem);
    delete t;
    return nullptr;
  }
  g_tables.push_back(t);
  return t;
}

void tables_release(SharedTables* t) {
  if (!t) return;
  std::lock_guard<std::mutex> lock(g_tables_mutex);
  if (--t->refs > 0) return;
  for (size_t i = 0; i < g_tables.size(); ++i)
    if (g_tables[i] == t) {
      g_tables.erase(g_tables.begin() + (long)i);
      break;
    }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(t->device);
  cudaEventSynchronize(t->ready);
  cudaEventDestroy(t->ready);
  cudaFree(t->mem);
  cudaSetDevice(cur);
  delete t;
}

int tables_live() {
  std::lock_guard<std::mutex> lock(g_tables_mutex);
  return (int)g_tables.size();
}

}  // namespace hamls
