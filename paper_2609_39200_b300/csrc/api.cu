// api.cu - the C ABI of the HAMLS library (include/hamls.h, include/hamls_debug.h).
//
// A plan owns one device arena sized at creation for its capacity M, its
// bandwidth N and degree K, plus the Shepard operator (sized at plan time
// after its members are counted: the one host wait of hamls_plan) and, once
// hamls_refit_prepare has run, the refit operator (sized the same way).
// hamls_replan, hamls_fit and hamls_refit never allocate. Every stage runs on
// the caller's stream; those three calls never wait for the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <chrono>
#include <new>
#include <thread>
#include "../../include/hamls.h"
#include "../../include/hamls_debug.h"
#include "common.cuh"
#include "kernels.h"

using namespace hamls;

static int dim_tan_host(int K) { return (K + 1) * (K + 2) / 2; }

namespace {

constexpr int NSTAGE = 9;

struct Arena {
  char* base = nullptr;
  size_t off = 0, cap = 0;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

int key_bands(int64_t M) {
  int b = 16;
  while ((int64_t)b * b * 4 < M && b < 4096) b *= 2;
  return b;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void reset_status_kernel(DevStatus* st, int full) {
  if (threadIdx.x == 0) {
    if (full) {
      st->flags = 0;
      st->tc_err = 0;
      for (int i = 0; i < C_NCOUNT; ++i) st->cnt[i] = 0;
      st->cnt[C_MIN_N] = ~0ull;
    } else {
      // per fit: the gather recounts n(q) and re-runs the guard
      st->cnt[C_REG] = st->cnt[C_REDO] = st->cnt[C_DROP] = st->cnt[C_BATCH] = st->cnt[C_REDO_LIST] = 0;
      st->cnt[C_REG_LIST] = 0;
      st->cnt[C_SUM_N] = st->cnt[C_MAX_N] = st->cnt[C_GUARD] = st->cnt[C_GUARD_LIST] = st->cnt[C_LIST_BATCH] = 0;
      st->cnt[C_MIN_N] = ~0ull;
    }
  }
}

}  // namespace

struct hamls_plan_s {
  int device = 0, num_sms = 148;
  int64_t Mcap = 0, M = 0;
  int N = 0, K = 0, m = 0, n_target = 0, MQ = 0, L = 0, M_aux = 0;
  hamls_params p;
  bool mixed = false, has_weights = false;
  Arena arena;
  GridTables g;                    // pointers into the shared tables of (device, N, form)
  SharedTables* tables = nullptr;
  // batched step 3 (hamls_quadrature_batch): spectra and folded spectra of up
  // to batch_cap value sets, allocated on first use and grown as needed
  void* batch_mem = nullptr;
  int batch_cap = 0;
  // refits of many value sets (hamls_refit_batch): transposed values, grid
  // values of each set (FP32, then FP64 for step 3), up to rb_cap sets
  void* rb_mem = nullptr;
  int rb_cap = 0;
  float *rb_yo = nullptr, *rb_yT = nullptr, *rb_fT = nullptr;
  double* rb_f = nullptr;
  float2* batch_F = nullptr;
  float* batch_G = nullptr;
  unsigned* batch_err = nullptr;
  // scattered nodes: the cell structure (B bands, P cells per band) follows
  // the current node count; Bcap is the largest one the arena holds
  int B = 0, P = 0, Bcap = 0;
  uint32_t *keys, *vals, *keys_alt, *vals_alt, *counts, *start;
  float4 *edge = nullptr, *aedge;  // band-edge tables of the node (current B) and auxiliary cells
  float4* edge_all = nullptr;      // the node tables of every B up to Bcap
  const uint32_t *perm = nullptr, *skeys = nullptr;
  double *px, *py, *pz, *sw, *sy;
  float4* pf;
  float* swf;
  // auxiliary grid
  int aB = 0, aP = 0;
  uint32_t *akeys, *avals, *akeys_alt, *avals_alt, *astart;
  const uint32_t *aperm = nullptr, *askeys = nullptr;
  double *ax, *ay, *az, *apx, *apy, *apz, *dn_aux;
  float* dn_auxf;
  float4* apf;
  uint32_t *tkeys, *tvals, *tkeys_alt, *tvals_alt;
  const uint32_t* tile_order = nullptr;
  // Shepard operator: CSR start in the arena; columns, weights and weight
  // sums in one allocation sized at plan time
  uint32_t* shep_start;
  void* shep_mem = nullptr;
  uint32_t* shep_col = nullptr;
  void *shep_w = nullptr, *shep_sw = nullptr;
  // values-only refit operator (hamls_refit_prepare): CSR rows over grid
  // nodes, original node indices, entries (float MIXED / double FP64), gamma
  void* op_mem = nullptr;
  size_t op_bytes = 0;
  uint32_t *op_rows = nullptr, *op_col = nullptr;
  void* op_val = nullptr;
  double* op_gamma = nullptr;
  float* op_yf = nullptr;          // MIXED: the values in FP32 for a refit
  uint32_t* op_long = nullptr;     // count, then the rows of more than 256 entries
  unsigned long long op_nnz = 0;
  bool op_valid = false;
  // grid nodes
  double *delta, *rho2, *fgrid, *chi, *tau;
  float *deltaf, *rho2f;
  uint32_t* redo_list;
  uint32_t* reg_list;
  int32_t* count;
  uint8_t* guarded;
  uint32_t *guard_list, *okeys, *ovals, *okeys_alt, *ovals_alt;
  const uint32_t* order = nullptr;
  void* mom;
  void* F;
  double2* fwd_ws = nullptr;       // hamls_forward: coefficients and recurrence factors in the plan's precision
  double* coeffs;
  // staging of host inputs
  double *in_nodes, *in_wts, *in_vals;
  DevStatus* st;
  DevStatus* st_host = nullptr;
  bool timing = false;
  cudaEvent_t ev[NSTAGE][2];
  bool ev_made = false;
  bool ev_used[NSTAGE];
  cudaStream_t last = 0;
  int64_t launches = 0;
  int radices[32];
  int nrad = 0;
};

namespace {

hamls_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HAMLS_OK;
  if (e == cudaErrorMemoryAllocation) return HAMLS_ERR_OOM;
  return HAMLS_ERR_CUDA;
}

#define HAMLS_TRY(expr)                              \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return cuda_status(_e);   \
  } while (0)

void carve(hamls_plan_s* P) {
  Arena& A = P->arena;
  A.off = 0;
  const int64_t M = P->Mcap;
  const int N = P->N, L = P->L, MQ = P->MQ, Ma = P->M_aux;
  const size_t ncoef = (size_t)(N + 1) * (N + 2) / 2;
  const int sortmax = (int)std::max<int64_t>(std::max<int64_t>(M, Ma), MQ);
  // (the grid tables are shared across plans: tables.cu)
  // nodes
  P->keys = A.take<uint32_t>(M);
  P->vals = A.take<uint32_t>(M);
  P->keys_alt = A.take<uint32_t>(M);
  P->vals_alt = A.take<uint32_t>(M);
  P->counts = A.take<uint32_t>((size_t)256 * radix_blocks(sortmax) + scan_partials(sortmax));
  P->start = A.take<uint32_t>((size_t)P->Bcap * 2 * P->Bcap + 1);
  // band-edge tables of every cell structure up to the capacity's (B = 16,
  // 32, ..., Bcap: B + 1 entries each, built once); a replan selects the one
  // of its node count, so no replan's work depends on an earlier one's (a
  // replan captured in a CUDA graph replays the same whatever ran before)
  {
    size_t ne = 0;
    for (int b = 16; b <= P->Bcap; b *= 2) ne += (size_t)b + 1;
    P->edge_all = A.take<float4>(ne);
  }
  P->aedge = A.take<float4>((size_t)P->aB + 1);
  P->px = A.take<double>(M);
  P->py = A.take<double>(M);
  P->pz = A.take<double>(M);
  P->sy = A.take<double>(M);
  P->sw = A.take<double>(M);
  P->pf = A.take<float4>(M);
  P->swf = A.take<float>(M);
  // aux
  P->akeys = A.take<uint32_t>(Ma);
  P->avals = A.take<uint32_t>(Ma);
  P->akeys_alt = A.take<uint32_t>(Ma);
  P->avals_alt = A.take<uint32_t>(Ma);
  P->astart = A.take<uint32_t>((size_t)P->aB * P->aP + 1);
  P->ax = A.take<double>(Ma);
  P->ay = A.take<double>(Ma);
  P->az = A.take<double>(Ma);
  P->apx = A.take<double>(Ma);
  P->apy = A.take<double>(Ma);
  P->apz = A.take<double>(Ma);
  P->dn_aux = A.take<double>(Ma);
  P->dn_auxf = A.take<float>(Ma);
  P->apf = A.take<float4>(Ma);
  P->tkeys = A.take<uint32_t>(Ma);
  P->tvals = A.take<uint32_t>(Ma);
  P->tkeys_alt = A.take<uint32_t>(Ma);
  P->tvals_alt = A.take<uint32_t>(Ma);
  P->shep_start = A.take<uint32_t>((size_t)MQ + 1);
  // grid nodes
  P->delta = A.take<double>(MQ);
  P->rho2 = A.take<double>(MQ);
  P->deltaf = A.take<float>(MQ);
  P->rho2f = A.take<float>(MQ);
  P->redo_list = A.take<uint32_t>(MQ);
  P->reg_list = A.take<uint32_t>(MQ);
  P->fgrid = A.take<double>(MQ);
  P->chi = A.take<double>(MQ);
  P->tau = A.take<double>(MQ);
  P->count = A.take<int32_t>(MQ);
  P->guarded = A.take<uint8_t>(MQ);
  P->guard_list = A.take<uint32_t>(MQ);
  P->okeys = A.take<uint32_t>(MQ);
  P->ovals = A.take<uint32_t>(MQ);
  P->okeys_alt = A.take<uint32_t>(MQ);
  P->ovals_alt = A.take<uint32_t>(MQ);
  P->mom = A.take<double>((size_t)MQ * mls_moment_slots(P->K) / (P->mixed ? 2 : 1) + 2);
  P->F = A.take<double2>((size_t)(N + 1) * (N + 1));
  P->fwd_ws = A.take<double2>(2 * ncoef);
  P->coeffs = A.take<double>(2 * ncoef);
  P->in_nodes = A.take<double>((size_t)3 * M);
  P->in_wts = A.take<double>(M);
  P->in_vals = A.take<double>(M);
  P->st = A.take<DevStatus>(1);
}

Cells node_cells(const hamls_plan_s* P) {
  Cells c;
  c.B = P->B;
  c.P = P->P;
  c.n = (int)P->M;
  c.start = P->start;
  c.edge = P->edge;
  c.pf = P->pf;
  c.px = P->px;
  c.py = P->py;
  c.pz = P->pz;
  c.perm = P->perm;
  return c;
}

Cells aux_cells(const hamls_plan_s* P) {
  Cells c;
  c.B = P->aB;
  c.P = P->aP;
  c.n = P->M_aux;
  c.start = P->astart;
  c.edge = P->aedge;
  c.pf = P->apf;
  c.px = P->apx;
  c.py = P->apy;
  c.pz = P->apz;
  c.perm = P->aperm;
  return c;
}

void stage_begin(hamls_plan_s* P, int i, cudaStream_t s) {
  if (P->timing) {
    cudaEventRecord(P->ev[i][0], s);
    P->ev_used[i] = true;
  }
}
void stage_end(hamls_plan_s* P, int i, cudaStream_t s) {
  if (P->timing) cudaEventRecord(P->ev[i][1], s);
}

SupportArgs support_args(hamls_plan_s* P) {
  SupportArgs a;
  a.nodes = node_cells(P);
  a.aux = aux_cells(P);
  a.n_target = P->n_target;
  a.m = P->m;
  a.N = P->N;
  a.eps = P->p.eps;
  a.weight_fn = P->p.weight_fn;
  a.rho_aux = P->p.aux_radius * sqrt(4.0 * M_PI / (double)P->M_aux);
  a.ring_t = P->g.t;
  a.ring_s = P->g.s;
  a.cphi = P->g.cphi;
  a.sphi = P->g.sphi;
  a.dn_aux_sorted = P->dn_aux;
  a.dn_aux_f = P->dn_auxf;
  a.delta = P->delta;
  a.rho2 = P->rho2;
  a.deltaf = P->deltaf;
  a.rho2f = P->rho2f;
  a.tf = P->g.tf;
  a.sf = P->g.sf;
  a.cpf = P->g.cpf;
  a.spf = P->g.spf;
  a.count = P->count;
  a.guarded = P->guarded;
  a.guard_list = P->guard_list;
  a.order_keys = P->okeys;
  a.order_vals = P->ovals;
  a.order = P->order;
  a.fp64 = P->mixed ? 0 : 1;
  a.tile_order = P->tile_order;
  a.shep_start = P->shep_start;
  a.shep_col = P->shep_col;
  a.shep_w = P->shep_w;
  a.shep_sw = P->shep_sw;
  a.num_sms = P->num_sms;
  a.st = P->st;
  return a;
}

// node-dependent part of the plan (Sec. 2.2: cell list, d_n, delta, n(q))
hamls_status build_nodes(hamls_plan_s* P, const double* nodes, const double* wts, int64_t M, cudaStream_t s) {
  P->M = M;
  // the cell structure depends on M alone (not on the capacity), so a fit
  // gives the same result in any plan that holds its nodes
  P->B = key_bands(M);
  P->P = 2 * P->B;
  {
    size_t off = 0;
    for (int b = 16; b < P->B; b *= 2) off += (size_t)b + 1;
    P->edge = P->edge_all + off;
  }
  P->op_valid = false;   // a refit operator belongs to the nodes it was built for
  P->has_weights = wts != nullptr;
  reset_status_kernel<<<1, 32, 0, s>>>(P->st, 1);
  ++P->launches;
  const double* dn = nodes;
  if (!is_device_ptr(nodes)) {
    HAMLS_TRY(cudaMemcpyAsync(P->in_nodes, nodes, (size_t)M * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    dn = P->in_nodes;
  }
  const double* dw = wts;
  if (wts && !is_device_ptr(wts)) {
    HAMLS_TRY(cudaMemcpyAsync(P->in_wts, wts, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, s));
    dw = P->in_wts;
  }
  stage_begin(P, 0, s);
  CellBuild cb;
  memset(&cb, 0, sizeof(cb));
  cb.n = (int)M;
  cb.B = P->B;
  cb.P = P->P;
  cb.xyz_aos = dn;
  cb.wts = dw;
  cb.keys = P->keys;
  cb.vals = P->vals;
  cb.keys_alt = P->keys_alt;
  cb.vals_alt = P->vals_alt;
  cb.counts = P->counts;
  cb.start = P->start;
  cb.px = P->px;
  cb.py = P->py;
  cb.pz = P->pz;
  cb.pf = P->pf;
  cb.sw = P->sw;
  cb.swf = P->swf;
  cb.st = P->st;
  cb.perm_out = &P->perm;
  cb.keys_out = &P->skeys;
  build_cells(cb, s, &P->launches);
  stage_end(P, 0, s);
  SupportArgs a = support_args(P);
  stage_begin(P, 1, s);
  run_aux_knn(a, s, &P->launches);
  stage_end(P, 1, s);
  stage_begin(P, 2, s);
  run_shepard(a, s, &P->launches);
  stage_end(P, 2, s);
  stage_begin(P, 3, s);
  bool alt = radix_sort_pairs(P->okeys, P->ovals, P->okeys_alt, P->ovals_alt, P->MQ, 3, P->counts, s,
                              &P->launches);
  P->order = alt ? P->ovals_alt : P->ovals;
  stage_end(P, 3, s);
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status build_static(hamls_plan_s* P, cudaStream_t s) {
  cudaError_t te = cudaSuccess;
  P->tables = tables_acquire(P->N, P->mixed, s, &P->launches, &te);
  if (!P->tables) return cuda_status(te == cudaSuccess ? cudaErrorMemoryAllocation : te);
  P->g = P->tables->g;
  build_edge_table(P->aB, P->aedge, s, &P->launches);
  {
    size_t off = 0;
    for (int b = 16; b <= P->Bcap; b *= 2) {
      build_edge_table(b, P->edge_all + off, s, &P->launches);
      off += (size_t)b + 1;
    }
  }
  fibonacci_points(P->ax, P->ay, P->az, P->M_aux, s, &P->launches);
  CellBuild cb;
  memset(&cb, 0, sizeof(cb));
  cb.n = P->M_aux;
  cb.B = P->aB;
  cb.P = P->aP;
  cb.ax = P->ax;
  cb.ay = P->ay;
  cb.az = P->az;
  cb.keys = P->akeys;
  cb.vals = P->avals;
  cb.keys_alt = P->akeys_alt;
  cb.vals_alt = P->avals_alt;
  cb.counts = P->counts;
  cb.start = P->astart;
  cb.px = P->apx;
  cb.py = P->apy;
  cb.pz = P->apz;
  cb.pf = P->apf;
  cb.st = P->st;
  cb.perm_out = &P->aperm;
  cb.keys_out = &P->askeys;
  build_cells(cb, s, &P->launches);
  // chain order of the auxiliary points for the k-NN: latitude bands about
  // 1.5 point spacings high (a band is 2.8/bt to 4/bt rad high), then
  // longitude; consecutive points then lie about one spacing apart
  const double spacing = sqrt(4.0 * M_PI / (double)P->M_aux);
  int bt = 2 * (int)lround(3.4 / (1.5 * spacing) / 2.0);
  bt = bt < 2 ? 2 : (bt > 4096 ? 4096 : bt);
  build_tile_order(P->apx, P->apy, P->apz, P->M_aux, bt, 8192, P->tkeys, P->tvals, P->tkeys_alt, P->tvals_alt,
                   P->counts, &P->tile_order, s, &P->launches);
  // the Shepard operator: count members per grid node, scan, size, fill
  shepard_rows(support_args(P), P->shep_start, nullptr, nullptr, nullptr, false, s, &P->launches);
  HAMLS_TRY(cudaMemsetAsync(P->shep_start + P->MQ, 0, sizeof(uint32_t), s));
  exclusive_scan_u32(P->shep_start, P->MQ + 1, P->counts, s, &P->launches);
  uint32_t nnz = 0;
  HAMLS_TRY(cudaMemcpyAsync(&nnz, P->shep_start + P->MQ, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HAMLS_TRY(cudaStreamSynchronize(s));
  const size_t wsz = P->mixed ? sizeof(float) : sizeof(double);
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_col = up((size_t)nnz * 4 + 4), b_w = up((size_t)nnz * wsz + wsz), b_sw = up((size_t)P->MQ * wsz);
  HAMLS_TRY(cudaMalloc(&P->shep_mem, b_col + b_w + b_sw));
  P->shep_col = reinterpret_cast<uint32_t*>(P->shep_mem);
  P->shep_w = reinterpret_cast<char*>(P->shep_mem) + b_col;
  P->shep_sw = reinterpret_cast<char*>(P->shep_mem) + b_col + b_w;
  shepard_rows(support_args(P), P->shep_start, P->shep_col, P->shep_w, P->shep_sw, true, s, &P->launches);
  return cuda_status(cudaGetLastError());
}

bool validate_params(const hamls_params& p) {
  if (!(p.eps > 0) || !(p.chi_target > 1) || !(p.chi_full > p.chi_target) || !(p.sobolev_s > 0)) return false;
  if (!(p.aux_radius > 0) || p.aux_points < 0 || !(p.pivot_floor >= 0) || !(p.fp64_pivot >= 0)) return false;
  if (p.precision != HAMLS_FP64 && p.precision != HAMLS_MIXED) return false;
  if (p.n_target < 0 || p.n_target > KNN_MAX) return false;
  if (p.weight_fn != 0 && p.weight_fn != 1) return false;
  return true;
}

void factor_radices(int L, int* r, int& n) {
  n = 0;
  int x = L;
  for (int p = 2; x > 1; ++p)
    while (x % p == 0) {
      r[n++] = p;
      x /= p;
    }
}

}  // namespace

extern "C" {

void hamls_default_params(hamls_params* p) {
  if (!p) return;
  p->n_target = 0;
  p->eps = 0.05;
  p->chi_target = 16.0;
  p->chi_full = 32.0;
  p->sobolev_s = 1.0;
  p->aux_points = 0;
  p->aux_radius = 3.0;
  p->pivot_floor = 1e-12;
  p->precision = HAMLS_FP64;
  p->fp64_pivot = 1e-4;
  p->weight_fn = 0;
}

const char* hamls_status_string(hamls_status s) {
  switch (s) {
    case HAMLS_OK: return "ok";
    case HAMLS_ERR_INVALID_ARG: return "invalid argument (or a node not on the unit sphere)";
    case HAMLS_ERR_OOM: return "device allocation failed";
    case HAMLS_ERR_CUDA: return "CUDA runtime error";
    case HAMLS_ERR_UNDERDETERMINED: return "fewer than m nodes in a support after the guard";
    case HAMLS_ERR_SUPPORT_TOO_LARGE: return "support radius reaches pi/2";
    case HAMLS_ERR_TIMEOUT: return "timed out waiting for the device";
    case HAMLS_ERR_NONFINITE: return "non-finite value";
    case HAMLS_ERR_CAPACITY: return "node count exceeds the plan capacity";
    case HAMLS_ERR_VORONOI: return "a Voronoi cell reaches 1.5 rad from its node or needs more than 32 edges";
  }
  return "unknown status";
}

// shape of a plan for (M, N, K, p): every size the arena depends on
static hamls_status plan_shape(hamls_plan_s* P, int64_t M, int N, int K, const hamls_params& p) {
  if (K < 1 || K > KMAX || N < 1 || N > 1024 || !validate_params(p)) return HAMLS_ERR_INVALID_ARG;
  const int m = dim_tan_host(K);
  const int n_target = p.n_target > 0 ? p.n_target : 4 * m;
  if (n_target > KNN_MAX || n_target < m) return HAMLS_ERR_INVALID_ARG;
  if (M < n_target || M >= (int64_t)1 << 31) return HAMLS_ERR_INVALID_ARG;
  P->p = p;
  P->mixed = p.precision == HAMLS_MIXED;
  P->Mcap = M;
  P->N = N;
  P->K = K;
  P->m = m;
  P->n_target = n_target;
  P->L = 2 * N + 2;
  P->MQ = (N + 1) * P->L;
  P->M_aux = (int)(p.aux_points > 0 ? p.aux_points : 2 * (int64_t)P->MQ);
  P->g.N = N;
  P->g.hc = N / 2 + 1;
  P->g.hcp = (P->g.hc + 7) / 8 * 8;
  P->Bcap = key_bands(M);
  P->B = P->Bcap;
  P->P = 2 * P->B;
  P->aB = key_bands(P->M_aux);
  P->aP = 2 * P->aB;
  factor_radices(P->L, P->radices, P->nrad);
  if (P->nrad > 32) return HAMLS_ERR_INVALID_ARG;
  return HAMLS_OK;
}

hamls_status hamls_plan_footprint(int64_t M, int N, int K, const hamls_params* pin, size_t* bytes) {
  if (!bytes) return HAMLS_ERR_INVALID_ARG;
  *bytes = 0;
  hamls_params p;
  if (pin) p = *pin;
  else hamls_default_params(&p);
  hamls_plan_s* P = new (std::nothrow) hamls_plan_s();
  if (!P) return HAMLS_ERR_OOM;
  hamls_status r = plan_shape(P, M, N, K, p);
  if (r == HAMLS_OK) {
    carve(P);   // measure only (no base address)
    // the Shepard operator: about pi (aux_radius)^2 auxiliary points per grid
    // node (a cap of radius aux_radius spacings), 4 B index + weight each,
    // with a quarter of slack, plus one weight sum per grid node
    const double wsz = P->mixed ? 4.0 : 8.0;
    const double per = 1.25 * M_PI * p.aux_radius * p.aux_radius + 4.0;
    // the grid tables count in full, as for the first plan of its (N, form)
    *bytes = P->arena.off + (size_t)((double)P->MQ * (per * (4.0 + wsz) + wsz)) + sizeof(DevStatus) +
             tables_bytes(N, P->mixed);
  }
  delete P;
  return r;
}

hamls_status hamls_plan(hamls_plan_t* out, const double* nodes_xyz, const double* node_weights, int64_t M,
                        int N, int K, const hamls_params* pin, cudaStream_t stream) {
  if (!out) return HAMLS_ERR_INVALID_ARG;
  *out = nullptr;
  hamls_params p;
  if (pin) p = *pin;
  else hamls_default_params(&p);
  if (!nodes_xyz) return HAMLS_ERR_INVALID_ARG;
  hamls_plan_s* P = new (std::nothrow) hamls_plan_s();
  if (!P) return HAMLS_ERR_OOM;
  {
    const hamls_status r = plan_shape(P, M, N, K, p);
    if (r != HAMLS_OK) {
      delete P;
      return r;
    }
  }
  cudaGetDevice(&P->device);
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  carve(P);   // measure
  P->arena.cap = P->arena.off;
  cudaError_t e = cudaMalloc((void**)&P->arena.base, P->arena.cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return HAMLS_ERR_OOM;
  }
  carve(P);   // assign
  e = cudaMallocHost((void**)&P->st_host, sizeof(DevStatus));
  if (e != cudaSuccess) {
    cudaFree(P->arena.base);
    delete P;
    return HAMLS_ERR_OOM;
  }
  for (int i = 0; i < NSTAGE; ++i) P->ev_used[i] = false;
  hamls_status s = build_static(P, stream);
  if (s == HAMLS_OK) s = build_nodes(P, nodes_xyz, node_weights, M, stream);
  if (s != HAMLS_OK) {
    hamls_destroy(P);
    return s;
  }
  *out = P;
  return HAMLS_OK;
}

hamls_status hamls_plan_reserve(hamls_plan_t* out, int64_t capacity, int N, int K, const hamls_params* pin,
                                cudaStream_t stream) {
  if (!out) return HAMLS_ERR_INVALID_ARG;
  *out = nullptr;
  hamls_params p;
  if (pin) p = *pin;
  else hamls_default_params(&p);
  hamls_plan_s* P = new (std::nothrow) hamls_plan_s();
  if (!P) return HAMLS_ERR_OOM;
  hamls_status r = plan_shape(P, capacity, N, K, p);
  if (r != HAMLS_OK) {
    delete P;
    return r;
  }
  cudaGetDevice(&P->device);
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  carve(P);
  P->arena.cap = P->arena.off;
  if (cudaMalloc((void**)&P->arena.base, P->arena.cap) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return HAMLS_ERR_OOM;
  }
  carve(P);
  if (cudaMallocHost((void**)&P->st_host, sizeof(DevStatus)) != cudaSuccess) {
    cudaFree(P->arena.base);
    delete P;
    return HAMLS_ERR_OOM;
  }
  for (int i = 0; i < NSTAGE; ++i) P->ev_used[i] = false;
  P->M = 0;   // no nodes until hamls_replan
  reset_status_kernel<<<1, 32, 0, stream>>>(P->st, 1);
  ++P->launches;
  r = build_static(P, stream);
  if (r == HAMLS_OK) r = cuda_status(cudaStreamSynchronize(stream));
  if (r != HAMLS_OK) {
    hamls_destroy(P);
    return r;
  }
  P->last = stream;
  *out = P;
  return HAMLS_OK;
}

hamls_status hamls_replan(hamls_plan_t P, const double* nodes_xyz, const double* node_weights, int64_t M,
                          cudaStream_t stream) {
  if (!P || !nodes_xyz) return HAMLS_ERR_INVALID_ARG;
  if (M > P->Mcap) return HAMLS_ERR_CAPACITY;
  if (M < P->n_target) return HAMLS_ERR_INVALID_ARG;
  return build_nodes(P, nodes_xyz, node_weights, M, stream);
}

static MlsArgs mls_args(hamls_plan_s* P) {
  MlsArgs a;
  memset(&a, 0, sizeof(a));
  a.nodes = node_cells(P);
  a.sy = P->sy;
  a.sw = P->has_weights ? P->sw : nullptr;
  a.swf = P->has_weights ? P->swf : nullptr;
  a.ring_t = P->g.t;
  a.ring_s = P->g.s;
  a.cphi = P->g.cphi;
  a.sphi = P->g.sphi;
  a.N = P->N;
  a.K = P->K;
  a.delta = P->delta;
  a.rho2 = P->rho2;
  a.deltaf = P->deltaf;
  a.rho2f = P->rho2f;
  a.tf = P->g.tf;
  a.sf = P->g.sf;
  a.cpf = P->g.cpf;
  a.spf = P->g.spf;
  a.order = P->order;
  a.MQ = P->MQ;
  a.fgrid = P->fgrid;
  a.chi = P->chi;
  a.tau = P->tau;
  a.chiT = P->p.chi_target;
  a.chiF = P->p.chi_full;
  a.floor_ = P->p.pivot_floor;
  a.fp64_pivot = P->p.fp64_pivot;
  a.weight_fn = P->p.weight_fn;
  for (int l = 0; l <= KMAX; ++l) a.mu[l] = pow((double)l * (l + 1), P->p.sobolev_s);
  a.mom = P->mom;
  a.redo_list = P->redo_list;
  a.reg_list = P->reg_list;
  a.m = P->m;
  a.count = P->count;
  a.guarded = P->guarded;
  a.guard_list = P->guard_list;
  a.st = P->st;
  a.num_sms = P->num_sms;
  return a;
}

// steps 1-2 of a fit on staged values: gather with n(q), guard, solves
static void run_step2(hamls_plan_s* P, cudaStream_t s) {
  MlsArgs a = mls_args(P);
  stage_begin(P, 5, s);
  run_mls(a, P->mixed, s, &P->launches, 1);
  run_guard(support_args(P), s, &P->launches);
  run_mls(a, P->mixed, s, &P->launches, 2);
  stage_end(P, 5, s);
}

// step 3 from the grid values: ring FFT, Legendre quadrature, coefficients out
static hamls_status run_step3(hamls_plan_s* P, double* coeffs, cudaStream_t s) {
  const bool dev_out = is_device_ptr(coeffs);
  QuadArgs q;
  memset(&q, 0, sizeof(q));
  q.g = &P->g;
  q.fgrid = P->fgrid;
  q.F = P->F;
  q.coeffs = dev_out ? coeffs : P->coeffs;
  for (int i = 0; i < P->nrad; ++i) q.radices[i] = P->radices[i];
  q.nrad = P->nrad;
  stage_begin(P, 6, s);
  run_quadrature(q, P->mixed, s, &P->launches, 1);
  stage_end(P, 6, s);
  stage_begin(P, 7, s);
  run_quadrature(q, P->mixed, s, &P->launches, 2);
  stage_end(P, 7, s);
  if (!dev_out) {
    const size_t ncoef = (size_t)(P->N + 1) * (P->N + 2) / 2;
    HAMLS_TRY(cudaMemcpyAsync(coeffs, P->coeffs, ncoef * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_fit(hamls_plan_t P, const double* values, double* coeffs, cudaStream_t s) {
  if (!P || !values || !coeffs) return HAMLS_ERR_INVALID_ARG;
  if (P->M <= 0) return HAMLS_ERR_INVALID_ARG;   // a reserved plan without nodes
  reset_status_kernel<<<1, 32, 0, s>>>(P->st, 0);
  ++P->launches;
  const double* dv = values;
  if (!is_device_ptr(values)) {
    HAMLS_TRY(cudaMemcpyAsync(P->in_vals, values, (size_t)P->M * sizeof(double), cudaMemcpyHostToDevice, s));
    dv = P->in_vals;
  }
  stage_begin(P, 4, s);
  stage_values(dv, P->perm, (int)P->M, P->sy, P->pf, !P->mixed, P->st, s, &P->launches);
  stage_end(P, 4, s);
  run_step2(P, s);
  return run_step3(P, coeffs, s);
}

hamls_status hamls_forward(hamls_plan_t P, const double* coeffs, const double* points, int64_t n_points,
                           double* values, cudaStream_t s) {
  if (!P || !coeffs || !values) return HAMLS_ERR_INVALID_ARG;
  const size_t ncoef = (size_t)(P->N + 1) * (P->N + 2) / 2;
  ForwardArgs a;
  memset(&a, 0, sizeof(a));
  a.N = P->N;
  a.mixed = P->mixed;
  a.a_rec = P->g.a_rec;
  a.b_rec = P->g.b_rec;
  a.cws = P->fwd_ws;
  a.abws = P->fwd_ws + ncoef;
  a.num_sms = P->num_sms;
  double* dv = values;
  if (points) {
    // arbitrary points: device arrays only (no staging of a caller-sized set)
    if (n_points < 0 || !is_device_ptr(points) || !is_device_ptr(values)) return HAMLS_ERR_INVALID_ARG;
    if (n_points == 0) return HAMLS_OK;
    a.px = points;
    a.py = points + 1;
    a.pz = points + 2;
    a.stride = 3;
    a.P = n_points;
  } else {
    // the plan's nodes, in sorted order (neighbours share a warp), written
    // back in the caller's order
    if (P->M <= 0 || n_points != P->M) return HAMLS_ERR_INVALID_ARG;
    a.px = P->px;
    a.py = P->py;
    a.pz = P->pz;
    a.stride = 1;
    a.P = P->M;
    a.perm = P->perm;
    if (!is_device_ptr(values)) dv = P->in_vals;
  }
  const double* dc = coeffs;
  if (!is_device_ptr(coeffs)) {
    HAMLS_TRY(cudaMemcpyAsync(P->coeffs, coeffs, 2 * ncoef * sizeof(double), cudaMemcpyHostToDevice, s));
    dc = P->coeffs;
  }
  a.coeffs = dc;
  a.out = dv;
  run_forward(a, s, &P->launches);
  if (dv != values)
    HAMLS_TRY(cudaMemcpyAsync(values, dv, (size_t)P->M * sizeof(double), cudaMemcpyDeviceToHost, s));
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_refit_prepare(hamls_plan_t P, cudaStream_t s) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  if (P->M <= 0) return HAMLS_ERR_INVALID_ARG;   // a reserved plan without nodes
  P->op_valid = false;
  // a fit with zero values: the Gram moments, n(q) and the guard for the nodes
  reset_status_kernel<<<1, 32, 0, s>>>(P->st, 0);
  ++P->launches;
  HAMLS_TRY(cudaMemsetAsync(P->in_vals, 0, (size_t)P->M * sizeof(double), s));
  stage_values(P->in_vals, P->perm, (int)P->M, P->sy, P->pf, !P->mixed, P->st, s, &P->launches);
  run_step2(P, s);
  // members per grid node (into the spare order-key buffer), their total
  MlsArgs a = mls_args(P);
  HAMLS_TRY(cudaMemsetAsync(&P->st->cnt[C_OP_TOTAL], 0, sizeof(unsigned long long), s));
  run_refit_operator(a, P->mixed, 0, nullptr, P->okeys_alt, nullptr, nullptr, &P->st->cnt[C_OP_TOTAL], s,
                     &P->launches);
  unsigned long long total = 0;
  HAMLS_TRY(cudaMemcpyAsync(&total, &P->st->cnt[C_OP_TOTAL], sizeof(total), cudaMemcpyDeviceToHost, s));
  HAMLS_TRY(cudaStreamSynchronize(s));
  if (total >= 0xFFFFFFFFull) return HAMLS_ERR_CAPACITY;
  // one allocation: CSR start, columns, values, gamma
  const size_t vsz = P->mixed ? sizeof(float) : sizeof(double);
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t nrow = (size_t)P->MQ + 1, ny = (size_t)value_moment_count(P->K);
  const size_t b_rows = up(nrow * 4), b_col = up(total * 4 + 4), b_val = up(total * vsz + vsz);
  const size_t b_gamma = up((size_t)P->MQ * ny * sizeof(double));
  const size_t b_long = up(((size_t)P->MQ + 1) * 4);
  const size_t need = b_rows + b_col + b_val + b_gamma + up((size_t)P->Mcap * sizeof(float)) + b_long;
  if (P->op_bytes < need) {
    if (P->op_mem) cudaFree(P->op_mem);
    P->op_mem = nullptr;
    P->op_bytes = 0;
    HAMLS_TRY(cudaMalloc(&P->op_mem, need));
    P->op_bytes = need;
  }
  char* base = reinterpret_cast<char*>(P->op_mem);
  P->op_rows = reinterpret_cast<uint32_t*>(base);
  P->op_col = reinterpret_cast<uint32_t*>(base + b_rows);
  P->op_val = base + b_rows + b_col;
  P->op_gamma = reinterpret_cast<double*>(base + b_rows + b_col + b_val);
  P->op_yf = reinterpret_cast<float*>(base + b_rows + b_col + b_val + b_gamma);
  P->op_long = reinterpret_cast<uint32_t*>(base + b_rows + b_col + b_val + b_gamma + up((size_t)P->Mcap * sizeof(float)));
  HAMLS_TRY(cudaMemcpyAsync(P->op_rows, P->okeys_alt, (size_t)P->MQ * 4, cudaMemcpyDeviceToDevice, s));
  HAMLS_TRY(cudaMemsetAsync(P->op_rows + P->MQ, 0, 4, s));
  exclusive_scan_u32(P->op_rows, P->MQ + 1, P->counts, s, &P->launches);
  run_refit_operator(a, P->mixed, 1, P->op_gamma, P->op_rows, P->op_col, P->op_val, nullptr, s, &P->launches);
  list_long_rows(P->MQ, P->op_rows, P->op_long + 1, P->op_long, s, &P->launches);
  P->op_nnz = total;
  P->op_valid = true;
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_refit(hamls_plan_t P, const double* values, double* coeffs, cudaStream_t s) {
  if (!P || !values || !coeffs) return HAMLS_ERR_INVALID_ARG;
  if (!P->op_valid) return HAMLS_ERR_INVALID_ARG;
  const double* dv = values;
  if (!is_device_ptr(values)) {
    HAMLS_TRY(cudaMemcpyAsync(P->in_vals, values, (size_t)P->M * sizeof(double), cudaMemcpyHostToDevice, s));
    dv = P->in_vals;
  }
  stage_begin(P, 5, s);
  run_refit_apply(P->MQ, P->mixed, P->op_rows, P->op_col, P->op_val, dv, P->perm, (int)P->M, P->op_yf, P->sy,
                  P->fgrid, P->st, s,
                  &P->launches);
  stage_end(P, 5, s);
  return run_step3(P, coeffs, s);
}

// step 3 of B grids (device), MIXED plans: workspace grown as needed
static hamls_status quad_batch_mixed(hamls_plan_s* P, const double* fgrid, double* coeffs, int B, cudaStream_t s) {
  const int N = P->N;
  if (B > P->batch_cap) {
    // workspace for B sets: spectra B (N+1)^2 complex FP32, folded spectra
    // 2 (N+1) x 2B x hcp FP32, an error word
    if (P->batch_mem) {
      HAMLS_TRY(cudaStreamSynchronize(P->last));
      HAMLS_TRY(cudaStreamSynchronize(s));
      cudaFree(P->batch_mem);
      P->batch_mem = nullptr;
      P->batch_cap = 0;
    }
    const size_t bF = ((size_t)B * (N + 1) * (N + 1) * sizeof(float2) + 255) & ~size_t(255);
    const size_t bG = ((size_t)2 * (N + 1) * 2 * B * P->g.hcp * sizeof(float) + 255) & ~size_t(255);
    HAMLS_TRY(cudaMalloc(&P->batch_mem, bF + bG + 256));
    P->batch_F = reinterpret_cast<float2*>(P->batch_mem);
    P->batch_G = reinterpret_cast<float*>(reinterpret_cast<char*>(P->batch_mem) + bF);
    P->batch_err = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(P->batch_mem) + bF + bG);
    P->batch_cap = B;
  }
  HAMLS_TRY(cudaMemsetAsync(P->batch_err, 0, sizeof(unsigned), s));
  stage_begin(P, 6, s);
  cudaError_t e = run_spectra_batch(P->g, P->radices, P->nrad, fgrid, B, P->batch_F, P->batch_G, s,
                                    &P->launches);
  stage_end(P, 6, s);
  if (e != cudaSuccess) return cuda_status(e);
  stage_begin(P, 7, s);
  e = tc_legendre(P->g, P->batch_G, B, P->tables->jobs, P->tables->njobs, coeffs, P->batch_err, s,
                  &P->launches);
  stage_end(P, 7, s);
  if (e != cudaSuccess) return cuda_status(e);
  // a tile that gave up waiting is reported by hamls_sync
  HAMLS_TRY(cudaMemcpyAsync(&P->st->tc_err, P->batch_err, sizeof(unsigned), cudaMemcpyDeviceToDevice, s));
  P->last = s;
  return cuda_status(cudaGetLastError());
}

// step 3 of one grid (device) into coeffs (device), FP64 or FP32 contraction
static void quad_one(hamls_plan_s* P, const double* fgrid, double* coeffs, cudaStream_t s) {
  QuadArgs q;
  memset(&q, 0, sizeof(q));
  q.g = &P->g;
  q.fgrid = fgrid;
  q.F = P->F;
  q.coeffs = coeffs;
  for (int i = 0; i < P->nrad; ++i) q.radices[i] = P->radices[i];
  q.nrad = P->nrad;
  run_quadrature(q, P->mixed, s, &P->launches);
}

hamls_status hamls_quadrature_batch(hamls_plan_t P, const double* fgrid, double* coeffs, int B, cudaStream_t s) {
  if (!P || !fgrid || !coeffs || B < 1 || B > 65535) return HAMLS_ERR_INVALID_ARG;
  if (!is_device_ptr(fgrid) || !is_device_ptr(coeffs)) return HAMLS_ERR_INVALID_ARG;
  const size_t ncoef = (size_t)(P->N + 1) * (P->N + 2) / 2;
  if (!P->mixed) {
    // the FP64 form: its own contraction per value set (the tensor cores
    // carry FP32 accuracy only)
    for (int b = 0; b < B; ++b) quad_one(P, fgrid + (size_t)b * P->MQ, coeffs + (size_t)b * ncoef * 2, s);
    P->last = s;
    return cuda_status(cudaGetLastError());
  }
  return quad_batch_mixed(P, fgrid, coeffs, B, s);
}

hamls_status hamls_refit_batch(hamls_plan_t P, const double* values, double* coeffs, int B, cudaStream_t s) {
  if (!P || !values || !coeffs || B < 1) return HAMLS_ERR_INVALID_ARG;
  if (!P->op_valid) return HAMLS_ERR_INVALID_ARG;
  if (!is_device_ptr(values) || !is_device_ptr(coeffs)) return HAMLS_ERR_INVALID_ARG;
  const size_t ncoef = (size_t)(P->N + 1) * (P->N + 2) / 2;
  const int64_t M = P->M;
  if (!P->mixed) {
    for (int b = 0; b < B; ++b) {
      run_refit_apply(P->MQ, false, P->op_rows, P->op_col, P->op_val, values + (size_t)b * M, P->perm, (int)M,
                      P->op_yf, P->sy, P->fgrid, P->st, s, &P->launches);
      quad_one(P, P->fgrid, coeffs + (size_t)b * ncoef * 2, s);
    }
    P->last = s;
    return cuda_status(cudaGetLastError());
  }
  const int chunk = B < 256 ? B : 256;
  if (chunk > P->rb_cap) {
    if (P->rb_mem) {
      HAMLS_TRY(cudaStreamSynchronize(P->last));
      HAMLS_TRY(cudaStreamSynchronize(s));
      cudaFree(P->rb_mem);
      P->rb_mem = nullptr;
      P->rb_cap = 0;
    }
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t by = up((size_t)P->Mcap * chunk * 4), bfT = up((size_t)P->MQ * chunk * 4);
    const size_t bf = up((size_t)P->MQ * chunk * 8);
    HAMLS_TRY(cudaMalloc(&P->rb_mem, 2 * by + bfT + bf));
    char* rb = reinterpret_cast<char*>(P->rb_mem);
    P->rb_yo = reinterpret_cast<float*>(rb);
    P->rb_yT = reinterpret_cast<float*>(rb + by);
    P->rb_fT = reinterpret_cast<float*>(rb + 2 * by);
    P->rb_f = reinterpret_cast<double*>(rb + 2 * by + bfT);
    P->rb_cap = chunk;
  }
  for (int b0 = 0; b0 < B; b0 += chunk) {
    const int nb = B - b0 < chunk ? B - b0 : chunk;
    stage_begin(P, 5, s);
    run_refit_apply_batch(P->MQ, P->op_rows, P->op_col, reinterpret_cast<const float*>(P->op_val),
                          values + (size_t)b0 * M, P->perm, (int)M, nb, P->rb_yo, P->rb_yT, P->rb_fT, P->rb_f,
                          P->op_long + 1, P->op_long, P->st, s, &P->launches);
    stage_end(P, 5, s);
    const hamls_status r = quad_batch_mixed(P, P->rb_f, coeffs + (size_t)b0 * ncoef * 2, nb, s);
    if (r != HAMLS_OK) return r;
  }
  P->last = s;
  return cuda_status(cudaGetLastError());
}

// Voronoi areas of the plan's nodes (Sec. 2.2, after Theorem 2.1): into the
// caller's buffer, or into the plan's node weights v_i. The FP32 remainders of
// the nodes go to the host-node staging buffer (M x 3 doubles), which a
// replan only needs before its cell build.
static float4* vor_scratch(hamls_plan_s* P) { return reinterpret_cast<float4*>(P->in_nodes); }

hamls_status hamls_voronoi_areas(hamls_plan_t P, double* areas, cudaStream_t s) {
  if (!P || !areas) return HAMLS_ERR_INVALID_ARG;
  if (P->M <= 0) return HAMLS_ERR_INVALID_ARG;   // a reserved plan without nodes
  const bool dev = is_device_ptr(areas);
  double* dst = dev ? areas : P->in_vals;
  stage_begin(P, 8, s);
  run_voronoi(node_cells(P), P->mixed, vor_scratch(P), dst, nullptr, nullptr, P->st, s, &P->launches);
  stage_end(P, 8, s);
  if (!dev) HAMLS_TRY(cudaMemcpyAsync(areas, dst, (size_t)P->M * sizeof(double), cudaMemcpyDeviceToHost, s));
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_voronoi_weights(hamls_plan_t P, cudaStream_t s) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  if (P->M <= 0) return HAMLS_ERR_INVALID_ARG;   // a reserved plan without nodes
  stage_begin(P, 8, s);
  run_voronoi(node_cells(P), P->mixed, vor_scratch(P), nullptr, P->sw, P->swf, P->st, s, &P->launches);
  stage_end(P, 8, s);
  P->has_weights = true;
  P->op_valid = false;   // the refit operator holds the old weights
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_sync(hamls_plan_t P, int timeout_ms) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  cudaStream_t s = P->last;
  HAMLS_TRY(cudaMemcpyAsync(P->st_host, P->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return cuda_status(e);
    if (timeout_ms >= 0) {
      auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
      if (ms > timeout_ms) return HAMLS_ERR_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  unsigned f = P->st_host->flags;
  const unsigned tc = P->st_host->tc_err;
  if (f) HAMLS_TRY(cudaMemsetAsync(&P->st->flags, 0, sizeof(unsigned), s));
  if (tc) HAMLS_TRY(cudaMemsetAsync(&P->st->tc_err, 0, sizeof(unsigned), s));
  if (tc && !f) return HAMLS_ERR_TIMEOUT;
  return hamls_status_from_flags(f);
}

hamls_status hamls_status_from_flags(uint32_t f) {
  if (f & ST_BADNODE) return HAMLS_ERR_INVALID_ARG;
  if (f & ST_NONFINITE) return HAMLS_ERR_NONFINITE;
  if (f & ST_SUPPORT) return HAMLS_ERR_SUPPORT_TOO_LARGE;
  if (f & (ST_UNDERDET | ST_KNN)) return HAMLS_ERR_UNDERDETERMINED;
  if (f & ST_VORONOI) return HAMLS_ERR_VORONOI;
  return HAMLS_OK;
}

hamls_status hamls_status_async(hamls_plan_t P, uint32_t* flags, cudaStream_t s) {
  if (!P || !flags) return HAMLS_ERR_INVALID_ARG;
  HAMLS_TRY(cudaMemcpyAsync(flags, &P->st->flags, sizeof(uint32_t), cudaMemcpyDefault, s));
  HAMLS_TRY(cudaMemsetAsync(&P->st->flags, 0, sizeof(uint32_t), s));
  P->last = s;
  return HAMLS_OK;
}

hamls_status hamls_stats(hamls_plan_t P, hamls_fit_stats* out) {
  if (!P || !out) return HAMLS_ERR_INVALID_ARG;
  HAMLS_TRY(cudaMemcpyAsync(P->st_host, P->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, P->last));
  HAMLS_TRY(cudaStreamSynchronize(P->last));
  const DevStatus& d = *P->st_host;
  out->sum_n = (int64_t)d.cnt[C_SUM_N];
  out->min_n = (int64_t)d.cnt[C_MIN_N];
  out->max_n = (int64_t)d.cnt[C_MAX_N];
  out->n_regularized = (int64_t)d.cnt[C_REG];
  out->n_guarded = (int64_t)d.cnt[C_GUARD];
  out->n_fp64_redo = (int64_t)d.cnt[C_REDO];
  out->n_dropped = (int64_t)d.cnt[C_DROP];
  out->grid_nodes = P->MQ;
  out->aux_points = P->M_aux;
  out->bands = P->B;
  out->cells = P->P;
  out->knn_candidates = (int64_t)d.cnt[C_KNN_CAND];
  out->knn_scans = (int64_t)d.cnt[C_KNN_SCAN];
  out->knn_exact_fallbacks = (int64_t)d.cnt[C_KNN_EXACT_FB];
  return HAMLS_OK;
}

hamls_status hamls_destroy(hamls_plan_t P) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  cudaStreamSynchronize(P->last);
  if (P->ev_made)
    for (int i = 0; i < NSTAGE; ++i) {
      cudaEventDestroy(P->ev[i][0]);
      cudaEventDestroy(P->ev[i][1]);
    }
  if (P->arena.base) cudaFree(P->arena.base);
  if (P->batch_mem) cudaFree(P->batch_mem);
  if (P->rb_mem) cudaFree(P->rb_mem);
  tables_release(P->tables);
  if (P->shep_mem) cudaFree(P->shep_mem);
  if (P->op_mem) cudaFree(P->op_mem);
  if (P->st_host) cudaFreeHost(P->st_host);
  delete P;
  return HAMLS_OK;
}

hamls_status hamls_set_timing(hamls_plan_t P, int enable) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  if (enable && !P->ev_made) {
    for (int i = 0; i < NSTAGE; ++i) {
      HAMLS_TRY(cudaEventCreate(&P->ev[i][0]));
      HAMLS_TRY(cudaEventCreate(&P->ev[i][1]));
    }
    P->ev_made = true;
  }
  P->timing = enable != 0;
  return HAMLS_OK;
}

hamls_status hamls_stage_times(hamls_plan_t P, float* ms, int capacity, int* n_out) {
  if (!P || !ms) return HAMLS_ERR_INVALID_ARG;
  if (n_out) *n_out = NSTAGE;
  for (int i = 0; i < NSTAGE && i < capacity; ++i) {
    ms[i] = -1.f;
    if (P->ev_made && P->ev_used[i]) {
      HAMLS_TRY(cudaEventSynchronize(P->ev[i][1]));
      float t = 0.f;
      if (cudaEventElapsedTime(&t, P->ev[i][0], P->ev[i][1]) == cudaSuccess) ms[i] = t;
      else cudaGetLastError();
    }
  }
  return HAMLS_OK;
}

int64_t hamls_launch_count(hamls_plan_t P, int reset) {
  if (!P) return -1;
  int64_t v = P->launches;
  if (reset) P->launches = 0;
  return v;
}

// ------------------------------------------------------------------ debug
static hamls_status copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!dst) return HAMLS_OK;
  HAMLS_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return HAMLS_OK;
}

hamls_status hamls_debug_cells(hamls_plan_t P, uint32_t* keys_sorted, uint32_t* perm, uint32_t* cell_start,
                               cudaStream_t s) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  hamls_status r;
  if ((r = copy_out(keys_sorted, P->skeys, P->M * 4, s)) != HAMLS_OK) return r;
  if ((r = copy_out(perm, P->perm, P->M * 4, s)) != HAMLS_OK) return r;
  if ((r = copy_out(cell_start, P->start, ((size_t)P->B * P->P + 1) * 4, s)) != HAMLS_OK) return r;
  P->last = s;
  return HAMLS_OK;
}

hamls_status hamls_debug_knn(hamls_plan_t P, const double* queries, int64_t nq, int n, double* c2_out,
                             cudaStream_t s) {
  if (!P || !queries || !c2_out || n < 1 || n > KNN_MAX || n > P->M || nq < 0) return HAMLS_ERR_INVALID_ARG;
  if (!is_device_ptr(queries) || !is_device_ptr(c2_out)) return HAMLS_ERR_INVALID_ARG;
  run_knn_queries(node_cells(P), queries, nq, n, c2_out, P->st, s, &P->launches);
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_debug_ball(hamls_plan_t P, const double* queries, const double* rho2, int64_t nq,
                              int64_t* count, int64_t* idsum, uint64_t* idhash, cudaStream_t s) {
  if (!P || !queries || !rho2 || !count || !idsum || !idhash || nq < 0) return HAMLS_ERR_INVALID_ARG;
  if (!is_device_ptr(queries) || !is_device_ptr(rho2) || !is_device_ptr(count) || !is_device_ptr(idsum) ||
      !is_device_ptr(idhash))
    return HAMLS_ERR_INVALID_ARG;
  run_ball_queries(node_cells(P), queries, rho2, nq, count, idsum, idhash, s, &P->launches);
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_debug_grid(hamls_plan_t P, double* delta, int32_t* count, double* chi, double* tau_tilde,
                              double* fgrid, cudaStream_t s) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  const size_t n = P->MQ;
  hamls_status r;
  if ((r = copy_out(delta, P->delta, n * 8, s)) != HAMLS_OK) return r;
  if ((r = copy_out(count, P->count, n * 4, s)) != HAMLS_OK) return r;
  if ((r = copy_out(chi, P->chi, n * 8, s)) != HAMLS_OK) return r;
  if ((r = copy_out(tau_tilde, P->tau, n * 8, s)) != HAMLS_OK) return r;
  if ((r = copy_out(fgrid, P->fgrid, n * 8, s)) != HAMLS_OK) return r;
  P->last = s;
  return HAMLS_OK;
}

__global__ void unsort_aux_kernel(const double* px, const double* py, const double* pz, const double* dn,
                                  const uint32_t* perm, int n, double* xyz, double* dn_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t o = perm[i];
  if (xyz) {
    xyz[3 * (size_t)o] = px[i];
    xyz[3 * (size_t)o + 1] = py[i];
    xyz[3 * (size_t)o + 2] = pz[i];
  }
  if (dn_out) dn_out[o] = dn[i];
}

hamls_status hamls_debug_aux(hamls_plan_t P, double* aux_xyz, double* dn_aux, cudaStream_t s) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  if ((aux_xyz && !is_device_ptr(aux_xyz)) || (dn_aux && !is_device_ptr(dn_aux))) return HAMLS_ERR_INVALID_ARG;
  unsort_aux_kernel<<<(P->M_aux + 255) / 256, 256, 0, s>>>(P->apx, P->apy, P->apz, P->dn_aux, P->aperm, P->M_aux,
                                                           aux_xyz, dn_aux);
  ++P->launches;
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_debug_quadrature(hamls_plan_t P, const double* fgrid, double* coeffs, cudaStream_t s) {
  if (!P || !fgrid || !coeffs) return HAMLS_ERR_INVALID_ARG;
  if (!is_device_ptr(fgrid) || !is_device_ptr(coeffs)) return HAMLS_ERR_INVALID_ARG;
  QuadArgs q;
  memset(&q, 0, sizeof(q));
  q.g = &P->g;
  q.fgrid = fgrid;
  q.F = P->F;
  q.coeffs = coeffs;
  for (int i = 0; i < P->nrad; ++i) q.radices[i] = P->radices[i];
  q.nrad = P->nrad;
  run_quadrature(q, P->mixed, s, &P->launches);
  P->last = s;
  return cuda_status(cudaGetLastError());
}

hamls_status hamls_debug_gl(hamls_plan_t P, double* t, double* w, cudaStream_t s) {
  if (!P) return HAMLS_ERR_INVALID_ARG;
  hamls_status r;
  if ((r = copy_out(t, P->g.t, (P->N + 1) * 8, s)) != HAMLS_OK) return r;
  if ((r = copy_out(w, P->g.w, (P->N + 1) * 8, s)) != HAMLS_OK) return r;
  P->last = s;
  return HAMLS_OK;
}

}  // extern "C"
