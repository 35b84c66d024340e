// kernels.h - host-side launchers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace hamls {

// SM count of the current device (grid sizing); set_smem_attr raises a
// kernel's dynamic shared-memory limit once per device (thread-safe)
int current_sm_count();
void set_smem_attr_once(const void* func, int bytes, unsigned* done_mask);

// ------------------------------------------------------------------ cells.cu
struct CellBuild {
  int n, B, P;
  const double* xyz_aos;            // n x 3 input (or NULL, then ax/ay/az)
  const double *ax, *ay, *az;
  const double* wts;                // optional per-point weights (AoS input only)
  uint32_t *keys, *vals, *keys_alt, *vals_alt, *counts;
  uint32_t* start;                  // B*P + 1
  double *px, *py, *pz, *sw;
  float4* pf;
  float* swf;
  DevStatus* st;
  const uint32_t** perm_out;        // receives the sorted -> original permutation
  const uint32_t** keys_out;        // receives the sorted keys
};
int radix_blocks(int n);
void build_cells(const CellBuild& cb, cudaStream_t s, int64_t* launches);
bool radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, int n, int bits,
                      uint32_t* counts, cudaStream_t s, int64_t* launches);
int scan_partials(int n);   // scratch words radix_sort_pairs needs after the counts (see cells.cu)
// the band-edge table of a cell structure with B bands (B + 1 entries)
void build_edge_table(int B, float4* out, cudaStream_t s, int64_t* launches);
// in-place exclusive scan of len words; part: (len + 1023) / 1024 + 1 words of scratch
void exclusive_scan_u32(uint32_t* a, int len, uint32_t* part, cudaStream_t s, int64_t* launches);
void launch_cell_keys(const double* xyz, int n, int B, int P, uint32_t* keys, uint32_t* vals, DevStatus* st,
                      cudaStream_t s);
void launch_csr(const uint32_t* sk, int n, int ncells, uint32_t* start, cudaStream_t s);
void stage_values(const double* y, const uint32_t* perm, int n, double* sy, float4* pf, bool write64,
                  DevStatus* st, cudaStream_t s, int64_t* launches);
void build_tile_order(const double* px, const double* py, const double* pz, int n, int B, int P, uint32_t* keys,
                      uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* counts,
                      const uint32_t** order_out, cudaStream_t s, int64_t* launches);

// ------------------------------------------------------------------- grid.cu
struct GridTables {
  int N;
  double *t, *w, *s;            // N+1: cos theta_k (descending), GL weight, sin theta_k
  double *cphi, *sphi;          // 2N+2
  double *a_rec, *b_rec;        // packed (N+1)(N+2)/2 recurrence coefficients
  double* A64;                  // folded Legendre quadrature matrix, ncoef x hc
  float* A32;
  double2* W64;                 // FFT twiddles exp(-2 pi i j / L), L = 2N+2
  float2* W32;
  float *tf, *sf, *cpf, *spf;   // FP32 copies of t, s, cphi, sphi (FP32 paths)
  int hc;                       // folded column count
  int hcp;                      // row length of A32: hc rounded up to a multiple of 8 (16-byte rows)
};

// Row of degree l within order m's block of the FP32 quadrature matrix: the
// even l - m first (l = m, m+2, ...), then the odd ones.
__host__ __device__ __forceinline__ int l32_row(int N, int m, int l) {
  const int i = l - m;
  return (i & 1) ? (N - m) / 2 + 1 + (i >> 1) : (i >> 1);
}
void build_grid_tables(GridTables& g, bool want32, bool want64, cudaStream_t s, int64_t* launches);

// ----------------------------------------------------------------- tcgemm.cu
// One CTA tile of the tensor-core product D = A B^T: rows [a_y, a_y + 128)
// of A (plus 128 blockIdx.y) at depth a_z, rows [b_y, b_y + nt) of B (nt a
// multiple of 32, at most 256); e0..e3 belong to the epilogue.
struct TcJob {
  int a_y, a_z, b_y, nt;
  int e0, e1, e2, e3;
};
// Tiles of the batched Legendre contraction at bandwidth N (out == nullptr:
// count only): one per order m, parity and block of at most 256 degrees.
int tc_legendre_jobs(int N, TcJob* out);
// coeffs (B x ncoef complex, each set packed as hamls_fit) of the B value
// sets whose folded spectra are G: 2(N+1) blocks (order m, parity) of 2B
// rows (set b: real part row 2b, imaginary 2b+1) of hcp FP32 (hc used)
cudaError_t tc_legendre(const GridTables& g, const float* G, int B, const TcJob* jobs, int njobs, double* coeffs,
                        unsigned* err, cudaStream_t s, int64_t* launches);

// ----------------------------------------------------------------- tables.cu
struct SharedTables {
  int device = 0, N = 0;
  bool mixed = false;
  GridTables g;
  void* mem = nullptr;
  cudaEvent_t ready = nullptr;
  int refs = 0;
  TcJob* jobs = nullptr;        // tensor-core Legendre tiles (mixed form)
  int njobs = 0;
};
// the tables of (current device, N, form), built on s by the first user; later
// users' streams wait for them. nullptr and *err on failure.
SharedTables* tables_acquire(int N, bool mixed, cudaStream_t s, int64_t* launches, cudaError_t* err);
void tables_release(SharedTables* t);
size_t tables_bytes(int N, bool mixed);
int tables_live();
void fibonacci_points(double* x, double* y, double* z, int n, cudaStream_t s, int64_t* launches);

// -------------------------------------------------------------------- knn.cu
struct SupportArgs {
  Cells nodes;                  // scattered nodes
  Cells aux;                    // auxiliary grid
  int n_target, m, N;
  int weight_fn;                // phi: 0 Wendland phi_{3,2}, 1 phi_{3,1}
  double eps, rho_aux;
  const double *ring_t, *ring_s, *cphi, *sphi;
  double* dn_aux_sorted;        // aux d_n (geodesic), sorted aux order
  float* dn_aux_f;              // the same in FP32
  double* delta;                // M_Q
  double* rho2;                 // M_Q
  float* deltaf;                // M_Q, FP32 copies for the FP32 paths
  float* rho2f;
  const float *tf, *sf, *cpf, *spf;
  int32_t* count;               // M_Q
  uint8_t* guarded;             // M_Q
  uint32_t* guard_list;         // work-order positions whose support holds fewer than m nodes
  const uint32_t* order;        // work order (position -> grid node)
  uint32_t* order_keys;         // M_Q (cost keys)
  uint32_t* order_vals;         // M_Q
  int fp64;                     // 1: FP64 Shepard, 0: FP32
  const uint32_t* tile_order;   // aux points (sorted positions) in tile order
  // the Shepard operator (CSR over grid nodes): auxiliary members of each
  // grid node's cap, their Wendland weights (double FP64 / float MIXED) and
  // the weight sums
  const uint32_t* shep_start;
  const uint32_t* shep_col;
  const void* shep_w;
  const void* shep_sw;
  int num_sms;
  DevStatus* st;
};
void run_aux_knn(const SupportArgs& a, cudaStream_t s, int64_t* launches);
// plan time: members per grid node (fill = false, into rows) or the operator
// itself (fill = true, rows = the CSR start array)
void shepard_rows(const SupportArgs& a, uint32_t* rows, uint32_t* col, void* w, void* sw, bool fill,
                  cudaStream_t s, int64_t* launches);
void run_shepard(const SupportArgs& a, cudaStream_t s, int64_t* launches);
// the guard of the listed work-order positions (Sec. 2.2): exact d_n at q
void run_guard(const SupportArgs& a, cudaStream_t s, int64_t* launches);
void run_knn_queries(const Cells& nodes, const double* q, int64_t nq, int n, double* c2_out, DevStatus* st,
                     cudaStream_t s, int64_t* launches);
void run_ball_queries(const Cells& nodes, const double* q, const double* rho2, int64_t nq, int64_t* count,
                      int64_t* idsum, uint64_t* idhash, cudaStream_t s, int64_t* launches);

// -------------------------------------------------------------------- mls.cu
struct MlsArgs {
  Cells nodes;
  const double* sy;             // sorted values (FP64 form)
  const double* sw;             // sorted node weights or NULL
  const float* swf;
  const double *ring_t, *ring_s, *cphi, *sphi;
  int N, K;
  const double* delta;
  const double* rho2;
  const float* deltaf;
  const float* rho2f;
  const float *tf, *sf, *cpf, *spf;
  const uint32_t* order;        // grid nodes, heaviest first
  int MQ;
  double* fgrid;
  double* chi;
  double* tau;
  double chiT, chiF, floor_, fp64_pivot;
  int weight_fn;                // phi: 0 Wendland phi_{3,2}, 1 phi_{3,1}
  double mu[KMAX + 1];
  void* mom;                    // per work-order position: moments (float MIXED, double FP64)
  uint32_t* redo_list;          // MIXED: work-order positions re-solved in FP64
  uint32_t* reg_list;           // work-order positions with chi > chi_T (solved again with tau)
  int m;                        // dim Pi_K^tan
  int32_t* count;               // M_Q: n(q) = #X(q), written by the gather
  const uint8_t* guarded;       // M_Q: support radius from the guard
  uint32_t* guard_list;         // work-order positions with n(q) < m
  DevStatus* st;
  int num_sms;
};
// part 1: gather every grid node (moments, n(q), guard list);
// part 2: gather the guard list again, then solve (and re-solve in FP64)
void run_mls(const MlsArgs& a, bool mixed, cudaStream_t s, int64_t* launches, int part);
// values-only refits: part 0 = row counts (rows[j], their sum added to
// *total); part 1 = gamma per grid node, then the operator (rows = CSR start)
void run_refit_operator(const MlsArgs& a, bool mixed, int part, double* gamma, uint32_t* rows, uint32_t* col,
                        void* val, unsigned long long* total, cudaStream_t s, int64_t* launches);
// f = A y over the plan's grid: y (node order) is gathered into the cell
// order of the operator's columns (perm: cell position -> node), as FP32 in
// yf (MIXED, float entries) or FP64 in ys (FP64, double entries)
void run_refit_apply(int MQ, bool mixed, const uint32_t* rows, const uint32_t* col, const void* val,
                     const double* y, const uint32_t* perm, int M, float* yf, double* ys, double* f, DevStatus* st,
                     cudaStream_t s, int64_t* launches);
// refits of B value sets (MIXED operator): y (B x M doubles, node order)
// through yo (M x B floats, node order), yT (the same in cell order) and fT
// (M_Q x B floats) to f (B x M_Q doubles); B <= 256
// (rows longer than 256 entries go to whole blocks: their list, from
// list_long_rows at prepare time)
void run_refit_apply_batch(int MQ, const uint32_t* rows, const uint32_t* col, const float* val, const double* y,
                           const uint32_t* perm, int M, int B, float* yo, float* yT, float* fT, double* f,
                           const uint32_t* long_list, const uint32_t* nlong, DevStatus* st, cudaStream_t s,
                           int64_t* launches);
void list_long_rows(int MQ, const uint32_t* rows, uint32_t* list, uint32_t* nlist, cudaStream_t s,
                    int64_t* launches);
int value_moment_count(int K);
int mls_moment_slots(int K);

// ------------------------------------------------------------------- quad.cu
struct QuadArgs {
  const GridTables* g;
  const double* fgrid;          // M_Q ring-major
  void* F;                      // (N+1) x (N+1) complex, T
  double* coeffs;               // (N+1)(N+2)/2 complex
  int radices[32];
  int nrad;
};
// part: 1 = ring FFT, 2 = Legendre contraction, 3 = both
void run_quadrature(const QuadArgs& a, bool mixed, cudaStream_t s, int64_t* launches, int part = 3);
// step 3 of B value sets (mixed form), first part: ring FFTs of fgrid
// (B x M_Q, set b at b M_Q) into F (B x (N+1)^2 complex FP32) and the folded
// spectra G (FP32); tc_legendre then contracts them
cudaError_t run_spectra_batch(const GridTables& g, const int* radices, int nrad, const double* fgrid, int B,
                              float2* F, float* G, cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------- forward.cu
// The forward transform f(x) = (F fhat)(x) at P points (Sec. 1): coeffs
// packed complex (device, 2 ncoef doubles); points at (px[i stride],
// py[i stride], pz[i stride]); out[perm ? perm[i] : i]; cws and abws hold
// ncoef complex values each (T2 copies of the coefficients and of the
// recurrence factors a_rec, b_rec).
struct ForwardArgs {
  int N;
  bool mixed;
  const double* coeffs;
  const double *a_rec, *b_rec;
  void* cws;
  void* abws;
  const double *px, *py, *pz;
  int64_t stride, P;
  const uint32_t* perm;
  double* out;
  int num_sms;
};
void run_forward(const ForwardArgs& a, cudaStream_t s, int64_t* launches);

// ---------------------------------------------------------------- voronoi.cu
// Area of the spherical Voronoi cell of every point of g (FP32 area when
// mixed, FP64 otherwise): written to out[perm[s]], sw[s] and swf[s] for the
// non-null ones; lo_scratch holds g.n float4 (overwritten).
void run_voronoi(const Cells& g, bool mixed, float4* lo_scratch, double* out, double* sw, float* swf,
                 DevStatus* st, cudaStream_t s, int64_t* launches);

}  // namespace hamls
