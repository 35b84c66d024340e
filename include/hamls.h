/*
 * hamls.h - C ABI of the B300 (sm_103a) HAMLS library: harmonic approximation
 * of scattered data on the sphere S^2 via moving least squares.
 *
 * The library computes Algorithm 1 of the paper ("Harmonic Approximation via
 * Moving Least Squares", Sec. 2):
 *   step 1  a product quadrature grid: Gauss-Legendre nodes t_k = cos(theta_k)
 *           (k = 0..N, north first) times phi_j = 2 pi j / (2N+2)
 *           (j = 0..2N+1); M_Q = (N+1)(2N+2) nodes, exact on Pi_{2N} (Sec. 2.1);
 *   step 2  the regularised MLS value f_j = M_y(q_j) at every grid node
 *           (Sec. 2.2, 2.3): support radius delta(q) = (1+eps) d~_n(q)
 *           (eq. adaptive_support_radius, smoothed over a Fibonacci auxiliary
 *           grid), Wendland weights (eq. weight_function_radial), tangent-plane
 *           polynomials of degree <= K, centre amplification chi
 *           (eq. chi via coupling), degree-adapted regularisation tau found by
 *           bisection (eq. regularized MLS amplification), smoothed tau~;
 *   step 3  the adjoint transform fhat = F^H W f on the grid: a DFT over
 *           every ring, then the associated-Legendre quadrature
 *           (eq. quadrature_based_approximation).
 *
 * Notation: N is the harmonic bandwidth (the paper's L), M the number of
 * scattered nodes (the paper's N), K the MLS degree, m = (K+1)(K+2)/2.
 *
 * Memory and ownership. Every pointer argument may be a device pointer or a
 * host pointer (pageable or pinned); the library detects which with
 * cudaPointerGetAttributes and stages host data through buffers the plan owns.
 * The caller owns all argument buffers; the plan owns every device allocation
 * it makes: inside hamls_plan, and the refit operator in hamls_refit_prepare;
 * hamls_replan, hamls_fit, hamls_refit and the Voronoi calls allocate nothing.
 * Calls are stream-ordered and asynchronous: inputs must stay valid, and
 * outputs must not be read, until the stream work is done (hamls_sync).
 * A plan must not be used from two streams at once.
 *
 * Errors. No exception crosses the ABI and the library never aborts the
 * process. Argument errors are returned immediately. Conditions found on the
 * device (too few nodes in a support, support radius >= pi/2, non-finite
 * values, nodes off the unit sphere, a Voronoi cell that cannot be formed)
 * are recorded in a device status word and returned by hamls_sync.
 */
#ifndef HAMLS_H
#define HAMLS_H

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hamls_plan_s* hamls_plan_t;

typedef enum {
  HAMLS_OK = 0,
  HAMLS_ERR_INVALID_ARG = 1,        /* bad argument, or a node not on the unit sphere */
  HAMLS_ERR_OOM = 2,                /* a device allocation failed (plan creation only) */
  HAMLS_ERR_CUDA = 3,               /* a CUDA runtime call failed */
  HAMLS_ERR_UNDERDETERMINED = 4,    /* fewer than m nodes in a support even after the guard */
  HAMLS_ERR_SUPPORT_TOO_LARGE = 5,  /* delta(q) >= pi/2: no open hemisphere (Sec. 2.3) */
  HAMLS_ERR_TIMEOUT = 6,            /* hamls_sync gave up waiting */
  HAMLS_ERR_NONFINITE = 7,          /* a value or node coordinate is NaN/Inf */
  HAMLS_ERR_CAPACITY = 8,           /* M exceeds the plan's capacity */
  HAMLS_ERR_VORONOI = 9             /* a Voronoi cell reaches 1.5 rad from its node or needs more
                                       than 32 edges (hamls_voronoi_areas/_weights) */
} hamls_status;

typedef enum { HAMLS_FP64 = 0, HAMLS_MIXED = 1 } hamls_precision;

/* Method parameters. hamls_default_params fills the defaults given here. */
typedef struct {
  int     n_target;     /* target neighbour count n; 0 => 4 m (Sec. 3.2, n = 4 dim Pi_K^tan) */
  double  eps;          /* delta = (1+eps) d~_n (eq. adaptive_support_radius); default 0.05 */
  double  chi_target;   /* chi_T > 1 (Sec. 2.3, choosing the regularization strength); default 16 */
  double  chi_full;     /* chi_full > chi_T, full regularisation from here on; default 32 */
  double  sobolev_s;    /* s in mu_j = (l(j)(l(j)+1))^s (eq. mls degree multipliers); default 1 */
  int64_t aux_points;   /* Fibonacci auxiliary grid size; 0 => 2 M_Q (Sec. 2.2, last paragraph) */
  double  aux_radius;   /* Shepard support radius in units of sqrt(4 pi / aux_points); default 3 */
  double  pivot_floor;  /* squared Cholesky pivot at or below which a direction is dropped; 1e-12 */
  int     precision;    /* hamls_precision; default HAMLS_FP64 */
  double  fp64_pivot;   /* MIXED only: squared FP32 pivot below which the local Cholesky is
                           redone in FP64; default 1e-4 */
  int     weight_fn;    /* phi of eq. weight_function_radial, for the MLS weights and the Shepard
                           weights of the support radius (Sec. 2.2 leaves the Wendland function
                           open): 0 = phi_{3,2}(r) = (1-r)^6 (35 r^2 + 18 r + 3), C^4 (default);
                           1 = phi_{3,1}(r) = (1-r)^4 (4 r + 1), C^2 (then the smoothed tau of
                           Sec. 2.3 is C^2, not C^3). Other values: HAMLS_ERR_INVALID_ARG */
} hamls_params;

/* Per-plan statistics of the last plan/replan and fit. */
typedef struct {
  int64_t sum_n;          /* sum over grid nodes of n(q) = #X(q) (eq. number_of_local_nodes) */
  int64_t min_n, max_n;
  int64_t n_regularized;  /* grid nodes with tau~ > 0 */
  int64_t n_guarded;      /* grid nodes whose support came from the exact-d_n guard; the guard
                             runs inside the first fit after a plan/replan */
  int64_t n_fp64_redo;    /* MIXED: grid nodes whose local solve ran in FP64 */
  int64_t n_dropped;      /* basis directions dropped by the pivot floor, summed */
  int64_t grid_nodes;     /* M_Q */
  int64_t aux_points;     /* size of the auxiliary grid */
  int32_t bands, cells;   /* neighbour structure: latitude bands and cells per band */
  int64_t knn_candidates; /* auxiliary k-NN: candidate nodes streamed, over all cap scans */
  int64_t knn_scans;      /* auxiliary k-NN: cap scans (one per point when the chained radius
                             already holds n nodes) */
  int64_t knn_exact_fallbacks;  /* auxiliary searches that needed all-FP64 distances */
} hamls_fit_stats;

/* Fill *p with the defaults listed in hamls_params. */
void hamls_default_params(hamls_params* p);

/*
 * hamls_plan - allocate a plan for up to M nodes at bandwidth N and degree K
 * and build everything that depends on the nodes only: the quadrature grid
 * (Sec. 2.1), the cell list over the nodes, d_n on the auxiliary grid and
 * delta(q) at every grid node (Sec. 2.2). n(q) = #X(q) is counted by the
 * fit's gather, which also applies the guard (exact d_n at q) where n(q) < m.
 *   out          receives the plan handle (NULL on failure)
 *   nodes_xyz    M x 3 doubles, row-major unit vectors x_i (host or device)
 *   node_weights M doubles v_i > 0 multiplying the MLS weights, e.g. Voronoi
 *                areas (Sec. 2.2, after Theorem 2.1); NULL means v_i = 1
 *   M            number of nodes, m <= M < 2^31
 *   N            bandwidth, 1 <= N <= 1024
 *   K            MLS degree, 1 <= K <= 4
 *   p            parameters, NULL for the defaults
 *   stream       CUDA stream for all work (0 = legacy default stream)
 * The smoothing of d_n onto the grid (Shepard, Sec. 2.2) uses a fixed radius
 * on fixed grids, so the plan stores it as a sparse operator; to size that
 * operator hamls_plan waits once for its stream. Later work stays asynchronous.
 * Returns HAMLS_OK, HAMLS_ERR_INVALID_ARG, HAMLS_ERR_OOM or HAMLS_ERR_CUDA.
 */
hamls_status hamls_plan(hamls_plan_t* out, const double* nodes_xyz, const double* node_weights,
                        int64_t M, int N, int K, const hamls_params* p, cudaStream_t stream);

/*
 * hamls_plan_footprint - device memory that hamls_plan(M, N, K, p) would
 * allocate, in bytes, without touching the device: the plan's arena exactly
 * and the Shepard operator (sized only at plan time, after its members are
 * counted) estimated with a quarter of slack. A refit operator
 * (hamls_refit_prepare) is not included. For admission by memory footprint
 * in a serving loop. Returns HAMLS_ERR_INVALID_ARG for shapes hamls_plan
 * rejects.
 */
hamls_status hamls_plan_footprint(int64_t M, int N, int K, const hamls_params* p, size_t* bytes);

/*
 * hamls_plan_reserve - a plan for up to `capacity` nodes at bandwidth N and
 * degree K without nodes yet: allocates what hamls_plan allocates for M =
 * capacity and builds the node-independent part (quadrature grid, auxiliary
 * grid, Shepard operator), waiting for `stream` once; hamls_replan then gives
 * it nodes (fits, refits and Voronoi calls return HAMLS_ERR_INVALID_ARG until
 * then). For pools of plans created ahead of a stream of fits.
 * Returns as hamls_plan.
 */
hamls_status hamls_plan_reserve(hamls_plan_t* out, int64_t capacity, int N, int K, const hamls_params* p,
                                cudaStream_t stream);

/*
 * hamls_replan - rebuild the node-dependent part of an existing plan for a new
 * node set of M' <= M (the plan's capacity) nodes, with no allocation.
 * Arguments as in hamls_plan. Returns HAMLS_ERR_CAPACITY if M' is too large.
 * The cell structure over the nodes is chosen from M' alone, so a fit gives
 * the same coefficients in every plan that can hold its nodes.
 */
hamls_status hamls_replan(hamls_plan_t plan, const double* nodes_xyz, const double* node_weights,
                          int64_t M, cudaStream_t stream);

/*
 * hamls_fit - Algorithm 1 steps 2 and 3 for one set of values at the plan's nodes.
 *   values  M doubles y_i (host or device)
 *   coeffs  (N+1)(N+2)/2 complex coefficients, interleaved (re, im) doubles,
 *           packed m-major: order m = 0..N starts at m(N+1) - m(m-1)/2 and
 *           holds l = m..N. Fully normalised complex spherical harmonics with
 *           the Condon-Shortley phase; for real data fhat_l^{-m} =
 *           (-1)^m conj(fhat_l^m) gives the negative orders.
 * Complex data (the paper allows y in C) is two calls, one per part.
 */
hamls_status hamls_fit(hamls_plan_t plan, const double* values, double* coeffs, cudaStream_t stream);

/*
 * hamls_forward - the forward transform of the problem statement (Sec. 1, the
 * sampling matrix F of eq. LSQR-Problem_Regularized): the values
 *   f(x) = sum_l fhat_l^0 Pbar_l^0(cos theta) + 2 Re sum_{m>=1} e^{i m phi} sum_{l>=m} fhat_l^m Pbar_l^m(cos theta)
 * of the real field with the plan's bandwidth N whose coefficients are
 * given in hamls_fit's packing (fully normalised, Condon-Shortley phase), at
 * points x. With F applied to a fit's coefficients at the plan's nodes, the
 * values minus the data are the fit's residual.
 *   coeffs    (N+1)(N+2)/2 complex = 2 (N+1)(N+2)/2 doubles (host or device)
 *   points    n_points x 3 doubles (device), unit vectors; or NULL for the
 *             plan's nodes (then n_points must equal their count M, and the
 *             values come in the node order of the last hamls_plan/hamls_replan)
 *   values    n_points doubles (device; host allowed with points == NULL)
 * FP64 plans evaluate in FP64; MIXED plans run the degree recurrence in FP32
 * with a carried binary exponent (the per-order seed and e^{i m phi} in FP64):
 * about 1e-6 of the field's scale. Allocates nothing (the plan holds the
 * workspace). HAMLS_ERR_INVALID_ARG for NULL coeffs/values, a host points or
 * values array with explicit points, a mismatched n_points, or a reserved
 * plan without nodes when points == NULL.
 */
hamls_status hamls_forward(hamls_plan_t plan, const double* coeffs, const double* points, int64_t n_points,
                           double* values, cudaStream_t stream);

/*
 * hamls_quadrature_batch - Algorithm 1 step 3 for B sets of grid values at
 * once (eq. quadrature_based_approximation): for value sets that share the
 * bandwidth N (refits of many value series, or fits of different plans of
 * the same N), the Legendre quadrature of all sets is one matrix product per
 * order m and parity, which MIXED plans run on the tensor cores (tcgen05,
 * 3xTF32 products with FP32 accumulation; relative error ~1e-6, as the FP32
 * contraction of hamls_fit). FP64 plans run the FP64 contraction set by set.
 *   fgrid   B x M_Q doubles (device): set b at b M_Q, grid nodes ring-major
 *           (k (2N+2) + j), e.g. the grid values of hamls_debug_grid
 *   coeffs  B x (N+1)(N+2)/2 complex (device), each set packed as hamls_fit
 *   B       1 <= B <= 65535
 * The first call with a given B allocates the workspace (spectra and folded
 * spectra, about B (N+1)^2 24 B; owned by the plan, reused by later calls of
 * B or fewer sets) and, when it grows, waits for the plan's stream. A tile
 * whose copies or products did not arrive within about 2 s is reported by
 * hamls_sync as HAMLS_ERR_TIMEOUT.
 */
hamls_status hamls_quadrature_batch(hamls_plan_t plan, const double* fgrid, double* coeffs, int B,
                                    cudaStream_t stream);

/*
 * Values-only refits: new values at the same nodes (a time series on fixed
 * stations). For fixed nodes every grid value f(q_j) = M_y(q_j) is linear in
 * the data y: the Gram matrix, chi and tau~ of the local problem depend on the
 * nodes only, and the data enter through the right-hand side (Sec. 2.3). The
 * plan can therefore keep the fit as a sparse operator
 *   f(q_j) = sum_{i in X(q_j)} A_ji y_i,
 * and a refit is that product followed by step 3 (ring FFT, Legendre).
 *
 * hamls_refit_prepare - build the operator for the plan's current nodes: runs
 *   the gather, the guard and the local solves once (n(q) statistics as for a
 *   fit), then the entries. It allocates the operator's device memory (reused
 *   by later calls when large enough; owned and freed by the plan): about
 *   sum_q n(q) * 8 B (MIXED) or 12 B (FP64), plus M_Q * (4 + 4 (K+1)(K+2)) B
 *   and 4 B per node of capacity,
 *   and waits once for its stream to size it. hamls_replan invalidates the
 *   operator. Returns HAMLS_ERR_CAPACITY beyond 2^32 - 1 entries, and
 *   HAMLS_ERR_OOM or HAMLS_ERR_CUDA as hamls_plan.
 * hamls_refit - coefficients for new values at the prepared nodes; arguments
 *   as hamls_fit. HAMLS_ERR_INVALID_ARG if no operator exists for the current
 *   nodes. FP64 plans reproduce hamls_fit up to rounding; MIXED plans store the
 *   entries in FP32 (computed from the FP32 moments with FP64 local solves)
 *   and sum their products with the FP32-rounded values in FP32. Non-finite
 *   values are reported by hamls_sync.
 */
hamls_status hamls_refit_prepare(hamls_plan_t plan, cudaStream_t stream);
hamls_status hamls_refit(hamls_plan_t plan, const double* values, double* coeffs, cudaStream_t stream);

/*
 * hamls_refit_batch - hamls_refit for B value sets at the prepared nodes at
 * once (a time series on fixed stations): the operator is read once for all
 * sets, and step 3 is hamls_quadrature_batch's (tensor cores, MIXED plans).
 *   values  B x M doubles (device): set b at b M, in the node order of the plan
 *   coeffs  B x (N+1)(N+2)/2 complex (device), each set packed as hamls_fit
 * MIXED plans take up to 256 sets per pass (more are done in passes) and
 * allocate their workspace on the first call with a larger pass (about
 * (8 M + 12 M_Q) bytes per set, plus hamls_quadrature_batch's; owned by the
 * plan), waiting for the stream when it grows. FP64 plans refit set by set.
 * HAMLS_ERR_INVALID_ARG without a prepared operator or for host pointers.
 */
hamls_status hamls_refit_batch(hamls_plan_t plan, const double* values, double* coeffs, int B, cudaStream_t stream);

/*
 * hamls_voronoi_areas - the area of the spherical Voronoi cell of every node
 * of the plan, V_i = { p in S^2 : p.x_i >= p.x_j for all j }: the weights v_i
 * by which the paper rescales the local MLS weights for ill-distributed nodes
 * (Sec. 2.2, the remark after Theorem 2.1; all experiments of Sec. 3 use them).
 *   areas   M doubles (host or device), in the node order of the last
 *           hamls_plan/hamls_replan; they sum to 4 pi
 * Exact duplicate nodes share their cell equally. Geometry in FP64 for FP64
 * plans, FP32 (on FP64 differences of the nodes) for mixed plans. A cell that
 * reaches 1.5 rad from its node (nodes confined to a small part of the
 * sphere) or needs more than 32 edges gets a NaN area, and hamls_sync returns
 * HAMLS_ERR_VORONOI. Allocates nothing; asynchronous on `stream`.
 * Returns HAMLS_OK, HAMLS_ERR_INVALID_ARG or HAMLS_ERR_CUDA.
 */
hamls_status hamls_voronoi_areas(hamls_plan_t plan, double* areas, cudaStream_t stream);

/*
 * hamls_voronoi_weights - compute the Voronoi areas of the plan's nodes (as in
 * hamls_voronoi_areas) and use them as the node weights v_i of the following
 * fits, in place of the weights given to hamls_plan/hamls_replan, until the
 * next hamls_replan. A refit operator prepared before is invalidated.
 * Allocates nothing; asynchronous on `stream`.
 */
hamls_status hamls_voronoi_weights(hamls_plan_t plan, cudaStream_t stream);

/* Wait (at most timeout_ms, < 0 = forever) for the plan's stream work and
 * return the first device-detected error, or HAMLS_OK. Clears the status. */
hamls_status hamls_sync(hamls_plan_t plan, int timeout_ms);

/*
 * hamls_status_async - the device status word without a host wait: enqueue on
 * `stream` a copy of the plan's status word (the conditions hamls_sync would
 * report, as bit flags) into *flags and clear the word on the device. *flags
 * may be device memory or host memory (pinned for an asynchronous copy); it
 * is valid once the stream has reached the copy. Called after each fit, it
 * gives every fit its own status even when the plan is replanned before the
 * host looks. hamls_status_from_flags maps a word to the status hamls_sync
 * would return for it.
 */
hamls_status hamls_status_async(hamls_plan_t plan, uint32_t* flags, cudaStream_t stream);
hamls_status hamls_status_from_flags(uint32_t flags);

/* Statistics of the last plan/replan and fit (synchronises the stream); the
 * n(q) figures (sum_n, min_n, max_n, n_guarded) come from the last fit. */
hamls_status hamls_stats(hamls_plan_t plan, hamls_fit_stats* out);

/* Release every resource of the plan (synchronises its last stream). */
hamls_status hamls_destroy(hamls_plan_t plan);

/* Static text for a status code. */
const char* hamls_status_string(hamls_status s);

/*
 * Stage timing. When enabled, hamls_replan and hamls_fit record CUDA events
 * around each stage on the caller's stream; hamls_stage_times returns the
 * elapsed milliseconds of the last call of each stage (synchronises):
 *   0 cell keys + sort + ranges, 1 auxiliary kNN, 2 Shepard + support radius,
 *   3 work order of the grid nodes, 4 value staging, 5 MLS (gather with n(q),
 *   guard, solve), 6 ring FFT, 7 Legendre quadrature.  n_out receives the count (8).
 */
hamls_status hamls_set_timing(hamls_plan_t plan, int enable);
hamls_status hamls_stage_times(hamls_plan_t plan, float* ms, int capacity, int* n_out);

/* Number of kernel launches the library made on the plan's behalf since the
 * last reset (reset with reset != 0). */
int64_t hamls_launch_count(hamls_plan_t plan, int reset);

/*
 * hamls_cells_noalloc - the cell-list build of hamls_plan (integer cell keys,
 * stable radix sort, CSR runs; the same output as hamls_debug_cells for the
 * same bands/cells) for callers that cannot allocate device memory. The paper
 * has no counterpart: this is a service of the library.
 *   nodes_xyz    M x 3 doubles, row-major unit vectors, device memory
 *   M            1 <= M <= 1,048,576 (larger M returns HAMLS_ERR_CAPACITY)
 *   bands,cells  key shape: bands even in [2, 4096], cells a multiple of 4 in [4, 8192]
 *   keys_sorted  M uint32 (device): sorted cell keys
 *   perm         M uint32 (device): sorted position -> original node index (stable)
 *   cell_start   bands*cells + 1 uint32 (device): first sorted position of each cell
 * It calls no allocator: the sort's scratch is a static device array of about
 * 8.3 MiB that every GPU loading the library keeps until the process exits.
 * The first call on a device looks up that array's device address (once per
 * device); make that first call before any stream capture. All calls share
 * the one array, so calls that overlap on the GPU (other streams, other host
 * threads) race: serialise them. `stream` must belong to the current device
 * (else HAMLS_ERR_INVALID_ARG). A CUDA error left pending by earlier work of
 * the caller is reported as HAMLS_ERR_CUDA before anything is launched and is
 * left pending. Nodes that are not unit vectors are filed in the north-pole
 * cell; no status is reported for them.
 */
hamls_status hamls_cells_noalloc(const double* nodes_xyz, int64_t M, int bands, int cells, uint32_t* keys_sorted,
                                 uint32_t* perm, uint32_t* cell_start, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HAMLS_H */
