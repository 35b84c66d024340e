/*
 * hamls_debug.h - inspection entry points of the HAMLS library.
 *
 * These calls expose intermediate results of a plan so that each stage of
 * Algorithm 1 can be checked on its own. They follow the conventions of
 * hamls.h: pointers may be host or device (output pointers to host memory are
 * filled by stream-ordered copies, valid after hamls_sync), the caller owns
 * all buffers, errors are returned as hamls_status.
 */
#ifndef HAMLS_DEBUG_H
#define HAMLS_DEBUG_H

#include "hamls.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Neighbour structure over the plan's nodes (no counterpart in the paper; it
 * serves the nearest-neighbour queries that Sec. 3.2 names as the only place
 * M enters the cost). keys_sorted[M], perm[M] (sorted position -> original
 * node index, stable), cell_start[bands*cells + 1] (CSR over cells). */
hamls_status hamls_debug_cells(hamls_plan_t plan, uint32_t* keys_sorted, uint32_t* perm,
                               uint32_t* cell_start, cudaStream_t stream);

/* d_n of eq. adaptive_support_radius as a squared chord: for each of nq query
 * unit vectors (nq x 3 doubles), the n-th smallest |x_i - q|^2 over the plan's
 * nodes, computed exactly in FP64 as ((dx*dx + dy*dy) + dz*dz). */
hamls_status hamls_debug_knn(hamls_plan_t plan, const double* queries, int64_t nq, int n,
                             double* c2_out, cudaStream_t stream);

/* The local node sets X(q) of eq. mls_local_node_set for given squared chord
 * radii: for query j, count_j = #{i : |x_i - q_j|^2 < rho2_j}, idsum_j = sum
 * of the original indices i, idhash_j = xor of splitmix64(i) over the set. */
hamls_status hamls_debug_ball(hamls_plan_t plan, const double* queries, const double* rho2,
                              int64_t nq, int64_t* count, int64_t* idsum, uint64_t* idhash,
                              cudaStream_t stream);

/* Per grid node (ring-major, index k (2N+2) + j) results of the last
 * plan/fit: support radius delta, n(q), centre amplification chi, applied
 * regularisation tau~, and the MLS value f. Any pointer may be NULL. */
hamls_status hamls_debug_grid(hamls_plan_t plan, double* delta, int32_t* count, double* chi,
                              double* tau_tilde, double* fgrid, cudaStream_t stream);

/* The Fibonacci auxiliary grid (aux_points x 3 doubles) and d_n there
 * (geodesic). Either pointer may be NULL. */
hamls_status hamls_debug_aux(hamls_plan_t plan, double* aux_xyz, double* dn_aux, cudaStream_t stream);

/* Algorithm 1 step 3 alone: coefficients (layout of hamls_fit) of the given
 * M_Q grid values, in the plan's precision. */
hamls_status hamls_debug_quadrature(hamls_plan_t plan, const double* fgrid, double* coeffs,
                                    cudaStream_t stream);

/* Gauss-Legendre nodes t_k (descending) and weights w_k, N+1 each. */
hamls_status hamls_debug_gl(hamls_plan_t plan, double* t, double* w, cudaStream_t stream);

/* The tensor-core product used by the batched Legendre contraction, alone:
 * C (M x N, row-major) = A (M x K) B (N x K)^T, all FP32 row-major device
 * arrays, K a multiple of 4, computed as 3xTF32 on tcgen05 (FP32
 * accumulation). Synchronises the stream; HAMLS_ERR_TIMEOUT if a tile gave
 * up waiting for its copies or products. */
hamls_status hamls_debug_tc_gemm(const float* A, const float* B, float* C, int M, int N, int K,
                                 cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HAMLS_DEBUG_H */
