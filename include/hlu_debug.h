/*
 * hlu_debug.h - host-only validation entry point of the GB300 H-LU library.
 *
 * Runs the library's task scheduler (the recursive H-LU of Algorithm 1
 * step II and the preconditioner application of step III, turned into task
 * DAGs) on the CPU with a sequential reference executor.  Needs no GPU; used
 * to check the DAG (any topological order gives bit-identical results) and the
 * quality of the factor on a CPU-only machine.
 */
#ifndef HLU_DEBUG_H
#define HLU_DEBUG_H
#include <stdint.h>

#include "hlu.h"
#ifdef __cplusplus
extern "C" {
#endif

/* hlu_debug_host_factor_solve - FP64 H-LU of A on the host, then x = (LU)_H^-1 b.
 * clusters: int32[nc*12], blocks: int32[nb*8] in the hlu_export_trees layout;
 * perm: int32[N]; CSR of A in the original DOF order (rowptr int64[N+1], col
 * int32[nnz], val double[nnz]); eps: truncation tolerance (Sec. 4 truncated
 * SVD, keep s_i > eps s_1); rank_cap: capacity of admissible blocks (0 = 64);
 * tile: block-tree nodes whose clusters both hold <= tile DOFs are factored as
 * one dense tile (0 keeps the block tree's own leaves); precision: HLU_FP64 (0) or
 * HLU_FP32 (1) arithmetic in the factor and the triangular solves;
 * order_seed: 0 executes tasks in program order, otherwise in a random
 * topological order drawn from that seed; b, x: host double[N*nrhs]
 * column-major (original order).
 * info (int64[10], may be NULL): factor tasks, solve tasks, max rank,
 * rank-capacity hits, status, arena elements, host scheduling microseconds,
 * 1000 x mean rank, DAG edges, widest truncation.
 * Returns 0, 1 (bad argument), 3 (zero pivot), 6 (internal error) or 7
 * (an A_H block exceeds the rank capacity). */
int hlu_debug_host_factor_solve(int32_t nc, const int32_t* clusters, int32_t nb,
                                const int32_t* blocks, const int32_t* perm, const int64_t* rowptr,
                                const int32_t* col, const double* val, double eps,
                                int32_t rank_cap, int32_t tile, int32_t precision, uint64_t order_seed,
                                int32_t nrhs,
                                const double* b, double* x, int64_t* info);

/* hlu_debug_host_factor_prefix - as hlu_debug_host_factor_solve, but executes
 * only the first `limit` tasks of the factorisation DAG (limit < 0: all) and,
 * when arena_out is not NULL, copies the whole arena (float or double elements
 * by precision) and the rank slots to arena_out / ranks_out instead of
 * solving.  Used with hlu_debug_factor_prefix to locate the first task whose
 * device result differs from the host's. */
int hlu_debug_host_factor_prefix(int32_t nc, const int32_t* clusters, int32_t nb, const int32_t* blocks,
                                 const int32_t* perm, const int64_t* rowptr, const int32_t* col,
                                 const double* val, double eps, int32_t rank_cap, int32_t tile,
                                 int32_t precision, uint64_t order_seed, int32_t nrhs, const double* b,
                                 double* x, int64_t* info, int64_t limit, void* arena_out,
                                 int32_t* ranks_out);

/* hlu_debug_factor_prefix - device counterpart (needs a GPU): A_H fill plus the
 * first `limit` tasks of the factorisation of a built handle at `precision`,
 * then the arena and rank slots are copied to host buffers.
 * sizes: int64[3] receives (arena elements, rank slots, factor tasks); pass
 * NULL buffers to query sizes only. */
int hlu_debug_factor_prefix(hlu_handle* h, int32_t precision, int64_t limit, void* arena_out,
                            int32_t* ranks_out, int64_t* sizes);

/* hlu_debug_task_record - copy factorisation task `idx` of a built handle (its
 * internal record, 136 bytes: kind, flags, operand views) to `out`. */
int hlu_debug_task_record(const hlu_handle* h, int64_t idx, void* out);

/* hlu_debug_factor_trace - factorise a built handle at `precision` with a
 * per-task trace (needs a GPU).  trace_out: uint64[4 x tasks], one row per
 * ready-queue slot in claim order: (problem << 40 | task index), the time
 * the slot was claimed, the time the task started and the time it ended
 * (globaltimer ns); pred_ptr_out: int64[tasks+1]
 * and pred_idx_out: int32[edges], the dependency DAG; tasks_out: the task
 * records (136 bytes each).  sizes: int64[2] receives (tasks, edges); pass
 * NULL trace_out to query sizes only.  Any other output may be NULL. */
int hlu_debug_factor_trace(hlu_handle* h, int32_t precision, uint64_t* trace_out, int64_t* pred_ptr_out,
                           int32_t* pred_idx_out, void* tasks_out, int64_t* sizes);

/* hlu_debug_solve_trace - one triangular solve (nrhs columns of the work
 * vector, 1..16, contents as they are) of a factored handle with a per-task
 * trace (needs a GPU); outputs and sizes as hlu_debug_factor_trace, for the
 * solve DAG. */
int hlu_debug_solve_trace(hlu_handle* h, int32_t nrhs, uint64_t* trace_out, int64_t* pred_ptr_out,
                          int32_t* pred_idx_out, void* tasks_out, int64_t* sizes);

/* hlu_debug_tf32_tile - the TF32 tensor-core tile product of HLU_TF32
 * factorisations on its own (needs a GPU): D = A B for A 64 x K (ld 64), B
 * K x 64 (ld K) and D 64 x 64 (ld 64), column-major FP32 device arrays,
 * computed by one CTA through the executor's tcgen05 pipeline (each operand
 * split into TF32 high and low parts, A_hi B_hi + A_hi B_lo + A_lo B_hi
 * accumulated in FP32 in tensor memory).  K in [1, 4096].
 * status_out (may be NULL) receives the device status (0, or 5 if an MMA
 * completion wait ran out, which the call returns as HLU_ERR_TIMEOUT).
 * Synchronous. */
int hlu_debug_tf32_tile(const float* A, const float* B, float* D, int32_t K, int32_t* status_out);

/* hlu_debug_truncate - one recompression task (Sec. 3: QR of both factors,
 * SVD of the small core, keep s_i > eps s_1, at most cap) run by the device
 * executor on its own (needs a GPU).  The sum X Y^T (X m x w, Y n x w, host
 * column-major FP64) enters as pieces of piece_cols columns (0: one piece),
 * in `precision` (HLU_FP64 or HLU_FP32) arithmetic.  flags: 1 = the first
 * piece is the target itself (its factors start in the outputs, as in an
 * update A += sum), 2 = each piece's Y is stored row-major (a transposed
 * view), 4 = piece q restricted to the quadrant ((q mod 4) / 2, q mod 2) of
 * the m x n target (rows split at m / 2, columns at n / 2; X and Y must be
 * zero outside).  Xo (m x cap), Yo (n x cap): host outputs, the first
 * *rank columns hold the kept factors (Yo's columns orthonormal).
 * status_out (int32[8], may be NULL): the executor status words ([2]
 * capacity hits, [4] largest rank asked for).  cap in [1, min(m, n, 64)]. */
int hlu_debug_truncate(int32_t precision, int32_t m, int32_t n, int32_t w, int32_t piece_cols, int32_t flags,
                       const double* X, const double* Y, double eps, int32_t cap, double* Xo, double* Yo,
                       int32_t* rank, int32_t* status_out);

/* hlu_debug_zero_dof - input for the zero-pivot path (needs a GPU): sets row
 * and column `dof` (original DOF order) of the handle's assembled matrix A to
 * zero, in place on the device.  A later hlu_factor then meets an exact zero
 * pivot in the dense diagonal block holding that DOF and returns
 * HLU_ERR_ZERO_PIVOT.  The matrix stays modified until the handle is
 * destroyed.  HLU_ERR_ARG for dof outside [0, N).  Synchronous. */
int hlu_debug_zero_dof(hlu_handle* h, int64_t dof);

/* hlu_debug_check_hazards - static race check of one task DAG (no GPU).
 * Builds the schedules from the exported trees (clusters int32[nc*12],
 * blocks int32[nb*8]; rank_cap 0 = 64, tile and nrhs_max (1..16) as the
 * library uses them) and picks one DAG by `which`: 0 the H-LU factorisation
 * (Algorithm 1 step II), 1 the triangular solve (step III), 2 / 3 / 4 the
 * Schulz inverse's start, step and apply.  Every operand is expanded to the
 * elements it may address at full capacity (factor arena, pivot vectors and
 * rank slots are separate spaces), and the DAG is replayed in program order:
 * each write after write, read after write or write after read on one
 * element must be ordered by the DAG's edges, taken transitively.
 * drop_edge: -1, or the index of one edge (in the DAG's predecessor list) to
 * remove before the check, a planted mistake that tests the check itself.
 * report (int64[11], required): tasks, element accesses, distinct conflicting
 * task pairs checked, pairs the edges leave unordered, then for the first
 * finding the earlier task (-1 for an out-of-range access), the later task,
 * the space (0 arena, 1 pivots, 2 rank slots) and the element, then accesses
 * outside their space, the DAG's edge count, and whether the dropped edge's
 * two tasks are still ordered through other edges (1 / 0; -1 without a
 * drop).
 * Returns 0 when every conflict is ordered and every access is in range, 9
 * when not (see report), 1 for a bad argument, 6 for an internal error or a
 * DAG too large to check in host memory (more than 40,000 tasks or 2^27
 * arena elements). */
int hlu_debug_check_hazards(int32_t nc, const int32_t* clusters, int32_t nb, const int32_t* blocks,
                            int32_t rank_cap, int32_t tile, int32_t nrhs_max, int32_t which, int64_t drop_edge,
                            int64_t* report);

/* hlu_debug_host_hinverse - the Schulz inverse's task DAGs (hlu_hinverse)
 * run by the host reference executor in FP64 (no GPU): A_H from the CSR
 * matrix (original order) and the exported trees, X_0 = alpha A_H, `iters`
 * Schulz steps, then x = X b for nrhs (1..16) columns of b (N x nrhs,
 * column-major, original order).  info: int64[5] (tasks of a step, tasks of
 * an apply, largest rank of X, capacity hits, status); may be NULL. */
int hlu_debug_host_hinverse(int32_t nc, const int32_t* clusters, int32_t nb, const int32_t* blocks,
                            const int32_t* perm, const int64_t* rowptr, const int32_t* col, const double* val,
                            double eps, int32_t rank_cap, int32_t tile, double alpha, int32_t iters, int32_t nrhs,
                            const double* b, double* x, int64_t* info);

/* hlu_debug_wait_timeout - fault injection for the bounded device waits (needs a
 * GPU).  Runs the task executor with one CTA on a two-task schedule in which
 * task 1 waits for itself: task 0 runs, and the CTA that claims queue slot 1
 * waits for a task that can never become ready.  The wait must give up after
 * limit_ms (0 < limit_ms <= 5000), record HLU_ERR_TIMEOUT, and the kernel must
 * return with the context still usable.
 * status_out: int32[2] receives (device status code, queue slot that gave up).
 * Returns HLU_ERR_TIMEOUT when the wait ran out as intended. */
int hlu_debug_wait_timeout(double limit_ms, int32_t* status_out);

#ifdef __cplusplus
}
#endif
#endif
