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
#ifdef __cplusplus
extern "C" {
#endif

/* hlu_debug_host_factor_solve - FP64 H-LU of A on the host, then x = (LU)_H^-1 b.
 * clusters: int32[nc*12], blocks: int32[nb*8] in the hlu_export_trees layout;
 * perm: int32[N]; CSR of A in the original DOF order (rowptr int64[N+1], col
 * int32[nnz], val double[nnz]); eps: truncation tolerance (Sec. 4 truncated
 * SVD, keep s_i > eps s_1); rank_cap: capacity of admissible blocks (0 = 32);
 * tile: block-tree nodes whose clusters both hold <= tile DOFs are factored as
 * one dense tile (0 keeps the block tree's own leaves);
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
                                int32_t rank_cap, int32_t tile, uint64_t order_seed, int32_t nrhs,
                                const double* b, double* x, int64_t* info);

/* hlu_debug_wait_timeout - fault injection for the bounded device waits (needs a
 * GPU).  Runs the task executor with one CTA on a two-task schedule in which
 * task 0 waits for task 1, a completion flag that nothing can set.  The wait
 * must give up after limit_ms (0 < limit_ms <= 5000), record HLU_ERR_TIMEOUT,
 * and the kernel must return with the context still usable.
 * status_out: int32[2] receives (device status code, task that gave up).
 * Returns HLU_ERR_TIMEOUT when the wait ran out as intended. */
int hlu_debug_wait_timeout(double limit_ms, int32_t* status_out);

#ifdef __cplusplus
}
#endif
#endif
