// Launch interface of the persistent task executor (exec.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "hlu_internal.h"

namespace hlu {

// One problem's schedule and data as seen by the executor.  Tasks become
// ready when their last predecessor finishes (dependency counters), and ready
// tasks are handed out through a FIFO queue shared by all problems of a launch.
struct ProbSched {
  const Task* tasks;
  const Term* terms;
  const Piece* pieces;
  const int64_t* succ_ptr;  // ntasks + 1
  const int32_t* succ_idx;
  int32_t* indeg;           // unfinished predecessors (reset before every launch)
  void* arena;
  int32_t* ranks;
  int32_t* piv;
  double eps;
  int64_t ntasks;
  int64_t limit;            // tasks with index >= limit are not run
  int32_t nrhs_slot;        // rank slot of the right-hand-side count, and its
  int32_t nrhs;             // value for this launch (read without a load)
  const int32_t* term_p;    // solve launches: each term's column count, resolved
                            // after the factorisation (-1: read it live); else null
  double alpha;             // scalar of TF_ALPHA tasks and PF_ALPHA pieces (Schulz start)
};
constexpr int kMaxBatch = 64;  // problems in one launch
// profile layout: per task kind (TK_NUM + 1 rows) tasks, wait cycles, run
// cycles; then truncation phases: stacking, QR, core, Jacobi, selection and
// Q application cycles, compressions, Jacobi sweeps, summed stack widths
constexpr int kProfTrunc = (TK_NUM + 1) * 3;
constexpr int kProfEntries = kProfTrunc + 8;

struct ExecArgs {
  ProbSched probs[kMaxBatch];
  int32_t nprobs;
  int64_t ntotal;               // tasks run in this launch (= queue slots)
  // ready queue: slot k holds (problem << 40 | task) + 1 once pushed, 0 before;
  // qctl[0] = next slot to claim, qctl[1] = next slot to fill
  unsigned long long* queue;
  unsigned long long* qctl;
  void* scratch;                // per-CTA scratch, scratch_stride elements each
  int64_t scratch_stride;
  int64_t trunc_rows;           // rows of the truncation stacks in the scratch
  int32_t* status;              // [0] status code, [1] failing slot, [2] rank-cap hits, [3] abort,
                                // [4] largest rank a truncation asked for (kRankMax + 1: more),
                                // [5] dense-route truncations handed to the stack route
  double* flops;                // accumulated algorithmic flops (may be null)
  unsigned long long wait_limit_ns;
  double jacobi_tol;            // truncation: Jacobi orthogonality tolerance
  int32_t compress_at;          // truncation: stack width that triggers a compression
  unsigned long long* prof;     // optional [kProfEntries] (layout above)
  int32_t tf32;                 // FP32 launches: tile products in TF32 on the tensor cores (tcgen05)
  unsigned long long* trace;    // optional [ntotal x 4] per slot: (problem << 40 | task), claim, start, end (ns)
};

size_t exec_smem_bytes(int elem_size);
template <class T>
int exec_blocks_per_sm();
template <class T>
cudaError_t exec_launch(const ExecArgs& a, int grid, cudaStream_t s);

// The FP32 executor whose tile products run in TF32 on the tensor cores
// (exec_tc.cu; launches with ExecArgs::tf32 set).
namespace tcx {
template <class T>
int exec_blocks_per_sm();
template <class T>
cudaError_t exec_launch(const ExecArgs& a, int grid, cudaStream_t s);
// D (64 x 64) = A (64 x K) B (K x 64), column-major FP32 device arrays, through
// the executor's TF32 tensor-core tile pipeline (one CTA); status[0] receives
// HLU_ERR_TIMEOUT (5) if an MMA completion wait ran out.
cudaError_t tc_tile_product(const float* A, const float* B, float* D, int K, int32_t* status,
                            unsigned long long wait_ns, cudaStream_t s);
}  // namespace tcx

constexpr int kExecThreads = 256;
constexpr int kTruncStack = 96;  // columns of a truncation stack; wider pieces are stacked in parts
// per-CTA scratch: two stacks (kTruncStack wide) and two outputs (kRankMax wide)
#ifdef __CUDACC__
#define HLU_HD __host__ __device__
#else
#define HLU_HD
#endif
HLU_HD inline int64_t trunc_scratch_elems(int64_t rows) { return rows * (2 * kTruncStack + 2 * kRankMax); }
inline int64_t trunc_scratch_bytes(int64_t rows, int elem_size) {
  int64_t b = trunc_scratch_elems(rows) * elem_size;
  return (b + 255) & ~int64_t(255);
}

}  // namespace hlu
