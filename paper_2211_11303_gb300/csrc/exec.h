// Launch interface of the persistent task executor (exec.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "hlu_internal.h"

namespace hlu {

struct ExecArgs {
  const Task* tasks;
  int64_t ntasks;
  const Term* terms;
  const Piece* pieces;
  const int64_t* pred_ptr;  // ntasks + 1
  const int32_t* pred_idx;
  int32_t* done;            // completion epoch per task
  int32_t epoch;            // value published on completion in this launch
  unsigned long long* ticket;  // next task index (zeroed before the launch)
  void* const* arenas;      // per problem (Task::prob)
  int32_t* const* ranks;
  int32_t* const* pivs;
  void* scratch;            // per-CTA scratch, scratch_stride elements each
  int64_t scratch_stride;
  int64_t trunc_rows;       // rows of the truncation stacks in the scratch
  double eps;
  int32_t* status;          // [0] status code, [1] failing task, [2] rank-cap hits, [3] abort
  double* flops;            // accumulated algorithmic flops (may be null)
  unsigned long long wait_limit_ns;
  unsigned long long* prof;  // optional [(TK_NUM + 1) x 3]: tasks, wait cycles, run cycles per kind
};

size_t exec_smem_bytes(int elem_size);
template <class T>
int exec_blocks_per_sm();
template <class T>
cudaError_t exec_launch(const ExecArgs& a, int grid, cudaStream_t s);

constexpr int kExecThreads = 256;
constexpr int kTruncStack = 96;  // columns of a truncation stack (>= rank cap + widest piece)
// per-CTA scratch: two stacks (kTruncStack wide) and two outputs (32 wide)
inline int64_t trunc_scratch_elems(int64_t rows) { return rows * (2 * kTruncStack + 2 * 32); }

}  // namespace hlu
