// Persistent task executor for the H-LU and H-solve DAGs (sm_103a).
//
// One launch runs a whole schedule.  Every task carries a counter of its
// unfinished predecessors; the CTA that finishes a task decrements the
// counters of its successors, and the one that brings a counter to zero
// appends that task to a FIFO ready queue.  Each CTA repeatedly claims the
// next queue slot, waits until the slot is filled, and runs the task with all
// its threads.  The queue holds every task of the launch exactly once, and a
// claimed slot is always filled while some task is still running, so the
// waits cannot deadlock on an acyclic schedule.  Every wait is bounded by a
// wall-clock limit (%globaltimer); when it runs out the CTA records
// HLU_ERR_TIMEOUT and all CTAs drain without executing further work.
//
// Data written by one CTA and read by another goes through L2 (ld.global.cg /
// st.global.cg); a task's writes are fenced before its successors' counters
// are decremented, and queue slots are published with st.release and read
// with ld.acquire at gpu scope.
//
// This file is compiled twice.  exec.cu itself (HLU_EXEC_TC == 0) builds the
// FP32 and FP64 executors with no tensor-core code; exec_tc.cu includes it
// with HLU_EXEC_TC == 1 and builds, in namespace hlu::tcx, the FP32 executor
// whose tile products run as TF32 MMAs on the tensor cores.  A kernel that
// allocates tensor memory is held to one CTA per SM, so the FP32 executor
// must not contain that code.
#include <cuda_runtime.h>

#include <cstdint>

#include <type_traits>

#include "launch_count.h"

#include "exec.h"
#include "hlu_internal.h"
#include "tc.cuh"

#ifndef HLU_EXEC_TC
#define HLU_EXEC_TC 0
#endif

namespace hlu {
#if HLU_EXEC_TC
namespace tcx {
#endif

#define NT 256

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tensor-core state of one CTA (TF32 tile products, factorisation launches
// with HLU_TF32): the accumulator's tensor-memory columns, the completion
// mbarrier and its phase (every thread keeps its own copy; all threads pass
// the same waits).
struct TcCtl {
  bool on = false;
  char* stage = nullptr;  // 1024-aligned staging buffer, tc::kTcStageBytes
  bool broken = false;   // a completion wait ran out: no further MMAs are issued
  uint32_t tmem = 0;
  uint64_t* bar = nullptr;
  uint32_t phase = 0;
  int32_t* status = nullptr;
  unsigned long long wait_ns = 0;
};

template <class T>
struct Ctx {
  T* arena;
  int32_t* ranks;
  int32_t* piv;
  const Term* terms;
  const Piece* pieces;
  T* scratch;
  int64_t rows_max;  // rows of the per-CTA truncation stacks
  double eps;
  int32_t* status;
  double flops;
  unsigned long long* tprof;  // truncation phase profile (shared memory) or null
  double jacobi_tol;
  int32_t compress_at;
  int32_t nrhs_slot, nrhs;  // the launch's right-hand-side count and its slot
  const int32_t* term_p;    // resolved term column counts (solve launches) or null
  TcCtl* tcc;               // tensor-core tile products (FP32 factorisations with TF32) or null
  double alpha;             // the launch's scalar for TF_ALPHA / PF_ALPHA
};

template <class T>
__device__ __forceinline__ T ldv(const Ctx<T>& c, const View& v, int64_t i, int64_t j) {
  return __ldcg(c.arena + v.off + i * v.rs + j * v.cs);
}
template <class T>
__device__ __forceinline__ void stv(const Ctx<T>& c, const View& v, int64_t i, int64_t j, T x) {
  __stcg(c.arena + v.off + i * v.rs + j * v.cs, x);
}
template <class T>
__device__ __forceinline__ int32_t ncols(const Ctx<T>& c, const View& v) {
  if (v.slot < 0) return v.cols;
  return v.slot == c.nrhs_slot ? c.nrhs : __ldcg(c.ranks + v.slot);
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block-wide sum; red: >= NT/32 elements of shared memory.
template <class T>
__device__ T block_sum(T x, T* red) {
  x = warp_sum(x);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  T s = 0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < NT / 32 ? red[threadIdx.x] : T(0);
    s = warp_sum(s);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------- GETRF
// Dense diagonal leaf, partial pivoting (first index of max |a|), in place;
// pivot vector p with A[p] = L U.
template <class T>
__device__ void task_getrf(Ctx<T>& c, const Task& t, char* smem) {
  const int n = t.a.rows;
  T* A = reinterpret_cast<T*>(smem);
  int* perm = reinterpret_cast<int*>(A + n * n);
  __shared__ int s_p;
  for (int idx = threadIdx.x; idx < n * n; idx += NT) A[idx] = ldv(c, t.a, idx % n, idx / n);
  for (int i = threadIdx.x; i < n; i += NT) perm[i] = i;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      T best = T(-1);
      int bi = n;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        T v = fabs(A[i + k * n]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        s_p = bi;
        if (!(best > T(0))) atomicCAS(c.status, 0, 3);
        if (bi != k && bi < n) {
          int tmp = perm[k];
          perm[k] = perm[bi];
          perm[bi] = tmp;
        }
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k && p < n)
      for (int j = threadIdx.x; j < n; j += NT) {
        T tmp = A[k + j * n];
        A[k + j * n] = A[p + j * n];
        A[p + j * n] = tmp;
      }
    __syncthreads();
    const T piv = A[k + k * n];
    if (piv != T(0)) {
      const T inv = T(1) / piv;
      for (int i = k + 1 + threadIdx.x; i < n; i += NT) A[i + k * n] *= inv;
    }
    __syncthreads();
    const int m = n - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += NT) {
      int i = k + 1 + idx % m, j = k + 1 + idx / m;
      A[i + j * n] -= A[i + k * n] * A[k + j * n];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += NT) stv(c, t.a, idx % n, idx / n, A[idx]);
  for (int i = threadIdx.x; i < n; i += NT) __stcg(c.piv + t.piv_off + i, perm[i]);
  if (threadIdx.x == 0) c.flops += 2.0 * n * n * n / 3.0;
}

// ---------------------------------------------------------------- small GEMM core
// Strided operand: element (i, j) at p[i * rs + j * cs].
template <class T>
struct Mat {
  const T* p;
  int64_t rs, cs;
};
template <class T>
__device__ __forceinline__ Mat<T> mat(const Ctx<T>& c, const View& v) {
  return Mat<T>{c.arena + v.off, v.rs, v.cs};
}
template <class T>
__device__ __forceinline__ Mat<T> matT(const Ctx<T>& c, const View& v) {
  return Mat<T>{c.arena + v.off, v.cs, v.rs};
}
template <class T>
__device__ __forceinline__ Mat<T> shift(Mat<T> m, int64_t di, int64_t dj) {
  m.p += di * m.rs + dj * m.cs;
  return m;
}

// 64 x 64 output tile in registers: thread t owns rows 4 (t % 16) .. +3 and
// columns 4 (t / 16) .. +3.  tile_mma adds A (tile rows [rlo, rlo + mrows),
// K columns) times B (K rows, ncols columns); operand chunks of KC along K
// are staged in shared memory with loads ordered along the operand's
// contiguous dimension.
constexpr int KC = 32;
// Staged chunk layout: element (x, kk) of an operand (x = tile row of A or
// tile column of B) sits at kk * kLds + x.  The pitch 72 keeps every group of
// four x 16-byte aligned for the vector reads of chunk_mma.  Operands stored
// contiguously along x are staged 64 consecutive x per K index; operands
// stored contiguously along K are staged, per warp, 4 consecutive K indices
// of 8 columns (16-byte global segments), which under pitch 72 puts the 32
// shared-memory stores of a warp into 32 distinct banks (staging 32
// consecutive K indices of one column under pitch 64 was a 32-way conflict).
constexpr int kLds = 72;
constexpr int kStage = KC * kLds;  // elements of one staged operand chunk
static_assert(KC == 32 && NT == 256, "chunk_coord assumes 64 x 32 chunks staged by 256 threads");
__device__ __forceinline__ void chunk_coord(bool x_contig, int e, int& x, int& kk) {
  if (x_contig) {
    x = e & 63;
    kk = e >> 6;
  } else {
    kk = ((e >> 5) & 7) * 4 + (e & 3);
    x = (e >> 8) * 8 + ((e >> 2) & 7);
  }
}
template <class T>
__device__ __forceinline__ void acc_zero(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}
// One K-chunk of a tile product: rows [rlo, rlo + mrows) of the tile get
// A (mrows x kc) times B (kc x ncols).
template <class T>
struct Chunk {
  Mat<T> A, B;
  int rlo, mrows, ncols, kc;
  int clo = 0;   // B's columns land on tile columns [clo, clo + ncols)
  T sg = T(1);   // sign applied to B
};
constexpr int kChunkRegs = 64 * KC / NT;

// Loads a chunk's operands into registers, ordered along each operand's
// contiguous dimension (the same element order chunk_stage stores).
template <class T>
__device__ __forceinline__ void chunk_fetch(const Chunk<T>& ch, T (&ra)[kChunkRegs], T (&rb)[kChunkRegs]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < kChunkRegs; ++q) {
    const int e = tid + q * NT;
    int r, kk;
    chunk_coord(ch.A.rs == 1, e, r, kk);
    const int ar = r - ch.rlo;
    ra[q] = (kk < ch.kc && ar >= 0 && ar < ch.mrows) ? __ldcg(ch.A.p + (int64_t)ar * ch.A.rs + (int64_t)kk * ch.A.cs)
                                                      : T(0);
  }
#pragma unroll
  for (int q = 0; q < kChunkRegs; ++q) {
    const int e = tid + q * NT;
    int cc, kk;
    chunk_coord(ch.B.rs != 1, e, cc, kk);
    const int bc = cc - ch.clo;
    rb[q] = (kk < ch.kc && bc >= 0 && bc < ch.ncols)
                ? ch.sg * __ldcg(ch.B.p + (int64_t)kk * ch.B.rs + (int64_t)bc * ch.B.cs)
                : T(0);
  }
}
template <class T>
__device__ __forceinline__ void chunk_stage(const Chunk<T>& ch, const T (&ra)[kChunkRegs],
                                            const T (&rb)[kChunkRegs], T* As, T* Bs) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < kChunkRegs; ++q) {
    const int e = tid + q * NT;
    int r, kk;
    chunk_coord(ch.A.rs == 1, e, r, kk);
    As[kk * kLds + r] = ra[q];
  }
#pragma unroll
  for (int q = 0; q < kChunkRegs; ++q) {
    const int e = tid + q * NT;
    int cc, kk;
    chunk_coord(ch.B.rs != 1, e, cc, kk);
    Bs[kk * kLds + cc] = rb[q];
  }
}
// four consecutive staged elements, 16-byte aligned (pitch and offsets are
// multiples of four elements, the staging buffers start 16-byte aligned)
__device__ __forceinline__ void lds4(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&v)[4]) {
  const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
  v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
}
template <class T>
__device__ __forceinline__ void chunk_mma(T (&acc)[4][4], const T* As, const T* Bs, int kc) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int kk = 0; kk < kc; ++kk) {
    T a[4], b[4];
    lds4(As + kk * kLds + tx * 4, a);
    lds4(Bs + kk * kLds + ty * 4, b);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
  }
}

// ---------------------------------------------------------------- TF32 tile products
// Waits (thread 0, bounded by the launch's wait limit) until the MMAs
// committed last have completed; false, with HLU_ERR_TIMEOUT recorded and the
// launch aborted, when the wait ran out.  Every thread returns the same value.
__device__ bool tc_wait(TcCtl* t) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 0;
    if (!t->broken) {
      const uint64_t t0 = gtimer();
      for (;;) {
        if (tc::mbar_try_wait(t->bar, t->phase)) {
          ok = 1;
          break;
        }
        if (gtimer() - t0 > t->wait_ns) {
          atomicCAS(t->status, 0, 5);
          atomicExch(t->status + 3, 1);
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  if (ok)
    t->phase ^= 1u;
  else
    t->broken = true;
  return ok;
}

// The chunk pipeline of tile_mma_seq on the fifth-generation tensor cores,
// with FP32 accuracy from TF32 MMAs by splitting each operand into a TF32
// part and the TF32 rounding of its remainder (x = x_hi + x_lo): the staged
// M = 128 A operand is [A_hi; A_lo] (64 rows each), the N = 128 B operand
// [B_hi, B_lo], so one M = 128, N = 128, K = 8 MMA per K step accumulates
// all four products in tensor memory; the result is
// A_hi B_hi + A_hi B_lo + A_lo B_hi (A_lo B_lo, below FP32 rounding, is
// left out).  Each 64 x 32 (A) and 32 x 64 (B) chunk is staged K-major in
// the core-matrix layout (A at t->stage, B 16 KB after it); one thread issues
// four MMAs.  The MMAs run while the next chunk's operands load into
// registers; the staging buffer is rewritten only after the MMAs reading it
// completed.  At the end the three 64 x 64 quadrants go through shared
// memory into every thread's 4 x 4 register tile (acc +=).
template <class Cursor>
__device__ void tile_mma_seq_tc(float (&acc)[4][4], Cursor& cur, TcCtl* t) {
  if (!cur.first()) return;
  const int tid = threadIdx.x;
  float ra[kChunkRegs], rb[kChunkRegs];
  Chunk<float> ch = cur.chunk();
  chunk_fetch(ch, ra, rb);
  char* Sb = t->stage;
  float* S = reinterpret_cast<float*>(Sb);
  bool first = true;
  __syncthreads();  // the staging buffer's previous readers are done
  for (;;) {
    if (!first && !tc_wait(t)) return;  // the buffer is still read by the MMAs
#pragma unroll
    for (int q = 0; q < kChunkRegs; ++q) {
      const int e = tid + q * NT;
      int r, kk;
      chunk_coord(ch.A.rs == 1, e, r, kk);
      const float hi = tc::to_tf32(ra[q]);
      *reinterpret_cast<float*>(Sb + tc::tc_offset(r, kk)) = hi;
      *reinterpret_cast<float*>(Sb + tc::tc_offset(64 + r, kk)) = tc::to_tf32(ra[q] - hi);
    }
#pragma unroll
    for (int q = 0; q < kChunkRegs; ++q) {
      const int e = tid + q * NT;
      int cc, kk;
      chunk_coord(ch.B.rs != 1, e, cc, kk);
      const float hi = tc::to_tf32(rb[q]);
      *reinterpret_cast<float*>(Sb + tc::kTcOperandBytes + tc::tc_offset(cc, kk)) = hi;
      *reinterpret_cast<float*>(Sb + tc::kTcOperandBytes + tc::tc_offset(64 + cc, kk)) = tc::to_tf32(rb[q] - hi);
    }
    tc::fence_async_shared();
    __syncthreads();
    if (tid == 0 && !t->broken) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(Sb), b0 = a0 + tc::kTcOperandBytes;
#pragma unroll
      for (int ks = 0; ks < tc::kTcChunkK / 8; ++ks)
        tc::mma_tf32(t->tmem, tc::smem_desc(a0 + ks * 2 * tc::kTcLBO), tc::smem_desc(b0 + ks * 2 * tc::kTcLBO),
                     !first || ks > 0);
      tc::mma_commit(t->bar);
    }
    first = false;
    const bool more = cur.next();
    if (more) {
      ch = cur.chunk();
      chunk_fetch(ch, ra, rb);
    }
    if (!more) break;
  }
  if (!tc_wait(t)) return;
  tc::fence_after_sync();
  // warp w reads lane quarter q = w % 4 (accumulator rows 32 q ..), columns
  // 32 (w / 4) ..: quarters 0, 1 hold A_hi rows (hi x hi in columns 0..63,
  // hi x lo in 64..127), quarters 2, 3 the A_lo rows (lo x hi in 0..63)
  const int w = tid >> 5, lane = tid & 31;
  const int q = w & 3, col0 = (w >> 2) * 32;
  float v[32];
  tc::tmem_ld32(t->tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0, v);
  if (q < 2) {
    float u[32];
    tc::tmem_ld32(t->tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(col0 + 64), u);
    const int row = q * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) S[row + (col0 + j) * 64] = v[j] + u[j];
  }
  __syncthreads();
  if (q >= 2) {
    const int row = (q - 2) * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) S[row + (col0 + j) * 64] += v[j];
  }
  tc::fence_before_sync();
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] += S[(tx * 4 + i) + (ty * 4 + j) * 64];
  __syncthreads();
}

// Software pipeline over a sequence of chunks: the operands of chunk j + 1
// are in flight (registers) while chunk j is multiplied from shared memory.
// Cursor: first() -> bool (a chunk exists), chunk() -> Chunk, next() -> bool.
// With tensor-core state switched on (FP32 only) the products run in TF32 on
// the tensor cores (tile_mma_seq_tc).
template <class T, class Cursor>
__device__ void tile_mma_seq(T (&acc)[4][4], Cursor& cur, T* As, T* Bs, TcCtl* tcc = nullptr) {
#if HLU_EXEC_TC
  if constexpr (std::is_same<T, float>::value) {
    if (tcc && tcc->on) {
      tile_mma_seq_tc(acc, cur, tcc);
      return;
    }
  }
#else
  (void)tcc;
#endif
  if (!cur.first()) return;
  T ra[kChunkRegs], rb[kChunkRegs];
  Chunk<T> ch = cur.chunk();
  chunk_fetch(ch, ra, rb);
  for (;;) {
    __syncthreads();
    chunk_stage(ch, ra, rb, As, Bs);
    __syncthreads();
    const int kc = ch.kc;
    const bool more = cur.next();
    if (more) {
      ch = cur.chunk();
      chunk_fetch(ch, ra, rb);
    }
    chunk_mma(acc, As, Bs, kc);
    if (!more) break;
  }
  __syncthreads();
}

// Chunks of one product A (tile rows [rlo, rlo + mrows), K columns) B.
template <class T>
struct ProductCursor {
  Mat<T> A, B;
  int rlo, mrows, ncols, K, l0;
  __device__ bool first() {
    l0 = 0;
    return K > 0 && mrows > 0;
  }
  __device__ bool next() {
    l0 += KC;
    return l0 < K;
  }
  __device__ Chunk<T> chunk() const {
    return Chunk<T>{shift(A, 0, l0), shift(B, l0, 0), rlo, mrows, ncols, min(KC, K - l0), 0, T(1)};
  }
};

// acc += A (tile rows [rlo, rlo + mrows), K columns) times B (K x ncols)
template <class T>
__device__ void tile_mma(T (&acc)[4][4], const Mat<T>& A, int rlo, int mrows, const Mat<T>& B, int ncols, int K,
                         T* As, T* Bs, TcCtl* tcc = nullptr) {
  ProductCursor<T> cur{A, B, rlo, mrows, ncols, K, 0};
  tile_mma_seq(acc, cur, As, Bs, tcc);
}
// C[rows i0.., cols j0..] (+)= sign * acc for the valid part of the tile
template <class T>
__device__ void tile_store(T (&acc)[4][4], const Ctx<T>& c, const View& C, int i0, int j0, int mrows, int ncols,
                           T sign, bool overwrite) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int r = tx * 4 + i, cc = ty * 4 + j;
      if (r < mrows && cc < ncols) {
        T base = overwrite ? T(0) : ldv(c, C, i0 + r, j0 + cc);
        stv(c, C, i0 + r, j0 + cc, base + sign * acc[i][j]);
      }
    }
}

// ---------------------------------------------------------------- leaf TRSM
// Triangle in shared memory; one warp per right-hand-side column, the column
// held in two registers per lane (rows lane and lane + 32), shuffles for the
// substitution.
template <class T>
__device__ void task_trsm(Ctx<T>& c, const Task& t, char* smem) {
  const int n = t.a.rows;
  const int k = ncols(c, t.b);
  T* A = reinterpret_cast<T*>(smem);
  int* perm = reinterpret_cast<int*>(A + n * n);
  T* dinv = reinterpret_cast<T*>(perm + 64);
  for (int b0 = threadIdx.x; b0 < n * n; b0 += 4 * NT) {  // loads first, then the stores
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = b0 + u * NT;
      v[u] = idx < n * n ? ldv(c, t.a, idx % n, idx / n) : T(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (b0 + u * NT < n * n) A[b0 + u * NT] = v[u];
  }
  if (t.type == TK_TRSM_L)
    for (int i = threadIdx.x; i < n; i += NT) perm[i] = __ldcg(c.piv + t.piv_off + i);
  __syncthreads();
  if (t.type != TK_TRSM_L)
    for (int i = threadIdx.x; i < n; i += NT) dinv[i] = T(1) / A[i + i * n];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = lane, r1 = lane + 32;
  for (int j = warp; j < k; j += NT / 32) {
    T v0 = 0, v1 = 0;
    if (t.type == TK_TRSM_L) {
      if (r0 < n) v0 = ldv(c, t.b, perm[r0], j);
      if (r1 < n) v1 = ldv(c, t.b, perm[r1], j);
      for (int l = 0; l < n; ++l) {
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31);
        if (r0 > l && r0 < n) v0 -= A[r0 + l * n] * x;
        if (r1 > l && r1 < n) v1 -= A[r1 + l * n] * x;
      }
    } else if (t.type == TK_TRSM_UT) {
      if (r0 < n) v0 = ldv(c, t.b, r0, j);
      if (r1 < n) v1 = ldv(c, t.b, r1, j);
      for (int l = 0; l < n; ++l) {
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31) * dinv[l];
        if (r0 == l) v0 = x;
        if (r1 == l) v1 = x;
        if (r0 > l && r0 < n) v0 -= A[l + r0 * n] * x;
        if (r1 > l && r1 < n) v1 -= A[l + r1 * n] * x;
      }
    } else {
      if (r0 < n) v0 = ldv(c, t.b, r0, j);
      if (r1 < n) v1 = ldv(c, t.b, r1, j);
      for (int l = n - 1; l >= 0; --l) {
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31) * dinv[l];
        if (r0 == l) v0 = x;
        if (r1 == l) v1 = x;
        if (r0 < l) v0 -= A[r0 + l * n] * x;
        if (r1 < l && r1 < n) v1 -= A[r1 + l * n] * x;
      }
    }
    if (r0 < n) stv(c, t.b, r0, j, v0);
    if (r1 < n) stv(c, t.b, r1, j, v1);
  }
  if (threadIdx.x == 0) c.flops += (double)n * n * k;
}

// ---------------------------------------------------------------- PROJ
// c (r x k) = a^T b, a: m x r, b: m x k: a 64 x 64 tile reduced over m.
template <class T>
__device__ void task_proj(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.a.rows, r = ncols(c, t.a), k = ncols(c, t.b);
  if (r == 0 || k == 0) return;
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + kStage;
  for (int i0 = 0; i0 < r; i0 += 64)
    for (int j0 = 0; j0 < k; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      tile_mma(acc, shift(matT(c, t.a), i0, 0), 0, min(64, r - i0), shift(mat(c, t.b), 0, j0), min(64, k - j0), m,
               As, Bs, c.tcc);
      tile_store(acc, c, t.c, i0, j0, min(64, r - i0), min(64, k - j0), T(1), true);
    }
  if (threadIdx.x == 0) c.flops += 2.0 * m * r * k;
}

// ---------------------------------------------------------------- ROWMV
// c (n x k) = [c] + sign * sum_t A_t B_t, A_t covering rows [roff, roff + rows).
// The terms (and their ranks) are staged in shared memory, kStageTerms at a
// time; all their chunks form one software pipeline per output tile.
constexpr int kStageTerms = 32;
template <class T>
struct TermCursor {
  const Ctx<T>* c;
  const Term* tm;
  const int* p;
  int nq, i0, j0, k, q, l0;
  __device__ bool valid(int qq) const {
    const int lo = max(tm[qq].roff, i0), hi = min(tm[qq].roff + tm[qq].A.rows, i0 + 64);
    return hi > lo && p[qq] > 0;
  }
  __device__ bool seek(int qq) {
    while (qq < nq && !valid(qq)) ++qq;
    q = qq;
    l0 = 0;
    return q < nq;
  }
  __device__ bool first() { return seek(0); }
  __device__ bool next() {
    l0 += KC;
    if (l0 < p[q]) return true;
    return seek(q + 1);
  }
  __device__ Chunk<T> chunk() const {
    const Term& t = tm[q];
    const int lo = max(t.roff, i0), hi = min(t.roff + t.A.rows, i0 + 64);
    return Chunk<T>{shift(mat(*c, t.A), lo - t.roff, l0), shift(mat(*c, t.B), l0, j0), lo - i0, hi - lo,
                    min(64, k - j0), min(KC, p[q] - l0), 0, T(1)};
  }
};

// acc += sum of the task's terms restricted to the 64 x 64 output tile (i0, j0);
// returns the flops (thread 0 only).
template <class T>
__device__ double rowmv_tile(const Ctx<T>& c, const Task& t, int i0, int j0, int k, T (&acc)[4][4], T* As, T* Bs) {
  __shared__ Term s_tm[kStageTerms];
  __shared__ int s_p[kStageTerms];
  double fl = 0;
  for (int qb = 0; qb < t.list_count; qb += kStageTerms) {
    const int nq = min(kStageTerms, t.list_count - qb);
    __syncthreads();
    {
      const int words = nq * (int)(sizeof(Term) / sizeof(int32_t));
      const int32_t* src = reinterpret_cast<const int32_t*>(c.terms + t.list_begin + qb);
      int32_t* dst = reinterpret_cast<int32_t*>(s_tm);
      for (int w = threadIdx.x; w < words; w += NT) dst[w] = __ldg(src + w);
    }
    // resolved column counts arrive with the terms (no dependent rank load)
    const int pq = (c.term_p && threadIdx.x < nq) ? __ldcg(c.term_p + t.list_begin + qb + threadIdx.x) : -1;
    __syncthreads();
    if (threadIdx.x < nq) s_p[threadIdx.x] = pq >= 0 ? pq : ncols(c, s_tm[threadIdx.x].A);
    __syncthreads();
    TermCursor<T> cur{&c, s_tm, s_p, nq, i0, j0, k, 0, 0};
    tile_mma_seq(acc, cur, As, Bs, c.tcc);
    if (threadIdx.x == 0)
      for (int q = 0; q < nq; ++q) {
        const int lo = max(s_tm[q].roff, i0), hi = min(s_tm[q].roff + s_tm[q].A.rows, i0 + 64);
        if (hi > lo) fl += 2.0 * (hi - lo) * min(64, k - j0) * s_p[q];
      }
  }
  return fl;
}

template <class T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc);

template <class T>
__device__ void task_rowmv(Ctx<T>& c, const Task& t, char* smem) {
  const int n = t.c.rows, k = ncols(c, t.b);
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + kStage;
  double fl = 0;
  const bool overwrite = (t.flags & TF_OVERWRITE) != 0;
  const int kx = min(t.c.cols, 64);
  if (n <= 64 && k <= kx && !overwrite) {
    // one output tile: its current values stream into shared memory (all
    // the view's columns, so the copy need not wait for the live count)
    // while the product runs; no other task touches them meanwhile
    T* Cs = Bs + kStage;
    const T* cg = c.arena + t.c.off;
    for (int idx = threadIdx.x; idx < n * kx; idx += NT)
      cp_async_elem(Cs + idx, cg + (int64_t)(idx % n) * t.c.rs + (int64_t)(idx / n) * t.c.cs);
    asm volatile("cp.async.commit_group;" ::: "memory");
    T acc[4][4];
    acc_zero(acc);
    fl = rowmv_tile(c, t, 0, 0, k, acc, As, Bs);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const T sg = T(t.sign);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = tx * 4 + i, cc = ty * 4 + j;
        if (r < n && cc < k) stv(c, t.c, r, cc, Cs[r + cc * n] + sg * acc[i][j]);
      }
    if (threadIdx.x == 0) {
      c.flops += fl;
      if (t.out_slot >= 0) __stcg(c.ranks + t.out_slot, k);
    }
    return;
  }
  for (int i0 = 0; i0 < n; i0 += 64)
    for (int j0 = 0; j0 < k; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      fl += rowmv_tile(c, t, i0, j0, k, acc, As, Bs);
      tile_store(acc, c, t.c, i0, j0, min(64, n - i0), min(64, k - j0), T(t.sign), (t.flags & TF_OVERWRITE) != 0);
    }
  if (threadIdx.x == 0) {
    c.flops += fl;
    if (t.out_slot >= 0) __stcg(c.ranks + t.out_slot, k);
  }
}

// ---------------------------------------------------------------- RSOLVE
// A leaf of a triangular solve with its late update: c -= sum_t A_t B_t, then
// the diagonal tile's triangle (L^-1 P or U^-1) in place.  The tile streams
// into shared memory (cp.async) while the update runs, and the updated
// right-hand side goes to the substitution through shared memory.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}

template <class T>
__device__ void task_rsolve(Ctx<T>& c, const Task& t, char* smem) {
  const int n = t.a.rows, k = ncols(c, t.b);
  const bool upper = (t.flags & TF_UPPER) != 0;
  if (n > 64 || k > 64) {  // not a leaf tile: update, then the plain leaf solve
    Task r = t;
    r.type = TK_ROWMV;
    r.flags = 0;
    r.out_slot = -1;
    task_rowmv(c, r, smem);
    __threadfence_block();
    __syncthreads();
    Task q = t;
    q.type = upper ? TK_TRSM_U : TK_TRSM_L;
    q.b = t.c;
    task_trsm(c, q, smem);
    return;
  }
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + kStage;
  T* A = Bs + kStage;  // the diagonal tile, n x n
  T* X = A + 64 * 64;   // updated right-hand side, n x k (ld n)
  T* dinv = X + 64 * 64;
  int* perm = reinterpret_cast<int*>(dinv + 64);
  // the tile and the right-hand side start moving now: the tile is read-only
  // factor data, and no other task touches this segment of the right-hand
  // side while this one runs.  All the view's columns are copied (the work
  // vector holds that many), so the copy need not wait for the live count.
  const T* tile = c.arena + t.a.off;
  for (int idx = threadIdx.x; idx < n * n; idx += NT)
    cp_async_elem(A + idx, tile + (int64_t)(idx % n) * t.a.rs + (int64_t)(idx / n) * t.a.cs);
  const int kx = min(t.c.cols, 64);
  const T* rhs = c.arena + t.c.off;
  for (int idx = threadIdx.x; idx < n * kx; idx += NT)
    cp_async_elem(X + idx, rhs + (int64_t)(idx % n) * t.c.rs + (int64_t)(idx / n) * t.c.cs);
  asm volatile("cp.async.commit_group;" ::: "memory");
  const int pv = (!upper && threadIdx.x < n) ? __ldcg(c.piv + t.piv_off + threadIdx.x) : 0;
  // the update, kept in registers
  T acc[4][4];
  acc_zero(acc);
  double fl = t.list_count > 0 ? rowmv_tile(c, t, 0, 0, k, acc, As, Bs) : 0.0;
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  if (t.list_count > 0) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const T sg = T(t.sign);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = tx * 4 + i, cc = ty * 4 + j;
        if (r < n && cc < k) X[r + cc * n] += sg * acc[i][j];
      }
  }
  if (!upper && threadIdx.x < n) perm[threadIdx.x] = pv;
  __syncthreads();
  if (upper)
    for (int i = threadIdx.x; i < n; i += NT) dinv[i] = T(1) / A[i + i * n];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = lane, r1 = lane + 32;
  for (int j = warp; j < k; j += NT / 32) {
    const T* xj = X + j * n;
    T v0 = 0, v1 = 0;
    if (!upper) {
      if (r0 < n) v0 = xj[perm[r0]];
      if (r1 < n) v1 = xj[perm[r1]];
      for (int l = 0; l < n; ++l) {
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31);
        if (r0 > l && r0 < n) v0 -= A[r0 + l * n] * x;
        if (r1 > l && r1 < n) v1 -= A[r1 + l * n] * x;
      }
    } else {
      if (r0 < n) v0 = xj[r0];
      if (r1 < n) v1 = xj[r1];
      for (int l = n - 1; l >= 0; --l) {
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31) * dinv[l];
        if (r0 == l) v0 = x;
        if (r1 == l) v1 = x;
        if (r0 < l) v0 -= A[r0 + l * n] * x;
        if (r1 < l && r1 < n) v1 -= A[r1 + l * n] * x;
      }
    }
    if (r0 < n) stv(c, t.c, r0, j, v0);
    if (r1 < n) stv(c, t.c, r1, j, v1);
  }
  if (threadIdx.x == 0) c.flops += fl + (double)n * n * k;
}

// ---------------------------------------------------------------- DADD
template <class T>
__device__ void task_dadd(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.c.rows, n = ncols(c, t.c), k = ncols(c, t.a);
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + kStage;
  for (int i0 = 0; i0 < m; i0 += 64)
    for (int j0 = 0; j0 < n; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      if (k > 0)
        tile_mma(acc, shift(mat(c, t.a), i0, 0), 0, min(64, m - i0), shift(matT(c, t.b), 0, j0), min(64, n - j0), k,
                 As, Bs, c.tcc);
      const T sg = (t.flags & TF_ALPHA) ? T(t.sign) * T(c.alpha) : T(t.sign);
      tile_store(acc, c, t.c, i0, j0, min(64, m - i0), min(64, n - j0), sg, (t.flags & TF_OVERWRITE) != 0);
    }
  if (threadIdx.x == 0) c.flops += 2.0 * m * n * k;
}

// ---------------------------------------------------------------- TRUNC
__device__ __forceinline__ void group_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Sum of products in twice the working precision: the Dot2 scheme of Ogita,
// Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26,
// 2005).  The rounding error of each product comes from an FMA, that of each
// addition from Knuth's TwoSum; the errors are summed separately.
struct Dot2f {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x, float y) {
    const float p = __fmul_rn(x, y);
    const float ep = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, ep));
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};
struct Dot1d {
  double s = 0.0;
  __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <class T>
struct AccurateDot;
template <>
struct AccurateDot<float> {
  using type = Dot2f;
};
template <>
struct AccurateDot<double> {
  using type = Dot1d;
};

// Householder QR of S (m x w, column-major, ld m, private scratch) in place by
// a group of NW warps (group thread gt in [0, 32 NW), named barrier `bar`).
// Reflector j is I - tau_j v v^T with v = (1, S[j+1:m, j]) stored below the
// diagonal; R is left on and above it.  Each warp owns trailing columns
// j + 1 + warp + k NW and updates them without further synchronisation; the
// owner of column j + 1 also leaves that column's new squared norm below the
// diagonal in s2[j + 1], so one barrier per column suffices.  Column j is
// scaled into its stored form one step later, when no warp reads it.
template <class T, int NW>
__device__ void house_qr_group(T* S, int m, int w, T* tau, T* s2, T* scb, int gt, int bar) {
  constexpr int NTG = NW * 32;
  const int wg = gt >> 5, lane = gt & 31;
  const int tmax = min(m, w);
  if (wg == 0) {
    T s = 0;
    #pragma unroll 4
    for (int i = 1 + lane; i < m; i += 32) {
      const T x = S[i];
      s += x * x;
    }
    s = warp_sum(s);
    if (lane == 0) s2[0] = s;
  }
  group_bar(bar, NTG);
  for (int j = 0; j < tmax; ++j) {
    T* cj = S + (int64_t)j * m;
    const T ss = s2[j];
    const T alpha = cj[j];
    T beta = alpha, sc = 0, tj = 0;
    if (ss > T(0)) {
      const T nrm = sqrt(alpha * alpha + ss);
      beta = alpha >= T(0) ? -nrm : nrm;
      sc = T(1) / (alpha - beta);
      tj = (beta - alpha) / beta;
    }
    if (gt == 0) {
      tau[j] = tj;
      scb[j] = sc;
      scb[kTruncStack + j] = beta;
    }
    for (int c0 = j + 1 + wg; c0 < w; c0 += 4 * NW) {
      T* col[4];
      T d[4], top[4];
      int nc = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int cc = c0 + q * NW;
        col[q] = S + (int64_t)(cc < w ? cc : c0) * m;
        if (cc < w) nc = q + 1;
        d[q] = 0;
        top[q] = col[q][j];
      }
      #pragma unroll 4
      for (int i = j + 1 + lane; i < m; i += 32) {
        const T v = cj[i];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nc) d[q] += v * col[q][i];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] = (top[q] + sc * warp_sum(d[q])) * tj;
      const bool own_next = c0 == j + 1;
      T nn = 0;
      // four rows per lane at a time: all loads issued before the stores
      for (int i0 = j + 1 + lane; i0 < m; i0 += 128) {
        T v[4], x[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          v[u] = i < m ? cj[i] * sc : T(0);
#pragma unroll
          for (int q = 0; q < 4; ++q) x[u][q] = (i < m && q < nc) ? col[q][i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          if (i < m)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q < nc) {
                const T y = x[u][q] - d[q] * v[u];
                col[q][i] = y;
                if (q == 0 && i > j + 1) nn += y * y;
              }
        }
      }
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nc) col[q][j] = top[q] - d[q];
      if (own_next) {
        nn = warp_sum(nn);
        if (lane == 0) s2[j + 1] = nn;
      }
    }
    group_bar(bar, NTG);
  }
  // Each column's reflector is scaled to a unit leading entry and its
  // diagonal becomes R's, in one pass at the end (column j is last read in
  // step j, which used it unscaled).  Thread gt visits elements gt, gt + NTG,
  // ... of the m x tmax block; its (row, column) advances without a division.
  const int tot = m * tmax;
  int ri = gt % m, rj = gt / m;
  for (int b0 = gt; b0 < tot; b0 += 8 * NTG) {
    T x[8];
    int xi[8], xj[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      xi[u] = ri;
      xj[u] = rj;
      x[u] = (b0 + u * NTG < tot && ri > rj) ? S[(int64_t)rj * m + ri] : T(0);
      ri += NTG;
      while (ri >= m) {
        ri -= m;
        ++rj;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (b0 + u * NTG < tot) {
        if (xi[u] > xj[u])
          S[(int64_t)xj[u] * m + xi[u]] = x[u] * scb[xj[u]];
        else if (xi[u] == xj[u])
          S[(int64_t)xj[u] * m + xi[u]] = scb[kTruncStack + xj[u]];
      }
  }
  group_bar(bar, NTG);
}

// O (m x r, column-major, ld) <- Q O with Q = H_0 ... H_{tmax-1} from
// house_qr_group; each warp of the group owns output columns and applies all
// reflectors to them, four columns at a time.
template <class T, int NW>
__device__ void apply_q_group(const T* S, int m, int tmax, const T* tau, T* O, int64_t ld, int r, int gt) {
  const int wg = gt >> 5, lane = gt & 31;
  for (int c0 = wg; c0 < r; c0 += 4 * NW) {
    T* col[4];
    int nc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cc = c0 + q * NW;
      col[q] = O + (int64_t)(cc < r ? cc : c0) * ld;
      if (cc < r) nc = q + 1;
    }
    for (int j = tmax - 1; j >= 0; --j) {
      const T tj = tau[j];
      if (tj == T(0)) continue;
      const T* cj = S + (int64_t)j * m;
      T d[4], top[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        d[q] = 0;
        top[q] = col[q][j];
      }
      #pragma unroll 4
      for (int i = j + 1 + lane; i < m; i += 32) {
        const T v = cj[i];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nc) d[q] += v * col[q][i];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] = (top[q] + warp_sum(d[q])) * tj;
      for (int i0 = j + 1 + lane; i0 < m; i0 += 128) {
        T v[4], x[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          v[u] = i < m ? cj[i] : T(0);
#pragma unroll
          for (int q = 0; q < 4; ++q) x[u][q] = (i < m && q < nc) ? col[q][i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 32 * u;
          if (i < m)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q < nc) col[q][i] = x[u][q] - d[q] * v[u];
        }
      }
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nc) col[q][j] = top[q] - d[q];
      __syncwarp();
    }
  }
}

// One-sided Jacobi SVD of G (p x q, column-major, ld p, shared memory):
// G <- G V with V (q x q, ld q, starts as I) accumulating the rotations,
// until all column pairs are orthogonal to `tol` or the sweeps stop making
// progress at the rounding floor.  A round-robin round has qq/2 disjoint
// pairs (qq = q rounded up to even); each pair is handled by a group of gs
// lanes.  nrm2 holds the squared column norms: recomputed at the start of a
// sweep, updated by each rotation (a' = a - t g, b' = b + t g), and exact
// again on return.
template <class T>
__device__ int jacobi_svd(T* G, T* V, int p, int q, T* nrm2, T tol, T negl_rel) {
  __shared__ int s_rot;
  __shared__ float s_off, s_prev;
  __shared__ T s_negl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qq = q + (q & 1);
  const int npairs = qq / 2;
  int gs = 32;
  while (gs > 1 && npairs * gs > NT) gs >>= 1;
  const int k = threadIdx.x / gs, lg = threadIdx.x % gs;
  auto norms = [&]() {
    for (int j = warp; j < q; j += NT / 32) {
      T acc = 0;
      for (int i = lane; i < p; i += 32) acc += G[i + j * p] * G[i + j * p];
      acc = warp_sum(acc);
      if (lane == 0) nrm2[j] = acc;
    }
  };
  if (threadIdx.x == 0) s_prev = 3.0e38f;
  int sweep = 0;
  for (; sweep < 20 && qq > 1; ++sweep) {
    norms();
    __syncthreads();
    if (threadIdx.x == 0) {
      s_rot = 0;
      s_off = 0.0f;
      T mx = 0;
      for (int j = 0; j < q; ++j) mx = max(mx, nrm2[j]);
      s_negl = negl_rel * negl_rel * mx;
    }
    __syncthreads();
    for (int rd = 0; rd < qq - 1; ++rd) {
      int a = 0, b = 0;
      bool act = k < npairs;
      if (act) {
        const int pa = k == 0 ? 0 : ((k - 1 + rd) % (qq - 1)) + 1;
        const int kb = qq - 1 - k;
        const int pb = kb == 0 ? 0 : ((kb - 1 + rd) % (qq - 1)) + 1;
        a = min(pa, pb);
        b = max(pa, pb);
        act = b < q;
      }
      // a column far below the truncation level is discarded whatever the
      // rotations do (they never raise the smaller norm of a pair), so
      // pairs involving one are skipped
      if (act) act = min(nrm2[a], nrm2[b]) > s_negl;
      T ga = 0;
      if (act)
        for (int i = lg; i < p; i += gs) ga += G[i + a * p] * G[i + b * p];
      for (int o = gs >> 1; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
      if (act && ga != T(0)) {
        const T al = nrm2[a], be = nrm2[b];
        const T ratio = fabs(ga) / sqrt(al * be);
        if (lg == 0) atomicMax(reinterpret_cast<int*>(&s_off), __float_as_int((float)ratio));
        if (ratio > tol) {
          const T zeta = (be - al) / (T(2) * ga);
          const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
          for (int i = lg; i < p; i += gs) {
            const T x = G[i + a * p], y = G[i + b * p];
            G[i + a * p] = cs * x - sn * y;
            G[i + b * p] = sn * x + cs * y;
          }
          for (int i = lg; i < q; i += gs) {
            const T x = V[i + a * q], y = V[i + b * q];
            V[i + a * q] = cs * x - sn * y;
            V[i + b * q] = sn * x + cs * y;
          }
          if (lg == 0) {
            nrm2[a] = al - tt * ga;
            nrm2[b] = be + tt * ga;
            s_rot = 1;
          }
        }
      }
      __syncthreads();
    }
    if (!s_rot) break;
    const bool stalled = sweep >= 2 && s_off < 100.0f * (float)tol && s_off > 0.25f * s_prev;
    __syncthreads();
    if (threadIdx.x == 0) s_prev = s_off;
    if (stalled) break;
    __syncthreads();
  }
  norms();
  __syncthreads();
  return sweep + 1;
}

constexpr int kDenseMax = 128;
constexpr int kDenseRank = 40;           // rows kept by the dense route's pivoted QR
constexpr int kCoreRank = kRankMax;      // rows kept by the stack route's pivoted QR of the core
constexpr int kCoreV = kTruncStack * kCoreRank + kCoreRank * kCoreRank;  // M (q x r') and V (r' x r')

// dynamic shared memory of the task bodies: max over task kinds of TRUNC
// (3 stack-wide vectors + G + V), GETRF/TRSM (64 x 64 + 64 ints), the fused
// leaf solve and the staged GEMM chunks (2 x KC x kLds)
__host__ __device__ constexpr size_t exec_smem_base(int elem_size) {
  const size_t trunc0 = (size_t)elem_size * (3 * kTruncStack + kTruncStack * kTruncStack + kCoreV);
  // dense truncation route (FP32 only)
  const size_t r0 = (size_t)4 * (kDenseMax * kDenseRank + kDenseRank * kDenseRank);
  const size_t region0 = r0 < (size_t)4 * 2 * kStage ? (size_t)4 * 2 * kStage : r0;
  const size_t dense = region0 + (size_t)4 * (kDenseMax * kDenseMax + 2 * kDenseMax) + sizeof(int) * kDenseMax;
  const size_t trunc = (elem_size == 4 && dense > trunc0) ? dense : trunc0;
  const size_t lu0 = (size_t)elem_size * (64 * 64 + 64) + 64 * sizeof(int);
  // fused leaf solve: staging chunks, tile, right-hand side, inverse diagonal, pivots
  const size_t rsolve = (size_t)elem_size * (2 * kStage + 2 * 64 * 64 + 64) + 64 * sizeof(int);
  const size_t lu = rsolve > lu0 ? rsolve : lu0;
  const size_t gemm = (size_t)elem_size * 2 * kStage;
  const size_t m = trunc > lu ? trunc : lu;
  return m > gemm ? m : gemm;
}
// the tensor-core staging buffer follows the task bodies' region, 1024-aligned
__host__ __device__ constexpr size_t exec_stage_offset() { return (exec_smem_base(4) + 1023) & ~(size_t)1023; }


// Householder QR with column pivoting of D (m x n, ld m, shared memory) in
// place, stopped after kmax steps or once the trailing block's squared
// Frobenius norm is <= rel2 ||D||_F^2.  perm[j] = original index of column j.
// Returns the number of reflectors r'; *tail2 receives the dropped norm^2.
template <class T>
__device__ int pivoted_qr(T* D, int m, int n, int kmax, T rel2, T* tau, T* nrm2, int* perm, T* tail2) {
  __shared__ int s_piv;
  __shared__ T s_tail, s_thr, s_beta, s_sc, s_tau;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = threadIdx.x; j < n; j += NT) perm[j] = j;
  const int kend = min(kmax, min(m, n));
  int k = 0;
  for (;; ++k) {
    for (int j = k + warp; j < n; j += NT / 32) {
      T acc = 0;
      for (int i = k + lane; i < m; i += 32) acc += D[i + j * m] * D[i + j * m];
      acc = warp_sum(acc);
      if (lane == 0) nrm2[j] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T tail = 0, best = T(-1);
      int piv = k;
      for (int j = k; j < n; ++j) {
        tail += nrm2[j];
        if (nrm2[j] > best) {
          best = nrm2[j];
          piv = j;
        }
      }
      if (k == 0) s_thr = rel2 * tail;
      s_tail = tail;
      s_piv = piv;
    }
    __syncthreads();
    if (k >= kend || s_tail <= s_thr) break;
    const int pv = s_piv;
    if (pv != k) {
      for (int i = threadIdx.x; i < m; i += NT) {
        const T x = D[i + k * m];
        D[i + k * m] = D[i + pv * m];
        D[i + pv * m] = x;
      }
      if (threadIdx.x == 0) {
        const int pp = perm[k];
        perm[k] = perm[pv];
        perm[pv] = pp;
      }
    }
    __syncthreads();
    if (warp == 0) {
      T ss = 0;
      for (int i = k + 1 + lane; i < m; i += 32) ss += D[i + k * m] * D[i + k * m];
      ss = warp_sum(ss);
      if (lane == 0) {
        const T alpha = D[k + k * m];
        T beta = alpha, sc = 0, tj = 0;
        if (ss > T(0)) {
          const T nrm = sqrt(alpha * alpha + ss);
          beta = alpha >= T(0) ? -nrm : nrm;
          sc = T(1) / (alpha - beta);
          tj = (beta - alpha) / beta;
        }
        s_beta = beta;
        s_sc = sc;
        s_tau = tj;
        tau[k] = tj;
      }
      __syncwarp();
      const T sc = s_sc;
      for (int i = k + 1 + lane; i < m; i += 32) D[i + k * m] *= sc;
      __syncwarp();
      if (lane == 0) D[k + k * m] = s_beta;
    }
    __syncthreads();
    const T tj = s_tau;
    if (tj != T(0))
      for (int j = k + 1 + warp; j < n; j += NT / 32) {
        T d = 0;
        for (int i = k + 1 + lane; i < m; i += 32) d += D[i + k * m] * D[i + j * m];
        d = (warp_sum(d) + D[k + j * m]) * tj;
        for (int i = k + 1 + lane; i < m; i += 32) D[i + j * m] -= d * D[i + k * m];
        __syncwarp();
        if (lane == 0) D[k + j * m] -= d;
      }
    __syncthreads();
  }
  *tail2 = s_tail;
  return k;
}

// stack width at which a truncation compresses before adding the next piece
// (the core SVD costs grow with the cube of the width); rank cap 32 + a
// 64-wide piece still fit the stack
constexpr int kStackCols = kTruncStack;
constexpr int kCompressAt = 48;

// Truncated SVD of the stacked factors SX (m x W) and SY (n x W) in compute
// type TC: Householder QR of both (concurrently, half of the CTA each), the
// core R_x R_y^T accumulated in twice the working precision, its one-sided
// Jacobi SVD, keep s_i > eps s_1 (at most cap); X <- Q_x U_r S_r and
// Y <- Q_y V_r are written to OX (ld ox) and OY (ld oy).  Workspace: tauX,
// tauY, sv (kStackCols each), G (kStackCols^2) and V (kCoreV) in shared
// memory.  The largest rank asked for goes to status[4].
// Returns r (the same in every thread); *fro receives ||X Y^T||_F.
template <class TC>
__device__ int compress_core(TC* SX, TC* SY, int m, int n, int W, int cap, double eps, TC* tauX, TC* tauY,
                             TC* sv, TC* G, TC* V, TC* OX, int64_t ox, TC* OY, int64_t oy, int32_t* status,
                             double* flops, double* fro, unsigned long long* tp, double jtol) {
  __shared__ TC s2x[kStackCols + 1], s2y[kStackCols + 1];
  __shared__ TC s_scbx[2 * kStackCols], s_scby[2 * kStackCols];  // reflector scales and R's diagonal
  long long t0 = tp && threadIdx.x == 0 ? clock64() : 0;
  auto lap = [&](int k) {
    if (tp && threadIdx.x == 0) {
      const long long t1 = clock64();
      tp[k] += (unsigned long long)(t1 - t0);
      t0 = t1;
    }
  };
  __shared__ int s_r;
  __shared__ int s_ord[kStackCols];
  __shared__ double s_fro;
  constexpr int kHalf = NT / 2;
  if (threadIdx.x < kHalf)
    house_qr_group<TC, kHalf / 32>(SX, m, W, tauX, s2x, s_scbx, threadIdx.x, 1);
  else
    house_qr_group<TC, kHalf / 32>(SY, n, W, tauY, s2y, s_scby, threadIdx.x - kHalf, 2);
  __syncthreads();
  lap(1);
  const int p = min(m, W), q = min(n, W);
  // the core R_x R_y^T: the target and its updates cancel inside these sums
  for (int idx = threadIdx.x; idx < p * q; idx += NT) {
    const int i = idx % p, j = idx / p;
    typename AccurateDot<TC>::type acc;
    for (int l = max(i, j); l < W; ++l) acc.add(SX[i + (int64_t)l * m], SY[j + (int64_t)l * n]);
    G[i + j * p] = acc.value();
  }
  __syncthreads();
  lap(2);
  // pivoted QR of the core down to the truncation floor (G ~ Q_G R' P^T with
  // r' rows kept), then the Jacobi SVD of M = P R'^T (q x r'): M V_M = W,
  // G ~ Q_G V_M W^T; X <- Q_x Q_G V_M S and Y <- Q_y W S^-1 below
  __shared__ TC s_tauG[kStackCols];
  __shared__ int s_perm[kStackCols];
  TC tail2 = 0;
  const TC rel = TC(0.1 * eps);
  const int rp = pivoted_qr(G, p, q, min(kCoreRank, min(p, q)), rel * rel / TC(min(p, q)), s_tauG, sv, s_perm,
                            &tail2);
  TC* M = V;
  TC* Vs = V + q * rp;
  for (int idx = threadIdx.x; idx < q * rp; idx += NT) {
    const int j = idx % q, i = idx / q;
    M[s_perm[j] + i * q] = j >= i ? G[i + j * p] : TC(0);
  }
  for (int idx = threadIdx.x; idx < rp * rp; idx += NT) Vs[idx] = (idx % rp == idx / rp) ? TC(1) : TC(0);
  __syncthreads();
  const int sweeps = rp > 0 ? jacobi_svd(M, Vs, q, rp, sv, TC(jtol), TC(0.01 * eps)) : 0;
  lap(3);
  if (tp && threadIdx.x == 0) {
    tp[5] += 1ULL;
    tp[6] += (unsigned long long)sweeps;
    tp[7] += (unsigned long long)W;
  }
  if (threadIdx.x == 0) {
    double f2 = 0;
    for (int j = 0; j < rp; ++j) {
      sv[j] = sqrt(sv[j]);
      s_ord[j] = j;
      f2 += (double)sv[j] * (double)sv[j];
    }
    s_fro = sqrt(f2);
    for (int j = 1; j < rp; ++j) {  // stable insertion sort, descending
      int x = s_ord[j], i = j - 1;
      while (i >= 0 && sv[s_ord[i]] < sv[x]) {
        s_ord[i + 1] = s_ord[i];
        --i;
      }
      s_ord[i + 1] = x;
    }
    TC smax = rp ? sv[s_ord[0]] : TC(0);
    int r = 0;
    if (smax > TC(0))
      while (r < rp && sv[s_ord[r]] > TC(eps) * smax) ++r;
    const bool more = rp == kCoreRank && tail2 > TC(eps * eps) * smax * smax;
    atomicMax(status + 4, more ? kCoreRank + 1 : r);
    if (r > cap || more) {
      r = min(r, cap);
      atomicAdd(status + 2, 1);
    }
    s_r = r;
    *flops += 2.0 * (m + n) * W * W + 4.0 * (double)p * q * rp + 6.0 * sweeps * (double)q * rp * rp +
              2.0 * (m + n) * W * r;
  }
  __syncthreads();
  const int r = s_r;
  *fro = s_fro;
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    OX[i + (int64_t)j * ox] = i < rp ? Vs[i + s_ord[j] * rp] * sv[s_ord[j]] : TC(0);
  }
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    OY[i + (int64_t)j * oy] = i < q ? M[i + s_ord[j] * q] / sv[s_ord[j]] : TC(0);
  }
  __syncthreads();
  apply_q_group<TC, NT / 32>(G, p, rp, s_tauG, OX, ox, r, threadIdx.x);
  __syncthreads();
  if (threadIdx.x < kHalf)
    apply_q_group<TC, kHalf / 32>(SX, m, p, tauX, OX, ox, r, threadIdx.x);
  else
    apply_q_group<TC, kHalf / 32>(SY, n, q, tauY, OY, oy, r, threadIdx.x - kHalf);
  __syncthreads();
  lap(4);
  return r;
}

// Stacks the pieces in compute type TC (compressing whenever the stack would
// pass kCompressAt columns) and leaves the final factors in OX (m x r) and
// OY (n x r) of the scratch.  Returns r; *ratio receives the largest
// ||X||_F ||Y||_F / ||X Y^T||_F over the compressions (how much cancellation
// the arithmetic had to survive).
template <class TC, class T>
__device__ int trunc_stack(Ctx<T>& c, const Task& t, TC* SX, TC* SY, TC* OX, TC* OY, TC* tauX, TC* tauY, TC* sv,
                           TC* G, TC* V, double* ratio) {
  const int m = t.a.rows, n = t.b.rows;
  __shared__ TC s_rx[NT / 32];
  double worst = 0;
  int W = 0;
  auto stack_norm = [&](int w_) -> double {
    TC px = 0, py = 0;
    #pragma unroll 4
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * w_; idx += NT) px += SX[idx] * SX[idx];
    #pragma unroll 4
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * w_; idx += NT) py += SY[idx] * SY[idx];
    TC sx = block_sum(px, s_rx);
    TC sy = block_sum(py, s_rx);
    return sqrt((double)sx) * sqrt((double)sy);
  };
  // a piece goes onto the stack in parts of at most kStackCols - W columns
  // (X Y^T is the sum over its columns), compressing first whenever the rest
  // of the piece would take the stack past compress_at columns; after a
  // compression W <= kRankMax < kStackCols, so every part is nonempty
  for (int q = 0; q < t.list_count; ++q) {
    const Piece& P = c.pieces[t.list_begin + q];
    const int w = ncols(c, P.X);
    for (int c0 = 0; c0 < w;) {
      if (W > 0 && W + (w - c0) > c.compress_at) {
        const double in = stack_norm(W);
        double fro = 0;
        const int r = compress_core(SX, SY, m, n, W, t.cap, c.eps, tauX, tauY, sv, G, V, OX, m, OY, n, c.status,
                                    &c.flops, &fro, c.tprof, c.jacobi_tol);
        if (fro > 0) worst = fmax(worst, in / fro);
        for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) SX[idx] = __ldcg(OX + idx);
        for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) SY[idx] = __ldcg(OY + idx);
        W = r;
        __syncthreads();
      }
      const int take = min(w - c0, kStackCols - W);
      const TC sg = (P.pad & PF_ALPHA) ? TC(P.sign) * TC(c.alpha) : TC(P.sign);
      for (int64_t idx = threadIdx.x; idx < (int64_t)m * take; idx += NT) SX[(int64_t)W * m + idx] = TC(0);
      for (int64_t idx = threadIdx.x; idx < (int64_t)n * take; idx += NT) SY[(int64_t)W * n + idx] = TC(0);
      __syncthreads();
      // four elements per thread at a time: all loads issued before the stores
      for (int64_t b0 = threadIdx.x; b0 < (int64_t)P.X.rows * take; b0 += 4 * NT) {
        TC v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t idx = b0 + (int64_t)u * NT;
          v[u] = idx < (int64_t)P.X.rows * take ? TC(ldv(c, P.X, idx % P.X.rows, c0 + idx / P.X.rows)) : TC(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t idx = b0 + (int64_t)u * NT;
          if (idx < (int64_t)P.X.rows * take)
            SX[(P.xoff + idx % P.X.rows) + (int64_t)(W + idx / P.X.rows) * m] = sg * v[u];
        }
      }
      for (int64_t b0 = threadIdx.x; b0 < (int64_t)P.Y.rows * take; b0 += 4 * NT) {
        TC v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t idx = b0 + (int64_t)u * NT;
          v[u] = idx < (int64_t)P.Y.rows * take ? TC(ldv(c, P.Y, idx % P.Y.rows, c0 + idx / P.Y.rows)) : TC(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t idx = b0 + (int64_t)u * NT;
          if (idx < (int64_t)P.Y.rows * take)
            SY[(P.yoff + idx % P.Y.rows) + (int64_t)(W + idx / P.Y.rows) * n] = v[u];
        }
      }
      W += take;
      c0 += take;
      __syncthreads();
    }
  }
  int r = 0;
  if (W > 0) {
    const double in = stack_norm(W);
    double fro = 0;
    r = compress_core(SX, SY, m, n, W, t.cap, c.eps, tauX, tauY, sv, G, V, OX, m, OY, n, c.status, &c.flops, &fro,
                      c.tprof, c.jacobi_tol);
    if (fro > 0) worst = fmax(worst, in / fro);
  }
  *ratio = worst;
  return r;
}

// ------------------------------------------------------------- dense TRUNC
// Targets with both sides up to kDenseMax whose pieces would need more than
// one compression of the stack take a dense route (FP32 factors): the sum
// D = sum sign X Y^T is formed in shared memory, a Householder QR with column
// pivoting stops once the trailing block's Frobenius norm is below
// 0.1 eps ||D||_F / sqrt(min(m, n)) (<= 0.1 eps s_1), and the one-sided Jacobi
// SVD of the remaining r' x n rows gives the truncation s_i > eps s_1.
constexpr int kStagePieces = 16;

// Chunks of sum_pieces sign X Y^T restricted to the 64 x 64 tile (i0, j0).
template <class T>
struct PieceCursor {
  const Ctx<T>* c;
  const Piece* pc;
  const int* w;
  int nq, i0, j0, q, l0;
  __device__ bool valid(int qq) const {
    const Piece& P = pc[qq];
    return w[qq] > 0 && max(P.xoff, i0) < min(P.xoff + P.X.rows, i0 + 64) &&
           max(P.yoff, j0) < min(P.yoff + P.Y.rows, j0 + 64);
  }
  __device__ bool seek(int qq) {
    while (qq < nq && !valid(qq)) ++qq;
    q = qq;
    l0 = 0;
    return q < nq;
  }
  __device__ bool first() { return seek(0); }
  __device__ bool next() {
    l0 += KC;
    if (l0 < w[q]) return true;
    return seek(q + 1);
  }
  __device__ Chunk<T> chunk() const {
    const Piece& P = pc[q];
    const int xl = max(P.xoff, i0), xh = min(P.xoff + P.X.rows, i0 + 64);
    const int yl = max(P.yoff, j0), yh = min(P.yoff + P.Y.rows, j0 + 64);
    const T sg = (P.pad & PF_ALPHA) ? T(P.sign) * T(c->alpha) : T(P.sign);
    return Chunk<T>{shift(mat(*c, P.X), xl - P.xoff, l0), shift(matT(*c, P.Y), l0, yl - P.yoff), xl - i0, xh - xl,
                    yh - yl, min(KC, w[q] - l0), yl - j0, sg};
  }
};

// Returns false, having written nothing but the shared memory, when the
// pivoted QR reached kDenseRank rows with a dropped tail above
// eps |R_00| (|R_00| <= s_1): the stack route then truncates the target.
template <class T>
__device__ bool task_trunc_dense(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.a.rows, n = t.b.rows;
  // shared memory: [region 0: staging chunks, later M (n x kDenseRank) and
  // V][D (m x n)][tau, nrm2 (kDenseMax each)][perm]
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + kStage;
  T* M = As;
  T* V = M + kDenseMax * kDenseRank;
  T* D = V + kDenseRank * kDenseRank;
  T* tau = D + kDenseMax * kDenseMax;
  T* nrm2 = tau + kDenseMax;
  int* perm = reinterpret_cast<int*>(nrm2 + kDenseMax);
  __shared__ Piece s_pc[kStagePieces];
  __shared__ int s_w[kStagePieces];
  __shared__ int s_ord[kDenseRank];
  __shared__ int s_r;
  unsigned long long* tp = c.tprof;
  long long t0 = tp && threadIdx.x == 0 ? clock64() : 0;
  // D = sum of the pieces, tile by tile, pieces staged kStagePieces at a time
  for (int i0 = 0; i0 < m; i0 += 64)
    for (int j0 = 0; j0 < n; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      for (int qb = 0; qb < t.list_count; qb += kStagePieces) {
        const int nq = min(kStagePieces, t.list_count - qb);
        __syncthreads();
        {
          const int words = nq * (int)(sizeof(Piece) / sizeof(int32_t));
          const int32_t* src = reinterpret_cast<const int32_t*>(c.pieces + t.list_begin + qb);
          int32_t* dst = reinterpret_cast<int32_t*>(s_pc);
          for (int w = threadIdx.x; w < words; w += NT) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        if (threadIdx.x < nq) s_w[threadIdx.x] = ncols(c, s_pc[threadIdx.x].X);
        __syncthreads();
        PieceCursor<T> cur{&c, s_pc, s_w, nq, i0, j0, 0, 0};
        tile_mma_seq(acc, cur, As, Bs, c.tcc);
      }
      const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = i0 + tx * 4 + i, cc = j0 + ty * 4 + j;
          if (r < m && cc < n) D[r + cc * m] = acc[i][j];
        }
    }
  __syncthreads();
  if (tp && threadIdx.x == 0) {
    const long long t1 = clock64();
    tp[0] += (unsigned long long)(t1 - t0);
    t0 = t1;
  }
  // pivoted QR down to the truncation floor
  const T rel = T(0.1 * c.eps);
  T tail2 = 0;
  const int rp = pivoted_qr(D, m, n, kDenseRank, rel * rel / T(min(m, n)), tau, nrm2, perm, &tail2);
  if (tp && threadIdx.x == 0) {
    const long long t1 = clock64();
    tp[1] += (unsigned long long)(t1 - t0);
    t0 = t1;
  }
  if (rp == kDenseRank && tail2 > T(c.eps * c.eps) * D[0] * D[0]) {
    if (threadIdx.x == 0) atomicAdd(c.status + 5, 1);
    __syncthreads();
    return false;
  }
  // M = P R'^T (n x r'), Jacobi SVD of its columns: M V = W
  for (int idx = threadIdx.x; idx < n * rp; idx += NT) {
    const int j = idx % n, i = idx / n;
    M[perm[j] + i * n] = j >= i ? D[i + j * m] : T(0);
  }
  for (int idx = threadIdx.x; idx < rp * rp; idx += NT) V[idx] = (idx % rp == idx / rp) ? T(1) : T(0);
  __syncthreads();
  int sweeps = 0;
  if (rp > 0) sweeps = jacobi_svd(M, V, n, rp, nrm2, T(c.jacobi_tol), T(0.01 * c.eps));
  if (tp && threadIdx.x == 0) {
    const long long t1 = clock64();
    tp[3] += (unsigned long long)(t1 - t0);
    tp[5] += 1ULL;
    tp[6] += (unsigned long long)sweeps;
    tp[7] += (unsigned long long)rp;
    t0 = t1;
  }
  if (threadIdx.x == 0) {
    for (int j = 0; j < rp; ++j) {
      nrm2[j] = sqrt(nrm2[j]);
      s_ord[j] = j;
    }
    for (int j = 1; j < rp; ++j) {  // stable insertion sort, descending
      int x = s_ord[j], i = j - 1;
      while (i >= 0 && nrm2[s_ord[i]] < nrm2[x]) {
        s_ord[i + 1] = s_ord[i];
        --i;
      }
      s_ord[i + 1] = x;
    }
    const T smax = rp ? nrm2[s_ord[0]] : T(0);
    int r = 0;
    if (smax > T(0))
      while (r < rp && nrm2[s_ord[r]] > T(c.eps) * smax) ++r;
    atomicMax(c.status + 4, r);
    if (r > t.cap) {
      r = min(r, t.cap);
      atomicAdd(c.status + 2, 1);
    }
    s_r = r;
    c.flops += 2.0 * (double)m * n * kDenseRank + 2.0 * (double)m * n * rp + 6.0 * sweeps * (double)n * rp * rp;
  }
  __syncthreads();
  const int r = s_r;
  // X = Q' [V_sel S; 0] through the scratch, Y = W_sel / s
  T* OX = c.scratch;
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    OX[i + (int64_t)j * m] = i < rp ? V[i + s_ord[j] * rp] * nrm2[s_ord[j]] : T(0);
  }
  __syncthreads();
  apply_q_group<T, NT / 32>(D, m, rp, tau, OX, m, r, threadIdx.x);
  __syncthreads();
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) stv(c, t.a, idx % m, idx / m, OX[idx]);
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    stv(c, t.b, i, j, M[i + s_ord[j] * n] / nrm2[s_ord[j]]);
  }
  __syncthreads();
  if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, r);
  if (tp && threadIdx.x == 0) tp[4] += (unsigned long long)(clock64() - t0);
  return true;
}

// (a, b) <- truncation of sum_pieces sign X Y^T (stack, compress, store).
// ------------------------------------------------------------- small TRUNC
// Q (m x tmax) of a Householder QR in place: S holds the reflectors of
// house_qr_group below its diagonal (unit leading entries implicit), and
// column j of S becomes column j of Q = H_0 ... H_{tmax-1} [I; 0], formed
// from the last reflector back (the recurrence of LAPACK's dorg2r).  Run by
// a group of NW warps (group thread gt, named barrier bar).
template <class T, int NW>
__device__ void orgqr_group(T* S, int m, int tmax, const T* tau, int gt, int bar) {
  constexpr int NTG = NW * 32;
  const int wg = gt >> 5, lane = gt & 31;
  for (int j = tmax - 1; j >= 0; --j) {
    const T tj = tau[j];
    T* cj = S + (int64_t)j * m;
    // H_j on the columns already formed: their row j is still zero
    if (tj != T(0))
      for (int cc = j + 1 + wg; cc < tmax; cc += NW) {
        T* col = S + (int64_t)cc * m;
        T d = 0;
        for (int i = j + 1 + lane; i < m; i += 32) d += cj[i] * col[i];
        d = warp_sum(d) * tj;
        for (int i = j + 1 + lane; i < m; i += 32) col[i] -= d * cj[i];
        if (lane == 0) col[j] = -d;
      }
    group_bar(bar, NTG);
    for (int i = gt; i < m; i += NTG) cj[i] = i < j ? T(0) : (i == j ? T(1) - tj : -tj * cj[i]);
    group_bar(bar, NTG);
  }
}

// Elements of T a small truncation needs in shared memory: both stacks,
// their reflector scalars, the core, its SVD and the two small factors.
__host__ __device__ constexpr int64_t trunc_small_elems(int m, int n, int W) {
  return (int64_t)(m + n) * W + 5LL * W * W + 10LL * W + 4LL * kTruncStack + 8;
}
template <class T>
__device__ __forceinline__ bool trunc_small_fits(int m, int n, int W) {
  return W > 0 && W <= kTruncStack &&
         trunc_small_elems(m, n, W) * (int64_t)sizeof(T) <= (int64_t)exec_smem_base(sizeof(T));
}

// A truncation whose whole stack fits in shared memory: the same
// recompression as the stack route (Householder QR of both stacks, core
// R_x R_y^T with Dot2, pivoted QR of the core, Jacobi SVD, s_i > eps s_1),
// in one compression of all W columns, with the stacks, reflectors and
// factors resident in shared memory; the kept factors X = Q_x Z_x and
// Y = Q_y Z_y go straight to the target views (Q_x, Q_y formed in place).
template <class T>
__device__ void task_trunc_small(Ctx<T>& c, const Task& t, char* smem, int W) {
  const int m = t.a.rows, n = t.b.rows;
  unsigned long long* tp = c.tprof;
  long long t0 = tp && threadIdx.x == 0 ? clock64() : 0;
  auto lap = [&](int k) {
    if (tp && threadIdx.x == 0) {
      const long long t1 = clock64();
      tp[k] += (unsigned long long)(t1 - t0);
      t0 = t1;
    }
  };
  T* SX = reinterpret_cast<T*>(smem);
  T* SY = SX + (int64_t)m * W;
  T* tauX = SY + (int64_t)n * W;
  T* tauY = tauX + W;
  T* sv = tauY + W;
  T* s2x = sv + W;
  T* s2y = s2x + W + 1;
  T* scbx = s2y + W + 1;
  T* scby = scbx + 2 * kTruncStack;
  T* tauG = scby + 2 * kTruncStack;
  T* G = tauG + W;
  T* V = G + W * W;
  T* Zx = V + 2 * W * W;
  T* Zy = Zx + W * W;
  int* perm = reinterpret_cast<int*>(Zy + W * W);
  int* ord = perm + W;
  __shared__ int s_r;
  for (int idx = threadIdx.x; idx < (m + n) * W; idx += NT) SX[idx] = T(0);
  __syncthreads();
  int w0 = 0;
  for (int q = 0; q < t.list_count; ++q) {
    const Piece& P = c.pieces[t.list_begin + q];
    const int w = ncols(c, P.X);
    const T sg = (P.pad & PF_ALPHA) ? T(P.sign) * T(c.alpha) : T(P.sign);
    // four elements per thread at a time: all loads issued before the stores
    const int64_t nx = (int64_t)P.X.rows * w, ny = (int64_t)P.Y.rows * w;
    for (int64_t b0 = threadIdx.x; b0 < nx; b0 += 4 * NT) {
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t idx = b0 + (int64_t)u * NT;
        v[u] = idx < nx ? ldv(c, P.X, idx % P.X.rows, idx / P.X.rows) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t idx = b0 + (int64_t)u * NT;
        if (idx < nx) SX[(P.xoff + idx % P.X.rows) + (int64_t)(w0 + idx / P.X.rows) * m] = sg * v[u];
      }
    }
    for (int64_t b0 = threadIdx.x; b0 < ny; b0 += 4 * NT) {
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t idx = b0 + (int64_t)u * NT;
        v[u] = idx < ny ? ldv(c, P.Y, idx % P.Y.rows, idx / P.Y.rows) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t idx = b0 + (int64_t)u * NT;
        if (idx < ny) SY[(P.yoff + idx % P.Y.rows) + (int64_t)(w0 + idx / P.Y.rows) * n] = v[u];
      }
    }
    w0 += w;
  }
  __syncthreads();
  lap(0);
  constexpr int kHalf = NT / 2;
  if (threadIdx.x < kHalf)
    house_qr_group<T, kHalf / 32>(SX, m, W, tauX, s2x, scbx, threadIdx.x, 1);
  else
    house_qr_group<T, kHalf / 32>(SY, n, W, tauY, s2y, scby, threadIdx.x - kHalf, 2);
  __syncthreads();
  lap(1);
  const int p = min(m, W), q = min(n, W);
  for (int idx = threadIdx.x; idx < p * q; idx += NT) {
    const int i = idx % p, j = idx / p;
    typename AccurateDot<T>::type acc;
    for (int l = max(i, j); l < W; ++l) acc.add(SX[i + (int64_t)l * m], SY[j + (int64_t)l * n]);
    G[i + j * p] = acc.value();
  }
  __syncthreads();
  lap(2);
  T tail2 = 0;
  const T rel = T(0.1 * c.eps);
  const int rp = pivoted_qr(G, p, q, min(kCoreRank, min(p, q)), rel * rel / T(min(p, q)), tauG, sv, perm, &tail2);
  T* M = V;
  T* Vs = V + q * rp;
  for (int idx = threadIdx.x; idx < q * rp; idx += NT) {
    const int j = idx % q, i = idx / q;
    M[perm[j] + i * q] = j >= i ? G[i + j * p] : T(0);
  }
  for (int idx = threadIdx.x; idx < rp * rp; idx += NT) Vs[idx] = (idx % rp == idx / rp) ? T(1) : T(0);
  __syncthreads();
  const int sweeps = rp > 0 ? jacobi_svd(M, Vs, q, rp, sv, T(c.jacobi_tol), T(0.01 * c.eps)) : 0;
  lap(3);
  if (tp && threadIdx.x == 0) {
    tp[5] += 1ULL;
    tp[6] += (unsigned long long)sweeps;
    tp[7] += (unsigned long long)W;
  }
  if (threadIdx.x == 0) {
    for (int j = 0; j < rp; ++j) {
      sv[j] = sqrt(sv[j]);
      ord[j] = j;
    }
    for (int j = 1; j < rp; ++j) {  // stable insertion sort, descending
      int x = ord[j], i = j - 1;
      while (i >= 0 && sv[ord[i]] < sv[x]) {
        ord[i + 1] = ord[i];
        --i;
      }
      ord[i + 1] = x;
    }
    const T smax = rp ? sv[ord[0]] : T(0);
    int r = 0;
    if (smax > T(0))
      while (r < rp && sv[ord[r]] > T(c.eps) * smax) ++r;
    const bool more = rp == kCoreRank && tail2 > T(c.eps * c.eps) * smax * smax;
    atomicMax(c.status + 4, more ? kCoreRank + 1 : r);
    if (r > t.cap || more) {
      r = min(r, t.cap);
      atomicAdd(c.status + 2, 1);
    }
    s_r = r;
    c.flops += 2.0 * (m + n) * W * W + 4.0 * (double)p * q * rp + 6.0 * sweeps * (double)q * rp * rp +
               2.0 * (m + n) * W * r;
  }
  __syncthreads();
  const int r = s_r;
  // Z_x = Q_G [V_M S; 0] (p x r), Z_y = W S^-1 (q x r), columns by descending s
  for (int idx = threadIdx.x; idx < p * r; idx += NT) {
    const int i = idx % p, j = idx / p;
    Zx[idx] = i < rp ? Vs[i + ord[j] * rp] * sv[ord[j]] : T(0);
  }
  for (int idx = threadIdx.x; idx < q * r; idx += NT) {
    const int i = idx % q, j = idx / q;
    Zy[idx] = M[i + ord[j] * q] / sv[ord[j]];
  }
  __syncthreads();
  apply_q_group<T, NT / 32>(G, p, rp, tauG, Zx, p, r, threadIdx.x);
  if (threadIdx.x < kHalf)
    orgqr_group<T, kHalf / 32>(SX, m, p, tauX, threadIdx.x, 1);
  else
    orgqr_group<T, kHalf / 32>(SY, n, q, tauY, threadIdx.x - kHalf, 2);
  __syncthreads();
  for (int e = threadIdx.x; e < m * r; e += NT) {
    const int i = e % m, j = e / m;
    T sum = 0;
    for (int l = 0; l < p; ++l) sum += SX[i + (int64_t)l * m] * Zx[l + j * p];
    stv(c, t.a, i, j, sum);
  }
  for (int e = threadIdx.x; e < n * r; e += NT) {
    const int i = e % n, j = e / n;
    T sum = 0;
    for (int l = 0; l < q; ++l) sum += SY[i + (int64_t)l * n] * Zy[l + j * q];
    stv(c, t.b, i, j, sum);
  }
  __syncthreads();
  lap(4);
  if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, r);
}

template <class T>
__device__ void task_trunc(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.a.rows, n = t.b.rows;
  if (m == 0 || n == 0) {
    if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, 0);
    return;
  }
  __shared__ int s_wsum;
  if (threadIdx.x == 0) s_wsum = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < t.list_count; q += NT) atomicAdd(&s_wsum, ncols(c, c.pieces[t.list_begin + q].X));
  __syncthreads();
  const int wsum = s_wsum;
  __syncthreads();
  // dense route when the stack would need more than one compression
  if (sizeof(T) == 4 && m <= kDenseMax && n <= kDenseMax && wsum > c.compress_at && task_trunc_dense(c, t, smem))
    return;
  if (wsum == 0) {
    if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, 0);
    return;
  }
  // the whole stack in shared memory, one compression
  if (trunc_small_fits<T>(m, n, wsum)) {
    task_trunc_small(c, t, smem, wsum);
    return;
  }
  const int64_t R = c.rows_max;
  T* SX = c.scratch;
  T* SY = SX + R * kStackCols;
  T* OX = SY + R * kStackCols;
  T* OY = OX + R * kRankMax;
  T* tauX = reinterpret_cast<T*>(smem);
  T* tauY = tauX + kStackCols;
  T* sv = tauY + kStackCols;
  T* G = sv + kStackCols;
  T* V = G + kStackCols * kStackCols;
  double ratio = 0;
  const int r = trunc_stack<T, T>(c, t, SX, SY, OX, OY, tauX, tauY, sv, G, V, &ratio);
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) stv(c, t.a, idx % m, idx / m, __ldcg(OX + idx));
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) stv(c, t.b, idx % n, idx / n, __ldcg(OY + idx));
  __syncthreads();
  if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, r);
}

// One task's body with the whole CTA.
template <class T>
__device__ void run_task(Ctx<T>& c, const Task& t, char* smem) {
  switch (t.type) {
    case TK_GETRF: task_getrf(c, t, smem); break;
    case TK_TRSM_L:
    case TK_TRSM_UT:
    case TK_TRSM_U: task_trsm(c, t, smem); break;
    case TK_PROJ: task_proj(c, t, smem); break;
    case TK_ROWMV: task_rowmv(c, t, smem); break;
    case TK_TRUNC: task_trunc(c, t, smem); break;
    case TK_DADD: task_dadd(c, t, smem); break;
    case TK_RSOLVE: task_rsolve(c, t, smem); break;
    default: break;
  }
}

// ---------------------------------------------------------------- executor
template <class T>
// two CTAs per SM for the plain executors; the tensor-core one is held to one
// by its tensor memory, so it may use the whole register file
#if HLU_EXEC_TC
#define EXEC_MIN_BLOCKS 1
#else
#define EXEC_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(NT, EXEC_MIN_BLOCKS) exec_kernel(const __grid_constant__ ExecArgs a) {
  // the tensor-core staging buffer at the start of dynamic shared memory is
  // 1024-byte aligned; the plain executors need 16 bytes
#if HLU_EXEC_TC
  extern __shared__ __align__(1024) char smem[];
#else
  extern __shared__ __align__(16) char smem[];
#endif
  __shared__ int64_t s_task;
  __shared__ int64_t s_succ[2];  // successor range of the running task
  __shared__ int s_prob;
  Ctx<T> c;
  TcCtl tcc;
  c.tcc = nullptr;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_tcbar;
  const bool use_tc = HLU_EXEC_TC && std::is_same<T, float>::value && a.tf32 != 0;
#if HLU_EXEC_TC
  if (use_tc) {
    // tensor memory for the 128 x 64 FP32 accumulator, held for the whole
    // persistent launch, and the MMA completion barrier
    if (threadIdx.x < 32) tc::tmem_alloc(&s_tmem, tc::kTcCols);
    if (threadIdx.x == 0) tc::mbar_init(&s_tcbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tcc.on = true;
    tcc.stage = smem + exec_stage_offset();
    tcc.tmem = s_tmem;
    tcc.bar = &s_tcbar;
    tcc.status = a.status;
    tcc.wait_ns = a.wait_limit_ns;
    c.tcc = &tcc;
  }
#endif
  c.scratch = reinterpret_cast<T*>(a.scratch) + (int64_t)blockIdx.x * a.scratch_stride;
  c.rows_max = a.trunc_rows;
  c.status = a.status;
  c.flops = 0;
  __shared__ unsigned long long s_prof[kProfEntries];
  if (threadIdx.x < kProfEntries) s_prof[threadIdx.x] = 0ULL;
  c.tprof = a.prof ? s_prof + kProfTrunc : nullptr;
  c.jacobi_tol = a.jacobi_tol > 0 ? a.jacobi_tol : (sizeof(T) == 4 ? 1e-6 : 1e-14);
  c.compress_at = a.compress_at >= 8 && a.compress_at <= kStackCols ? a.compress_at : kCompressAt;
  long long t_begin = 0, t_waited = 0;
  unsigned long long g_begin = 0, g_waited = 0;
  int64_t slot_cur = 0;
  volatile int32_t* abort_flag = (volatile int32_t*)a.status + 3;
  for (;;) {
    // claim the next queue slot and wait (bounded) until a finished task
    // pushes a ready task into it
    if (threadIdx.x == 0) {
      t_begin = clock64();
      if (a.trace) g_begin = gtimer();
      const int64_t k = (int64_t)atomicAdd(a.qctl, 1ULL);
      slot_cur = k;
      s_task = -1;
      if (k < a.ntotal && !*abort_flag) {
        unsigned long long v = ld_acquire_u64(a.queue + k);
        if (!v) {
          const uint64_t t0 = gtimer();
          for (;;) {
            __nanosleep(32);
            v = ld_acquire_u64(a.queue + k);
            if (v || *abort_flag) break;
            if (gtimer() - t0 > a.wait_limit_ns) {
              atomicCAS(a.status, 0, 5);
              atomicCAS(a.status + 1, -1, (int32_t)k);
              *abort_flag = 1;
              break;
            }
          }
        }
        if (v) {
          const unsigned long long code = v - 1ULL;
          s_prob = (int)(code >> 40);
          s_task = (int64_t)(code & ((1ULL << 40) - 1ULL));
        }
      }
      t_waited = clock64();
      if (a.trace) g_waited = gtimer();
    }
    __syncthreads();
    const int64_t ti = s_task;
    if (ti < 0) break;
    const ProbSched& P = a.probs[s_prob];
    if (threadIdx.x == 0) {  // the successor range streams in while the task runs
      const unsigned d = (unsigned)__cvta_generic_to_shared(s_succ);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(P.succ_ptr + ti) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 8u), "l"(P.succ_ptr + ti + 1) : "memory");
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int ttype = P.tasks[ti].type;
    if (ttype >= 0 && ttype < TK_NUM) {
      const Task t = P.tasks[ti];
      c.arena = reinterpret_cast<T*>(P.arena);
      c.ranks = P.ranks;
      c.piv = P.piv;
      c.terms = P.terms;
      c.pieces = P.pieces;
      c.eps = P.eps;
      c.nrhs_slot = P.nrhs_slot;
      c.nrhs = P.nrhs;
      c.term_p = P.term_p;
      c.alpha = P.alpha;
      run_task(c, t, smem);
    }
    if (threadIdx.x == 0) asm volatile("cp.async.wait_all;" ::: "memory");
    __threadfence();
    __syncthreads();
    // release the successors: the last predecessor to finish pushes a task
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const int64_t e0 = s_succ[0], e1 = s_succ[1];
      for (int64_t eb = e0; eb < e1; eb += 32) {
        const int64_t e = eb + lane;
        bool push = false;
        int32_t sx = 0;
        if (e < e1) {
          sx = P.succ_idx[e];
          if (sx < P.limit) push = atomicSub(P.indeg + sx, 1) == 1;
        }
        const unsigned mask = __ballot_sync(0xffffffffu, push);
        if (mask) {
          __threadfence();
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(a.qctl + 1, (unsigned long long)__popc(mask));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (push) {
            const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
            st_release_u64(a.queue + slot, ((((unsigned long long)s_prob) << 40) | (unsigned long long)sx) + 1ULL);
          }
        }
      }
    }
    if (threadIdx.x == 0) {
      if (a.trace) {
        unsigned long long* tr = a.trace + 4 * slot_cur;
        tr[0] = ((unsigned long long)s_prob << 40) | (unsigned long long)ti;
        tr[1] = g_begin;
        tr[2] = g_waited;
        tr[3] = gtimer();
      }
      if (a.prof) {
        const int k = (ttype >= 0 && ttype < TK_NUM) ? ttype : TK_NUM;
        long long t_end = clock64();
        s_prof[3 * k + 0] += 1ULL;
        s_prof[3 * k + 1] += (unsigned long long)(t_waited - t_begin);
        s_prof[3 * k + 2] += (unsigned long long)(t_end - t_waited);
      }
    }
    __syncthreads();
  }
#if HLU_EXEC_TC
  if (use_tc) {
    __syncthreads();
    if (tcc.broken && threadIdx.x == 0) {
      // a completion wait ran out: wait once more (bounded) for the MMAs in
      // flight before the accumulator columns are released
      const uint64_t t0 = gtimer();
      while (!tc::mbar_try_wait(tcc.bar, tcc.phase) && gtimer() - t0 < a.wait_limit_ns) {
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(tcc.tmem, tc::kTcCols);
  }
#else
  (void)use_tc;
#endif
  if (threadIdx.x == 0 && a.flops) atomicAdd(a.flops, c.flops);
  if (a.prof && threadIdx.x < kProfEntries) {
    unsigned long long v = s_prof[threadIdx.x];
    if (v) atomicAdd(a.prof + threadIdx.x, v);
  }
}

#if HLU_EXEC_TC
// One 64 x 64 tile product D = A B (A: 64 x K, ld 64; B: K x 64, ld K; D:
// 64 x 64, ld 64; column-major FP32) through the TF32 tensor-core pipeline of
// the executor, by one CTA: checks that path on its own.
__global__ void __launch_bounds__(NT, 1)
    tc_tile_kernel(const float* A, const float* B, float* D, int K, int32_t* status, unsigned long long wait_ns) {
  extern __shared__ __align__(1024) char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  if (threadIdx.x < 32) tc::tmem_alloc(&s_tmem, tc::kTcCols);
  if (threadIdx.x == 0) tc::mbar_init(&s_bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  TcCtl t;
  t.on = true;
  t.stage = smem;
  t.tmem = s_tmem;
  t.bar = &s_bar;
  t.status = status;
  t.wait_ns = wait_ns;
  float acc[4][4];
  acc_zero(acc);
  ProductCursor<float> cur{Mat<float>{A, 1, 64}, Mat<float>{B, 1, K}, 0, 64, 64, K, 0};
  tile_mma_seq_tc(acc, cur, &t);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) D[(tx * 4 + i) + (ty * 4 + j) * 64] = acc[i][j];
  __syncthreads();
  if (t.broken && threadIdx.x == 0) {
    const uint64_t t0 = gtimer();
    while (!tc::mbar_try_wait(t.bar, t.phase) && gtimer() - t0 < wait_ns) {
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(t.tmem, tc::kTcCols);
}

cudaError_t tc_tile_product(const float* A, const float* B, float* D, int K, int32_t* status,
                            unsigned long long wait_ns, cudaStream_t s) {
  note_launch();
  cudaError_t e = cudaFuncSetAttribute(tc_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc::kTcStageBytes);
  if (e != cudaSuccess) return e;
  tc_tile_kernel<<<1, NT, tc::kTcStageBytes, s>>>(A, B, D, K, status, wait_ns);
  return cudaGetLastError();
}
#endif

size_t exec_smem_bytes(int elem_size) {
#if HLU_EXEC_TC
  if (elem_size == 4) return exec_stage_offset() + tc::kTcStageBytes;
#endif
  return exec_smem_base(elem_size);
}

template <class T>
int exec_blocks_per_sm() {
  int nb = 0;
  size_t sm = exec_smem_bytes(sizeof(T));
  if (cudaFuncSetAttribute(exec_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, exec_kernel<T>, NT, sm) != cudaSuccess) return 0;
  return nb;
}

template <class T>
cudaError_t exec_launch(const ExecArgs& a, int grid, cudaStream_t s) {
  size_t sm = exec_smem_bytes(sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(exec_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  note_launch();
  exec_kernel<T><<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t exec_launch<float>(const ExecArgs&, int, cudaStream_t);
template int exec_blocks_per_sm<float>();
#if !HLU_EXEC_TC
template cudaError_t exec_launch<double>(const ExecArgs&, int, cudaStream_t);
template int exec_blocks_per_sm<double>();
#endif

#if HLU_EXEC_TC
}  // namespace tcx
#endif
}  // namespace hlu
