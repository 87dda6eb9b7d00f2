// Persistent task executor for the H-LU and H-solve DAGs (sm_103a).
//
// One launch runs a whole schedule.  Each CTA repeatedly takes the next task
// index from a global ticket counter (tickets follow a topological order), waits
// until every predecessor has published completion for the current epoch,
// runs the task with all its threads, and publishes its own completion.  A CTA
// only ever waits on tasks with smaller tickets, which were taken by CTAs that
// are already running, so the waits cannot deadlock.  Every wait is bounded by
// a wall-clock limit (%globaltimer); when it runs out the CTA records
// HLU_ERR_TIMEOUT and all CTAs drain without executing further work.
//
// Data written by one CTA and read by another goes through L2 (ld.global.cg /
// st.global.cg); completion flags use st.release / ld.acquire at gpu scope.
#include <cuda_runtime.h>

#include <cstdint>

#include "launch_count.h"

#include "exec.h"
#include "hlu_internal.h"

namespace hlu {

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
  return v.slot >= 0 ? __ldcg(c.ranks + v.slot) : v.cols;
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
template <class T>
__device__ __forceinline__ void acc_zero(T (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
}
template <class T>
__device__ void tile_mma(T (&acc)[4][4], const Mat<T>& A, int rlo, int mrows, const Mat<T>& B, int ncols, int K,
                         T* As, T* Bs) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int l0 = 0; l0 < K; l0 += KC) {
    const int kc = min(KC, K - l0);
    __syncthreads();
    if (A.rs == 1) {
      for (int e = tid; e < 64 * KC; e += NT) {
        int r = e & 63, kk = e >> 6;
        int ar = r - rlo;
        As[kk * 64 + r] = (kk < kc && ar >= 0 && ar < mrows) ? __ldcg(A.p + ar + (int64_t)(l0 + kk) * A.cs) : T(0);
      }
    } else {
      for (int e = tid; e < 64 * KC; e += NT) {
        int kk = e % KC, r = e / KC;
        int ar = r - rlo;
        As[kk * 64 + r] =
            (kk < kc && ar >= 0 && ar < mrows) ? __ldcg(A.p + (int64_t)ar * A.rs + (int64_t)(l0 + kk) * A.cs) : T(0);
      }
    }
    if (B.rs == 1) {
      for (int e = tid; e < 64 * KC; e += NT) {
        int kk = e % KC, cc = e / KC;
        Bs[kk * 64 + cc] = (kk < kc && cc < ncols) ? __ldcg(B.p + (l0 + kk) + (int64_t)cc * B.cs) : T(0);
      }
    } else {
      for (int e = tid; e < 64 * KC; e += NT) {
        int cc = e & 63, kk = e >> 6;
        Bs[kk * 64 + cc] =
            (kk < kc && cc < ncols) ? __ldcg(B.p + (int64_t)(l0 + kk) * B.rs + (int64_t)cc * B.cs) : T(0);
      }
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk * 64 + tx * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk * 64 + ty * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
  }
  __syncthreads();
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
  for (int idx = threadIdx.x; idx < n * n; idx += NT) A[idx] = ldv(c, t.a, idx % n, idx / n);
  if (t.type == TK_TRSM_L)
    for (int i = threadIdx.x; i < n; i += NT) perm[i] = __ldcg(c.piv + t.piv_off + i);
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
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31) / A[l + l * n];
        if (r0 == l) v0 = x;
        if (r1 == l) v1 = x;
        if (r0 > l && r0 < n) v0 -= A[l + r0 * n] * x;
        if (r1 > l && r1 < n) v1 -= A[l + r1 * n] * x;
      }
    } else {
      if (r0 < n) v0 = ldv(c, t.b, r0, j);
      if (r1 < n) v1 = ldv(c, t.b, r1, j);
      for (int l = n - 1; l >= 0; --l) {
        T x = __shfl_sync(0xffffffffu, l < 32 ? v0 : v1, l & 31) / A[l + l * n];
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
  T* Bs = As + 64 * KC;
  for (int i0 = 0; i0 < r; i0 += 64)
    for (int j0 = 0; j0 < k; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      tile_mma(acc, shift(matT(c, t.a), i0, 0), 0, min(64, r - i0), shift(mat(c, t.b), 0, j0), min(64, k - j0), m,
               As, Bs);
      tile_store(acc, c, t.c, i0, j0, min(64, r - i0), min(64, k - j0), T(1), true);
    }
  if (threadIdx.x == 0) c.flops += 2.0 * m * r * k;
}

// ---------------------------------------------------------------- ROWMV
// c (n x k) = [c] + sign * sum_t A_t B_t, A_t covering rows [roff, roff + rows).
template <class T>
__device__ void task_rowmv(Ctx<T>& c, const Task& t, char* smem) {
  const int n = t.c.rows, k = ncols(c, t.b);
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + 64 * KC;
  double fl = 0;
  for (int i0 = 0; i0 < n; i0 += 64)
    for (int j0 = 0; j0 < k; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      for (int q = 0; q < t.list_count; ++q) {
        const Term& tm = c.terms[t.list_begin + q];
        const int p = ncols(c, tm.A);
        // term rows [roff, roff + rows) intersected with tile rows [i0, i0 + 64)
        int lo = max(tm.roff, i0), hi = min(tm.roff + tm.A.rows, i0 + 64);
        if (hi <= lo || p == 0) continue;
        tile_mma(acc, shift(mat(c, tm.A), lo - tm.roff, 0), lo - i0, hi - lo, shift(mat(c, tm.B), 0, j0),
                 min(64, k - j0), p, As, Bs);
        fl += 2.0 * (hi - lo) * min(64, k - j0) * p;
      }
      tile_store(acc, c, t.c, i0, j0, min(64, n - i0), min(64, k - j0), T(t.sign), (t.flags & TF_OVERWRITE) != 0);
    }
  if (threadIdx.x == 0) {
    c.flops += fl;
    if (t.out_slot >= 0) __stcg(c.ranks + t.out_slot, k);
  }
}

// ---------------------------------------------------------------- RSOLVE
// One tile of a left-looking triangular solve: c -= sum_t A_t B_t, then the
// diagonal tile's triangle (L^-1 P or U^-1) in place.
template <class T>
__device__ void task_rsolve(Ctx<T>& c, const Task& t, char* smem) {
  if (t.list_count > 0) {
    Task r = t;
    r.type = TK_ROWMV;
    r.flags = 0;
    r.out_slot = -1;
    task_rowmv(c, r, smem);
    __threadfence_block();
    __syncthreads();
  }
  Task s = t;
  s.type = (t.flags & TF_UPPER) ? TK_TRSM_U : TK_TRSM_L;
  s.b = t.c;
  task_trsm(c, s, smem);
}

// ---------------------------------------------------------------- DADD
template <class T>
__device__ void task_dadd(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.c.rows, n = ncols(c, t.c), k = ncols(c, t.a);
  T* As = reinterpret_cast<T*>(smem);
  T* Bs = As + 64 * KC;
  for (int i0 = 0; i0 < m; i0 += 64)
    for (int j0 = 0; j0 < n; j0 += 64) {
      T acc[4][4];
      acc_zero(acc);
      if (k > 0)
        tile_mma(acc, shift(mat(c, t.a), i0, 0), 0, min(64, m - i0), shift(matT(c, t.b), 0, j0), min(64, n - j0), k,
                 As, Bs);
      tile_store(acc, c, t.c, i0, j0, min(64, m - i0), min(64, n - j0), T(t.sign), (t.flags & TF_OVERWRITE) != 0);
    }
  if (threadIdx.x == 0) c.flops += 2.0 * m * n * k;
}

// ---------------------------------------------------------------- TRUNC
// Householder QR of S (m x w, column-major, ld m, this CTA's private scratch)
// in place.  Every step uses the whole CTA: the norm is a block reduction and
// the reflector is applied to groups of 8 columns at once.
template <class T>
__device__ void house_qr(T* S, int m, int w, T* tau, T* red) {
  const int tmax = min(m, w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ T s_scale;
  __shared__ T s_d[8];
  __shared__ T s_part[NT / 32][8];
  for (int j = 0; j < tmax; ++j) {
    T* cj = S + (int64_t)j * m;
    T part = 0;
    for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
      T x = cj[i];
      part += x * x;
    }
    T s2 = block_sum(part, red);
    if (threadIdx.x == 0) {
      T alpha = cj[j];
      if (s2 == T(0)) {
        tau[j] = 0;
        s_scale = 0;
      } else {
        T nrm = sqrt(alpha * alpha + s2);
        T beta = alpha >= T(0) ? -nrm : nrm;
        s_scale = T(1) / (alpha - beta);
        tau[j] = (beta - alpha) / beta;
        cj[j] = beta;
      }
    }
    __syncthreads();
    const T sc = s_scale;
    if (sc != T(0))
      for (int i = j + 1 + threadIdx.x; i < m; i += NT) cj[i] *= sc;
    __syncthreads();
    const T tj = tau[j];
    if (tj == T(0)) continue;
    for (int c0 = j + 1; c0 < w; c0 += 8) {
      const int nc = min(8, w - c0);
      T d[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) d[q] = 0;
      for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
        T v = cj[i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nc) d[q] += v * S[i + (int64_t)(c0 + q) * m];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        T x = warp_sum(d[q]);
        if (lane == 0) s_part[warp][q] = x;
      }
      __syncthreads();
      if (threadIdx.x < nc) {
        T tot = S[j + (int64_t)(c0 + threadIdx.x) * m];
        for (int w8 = 0; w8 < NT / 32; ++w8) tot += s_part[w8][threadIdx.x];
        s_d[threadIdx.x] = tot * tj;
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
        T v = cj[i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nc) S[i + (int64_t)(c0 + q) * m] -= s_d[q] * v;
      }
      if (threadIdx.x < nc) S[j + (int64_t)(c0 + threadIdx.x) * m] -= s_d[threadIdx.x];
      __syncthreads();
    }
  }
}

// O (m x r, column-major, ld) <- Q O, Q = H_0 ... H_{t-1}; CTA-wide per
// reflector, output columns in groups of 8 (tall stacks).
template <class T>
__device__ void apply_q(const T* S, int m, int tmax, const T* tau, T* O, int64_t ld, int r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ T s_d[8];
  __shared__ T s_part[NT / 32][8];
  for (int j = tmax - 1; j >= 0; --j) {
    const T tj = tau[j];
    if (tj == T(0)) continue;
    const T* cj = S + (int64_t)j * m;
    for (int c0 = 0; c0 < r; c0 += 8) {
      const int nc = min(8, r - c0);
      T d[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) d[q] = 0;
      for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
        T v = cj[i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nc) d[q] += v * __ldcg(O + i + (int64_t)(c0 + q) * ld);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        T x = warp_sum(d[q]);
        if (lane == 0) s_part[warp][q] = x;
      }
      __syncthreads();
      if (threadIdx.x < nc) {
        T tot = __ldcg(O + j + (int64_t)(c0 + threadIdx.x) * ld);
        for (int w8 = 0; w8 < NT / 32; ++w8) tot += s_part[w8][threadIdx.x];
        s_d[threadIdx.x] = tot * tj;
      }
      __syncthreads();
      for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
        T v = cj[i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nc) {
            T* p = O + i + (int64_t)(c0 + q) * ld;
            __stcg(p, __ldcg(p) - s_d[q] * v);
          }
      }
      if (threadIdx.x < nc) {
        T* p = O + j + (int64_t)(c0 + threadIdx.x) * ld;
        __stcg(p, __ldcg(p) - s_d[threadIdx.x]);
      }
      __syncthreads();
    }
  }
}

// Householder QR of S (m x w, column-major, ld m) by one warp, no block
// barriers: lanes stride over rows, columns are updated one after another.
template <class T>
__device__ void house_qr_warp(T* S, int m, int w, T* tau) {
  const int lane = threadIdx.x & 31;
  const int tmax = min(m, w);
  for (int j = 0; j < tmax; ++j) {
    T* cj = S + (int64_t)j * m;
    T s2 = 0;
    for (int i = j + 1 + lane; i < m; i += 32) {
      T x = cj[i];
      s2 += x * x;
    }
    s2 = warp_sum(s2);
    const T alpha = cj[j];
    __syncwarp();
    if (s2 == T(0)) {
      if (lane == 0) tau[j] = 0;
      __syncwarp();
      continue;
    }
    const T nrm = sqrt(alpha * alpha + s2);
    const T beta = alpha >= T(0) ? -nrm : nrm;
    const T sc = T(1) / (alpha - beta);
    const T tj = (beta - alpha) / beta;
    for (int i = j + 1 + lane; i < m; i += 32) cj[i] *= sc;
    if (lane == 0) {
      cj[j] = beta;
      tau[j] = tj;
    }
    __syncwarp();
    for (int cc = j + 1; cc < w; ++cc) {
      T* col = S + (int64_t)cc * m;
      T d = 0;
      for (int i = j + 1 + lane; i < m; i += 32) d += cj[i] * col[i];
      d = warp_sum(d);
      d = (d + col[j]) * tj;
      __syncwarp();
      for (int i = j + 1 + lane; i < m; i += 32) col[i] -= d * cj[i];
      if (lane == 0) col[j] -= d;
      __syncwarp();
    }
  }
}

// O (m x r, column-major, ld) <- Q O, one warp per column (short stacks).
template <class T>
__device__ void apply_q_warp(const T* S, int m, int tmax, const T* tau, T* O, int64_t ld, int r, int warp0,
                             int nwarps) {
  const int warp = (threadIdx.x >> 5) - warp0, lane = threadIdx.x & 31;
  if (warp < 0 || warp >= nwarps) return;
  for (int cc = warp; cc < r; cc += nwarps) {
    T* col = O + (int64_t)cc * ld;
    for (int j = tmax - 1; j >= 0; --j) {
      const T tj = tau[j];
      if (tj == T(0)) continue;
      const T* cj = S + (int64_t)j * m;
      T d = 0;
      for (int i = j + 1 + lane; i < m; i += 32) d += cj[i] * __ldcg(col + i);
      d = warp_sum(d);
      d = (d + __ldcg(col + j)) * tj;
      __syncwarp();
      for (int i = j + 1 + lane; i < m; i += 32) __stcg(col + i, __ldcg(col + i) - d * cj[i]);
      if (lane == 0) __stcg(col + j, __ldcg(col + j) - d);
      __syncwarp();
    }
  }
}

// stacked factors up to this many rows use the warp-level QR and apply
constexpr int kWarpQrRows = 768;
constexpr int kStackCols = kTruncStack;
// a stack wider than this is compressed before the next piece is added
// (Jacobi cost grows with the cube of the width); rank cap 32 + a 64-wide
// piece still fit the stack
constexpr int kCompressAt = 48;

// Truncated SVD of the stacked factors SX (m x W) and SY (n x W) in compute
// type TC: QR of both, one-sided Jacobi SVD of the core R_x R_y^T, keep
// s_i > eps s_1 (at most cap); X <- Q_x U_r S_r and Y <- Q_y V_r are written
// to OX (ld ox) and OY (ld oy).  Workspace: tauX, tauY, sv (kStackCols each)
// and G, V (kStackCols^2 each), in shared or global memory.  Returns r (the
// same in every thread); *fro receives ||X Y^T||_F.
template <class TC>
__device__ int compress_core(TC* SX, TC* SY, int m, int n, int W, int cap, double eps, TC* tauX, TC* tauY,
                             TC* sv, TC* G, TC* V, TC* OX, int64_t ox, TC* OY, int64_t oy, int32_t* cap_hits,
                             double* flops, double* fro) {
  __shared__ int s_rot;
  __shared__ int s_r;
  __shared__ int s_ord[kStackCols];
  __shared__ TC s_red[NT / 32];
  __shared__ double s_fro;
  __shared__ float s_off, s_prev;
  const bool small = max(m, n) <= kWarpQrRows;
  if (small) {
    const int wq = threadIdx.x >> 5;
    if (wq == 0) house_qr_warp(SX, m, W, tauX);
    if (wq == 1) house_qr_warp(SY, n, W, tauY);
    __syncthreads();
  } else {
    house_qr(SX, m, W, tauX, s_red);
    house_qr(SY, n, W, tauY, s_red);
  }
  const int p = min(m, W), q = min(n, W);
  // the core is accumulated in FP64: the target and its updates cancel inside
  // this sum, and FP32 accumulation there costs the truncation its accuracy
  for (int idx = threadIdx.x; idx < p * q; idx += NT) {
    int i = idx % p, j = idx / p;
    double acc = 0;
    for (int l = max(i, j); l < W; ++l) acc += (double)SX[i + (int64_t)l * m] * (double)SY[j + (int64_t)l * n];
    G[i + j * p] = (TC)acc;
  }
  for (int idx = threadIdx.x; idx < q * q; idx += NT) V[idx] = (idx % q == idx / q) ? TC(1) : TC(0);
  __syncthreads();
  // stop when every pair is orthogonal to tol, or when a sweep no longer
  // reduces the largest off-diagonal measure while it is already small (the
  // rounding floor)
  const TC tol = sizeof(TC) == 4 ? TC(1e-6) : TC(1e-14);
  const int qq = q + (q & 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_prev = 3.0e38f;
  for (int sweep = 0; sweep < 20 && qq > 1; ++sweep) {
    if (threadIdx.x == 0) {
      s_rot = 0;
      s_off = 0.0f;
    }
    __syncthreads();
    for (int rd = 0; rd < qq - 1; ++rd) {
      for (int k = warp; k < qq / 2; k += NT / 32) {
        int pa = k == 0 ? 0 : ((k - 1 + rd) % (qq - 1)) + 1;
        int kb = qq - 1 - k;
        int pb = kb == 0 ? 0 : ((kb - 1 + rd) % (qq - 1)) + 1;
        int a = min(pa, pb), b = max(pa, pb);
        if (b >= q) continue;
        TC al = 0, be = 0, ga = 0;
        for (int i = lane; i < p; i += 32) {
          TC x = G[i + a * p], y = G[i + b * p];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == TC(0)) continue;
        const TC ratio = fabs(ga) / sqrt(al * be);
        if (lane == 0) atomicMax(reinterpret_cast<int*>(&s_off), __float_as_int((float)ratio));
        if (ratio <= tol) continue;
        TC zeta = (be - al) / (TC(2) * ga);
        TC tt = (zeta >= TC(0) ? TC(1) : TC(-1)) / (fabs(zeta) + sqrt(TC(1) + zeta * zeta));
        TC cs = TC(1) / sqrt(TC(1) + tt * tt), sn = cs * tt;
        for (int i = lane; i < p; i += 32) {
          TC x = G[i + a * p], y = G[i + b * p];
          G[i + a * p] = cs * x - sn * y;
          G[i + b * p] = sn * x + cs * y;
        }
        for (int i = lane; i < q; i += 32) {
          TC x = V[i + a * q], y = V[i + b * q];
          V[i + a * q] = cs * x - sn * y;
          V[i + b * q] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
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
  for (int j = warp; j < q; j += NT / 32) {
    TC acc = 0;
    for (int i = lane; i < p; i += 32) acc += G[i + j * p] * G[i + j * p];
    acc = warp_sum(acc);
    if (lane == 0) sv[j] = sqrt(acc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f2 = 0;
    for (int j = 0; j < q; ++j) {
      s_ord[j] = j;
      f2 += (double)sv[j] * (double)sv[j];
    }
    s_fro = sqrt(f2);
    for (int j = 1; j < q; ++j) {  // stable insertion sort, descending
      int x = s_ord[j], i = j - 1;
      while (i >= 0 && sv[s_ord[i]] < sv[x]) {
        s_ord[i + 1] = s_ord[i];
        --i;
      }
      s_ord[i + 1] = x;
    }
    TC smax = q ? sv[s_ord[0]] : TC(0);
    int r = 0;
    if (smax > TC(0))
      while (r < q && sv[s_ord[r]] > TC(eps) * smax) ++r;
    if (r > cap) {
      r = cap;
      atomicAdd(cap_hits, 1);
    }
    s_r = r;
    *flops += 2.0 * (m + n) * W * W + 21.0 * (double)q * q * q + 2.0 * (m + n) * W * r;
  }
  __syncthreads();
  const int r = s_r;
  *fro = s_fro;
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) {
    int i = (int)(idx % m), j = (int)(idx / m);
    __stcg(OX + i + (int64_t)j * ox, i < p ? G[i + s_ord[j] * p] : TC(0));
  }
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) {
    int i = (int)(idx % n), j = (int)(idx / n);
    __stcg(OY + i + (int64_t)j * oy, i < q ? V[i + s_ord[j] * q] : TC(0));
  }
  __syncthreads();
  if (small) {
    apply_q_warp(SX, m, min(m, W), tauX, OX, ox, r, 0, NT / 64);
    apply_q_warp(SY, n, min(n, W), tauY, OY, oy, r, NT / 64, NT / 64);
  } else {
    apply_q(SX, m, min(m, W), tauX, OX, ox, r);
    apply_q(SY, n, min(n, W), tauY, OY, oy, r);
  }
  __syncthreads();
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
  __shared__ double s_nx, s_ny;
  __shared__ TC s_rx[NT / 32];
  double worst = 0;
  int W = 0;
  int32_t* cap_hits = c.status + 2;
  auto stack_norm = [&](int w_) -> double {
    TC px = 0, py = 0;
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * w_; idx += NT) px += SX[idx] * SX[idx];
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * w_; idx += NT) py += SY[idx] * SY[idx];
    TC sx = block_sum(px, s_rx);
    TC sy = block_sum(py, s_rx);
    return sqrt((double)sx) * sqrt((double)sy);
  };
  for (int q = 0; q < t.list_count; ++q) {
    const Piece& P = c.pieces[t.list_begin + q];
    const int w = ncols(c, P.X);
    if (w == 0) continue;
    if (W > 0 && W + w > kCompressAt) {
      const double in = stack_norm(W);
      double fro = 0;
      const int r = compress_core(SX, SY, m, n, W, t.cap, c.eps, tauX, tauY, sv, G, V, OX, m, OY, n, cap_hits,
                                  &c.flops, &fro);
      if (fro > 0) worst = fmax(worst, in / fro);
      for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) SX[idx] = __ldcg(OX + idx);
      for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) SY[idx] = __ldcg(OY + idx);
      W = r;
      __syncthreads();
    }
    const TC sg = TC(P.sign);
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * w; idx += NT) SX[(int64_t)W * m + idx] = TC(0);
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * w; idx += NT) SY[(int64_t)W * n + idx] = TC(0);
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)P.X.rows * w; idx += NT) {
      int i = (int)(idx % P.X.rows), j = (int)(idx / P.X.rows);
      SX[(P.xoff + i) + (int64_t)(W + j) * m] = sg * TC(ldv(c, P.X, i, j));
    }
    for (int64_t idx = threadIdx.x; idx < (int64_t)P.Y.rows * w; idx += NT) {
      int i = (int)(idx % P.Y.rows), j = (int)(idx / P.Y.rows);
      SY[(P.yoff + i) + (int64_t)(W + j) * n] = TC(ldv(c, P.Y, i, j));
    }
    W += w;
    __syncthreads();
  }
  int r = 0;
  if (W > 0) {
    const double in = stack_norm(W);
    double fro = 0;
    r = compress_core(SX, SY, m, n, W, t.cap, c.eps, tauX, tauY, sv, G, V, OX, m, OY, n, cap_hits, &c.flops, &fro);
    if (fro > 0) worst = fmax(worst, in / fro);
  }
  *ratio = worst;
  (void)s_nx;
  (void)s_ny;
  return r;
}

// (a, b) <- truncation of sum_pieces sign X Y^T (stack, compress, store).
template <class T>
__device__ void task_trunc(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.a.rows, n = t.b.rows;
  if (m == 0 || n == 0) {
    if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, 0);
    return;
  }
  const int64_t R = c.rows_max;
  T* SX = c.scratch;
  T* SY = SX + R * kStackCols;
  T* OX = SY + R * kStackCols;
  T* OY = OX + R * 32;
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

// ---------------------------------------------------------------- executor
template <class T>
__global__ void __launch_bounds__(NT, 2) exec_kernel(const __grid_constant__ ExecArgs a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int64_t s_task;
  __shared__ int s_skip;
  __shared__ int s_prob;
  Ctx<T> c;
  c.scratch = reinterpret_cast<T*>(a.scratch) + (int64_t)blockIdx.x * a.scratch_stride;
  c.rows_max = a.trunc_rows;
  c.status = a.status;
  c.flops = 0;
  __shared__ unsigned long long s_prof[TK_NUM + 1][3];  // count, wait cycles, run cycles
  if (threadIdx.x < (TK_NUM + 1) * 3) (&s_prof[0][0])[threadIdx.x] = 0ULL;
  long long t_begin = 0, t_waited = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t tk = (int64_t)atomicAdd(a.ticket, 1ULL);
      if (tk >= a.ntotal) {
        s_task = -1;
      } else if (a.order) {
        const int64_t code = a.order[tk];
        s_prob = (int)(code >> 40);
        s_task = code & ((int64_t(1) << 40) - 1);
      } else {
        s_prob = 0;
        s_task = tk;
      }
      t_begin = clock64();
    }
    __syncthreads();
    const int64_t ti = s_task;
    if (ti < 0) break;
    const ProbSched& P = a.probs[s_prob];
    // wait for the predecessors (lanes of warp 0 in parallel, bounded)
    if (threadIdx.x < 32) {
      int bad = 0;
      const int64_t e0 = P.pred_ptr[ti], e1 = P.pred_ptr[ti + 1];
      for (int64_t e = e0 + threadIdx.x; e < e1; e += 32) {
        const int32_t* flag = P.done + P.pred_idx[e];
        if (ld_acquire(flag) == P.epoch) continue;
        const uint64_t t0 = gtimer();
        for (;;) {
          if (ld_acquire(flag) == P.epoch) break;
          if (*((volatile int32_t*)a.status + 3)) {
            bad = 1;
            break;
          }
          if (gtimer() - t0 > a.wait_limit_ns) {
            atomicCAS(a.status, 0, 5);
            atomicCAS(a.status + 1, -1, (int32_t)ti);
            *((volatile int32_t*)a.status + 3) = 1;
            bad = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      bad = __any_sync(0xffffffffu, bad);
      if (threadIdx.x == 0) s_skip = bad || *((volatile int32_t*)a.status + 3);
      __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) t_waited = clock64();
    const int ttype = P.tasks[ti].type;
    if (!s_skip && ttype >= 0 && ttype < TK_NUM) {
      const Task t = P.tasks[ti];
      c.arena = reinterpret_cast<T*>(P.arena);
      c.ranks = P.ranks;
      c.piv = P.piv;
      c.terms = P.terms;
      c.pieces = P.pieces;
      c.eps = P.eps;
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
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      st_release(P.done + ti, P.epoch);
      if (a.prof) {
        const int k = (ttype >= 0 && ttype < TK_NUM) ? ttype : TK_NUM;
        long long t_end = clock64();
        s_prof[k][0] += 1ULL;
        s_prof[k][1] += (unsigned long long)(t_waited - t_begin);
        s_prof[k][2] += (unsigned long long)(t_end - t_waited);
      }
    }
  }
  if (threadIdx.x == 0 && a.flops) atomicAdd(a.flops, c.flops);
  if (a.prof && threadIdx.x < (TK_NUM + 1) * 3) {
    unsigned long long v = (&s_prof[0][0])[threadIdx.x];
    if (v) atomicAdd(a.prof + threadIdx.x, v);
  }
}

size_t exec_smem_bytes(int elem_size) {
  // max over task kinds: TRUNC (3 stack-wide vectors + G + V), GETRF/TRSM
  // (64 x 64 + 64 ints), staged GEMM chunks (2 x 64 x KC)
  size_t trunc = (size_t)elem_size * (3 * kTruncStack + 2 * kTruncStack * kTruncStack);
  size_t lu = (size_t)elem_size * 64 * 64 + 64 * sizeof(int);
  size_t gemm = (size_t)elem_size * 2 * 64 * KC;
  size_t m = trunc > lu ? trunc : lu;
  return m > gemm ? m : gemm;
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
template cudaError_t exec_launch<double>(const ExecArgs&, int, cudaStream_t);
template int exec_blocks_per_sm<float>();
template int exec_blocks_per_sm<double>();

}  // namespace hlu
