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
  int64_t scratch_half;  // elements of the X half of the per-CTA scratch
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

// ---------------------------------------------------------------- leaf TRSM
// One thread per right-hand-side column, triangle in shared memory.
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
  T v[64];
  for (int j = threadIdx.x; j < k; j += NT) {
    if (t.type == TK_TRSM_L) {
      for (int i = 0; i < n; ++i) v[i] = ldv(c, t.b, perm[i], j);
      for (int i = 0; i < n; ++i) {
        T s = v[i];
        for (int l = 0; l < i; ++l) s -= A[i + l * n] * v[l];
        v[i] = s;
      }
    } else if (t.type == TK_TRSM_UT) {
      for (int i = 0; i < n; ++i) v[i] = ldv(c, t.b, i, j);
      for (int i = 0; i < n; ++i) {
        T s = v[i];
        for (int l = 0; l < i; ++l) s -= A[l + i * n] * v[l];
        v[i] = s / A[i + i * n];
      }
    } else {
      for (int i = 0; i < n; ++i) v[i] = ldv(c, t.b, i, j);
      for (int i = n - 1; i >= 0; --i) {
        T s = v[i];
        for (int l = i + 1; l < n; ++l) s -= A[i + l * n] * v[l];
        v[i] = s / A[i + i * n];
      }
    }
    for (int i = 0; i < n; ++i) stv(c, t.b, i, j, v[i]);
  }
  if (threadIdx.x == 0) c.flops += (double)n * n * k;
}

// ---------------------------------------------------------------- PROJ
// c (r x k) = a^T b, a: m x r, b: m x k.  Threads split outputs x row groups.
template <class T>
__device__ void task_proj(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.a.rows, r = ncols(c, t.a), k = ncols(c, t.b);
  const int no = r * k;
  T* part = reinterpret_cast<T*>(smem);
  if (no == 0) return;
  if (no >= NT) {
    for (int o = threadIdx.x; o < no; o += NT) {
      int i = o % r, j = o / r;
      T s = 0;
      for (int l = 0; l < m; ++l) s += ldv(c, t.a, l, i) * ldv(c, t.b, l, j);
      stv(c, t.c, i, j, s);
    }
  } else {
    const int G = NT / no;
    const int o = threadIdx.x % no, g = threadIdx.x / no;
    T s = 0;
    if (g < G) {
      int i = o % r, j = o / r;
      for (int l = g; l < m; l += G) s += ldv(c, t.a, l, i) * ldv(c, t.b, l, j);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < no) {
      T tot = 0;
      for (int q = 0; q < G; ++q) tot += part[threadIdx.x + q * no];
      stv(c, t.c, threadIdx.x % r, threadIdx.x / r, tot);
    }
  }
  if (threadIdx.x == 0) c.flops += 2.0 * m * r * k;
}

// ---------------------------------------------------------------- ROWMV
// c (n x k) = [c] + sign * sum_t A_t B_t.
template <class T>
__device__ void task_rowmv(Ctx<T>& c, const Task& t) {
  const int n = t.c.rows, k = ncols(c, t.b);
  const int no = n * k;
  const T sg = T(t.sign);
  double fl = 0;
  for (int o = threadIdx.x; o < no; o += NT) {
    int i = o % n, j = o / n;
    T acc = 0;
    for (int q = 0; q < t.list_count; ++q) {
      const Term& tm = c.terms[t.list_begin + q];
      const int ii = i - tm.roff;
      if (ii < 0 || ii >= tm.A.rows) continue;
      const int p = ncols(c, tm.A);
      for (int l = 0; l < p; ++l) acc += ldv(c, tm.A, ii, l) * ldv(c, tm.B, l, j);
    }
    T base = (t.flags & TF_OVERWRITE) ? T(0) : ldv(c, t.c, i, j);
    stv(c, t.c, i, j, base + sg * acc);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < t.list_count; ++q) {
      const Term& tm = c.terms[t.list_begin + q];
      fl += 2.0 * tm.A.rows * k * ncols(c, tm.A);
    }
    c.flops += fl;
    if (t.out_slot >= 0) __stcg(c.ranks + t.out_slot, k);
  }
}

// ---------------------------------------------------------------- DADD
template <class T>
__device__ void task_dadd(Ctx<T>& c, const Task& t) {
  const int m = t.c.rows, n = ncols(c, t.c), k = ncols(c, t.a);
  const T sg = T(t.sign);
  for (int o = threadIdx.x; o < m * n; o += NT) {
    int i = o % m, j = o / m;
    T s = 0;
    for (int l = 0; l < k; ++l) s += ldv(c, t.a, i, l) * ldv(c, t.b, j, l);
    T base = (t.flags & TF_OVERWRITE) ? T(0) : ldv(c, t.c, i, j);
    stv(c, t.c, i, j, base + sg * s);
  }
  if (threadIdx.x == 0) c.flops += 2.0 * m * n * k;
}

// ---------------------------------------------------------------- TRUNC
// Householder QR of S (m x w, column-major, ld m) in place, by the whole CTA.
template <class T>
__device__ void house_qr(T* S, int m, int w, T* tau, T* red) {
  const int tmax = min(m, w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ T s_scale;
  for (int j = 0; j < tmax; ++j) {
    T* cj = S + (int64_t)j * m;
    T part = 0;
    for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
      T x = __ldcg(cj + i);
      part += x * x;
    }
    T s2 = block_sum(part, red);
    if (threadIdx.x == 0) {
      T alpha = __ldcg(cj + j);
      if (s2 == T(0)) {
        tau[j] = 0;
        s_scale = 0;
      } else {
        T nrm = sqrt(alpha * alpha + s2);
        T beta = alpha >= T(0) ? -nrm : nrm;
        s_scale = T(1) / (alpha - beta);
        tau[j] = (beta - alpha) / beta;
        __stcg(cj + j, beta);
      }
    }
    __syncthreads();
    const T sc = s_scale;
    if (sc != T(0))
      for (int i = j + 1 + threadIdx.x; i < m; i += NT) __stcg(cj + i, __ldcg(cj + i) * sc);
    __syncthreads();
    const T tj = tau[j];
    if (tj != T(0)) {
      for (int cc = j + 1 + warp; cc < w; cc += NT / 32) {
        T* col = S + (int64_t)cc * m;
        T d = 0;
        for (int i = j + 1 + lane; i < m; i += 32) d += __ldcg(cj + i) * __ldcg(col + i);
        d = warp_sum(d);
        d = (d + __ldcg(col + j)) * tj;
        if (lane == 0) __stcg(col + j, __ldcg(col + j) - d);
        for (int i = j + 1 + lane; i < m; i += 32) __stcg(col + i, __ldcg(col + i) - d * __ldcg(cj + i));
      }
    }
    __syncthreads();
  }
}

// out (column-major view, m x r) <- Q out, Q = H_0 ... H_{t-1}; one warp per column.
template <class T>
__device__ void apply_q(const Ctx<T>& c, const T* S, int m, int tmax, const T* tau, const View& out,
                        int r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int cc = warp; cc < r; cc += NT / 32) {
    for (int j = tmax - 1; j >= 0; --j) {
      const T tj = tau[j];
      if (tj == T(0)) continue;
      const T* cj = S + (int64_t)j * m;
      T d = 0;
      for (int i = j + 1 + lane; i < m; i += 32) d += __ldcg(cj + i) * ldv(c, out, i, cc);
      d = warp_sum(d);
      d = (d + ldv(c, out, j, cc)) * tj;
      __syncwarp();
      if (lane == 0) stv(c, out, j, cc, ldv(c, out, j, cc) - d);
      for (int i = j + 1 + lane; i < m; i += 32) stv(c, out, i, cc, ldv(c, out, i, cc) - d * __ldcg(cj + i));
      __syncwarp();
    }
  }
}

template <class T>
__device__ void task_trunc(Ctx<T>& c, const Task& t, char* smem) {
  const int m = t.a.rows, n = t.b.rows;
  __shared__ int s_W;
  __shared__ int s_colstart[64];
  __shared__ int s_rot;
  __shared__ int s_r;
  __shared__ int s_ord[64];
  __shared__ T s_red[NT / 32];
  if (threadIdx.x == 0) {
    int W = 0;
    for (int q = 0; q < t.list_count && q < 64; ++q) {
      s_colstart[q] = W;
      W += ncols(c, c.pieces[t.list_begin + q].X);
    }
    s_W = W;
  }
  __syncthreads();
  const int W = s_W;
  if (W == 0 || m == 0 || n == 0) {
    if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, 0);
    return;
  }
  T* SX = c.scratch;
  T* SY = c.scratch + c.scratch_half;
  // stack the pieces (zero outside each piece's rows)
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * W; idx += NT) __stcg(SX + idx, T(0));
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * W; idx += NT) __stcg(SY + idx, T(0));
  __syncthreads();
  for (int q = 0; q < t.list_count; ++q) {
    const Piece& P = c.pieces[t.list_begin + q];
    const int w = ncols(c, P.X);
    const int c0 = s_colstart[q];
    const T sg = T(P.sign);
    for (int64_t idx = threadIdx.x; idx < (int64_t)P.X.rows * w; idx += NT) {
      int i = (int)(idx % P.X.rows), j = (int)(idx / P.X.rows);
      __stcg(SX + (P.xoff + i) + (int64_t)(c0 + j) * m, sg * ldv(c, P.X, i, j));
    }
    for (int64_t idx = threadIdx.x; idx < (int64_t)P.Y.rows * w; idx += NT) {
      int i = (int)(idx % P.Y.rows), j = (int)(idx / P.Y.rows);
      __stcg(SY + (P.yoff + i) + (int64_t)(c0 + j) * n, ldv(c, P.Y, i, j));
    }
  }
  __syncthreads();
  T* tauX = reinterpret_cast<T*>(smem);
  T* tauY = tauX + 64;
  T* G = tauY + 64;           // p x q
  T* V = G + 64 * 64;         // q x q
  T* sv = V + 64 * 64;        // q
  house_qr(SX, m, W, tauX, s_red);
  house_qr(SY, n, W, tauY, s_red);
  const int p = min(m, W), q = min(n, W);
  // core G = R_x R_y^T
  for (int idx = threadIdx.x; idx < p * q; idx += NT) {
    int i = idx % p, j = idx / p;
    T s = 0;
    for (int l = max(i, j); l < W; ++l) s += __ldcg(SX + i + (int64_t)l * m) * __ldcg(SY + j + (int64_t)l * n);
    G[i + j * p] = s;
  }
  for (int idx = threadIdx.x; idx < q * q; idx += NT) V[idx] = (idx % q == idx / q) ? T(1) : T(0);
  __syncthreads();
  // one-sided Jacobi on the columns of G, round-robin pairing
  const T tol = sizeof(T) == 4 ? T(1e-5) : T(1e-13);
  const int qq = q + (q & 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int sweep = 0; sweep < 24 && qq > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int rd = 0; rd < qq - 1; ++rd) {
      for (int k = warp; k < qq / 2; k += NT / 32) {
        int pa = k == 0 ? 0 : ((k - 1 + rd) % (qq - 1)) + 1;
        int kb = qq - 1 - k;
        int pb = kb == 0 ? 0 : ((kb - 1 + rd) % (qq - 1)) + 1;
        int a = min(pa, pb), b = max(pa, pb);
        if (b >= q) continue;
        T al = 0, be = 0, ga = 0;
        for (int i = lane; i < p; i += 32) {
          T x = G[i + a * p], y = G[i + b * p];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == T(0) || fabs(ga) <= tol * sqrt(al * be)) continue;
        T zeta = (be - al) / (T(2) * ga);
        T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
        for (int i = lane; i < p; i += 32) {
          T x = G[i + a * p], y = G[i + b * p];
          G[i + a * p] = cs * x - sn * y;
          G[i + b * p] = sn * x + cs * y;
        }
        for (int i = lane; i < q; i += 32) {
          T x = V[i + a * q], y = V[i + b * q];
          V[i + a * q] = cs * x - sn * y;
          V[i + b * q] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  for (int j = warp; j < q; j += NT / 32) {
    T s = 0;
    for (int i = lane; i < p; i += 32) s += G[i + j * p] * G[i + j * p];
    s = warp_sum(s);
    if (lane == 0) sv[j] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < q; ++j) s_ord[j] = j;
    for (int j = 1; j < q; ++j) {  // stable insertion sort, descending
      int x = s_ord[j], i = j - 1;
      while (i >= 0 && sv[s_ord[i]] < sv[x]) {
        s_ord[i + 1] = s_ord[i];
        --i;
      }
      s_ord[i + 1] = x;
    }
    T smax = q ? sv[s_ord[0]] : T(0);
    int r = 0;
    if (smax > T(0))
      while (r < q && sv[s_ord[r]] > T(c.eps) * smax) ++r;
    if (r > t.cap) {
      r = t.cap;
      atomicAdd(c.status + 2, 1);
    }
    s_r = r;
    c.flops += 2.0 * (m + n) * W * W + 21.0 * (double)q * q * q + 2.0 * (m + n) * W * r;
  }
  __syncthreads();
  const int r = s_r;
  for (int64_t idx = threadIdx.x; idx < (int64_t)m * r; idx += NT) {
    int i = (int)(idx % m), j = (int)(idx / m);
    stv(c, t.a, i, j, i < p ? G[i + s_ord[j] * p] : T(0));
  }
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * r; idx += NT) {
    int i = (int)(idx % n), j = (int)(idx / n);
    stv(c, t.b, i, j, i < q ? V[i + s_ord[j] * q] : T(0));
  }
  __syncthreads();
  apply_q(c, SX, m, min(m, W), tauX, t.a, r);
  apply_q(c, SY, n, min(n, W), tauY, t.b, r);
  __syncthreads();
  if (threadIdx.x == 0) __stcg(c.ranks + t.out_slot, r);
}

// ---------------------------------------------------------------- executor
template <class T>
__global__ void __launch_bounds__(NT, 2) exec_kernel(ExecArgs a) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int64_t s_task;
  __shared__ int s_skip;
  Ctx<T> c;
  c.terms = a.terms;
  c.pieces = a.pieces;
  c.scratch = reinterpret_cast<T*>(a.scratch) + (int64_t)blockIdx.x * a.scratch_stride;
  c.scratch_half = a.scratch_stride / 2;
  c.eps = a.eps;
  c.status = a.status;
  c.flops = 0;
  for (;;) {
    if (threadIdx.x == 0) s_task = (int64_t)atomicAdd(a.ticket, 1ULL);
    __syncthreads();
    const int64_t ti = s_task;
    if (ti >= a.ntasks) break;
    // wait for the predecessors (lanes of warp 0 in parallel, bounded)
    if (threadIdx.x < 32) {
      int bad = 0;
      const int64_t e0 = a.pred_ptr[ti], e1 = a.pred_ptr[ti + 1];
      for (int64_t e = e0 + threadIdx.x; e < e1; e += 32) {
        const int32_t* flag = a.done + a.pred_idx[e];
        if (ld_acquire(flag) == a.epoch) continue;
        const uint64_t t0 = gtimer();
        for (;;) {
          if (ld_acquire(flag) == a.epoch) break;
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
    if (!s_skip && a.tasks[ti].type >= 0 && a.tasks[ti].type < TK_NUM) {
      const Task t = a.tasks[ti];
      c.arena = reinterpret_cast<T*>(a.arenas[t.prob]);
      c.ranks = a.ranks[t.prob];
      c.piv = a.pivs[t.prob];
      switch (t.type) {
        case TK_GETRF: task_getrf(c, t, smem); break;
        case TK_TRSM_L:
        case TK_TRSM_UT:
        case TK_TRSM_U: task_trsm(c, t, smem); break;
        case TK_PROJ: task_proj(c, t, smem); break;
        case TK_ROWMV: task_rowmv(c, t); break;
        case TK_TRUNC: task_trunc(c, t, smem); break;
        case TK_DADD: task_dadd(c, t); break;
        default: break;
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) st_release(a.done + ti, a.epoch);
  }
  if (threadIdx.x == 0 && a.flops) atomicAdd(a.flops, c.flops);
}

size_t exec_smem_bytes(int elem_size) {
  // max over task kinds: GETRF/TRSM 64x64 + 64 ints; TRUNC 2*64 + 2*64*64 + 64
  size_t trunc = (size_t)elem_size * (128 + 2 * 64 * 64 + 64);
  size_t lu = (size_t)elem_size * 64 * 64 + 64 * sizeof(int);
  size_t proj = (size_t)elem_size * NT;
  size_t m = trunc > lu ? trunc : lu;
  return m > proj ? m : proj;
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
  exec_kernel<T><<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t exec_launch<float>(const ExecArgs&, int, cudaStream_t);
template cudaError_t exec_launch<double>(const ExecArgs&, int, cudaStream_t);
template int exec_blocks_per_sm<float>();
template int exec_blocks_per_sm<double>();

}  // namespace hlu
