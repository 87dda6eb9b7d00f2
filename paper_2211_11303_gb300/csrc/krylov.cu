// FP64 Krylov kernels: CSR SpMV (multi-column), CGS2 Gram-Schmidt pieces,
// Givens rotations and the final least-squares update of restarted flexible
// GMRES (Sec. 4, Example 1), plus the permute-and-cast kernels that move FP64
// vectors in and out of the triangular solves of Algorithm 1 step III.
#include <cuda_runtime.h>

#include <cstdint>

#include "launch_count.h"

#include "krylov.h"

namespace hlu {

static int gridn(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

// y[:, r] = A x[:, r]; one warp per row, lanes over the row's entries
__global__ void k_spmv(int64_t N, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                       int64_t ldx, double* y, int64_t ldy, int nrhs) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < N; row += nw) {
    int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
    for (int r = 0; r < nrhs; ++r) {
      double s = 0;
      for (int64_t e = e0 + lane; e < e1; e += 32) s += val[e] * x[col[e] + r * ldx];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) y[row + r * ldy] = s;
    }
  }
}

cudaError_t spmv(const int64_t* rowptr, const int32_t* col, const double* val, int64_t N, const double* x,
                 int64_t ldx, double* y, int64_t ldy, int nrhs, cudaStream_t s) {
  int64_t threads = N * 32;
  note_launch();
  k_spmv<<<gridn(threads, 256), 256, 0, s>>>(N, rowptr, col, val, x, ldx, y, ldy, nrhs);
  return cudaGetLastError();
}

// out = b - A x
__global__ void k_residual(int64_t N, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
                           int64_t ldx, const double* b, int64_t ldb, double* out, int64_t ldo, int nrhs) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < N; row += nw) {
    int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
    for (int r = 0; r < nrhs; ++r) {
      double s = 0;
      for (int64_t e = e0 + lane; e < e1; e += 32) s += val[e] * x[col[e] + r * ldx];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) out[row + r * ldo] = b[row + r * ldb] - s;
    }
  }
}

cudaError_t residual(const int64_t* rowptr, const int32_t* col, const double* val, int64_t N, const double* x,
                     int64_t ldx, const double* b, int64_t ldb, double* out, int64_t ldo, int nrhs, cudaStream_t s) {
  note_launch();
  k_residual<<<gridn(N * 32, 256), 256, 0, s>>>(N, rowptr, col, val, x, ldx, b, ldb, out, ldo, nrhs);
  return cudaGetLastError();
}

// partial[(r * nk + k) * nblk + blk] = sum over the block's rows of V_r[:, k] . w_r
// V_r = V + r * ldr, column k at + k * N.  Deterministic two-stage reduction.
#define DOT_CHUNK 4096
__global__ void k_multidot(int64_t N, const double* V, int64_t ldr, int nk, const double* w, int64_t ldw,
                           double* partial, int nblk) {
  __shared__ double red[32];
  const int blk = blockIdx.x, r = blockIdx.y;
  const int64_t i0 = (int64_t)blk * DOT_CHUNK;
  const int64_t i1 = (N < i0 + DOT_CHUNK) ? N : i0 + DOT_CHUNK;
  const double* Vr = V + r * ldr;
  const double* wr = w + r * ldw;
  for (int k = 0; k < nk; ++k) {
    double s = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += Vr[i + k * N] * wr[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
      partial[((int64_t)r * nk + k) * nblk + blk] = t;
    }
    __syncthreads();
  }
}
__global__ void k_reduce_partial(int nrhs, int nk, int nblk, const double* partial, double* out, int64_t ldo) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nrhs * nk) return;
  int r = id / nk, k = id % nk;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)id * nblk + b];
  out[k + r * ldo] = s;
}

cudaError_t multidot(int64_t N, const double* V, int64_t ldr, int nk, const double* w, int64_t ldw, int nrhs,
                     double* partial, double* out, int64_t ldo, cudaStream_t s) {
  int nblk = (int)((N + DOT_CHUNK - 1) / DOT_CHUNK);
  dim3 g(nblk, nrhs);
  note_launch();
  k_multidot<<<g, 256, 0, s>>>(N, V, ldr, nk, w, ldw, partial, nblk);
  note_launch();
  k_reduce_partial<<<gridn((int64_t)nrhs * nk, 128), 128, 0, s>>>(nrhs, nk, nblk, partial, out, ldo);
  return cudaGetLastError();
}
int multidot_partials(int64_t N, int nk, int nrhs) { return (int)((N + DOT_CHUNK - 1) / DOT_CHUNK) * nk * nrhs; }

// w_r -= V_r[:, 0..nk) h_r
__global__ void k_multiaxpy(int64_t N, const double* V, int64_t ldr, int nk, const double* h, int64_t ldh, double* w,
                            int64_t ldw, int nrhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) {
      double s = 0;
      const double* Vr = V + r * ldr;
      for (int k = 0; k < nk; ++k) s += Vr[i + k * N] * h[k + r * ldh];
      w[i + r * ldw] -= s;
    }
}
cudaError_t multiaxpy(int64_t N, const double* V, int64_t ldr, int nk, const double* h, int64_t ldh, double* w,
                      int64_t ldw, int nrhs, cudaStream_t s) {
  note_launch();
  k_multiaxpy<<<gridn(N, 256), 256, 0, s>>>(N, V, ldr, nk, h, ldh, w, ldw, nrhs);
  return cudaGetLastError();
}

// out_r = w_r / nrm_r (zero when the norm is zero)
__global__ void k_scale(int64_t N, const double* w, int64_t ldw, const double* nrm, double* out, int64_t ldo, int nrhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) {
      double d = nrm[r];
      out[i + r * ldo] = d > 0 ? w[i + r * ldw] / d : 0.0;
    }
}
cudaError_t scale_cols(int64_t N, const double* w, int64_t ldw, const double* nrm, double* out, int64_t ldo, int nrhs,
                       cudaStream_t s) {
  note_launch();
  k_scale<<<gridn(N, 256), 256, 0, s>>>(N, w, ldw, nrm, out, ldo, nrhs);
  return cudaGetLastError();
}

__global__ void k_sqrt_inplace(double* v, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = sqrt(v[i]);
}
cudaError_t sqrt_inplace(double* v, int n, cudaStream_t s) {
  note_launch();
  k_sqrt_inplace<<<(n + 127) / 128, 128, 0, s>>>(v, n);
  return cudaGetLastError();
}

// Hessenberg column j of every right-hand side: H[0..j] = h1 + h2 (CGS2),
// H[j+1] = hn; apply earlier rotations, build a new one, update g.
// Layout per r: H (m+1) x m column-major at H + r*(m+1)*m; cs, sn, g per r.
__global__ void k_givens(int nrhs, int m, int j, const double* h1, const double* h2, int64_t ldh, const double* hn,
                         double* H, double* cs, double* sn, double* g, double* est) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double* Hr = H + (int64_t)r * (m + 1) * m;
  double* col = Hr + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h1[i + r * ldh] + h2[i + r * ldh];
  col[j + 1] = hn[r];
  double* c = cs + (int64_t)r * m;
  double* s = sn + (int64_t)r * m;
  double* gr = g + (int64_t)r * (m + 1);
  for (int i = 0; i < j; ++i) {
    double t = c[i] * col[i] + s[i] * col[i + 1];
    col[i + 1] = -s[i] * col[i] + c[i] * col[i + 1];
    col[i] = t;
  }
  double a = col[j], b = col[j + 1];
  double rho = hypot(a, b);
  if (rho == 0.0) {
    c[j] = 1.0;
    s[j] = 0.0;
  } else {
    c[j] = a / rho;
    s[j] = b / rho;
  }
  col[j] = rho;
  col[j + 1] = 0.0;
  gr[j + 1] = -s[j] * gr[j];
  gr[j] = c[j] * gr[j];
  est[r] = fabs(gr[j + 1]);
}
cudaError_t givens(int nrhs, int m, int j, const double* h1, const double* h2, int64_t ldh, const double* hn, double* H,
                   double* cs, double* sn, double* g, double* est, cudaStream_t s) {
  note_launch();
  k_givens<<<(nrhs + 31) / 32, 32, 0, s>>>(nrhs, m, j, h1, h2, ldh, hn, H, cs, sn, g, est);
  return cudaGetLastError();
}

// back substitution y = R^-1 g for columns r with jr[r] steps (0: skip)
__global__ void k_backsub(int nrhs, int m, const int* jr, const double* H, const double* g, double* y) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  int J = jr[r];
  const double* Hr = H + (int64_t)r * (m + 1) * m;
  const double* gr = g + (int64_t)r * (m + 1);
  double* yr = y + (int64_t)r * m;
  for (int i = 0; i < m; ++i) yr[i] = 0.0;
  for (int i = J - 1; i >= 0; --i) {
    double t = gr[i];
    for (int k = i + 1; k < J; ++k) t -= Hr[i + (int64_t)k * (m + 1)] * yr[k];
    yr[i] = t / Hr[i + (int64_t)i * (m + 1)];
  }
}
cudaError_t backsub(int nrhs, int m, const int* jr, const double* H, const double* g, double* y, cudaStream_t s) {
  note_launch();
  k_backsub<<<(nrhs + 31) / 32, 32, 0, s>>>(nrhs, m, jr, H, g, y);
  return cudaGetLastError();
}

// g_r = (beta_r, 0, ...)
__global__ void k_init_g(int nrhs, int m, const double* beta, double* g) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  for (int i = 0; i <= m; ++i) g[(int64_t)r * (m + 1) + i] = 0.0;
  g[(int64_t)r * (m + 1)] = beta[r];
}
cudaError_t init_g(int nrhs, int m, const double* beta, double* g, cudaStream_t s) {
  note_launch();
  k_init_g<<<(nrhs + 31) / 32, 32, 0, s>>>(nrhs, m, beta, g);
  return cudaGetLastError();
}

// x_r += Z_r[:, 0..m) y_r
__global__ void k_xupdate(int64_t N, const double* Z, int64_t ldzr, int m, const double* y, double* x, int64_t ldx,
                          int nrhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    for (int r = 0; r < nrhs; ++r) {
      double s = 0;
      const double* Zr = Z + r * ldzr;
      const double* yr = y + (int64_t)r * m;
      for (int k = 0; k < m; ++k) {
        double yk = yr[k];
        if (yk != 0.0) s += Zr[i + k * N] * yk;
      }
      x[i + r * ldx] += s;
    }
}
cudaError_t xupdate(int64_t N, const double* Z, int64_t ldzr, int m, const double* y, double* x, int64_t ldx, int nrhs,
                    cudaStream_t s) {
  note_launch();
  k_xupdate<<<gridn(N, 256), 256, 0, s>>>(N, Z, ldzr, m, y, x, ldx, nrhs);
  return cudaGetLastError();
}

// work (T, permuted, column-major N x nrhs) <- b[perm[i] + r ldb]
template <class T>
__global__ void k_gather_cast(int64_t N, const int32_t* perm, const double* b, int64_t ldb, T* work, int nrhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = perm[i];
    for (int r = 0; r < nrhs; ++r) work[i + r * N] = (T)b[p + r * ldb];
  }
}
template <class T>
__global__ void k_scatter_cast(int64_t N, const int32_t* perm, const T* work, double* x, int64_t ldx, int nrhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = perm[i];
    for (int r = 0; r < nrhs; ++r) x[p + r * ldx] = (double)work[i + r * N];
  }
}
template <class T>
cudaError_t gather_cast(int64_t N, const int32_t* perm, const double* b, int64_t ldb, T* work, int nrhs, cudaStream_t s) {
  note_launch();
  k_gather_cast<T><<<gridn(N, 256), 256, 0, s>>>(N, perm, b, ldb, work, nrhs);
  return cudaGetLastError();
}
template <class T>
cudaError_t scatter_cast(int64_t N, const int32_t* perm, const T* work, double* x, int64_t ldx, int nrhs, cudaStream_t s) {
  note_launch();
  k_scatter_cast<T><<<gridn(N, 256), 256, 0, s>>>(N, perm, work, x, ldx, nrhs);
  return cudaGetLastError();
}
template cudaError_t gather_cast<float>(int64_t, const int32_t*, const double*, int64_t, float*, int, cudaStream_t);
template cudaError_t gather_cast<double>(int64_t, const int32_t*, const double*, int64_t, double*, int, cudaStream_t);
template cudaError_t scatter_cast<float>(int64_t, const int32_t*, const float*, double*, int64_t, int, cudaStream_t);
template cudaError_t scatter_cast<double>(int64_t, const int32_t*, const double*, double*, int64_t, int, cudaStream_t);

__global__ void k_set_int(int32_t* p, int32_t v) { *p = v; }
cudaError_t set_int(int32_t* p, int32_t v, cudaStream_t s) {
  note_launch();
  k_set_int<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

}  // namespace hlu
