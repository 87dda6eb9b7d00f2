// FP64 Krylov building blocks (krylov.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hlu {
cudaError_t spmv(const int64_t* rowptr, const int32_t* col, const double* val, int64_t N, const double* x,
                 int64_t ldx, double* y, int64_t ldy, int nrhs, cudaStream_t s);
cudaError_t residual(const int64_t* rowptr, const int32_t* col, const double* val, int64_t N, const double* x,
                     int64_t ldx, const double* b, int64_t ldb, double* out, int64_t ldo, int nrhs, cudaStream_t s);
cudaError_t multidot(int64_t N, const double* V, int64_t ldr, int nk, const double* w, int64_t ldw, int nrhs,
                     double* partial, double* out, int64_t ldo, cudaStream_t s);
int multidot_partials(int64_t N, int nk, int nrhs);
cudaError_t multiaxpy(int64_t N, const double* V, int64_t ldr, int nk, const double* h, int64_t ldh, double* w,
                      int64_t ldw, int nrhs, cudaStream_t s);
cudaError_t scale_cols(int64_t N, const double* w, int64_t ldw, const double* nrm, double* out, int64_t ldo, int nrhs,
                       cudaStream_t s);
cudaError_t sqrt_inplace(double* v, int n, cudaStream_t s);
cudaError_t givens(int nrhs, int m, int j, const double* h1, const double* h2, int64_t ldh, const double* hn, double* H,
                   double* cs, double* sn, double* g, double* est, cudaStream_t s);
cudaError_t backsub(int nrhs, int m, const int* jr, const double* H, const double* g, double* y, cudaStream_t s);
cudaError_t init_g(int nrhs, int m, const double* beta, double* g, cudaStream_t s);
cudaError_t xupdate(int64_t N, const double* Z, int64_t ldzr, int m, const double* y, double* x, int64_t ldx, int nrhs,
                    cudaStream_t s);
template <class T>
cudaError_t gather_cast(int64_t N, const int32_t* perm, const double* b, int64_t ldb, T* work, int nrhs, cudaStream_t s);
template <class T>
cudaError_t scatter_cast(int64_t N, const int32_t* perm, const T* work, double* x, int64_t ldx, int nrhs, cudaStream_t s);
cudaError_t set_int(int32_t* p, int32_t v, cudaStream_t s);
}  // namespace hlu
