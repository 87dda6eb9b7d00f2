// Test driver: the library's host-side code (task scheduler, host reference
// executor, race check of the DAGs, Schulz inverse on the host) built with
// AddressSanitizer and UndefinedBehaviorSanitizer by tests/test_host_sanitizers.py.
//
// Input file (little-endian): int32 nc, nb, N, nrhs, tile; int64 nnz;
// clusters int32[nc*12]; blocks int32[nb*8]; perm int32[N]; rowptr
// int64[N+1]; col int32[nnz]; val double[nnz]; b double[N*nrhs].
// Output file: the solutions, double[N*nrhs] each, of: FP64 in program order,
// FP64 in a random topological order, FP32 in program order, and the
// Schulz inverse after two steps.  Exit 0 when every call succeeds.
#include <cmath>
#include <cstdio>
#include <vector>

#include "../include/hlu_debug.h"

template <class T>
static bool rd(FILE* f, std::vector<T>& v, size_t n) {
  v.resize(n);
  return n == 0 || fread(v.data(), sizeof(T), n, f) == n;
}

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[5];
  int64_t nnz = 0;
  if (fread(hdr, sizeof(int32_t), 5, f) != 5 || fread(&nnz, sizeof(int64_t), 1, f) != 1) return 2;
  const int32_t nc = hdr[0], nb = hdr[1], N = hdr[2], nrhs = hdr[3], tile = hdr[4];
  std::vector<int32_t> C, B, perm, col;
  std::vector<int64_t> rowptr;
  std::vector<double> val, b;
  if (!rd(f, C, (size_t)nc * 12) || !rd(f, B, (size_t)nb * 8) || !rd(f, perm, (size_t)N) ||
      !rd(f, rowptr, (size_t)N + 1) || !rd(f, col, (size_t)nnz) || !rd(f, val, (size_t)nnz) ||
      !rd(f, b, (size_t)N * nrhs))
    return 2;
  fclose(f);

  std::vector<double> out;
  std::vector<double> x((size_t)N * nrhs);
  int64_t info[10];
  const struct {
    int32_t precision;
    uint64_t seed;
  } runs[3] = {{0, 0}, {0, 3}, {1, 0}};
  for (const auto& r : runs) {
    int st = hlu_debug_host_factor_solve(nc, C.data(), nb, B.data(), perm.data(), rowptr.data(), col.data(),
                                         val.data(), 1e-4, 32, tile, r.precision, r.seed, nrhs, b.data(), x.data(),
                                         info);
    printf("factor_solve precision %d seed %llu: status %d, %lld factor tasks\n", r.precision,
           (unsigned long long)r.seed, st, (long long)info[0]);
    if (st != 0) return 3;
    out.insert(out.end(), x.begin(), x.end());
  }
  for (int32_t which = 0; which <= 4; ++which) {
    int64_t rep[11];
    int st = hlu_debug_check_hazards(nc, C.data(), nb, B.data(), 32, tile, 16, which, -1, rep);
    printf("hazards dag %d: status %d, %lld tasks, %lld unordered\n", which, st, (long long)rep[0],
           (long long)rep[3]);
    if (st != 0 && st != 6) return 4;  // 6: too large for the check, refused before any work
  }
  // Schulz start X_0 = alpha A with alpha = 1 / (||A||_1 ||A||_inf)
  std::vector<double> colsum(N, 0.0);
  double rmax = 0.0;
  for (int32_t i = 0; i < N; ++i) {
    double rs = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      rs += std::fabs(val[e]);
      colsum[col[e]] += std::fabs(val[e]);
    }
    rmax = rs > rmax ? rs : rmax;
  }
  double cmax = 0.0;
  for (double c : colsum) cmax = c > cmax ? c : cmax;
  int st = hlu_debug_host_hinverse(nc, C.data(), nb, B.data(), perm.data(), rowptr.data(), col.data(), val.data(),
                                   1e-6, 32, tile, 1.0 / (rmax * cmax), 2, nrhs, b.data(), x.data(), info);
  printf("hinverse: status %d, %lld step tasks\n", st, (long long)info[0]);
  if (st != 0) return 5;
  out.insert(out.end(), x.begin(), x.end());

  FILE* g = fopen(argv[2], "wb");
  if (!g || fwrite(out.data(), sizeof(double), out.size(), g) != out.size()) return 6;
  fclose(g);
  return 0;
}
