// Debug / validation entry points that need no GPU: the task scheduler plus
// the host reference executor, driven from exported tree arrays.
#include <algorithm>
#include <cstring>
#include <exception>
#include <vector>

#include "../../include/hlu_debug.h"
#include "host_exec.h"
#include "hlu_internal.h"

namespace hlu {

void trees_from_export(int32_t nc, const int32_t* cl, int32_t nb, const int32_t* bl,
                       std::vector<Cluster>& C, std::vector<Block>& B) {
  C.resize(nc);
  for (int32_t i = 0; i < nc; ++i) {
    const int32_t* r = cl + (int64_t)12 * i;
    Cluster& c = C[i];
    c.off = r[0];
    c.size = r[1];
    for (int k = 0; k < 3; ++k) {
      c.lo[k] = r[2 + k];
      c.hi[k] = r[5 + k];
    }
    c.son[0] = r[8];
    c.son[1] = r[9];
    c.level = r[10];
    c.parent = r[11];
  }
  // leaf ranges: leaves in id (= DFS pre-order = index) order
  int32_t nl = 0;
  for (int32_t i = 0; i < nc; ++i)
    if (C[i].son[0] < 0) {
      C[i].leaf_begin = nl;
      C[i].leaf_end = ++nl;
    }
  for (int32_t i = nc - 1; i >= 0; --i)
    if (C[i].son[0] >= 0) {
      C[i].leaf_begin = C[C[i].son[0]].leaf_begin;
      C[i].leaf_end = C[C[i].son[1]].leaf_end;
    }
  B.resize(nb);
  for (int32_t i = 0; i < nb; ++i) {
    const int32_t* r = bl + (int64_t)8 * i;
    Block& b = B[i];
    b.row = r[0];
    b.col = r[1];
    b.kind = r[2];
    for (int k = 0; k < 4; ++k) b.son[k] = r[3 + k];
    b.parent = r[7];
  }
}

}  // namespace hlu

using namespace hlu;

extern "C" int hlu_debug_host_factor_prefix(int32_t nc, const int32_t* clusters, int32_t nb,
                                            const int32_t* blocks, const int32_t* perm, const int64_t* rowptr,
                                            const int32_t* col, const double* val, double eps, int32_t rank_cap,
                                            int32_t tile, int32_t precision, uint64_t order_seed, int32_t nrhs,
                                            const double* b, double* x, int64_t* info, int64_t limit,
                                            void* arena_out, int32_t* ranks_out);

extern "C" int hlu_debug_host_factor_solve(int32_t nc, const int32_t* clusters, int32_t nb,
                                           const int32_t* blocks, const int32_t* perm,
                                           const int64_t* rowptr, const int32_t* col,
                                           const double* val, double eps, int32_t rank_cap,
                                           int32_t tile, int32_t precision, uint64_t order_seed, int32_t nrhs, const double* b,
                                           double* x, int64_t* info) {
  return hlu_debug_host_factor_prefix(nc, clusters, nb, blocks, perm, rowptr, col, val, eps, rank_cap, tile,
                                      precision, order_seed, nrhs, b, x, info, -1, nullptr, nullptr);
}

extern "C" int hlu_debug_host_factor_prefix(int32_t nc, const int32_t* clusters, int32_t nb,
                                            const int32_t* blocks, const int32_t* perm, const int64_t* rowptr,
                                            const int32_t* col, const double* val, double eps, int32_t rank_cap,
                                            int32_t tile, int32_t precision, uint64_t order_seed, int32_t nrhs,
                                            const double* b, double* x, int64_t* info, int64_t limit,
                                            void* arena_out, int32_t* ranks_out) {
  try {
    if (!clusters || !blocks || !perm || !rowptr || !col || !val || nrhs < 1 || eps <= 0)
      return 1;
    std::vector<Cluster> C;
    std::vector<Block> B;
    trees_from_export(nc, clusters, nb, blocks, C, B);
    const int32_t N = C[0].size;
    ArenaLayout L;
    Schedule F, S;
    SchedStats st;
    std::vector<Block> FB;
    build_schedules(C, B, rank_cap > 0 ? rank_cap : kRankMax, nrhs, tile, L, F, S, st, &FB);
    B = FB;
    std::vector<double> arena(L.total, 0.0);
    std::vector<int32_t> ranks(L.n_slots, 0), piv(std::max<int64_t>(L.piv_total, 1), 0);
    // identity
    for (int32_t i = 0; i < L.ident_n; ++i) arena[L.ident_off + i + (int64_t)i * L.ident_n] = 1.0;
    // A_H (Alg. 1 step I): permuted CSR -> dense leaves and exact low-rank blocks
    std::vector<int32_t> iperm(N);
    for (int32_t i = 0; i < N; ++i) iperm[perm[i]] = i;
    for (size_t bi = 0; bi < B.size(); ++bi) {
      const Block& bk = B[bi];
      if (bk.kind == KIND_SUB) continue;
      const Cluster& R = C[bk.row];
      const Cluster& Q = C[bk.col];
      int32_t kk = 0;
      for (int32_t i = 0; i < R.size; ++i) {
        int32_t orow = perm[R.off + i];
        bool any = false;
        for (int64_t e = rowptr[orow]; e < rowptr[orow + 1]; ++e) {
          int32_t j = iperm[col[e]] - Q.off;
          if (j < 0 || j >= Q.size) continue;
          if (bk.kind == KIND_DENSE) {
            arena[L.dense_off[bi] + i + (int64_t)j * R.size] = val[e];
          } else {
            if (!any) {
              if (kk >= L.cap[bi]) return 7;
              arena[L.x_off[bi] + i + (int64_t)kk * R.size] = 1.0;
              any = true;
            }
            arena[L.y_off[bi] + j + (int64_t)kk * Q.size] = val[e];
          }
        }
        if (any) ++kk;
      }
      if (bk.kind == KIND_ADM) ranks[L.slot[bi]] = kk;
    }
    int32_t cap_hits = 0;
    int st1 = 0, st2 = 0;
    if (precision == 1) {
      std::vector<float> af(arena.begin(), arena.end());
      st1 = host_execute<float>(F, af.data(), ranks.data(), piv.data(), eps, order_seed, &cap_hits, limit);
      if (arena_out) {
        std::memcpy(arena_out, af.data(), sizeof(float) * af.size());
        if (ranks_out) std::memcpy(ranks_out, ranks.data(), sizeof(int32_t) * ranks.size());
        return st1;
      }
      ranks[L.nrhs_slot] = nrhs;
      for (int32_t j = 0; j < nrhs; ++j)
        for (int32_t i = 0; i < N; ++i) af[L.work_off + i + (int64_t)j * N] = (float)b[perm[i] + (int64_t)j * N];
      st2 = host_execute<float>(S, af.data(), ranks.data(), piv.data(), eps, order_seed, &cap_hits);
      for (int32_t j = 0; j < nrhs; ++j)
        for (int32_t i = 0; i < N; ++i) x[perm[i] + (int64_t)j * N] = af[L.work_off + i + (int64_t)j * N];
    } else {
      st1 = host_execute<double>(F, arena.data(), ranks.data(), piv.data(), eps, order_seed, &cap_hits, limit);
      if (arena_out) {
        std::memcpy(arena_out, arena.data(), sizeof(double) * arena.size());
        if (ranks_out) std::memcpy(ranks_out, ranks.data(), sizeof(int32_t) * ranks.size());
        return st1;
      }
      // solve: work vector in permuted order
      ranks[L.nrhs_slot] = nrhs;
      for (int32_t j = 0; j < nrhs; ++j)
        for (int32_t i = 0; i < N; ++i) arena[L.work_off + i + (int64_t)j * N] = b[perm[i] + (int64_t)j * N];
      st2 = host_execute<double>(S, arena.data(), ranks.data(), piv.data(), eps, order_seed, &cap_hits);
      for (int32_t j = 0; j < nrhs; ++j)
        for (int32_t i = 0; i < N; ++i) x[perm[i] + (int64_t)j * N] = arena[L.work_off + i + (int64_t)j * N];
    }
    if (info) {
      int32_t rmax = 0;
      int64_t rsum = 0, nadm = 0;
      for (size_t bi = 0; bi < B.size(); ++bi)
        if (B[bi].kind == KIND_ADM) {
          rmax = std::max(rmax, ranks[L.slot[bi]]);
          rsum += ranks[L.slot[bi]];
          ++nadm;
        }
      info[0] = (int64_t)F.tasks.size();
      info[1] = (int64_t)S.tasks.size();
      info[2] = rmax;
      info[3] = cap_hits;
      info[4] = st1 ? st1 : st2;
      info[5] = L.total;
      info[6] = (int64_t)(st.host_ms * 1000);
      info[7] = nadm ? (rsum * 1000) / nadm : 0;
      info[8] = F.n_edges;
      info[9] = L.wmax;
    }
    return st1 ? st1 : st2;
  } catch (const std::exception&) {
    return 6;
  }
}

// The Schulz inverse's schedules run by the host reference executor (FP64):
// A_H into copy 0, X_0 = alpha A_H, `iters` Schulz steps, then x = X b.
extern "C" int hlu_debug_host_hinverse(int32_t nc, const int32_t* clusters, int32_t nb, const int32_t* blocks,
                                       const int32_t* perm, const int64_t* rowptr, const int32_t* col,
                                       const double* val, double eps, int32_t rank_cap, int32_t tile,
                                       double alpha, int32_t iters, int32_t nrhs, const double* b, double* x,
                                       int64_t* info) {
  try {
    if (!clusters || !blocks || !perm || !rowptr || !col || !val || nrhs < 1 || nrhs > 16 || eps <= 0 || iters < 0)
      return 1;
    std::vector<Cluster> C;
    std::vector<Block> B;
    trees_from_export(nc, clusters, nb, blocks, C, B);
    const int32_t N = C[0].size;
    std::vector<Block> FB = factor_tree(C, B, tile);
    ArenaLayout L;
    std::vector<Block> Bx;
    Schedule S0, S1, S2;
    SchedStats st;
    build_inverse_schedules(C, FB, rank_cap > 0 ? rank_cap : kRankMax, 16, tile, L, Bx, S0, S1, S2, st);
    std::vector<double> arena(L.total, 0.0);
    std::vector<int32_t> ranks(std::max(L.n_slots, 1), 0), piv(1, 0);
    for (int32_t i = 0; i < L.ident_n; ++i) arena[L.ident_off + i + (int64_t)i * L.ident_n] = 1.0;
    std::vector<int32_t> iperm(N);
    for (int32_t i = 0; i < N; ++i) iperm[perm[i]] = i;
    for (size_t bi = 0; bi < FB.size(); ++bi) {  // A_H: copy 0
      const Block& bk = Bx[bi];
      if (bk.kind == KIND_SUB) continue;
      const Cluster& R = C[bk.row];
      const Cluster& Q = C[bk.col];
      int32_t kk = 0;
      for (int32_t i = 0; i < R.size; ++i) {
        const int32_t orow = perm[R.off + i];
        bool any = false;
        for (int64_t e = rowptr[orow]; e < rowptr[orow + 1]; ++e) {
          const int32_t j = iperm[col[e]] - Q.off;
          if (j < 0 || j >= Q.size) continue;
          if (bk.kind == KIND_DENSE) {
            arena[L.dense_off[bi] + i + (int64_t)j * R.size] = val[e];
          } else {
            if (!any) {
              if (kk >= L.cap[bi]) return 7;
              arena[L.x_off[bi] + i + (int64_t)kk * R.size] = 1.0;
              any = true;
            }
            arena[L.y_off[bi] + j + (int64_t)kk * Q.size] = val[e];
          }
        }
        if (any) ++kk;
      }
      if (bk.kind == KIND_ADM) ranks[L.slot[bi]] = kk;
    }
    int32_t cap_hits = 0;
    int stt = host_execute<double>(S0, arena.data(), ranks.data(), piv.data(), eps, 0, &cap_hits, -1, alpha);
    for (int32_t k = 0; k < iters && !stt; ++k)
      stt = host_execute<double>(S1, arena.data(), ranks.data(), piv.data(), eps, 0, &cap_hits);
    ranks[L.nrhs_slot] = nrhs;
    for (int32_t j = 0; j < nrhs; ++j)
      for (int32_t i = 0; i < N; ++i) arena[L.work_off + i + (int64_t)j * N] = b[perm[i] + (int64_t)j * N];
    if (!stt) stt = host_execute<double>(S2, arena.data(), ranks.data(), piv.data(), eps, 0, &cap_hits);
    for (int32_t j = 0; j < nrhs; ++j)
      for (int32_t i = 0; i < N; ++i) x[perm[i] + (int64_t)j * N] = arena[L.out_off + i + (int64_t)j * N];
    if (info) {
      int32_t rmax = 0;
      for (size_t bi = FB.size(); bi < 2 * FB.size(); ++bi)
        if (Bx[bi].kind == KIND_ADM) rmax = std::max(rmax, ranks[L.slot[bi]]);
      info[0] = (int64_t)S1.tasks.size();
      info[1] = (int64_t)S2.tasks.size();
      info[2] = rmax;
      info[3] = cap_hits;
      info[4] = stt;
    }
    return stt;
  } catch (const std::exception&) {
    return 6;
  }
}
