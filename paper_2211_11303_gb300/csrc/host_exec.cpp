// Host reference executor of the task DAG (sequential C++, one task at a time).
//
// It runs the same schedules as the device executor, task by task, with plain
// loops.  It exists to validate the scheduler without a GPU: executing the DAG
// in any topological order must give bit-identical results, and the resulting
// preconditioner must be as good as the recursive H-LU it encodes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <stdexcept>
#include <vector>

#include "hlu_internal.h"
#include "host_exec.h"

namespace hlu {
namespace {

template <class T>
struct HostCtx {
  T* arena;
  int32_t* ranks;
  int32_t* piv;
  const Term* terms;
  const Piece* pieces;
  double eps;
  double alpha = 0.0;
  int32_t status = 0;
  int32_t cap_hits = 0;
};

template <class T>
inline int32_t ncols(const HostCtx<T>& c, const View& v) {
  return v.slot >= 0 ? c.ranks[v.slot] : v.cols;
}
template <class T>
inline T& at(HostCtx<T>& c, const View& v, int64_t i, int64_t j) {
  return c.arena[v.off + i * v.rs + j * v.cs];
}

template <class T>
void h_getrf(HostCtx<T>& c, const Task& t) {
  int n = t.a.rows;
  std::vector<T> A(n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) A[i + j * n] = at(c, t.a, i, j);
  int32_t* p = c.piv + t.piv_off;
  for (int i = 0; i < n; ++i) p[i] = i;
  for (int k = 0; k < n; ++k) {
    int q = k;
    T best = std::fabs(A[k + k * n]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i + k * n]) > best) {
        best = std::fabs(A[i + k * n]);
        q = i;
      }
    if (best == T(0)) {
      c.status = 3;
      continue;
    }
    if (q != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k + j * n], A[q + j * n]);
      std::swap(p[k], p[q]);
    }
    T inv = T(1) / A[k + k * n];
    for (int i = k + 1; i < n; ++i) A[i + k * n] *= inv;
    for (int j = k + 1; j < n; ++j)
      for (int i = k + 1; i < n; ++i) A[i + j * n] -= A[i + k * n] * A[k + j * n];
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) at(c, t.a, i, j) = A[i + j * n];
}

template <class T>
void h_trsm(HostCtx<T>& c, const Task& t) {
  int n = t.a.rows;
  int k = ncols(c, t.b);
  std::vector<T> V(n);
  const int32_t* p = c.piv + t.piv_off;
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < n; ++i) V[i] = at(c, t.b, i, j);
    if (t.type == TK_TRSM_L) {
      std::vector<T> W(n);
      for (int i = 0; i < n; ++i) W[i] = V[p[i]];
      for (int i = 0; i < n; ++i)
        for (int l = 0; l < i; ++l) W[i] -= at(c, t.a, i, l) * W[l];
      V = W;
    } else if (t.type == TK_TRSM_UT) {
      for (int i = 0; i < n; ++i) {
        for (int l = 0; l < i; ++l) V[i] -= at(c, t.a, l, i) * V[l];
        V[i] /= at(c, t.a, i, i);
      }
    } else {
      for (int i = n - 1; i >= 0; --i) {
        for (int l = i + 1; l < n; ++l) V[i] -= at(c, t.a, i, l) * V[l];
        V[i] /= at(c, t.a, i, i);
      }
    }
    for (int i = 0; i < n; ++i) at(c, t.b, i, j) = V[i];
  }
}

template <class T>
void h_proj(HostCtx<T>& c, const Task& t) {
  int m = t.a.rows, r = ncols(c, t.a), k = ncols(c, t.b);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < k; ++j) {
      T s = 0;
      for (int l = 0; l < m; ++l) s += at(c, t.a, l, i) * at(c, t.b, l, j);
      at(c, t.c, i, j) = s;
    }
}

template <class T>
void h_rowmv(HostCtx<T>& c, const Task& t) {
  int n = t.c.rows, k = ncols(c, t.b);
  std::vector<T> acc((size_t)n * k, T(0));
  for (int q = 0; q < t.list_count; ++q) {
    const Term& tm = c.terms[t.list_begin + q];
    int p = ncols(c, tm.A);
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < tm.A.rows; ++i) {
        T s = 0;
        for (int l = 0; l < p; ++l) s += at(c, tm.A, i, l) * at(c, tm.B, l, j);
        acc[(tm.roff + i) + (size_t)j * n] += s;
      }
  }
  T sg = T(t.sign);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < n; ++i) {
      T base = (t.flags & TF_OVERWRITE) ? T(0) : at(c, t.c, i, j);
      at(c, t.c, i, j) = base + sg * acc[i + (size_t)j * n];
    }
  if (t.out_slot >= 0) c.ranks[t.out_slot] = k;
}

template <class T>
void h_dadd(HostCtx<T>& c, const Task& t) {
  int m = t.c.rows, n = ncols(c, t.c), k = ncols(c, t.a);
  T sg = (t.flags & TF_ALPHA) ? T(t.sign) * T(c.alpha) : T(t.sign);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      T s = 0;
      for (int l = 0; l < k; ++l) s += at(c, t.a, i, l) * at(c, t.b, j, l);
      T base = (t.flags & TF_OVERWRITE) ? T(0) : at(c, t.c, i, j);
      at(c, t.c, i, j) = base + sg * s;
    }
}

// Householder QR of S (m x w, column-major, ld m) in place: R in the upper
// triangle, reflector tails below, tau[] the reflector scalars.
template <class T>
void h_house(std::vector<T>& S, int m, int w, std::vector<T>& tau) {
  int t = std::min(m, w);
  tau.assign(t, T(0));
  for (int j = 0; j < t; ++j) {
    T alpha = S[j + (size_t)j * m];
    T s2 = 0;
    for (int i = j + 1; i < m; ++i) s2 += S[i + (size_t)j * m] * S[i + (size_t)j * m];
    if (s2 == T(0)) {
      tau[j] = 0;
      continue;
    }
    T nrm = std::sqrt(alpha * alpha + s2);
    T beta = alpha >= 0 ? -nrm : nrm;
    T scale = T(1) / (alpha - beta);
    for (int i = j + 1; i < m; ++i) S[i + (size_t)j * m] *= scale;
    tau[j] = (beta - alpha) / beta;
    S[j + (size_t)j * m] = beta;
    for (int cc = j + 1; cc < w; ++cc) {
      T d = S[j + (size_t)cc * m];
      for (int i = j + 1; i < m; ++i) d += S[i + (size_t)j * m] * S[i + (size_t)cc * m];
      d *= tau[j];
      S[j + (size_t)cc * m] -= d;
      for (int i = j + 1; i < m; ++i) S[i + (size_t)cc * m] -= d * S[i + (size_t)j * m];
    }
  }
}
// B (m x r, ld m) <- Q B with Q = H_0 ... H_{t-1} from h_house.
template <class T>
void h_applyq(const std::vector<T>& S, int m, const std::vector<T>& tau, std::vector<T>& Bm, int r) {
  int t = (int)tau.size();
  for (int j = t - 1; j >= 0; --j) {
    if (tau[j] == T(0)) continue;
    for (int cc = 0; cc < r; ++cc) {
      T d = Bm[j + (size_t)cc * m];
      for (int i = j + 1; i < m; ++i) d += S[i + (size_t)j * m] * Bm[i + (size_t)cc * m];
      d *= tau[j];
      Bm[j + (size_t)cc * m] -= d;
      for (int i = j + 1; i < m; ++i) Bm[i + (size_t)cc * m] -= d * S[i + (size_t)j * m];
    }
  }
}

// One-sided Jacobi: G (p x q, ld p) -> G V with orthogonal columns; V (q x q).
template <class T>
void h_jacobi(std::vector<T>& G, int p, int q, std::vector<T>& V) {
  V.assign((size_t)q * q, T(0));
  for (int i = 0; i < q; ++i) V[i + (size_t)i * q] = 1;
  const T tol = sizeof(T) == 4 ? T(1e-6) : T(1e-14);
  double prev = 3e38;
  for (int sweep = 0; sweep < 20; ++sweep) {
    bool rot = false;
    double off = 0;
    for (int a = 0; a < q - 1; ++a)
      for (int b = a + 1; b < q; ++b) {
        T al = 0, be = 0, ga = 0;
        for (int i = 0; i < p; ++i) {
          T x = G[i + (size_t)a * p], y = G[i + (size_t)b * p];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        if (ga == T(0)) continue;
        T ratio = std::fabs(ga) / std::sqrt(al * be);
        off = std::max(off, (double)ratio);
        if (ratio <= tol) continue;
        rot = true;
        T zeta = (be - al) / (2 * ga);
        T tt = (zeta >= 0 ? T(1) : T(-1)) / (std::fabs(zeta) + std::sqrt(T(1) + zeta * zeta));
        T cs = T(1) / std::sqrt(T(1) + tt * tt), sn = cs * tt;
        for (int i = 0; i < p; ++i) {
          T x = G[i + (size_t)a * p], y = G[i + (size_t)b * p];
          G[i + (size_t)a * p] = cs * x - sn * y;
          G[i + (size_t)b * p] = sn * x + cs * y;
        }
        for (int i = 0; i < q; ++i) {
          T x = V[i + (size_t)a * q], y = V[i + (size_t)b * q];
          V[i + (size_t)a * q] = cs * x - sn * y;
          V[i + (size_t)b * q] = sn * x + cs * y;
        }
      }
    if (!rot) break;
    if (sweep >= 2 && off < 100.0 * (double)tol && off > 0.25 * prev) break;
    prev = off;
  }
}

// Truncated SVD of X Y^T (SX: m x W, SY: n x W, column-major): returns the
// new factors (m x r, n x r) with s_i > eps s_1 kept, at most cap.
template <class T>
int h_compress(double eps, int32_t* cap_hits, std::vector<T> SX, std::vector<T> SY, int m, int n, int W, int cap,
               std::vector<T>& BX, std::vector<T>& BY, double* fro) {
  std::vector<T> tx, ty;
  h_house(SX, m, W, tx);
  h_house(SY, n, W, ty);
  int p = std::min(m, W), q = std::min(n, W);
  std::vector<T> G((size_t)p * q, T(0));
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) {
      double s = 0;  // FP64 accumulation: cancellation between target and update
      for (int l = std::max(i, j); l < W; ++l) s += (double)SX[i + (size_t)l * m] * (double)SY[j + (size_t)l * n];
      G[i + (size_t)j * p] = (T)s;
    }
  std::vector<T> V;
  h_jacobi(G, p, q, V);
  std::vector<T> sv(q);
  double f2 = 0;
  for (int j = 0; j < q; ++j) {
    T s = 0;
    for (int i = 0; i < p; ++i) s += G[i + (size_t)j * p] * G[i + (size_t)j * p];
    sv[j] = std::sqrt(s);
    f2 += (double)sv[j] * (double)sv[j];
  }
  *fro = std::sqrt(f2);
  std::vector<int> ord(q);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  T smax = q ? sv[ord[0]] : T(0);
  int r = 0;
  if (smax > T(0))
    while (r < q && sv[ord[r]] > T(eps) * smax) ++r;
  if (r > cap) {
    r = cap;
    (*cap_hits)++;
  }
  BX.assign((size_t)m * r, T(0));
  BY.assign((size_t)n * r, T(0));
  for (int j = 0; j < r; ++j) {
    for (int i = 0; i < p; ++i) BX[i + (size_t)j * m] = G[i + (size_t)ord[j] * p];
    for (int i = 0; i < q; ++i) BY[i + (size_t)j * n] = V[i + (size_t)ord[j] * q];
  }
  h_applyq(SX, m, tx, BX, r);
  h_applyq(SY, n, ty, BY, r);
  return r;
}

// pieces are stacked, compressing whenever the stack would pass 48 columns
// (the device executor's order of operations); *ratio receives the largest
// ||X|| ||Y|| / ||X Y^T|| over the compressions
constexpr int kHostCompressAt = 48;
template <class TC, class T>
int h_trunc_stack(HostCtx<T>& c, const Task& t, std::vector<TC>& SX, std::vector<TC>& SY, double* ratio) {
  const int m = t.a.rows, n = t.b.rows;
  int W = 0;
  double worst = 0;
  auto norms = [&](int w_) {
    double nx = 0, ny = 0;
    for (size_t i = 0; i < (size_t)m * w_; ++i) nx += (double)SX[i] * SX[i];
    for (size_t i = 0; i < (size_t)n * w_; ++i) ny += (double)SY[i] * SY[i];
    return std::sqrt(nx) * std::sqrt(ny);
  };
  for (int q = 0; q < t.list_count; ++q) {
    const Piece& P = c.pieces[t.list_begin + q];
    int w = ncols(c, P.X);
    if (w == 0) continue;
    if (W > 0 && W + w > kHostCompressAt) {
      std::vector<TC> BX, BY;
      double in = norms(W), fro = 0;
      W = h_compress(c.eps, &c.cap_hits, SX, SY, m, n, W, t.cap, BX, BY, &fro);
      if (fro > 0) worst = std::max(worst, in / fro);
      SX = BX;
      SY = BY;
    }
    SX.resize((size_t)m * (W + w), TC(0));
    SY.resize((size_t)n * (W + w), TC(0));
    for (int j = 0; j < w; ++j) {
      const TC sg = (P.pad & PF_ALPHA) ? TC(P.sign) * TC(c.alpha) : TC(P.sign);
      for (int i = 0; i < P.X.rows; ++i) SX[(P.xoff + i) + (size_t)(W + j) * m] = sg * TC(at(c, P.X, i, j));
      for (int i = 0; i < P.Y.rows; ++i) SY[(P.yoff + i) + (size_t)(W + j) * n] = TC(at(c, P.Y, i, j));
    }
    W += w;
  }
  int r = 0;
  if (W > 0) {
    std::vector<TC> BX, BY;
    double in = norms(W), fro = 0;
    r = h_compress(c.eps, &c.cap_hits, SX, SY, m, n, W, t.cap, BX, BY, &fro);
    if (fro > 0) worst = std::max(worst, in / fro);
    SX = BX;
    SY = BY;
  }
  *ratio = worst;
  return r;
}

template <class T>
void h_trunc(HostCtx<T>& c, const Task& t) {
  int m = t.a.rows, n = t.b.rows;
  if (m == 0 || n == 0) {
    c.ranks[t.out_slot] = 0;
    return;
  }
  std::vector<T> SX, SY;
  double ratio = 0;
  int r = h_trunc_stack<T, T>(c, t, SX, SY, &ratio);
  for (int j = 0; j < r; ++j) {
    for (int i = 0; i < m; ++i) at(c, t.a, i, j) = SX[i + (size_t)j * m];
    for (int i = 0; i < n; ++i) at(c, t.b, i, j) = SY[i + (size_t)j * n];
  }
  c.ranks[t.out_slot] = r;
}

template <class T>
void h_rsolve(HostCtx<T>& c, const Task& t) {
  Task r = t;
  r.type = TK_ROWMV;
  r.flags = 0;
  r.out_slot = -1;
  h_rowmv(c, r);
  Task s = t;
  s.type = (t.flags & TF_UPPER) ? TK_TRSM_U : TK_TRSM_L;
  s.b = t.c;
  h_trsm(c, s);
}

template <class T>
void run_task(HostCtx<T>& c, const Task& t) {
  switch (t.type) {
    case TK_GETRF: h_getrf(c, t); break;
    case TK_TRSM_L:
    case TK_TRSM_UT:
    case TK_TRSM_U: h_trsm(c, t); break;
    case TK_PROJ: h_proj(c, t); break;
    case TK_ROWMV: h_rowmv(c, t); break;
    case TK_TRUNC: h_trunc(c, t); break;
    case TK_DADD: h_dadd(c, t); break;
    case TK_RSOLVE: h_rsolve(c, t); break;
    case TK_FENCE: break;
    default: throw std::logic_error("task type");
  }
}

// A topological order: program order, or a random one (Kahn's algorithm with a
// random choice among ready tasks) to check that the edges are sufficient.
std::vector<int64_t> exec_order(const Schedule& S, uint64_t seed) {
  int64_t n = (int64_t)S.tasks.size();
  std::vector<int64_t> order(n);
  if (seed == 0) {
    std::iota(order.begin(), order.end(), 0);
    return order;
  }
  std::vector<int32_t> indeg(n, 0);
  std::vector<std::vector<int32_t>> succ(n);
  for (int64_t t = 0; t < n; ++t)
    for (int64_t e = S.pred_ptr[t]; e < S.pred_ptr[t + 1]; ++e) {
      succ[S.pred_idx[e]].push_back((int32_t)t);
      indeg[t]++;
    }
  std::vector<int32_t> ready;
  for (int64_t t = 0; t < n; ++t)
    if (!indeg[t]) ready.push_back((int32_t)t);
  std::mt19937_64 rng(seed);
  int64_t k = 0;
  while (!ready.empty()) {
    size_t i = rng() % ready.size();
    int32_t t = ready[i];
    ready[i] = ready.back();
    ready.pop_back();
    order[k++] = t;
    for (int32_t s : succ[t])
      if (--indeg[s] == 0) ready.push_back(s);
  }
  if (k != n) throw std::logic_error("schedule has a cycle");
  return order;
}

}  // namespace

template <class T>
int host_execute(const Schedule& S, T* arena, int32_t* ranks, int32_t* piv, double eps,
                 uint64_t order_seed, int32_t* cap_hits, int64_t limit, double alpha) {
  HostCtx<T> c;
  c.arena = arena;
  c.ranks = ranks;
  c.piv = piv;
  c.terms = S.terms.data();
  c.pieces = S.pieces.data();
  c.eps = eps;
  c.alpha = alpha;
  for (int64_t t : exec_order(S, order_seed)) {
    if (limit >= 0 && t >= limit) continue;
    run_task(c, S.tasks[t]);
  }
  if (cap_hits) *cap_hits += c.cap_hits;
  return c.status;
}

template int host_execute<double>(const Schedule&, double*, int32_t*, int32_t*, double, uint64_t,
                                  int32_t*, int64_t, double);
template int host_execute<float>(const Schedule&, float*, int32_t*, int32_t*, double, uint64_t,
                                 int32_t*, int64_t, double);

}  // namespace hlu
