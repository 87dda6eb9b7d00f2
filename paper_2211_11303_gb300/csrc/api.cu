// C ABI of the GB300 H-LU library (declarations and documentation in
// include/hlu.h).  Host orchestration only: every step of the numerical path
// runs in the kernels of build.cu, exec.cu and krylov.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "../../include/hlu.h"
#include "build.h"
#include "devmem.h"
#include "exec.h"
#include "hlu_internal.h"
#include "host_exec.h"
#include "krylov.h"
#include "launch_count.h"

#include <nvtx3/nvToolsExt.h>

namespace {
// One NVTX range per public call (build, factor, solve, GMRES, Richardson,
// Schulz inverse, batched calls), named after the call, for profilers that
// filter by range (ncu --nvtx); without a profiler attached each push and
// pop is a test of an unset function pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using namespace hlu;

namespace hlu {
std::atomic<int64_t> g_launches{0};
}

namespace {

thread_local std::string g_err;
double g_wait_limit_ms = 20000.0;
double g_jacobi_tol = 0.0;  // 0: default of the factor precision
int32_t g_compress_at = 0;  // 0: default
int32_t g_tile = 64;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HLU_ERR_OOM : HLU_ERR_CUDA;
}
#define CKR(x, where)                                \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

template <class T>
cudaError_t upload(T** d, const std::vector<T>& h) {
  *d = nullptr;
  size_t bytes = sizeof(T) * std::max<size_t>(h.size(), 1);
  cudaError_t e = dev_malloc(d, bytes);
  if (e != cudaSuccess) return e;
  if (!h.empty()) e = cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
  return e;
}

// A schedule on the device.  The task arrays and the DAG are shared
// (read-only) between handles with the same block tree; the dependency
// counters and the ready queue belong to one handle.
struct DevSched {
  Task* tasks = nullptr;
  Term* terms = nullptr;
  Piece* pieces = nullptr;
  int64_t* pred_ptr = nullptr;
  int32_t* pred_idx = nullptr;
  int64_t* succ_ptr = nullptr;
  int32_t* succ_idx = nullptr;
  int32_t* indeg0 = nullptr;            // predecessor counts
  unsigned long long* roots = nullptr;  // tasks without predecessors, as queue entries (index + 1)
  std::vector<int32_t> h_roots;         // the same, ascending
  int32_t* indeg = nullptr;             // per handle: counters of the running launch
  unsigned long long* queue = nullptr;  // per handle: ready queue, ntasks slots
  unsigned long long* qctl = nullptr;   // per handle: claim / fill positions
  int64_t ntasks = 0;
  int64_t nterms = 0;
  bool owns_data = true;
  cudaError_t load(const Schedule& S) {
    ntasks = (int64_t)S.tasks.size();
    nterms = (int64_t)S.terms.size();
    cudaError_t e;
    if ((e = upload(&tasks, S.tasks)) != cudaSuccess) return e;
    if ((e = upload(&terms, S.terms)) != cudaSuccess) return e;
    if ((e = upload(&pieces, S.pieces)) != cudaSuccess) return e;
    if ((e = upload(&pred_ptr, S.pred_ptr)) != cudaSuccess) return e;
    if ((e = upload(&pred_idx, S.pred_idx)) != cudaSuccess) return e;
    // successor lists (edges sorted by predecessor, successors ascending)
    const int64_t ne = S.pred_ptr.empty() ? 0 : S.pred_ptr[ntasks];
    std::vector<int64_t> sp(ntasks + 1, 0);
    std::vector<int32_t> si(std::max<int64_t>(ne, 0)), in0(ntasks);
    for (int64_t t = 0; t < ntasks; ++t) {
      in0[t] = (int32_t)(S.pred_ptr[t + 1] - S.pred_ptr[t]);
      for (int64_t q = S.pred_ptr[t]; q < S.pred_ptr[t + 1]; ++q) ++sp[S.pred_idx[q] + 1];
    }
    for (int64_t t = 0; t < ntasks; ++t) sp[t + 1] += sp[t];
    std::vector<int64_t> fill(sp.begin(), sp.end() - 1);
    for (int64_t t = 0; t < ntasks; ++t)
      for (int64_t q = S.pred_ptr[t]; q < S.pred_ptr[t + 1]; ++q) si[fill[S.pred_idx[q]]++] = (int32_t)t;
    std::vector<unsigned long long> rq;
    h_roots.clear();
    for (int64_t t = 0; t < ntasks; ++t)
      if (in0[t] == 0) {
        h_roots.push_back((int32_t)t);
        rq.push_back((unsigned long long)t + 1ULL);
      }
    if ((e = upload(&succ_ptr, sp)) != cudaSuccess) return e;
    if ((e = upload(&succ_idx, si)) != cudaSuccess) return e;
    if ((e = upload(&indeg0, in0)) != cudaSuccess) return e;
    if ((e = upload(&roots, rq)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  cudaError_t alloc_state() {
    cudaError_t e = dev_malloc(&indeg, sizeof(int32_t) * std::max<int64_t>(ntasks, 1));
    if (e != cudaSuccess) return e;
    if ((e = dev_malloc(&queue, sizeof(unsigned long long) * std::max<int64_t>(ntasks, 1))) != cudaSuccess) return e;
    return dev_malloc(&qctl, sizeof(unsigned long long) * 2);
  }
  // a per-handle view of shared task data
  DevSched share() const {
    DevSched d = *this;
    d.indeg = nullptr;
    d.queue = nullptr;
    d.qctl = nullptr;
    d.owns_data = false;
    return d;
  }
  // tasks run by a launch limited to the first `limit` tasks, and its roots
  int64_t run_count(int64_t limit) const { return limit >= 0 ? std::min(limit, ntasks) : ntasks; }
  int64_t root_count(int64_t limit) const {
    if (limit < 0) return (int64_t)h_roots.size();
    return std::lower_bound(h_roots.begin(), h_roots.end(), limit) - h_roots.begin();
  }
  void free_all() {
    if (owns_data)
      for (void* p : {(void*)tasks, (void*)terms, (void*)pieces, (void*)pred_ptr, (void*)pred_idx,
                      (void*)succ_ptr,
                      (void*)succ_idx, (void*)indeg0, (void*)roots})
        if (p) dev_free(p);
    for (void* p : {(void*)indeg, (void*)queue, (void*)qctl})
      if (p) dev_free(p);
    *this = DevSched();
  }
};

// Everything derived from a block tree alone: the arena layout, the two task
// DAGs (on the device), the factor tree and the A_H fill descriptors.
struct SchedBundle {
  uint64_t key = 0;
  ArenaLayout L;
  SchedStats st;
  std::vector<Block> FB;
  DevSched dF, dS;  // shared data, no flags
  FillDesc* d_fill_dense = nullptr;
  FillDesc* d_fill_lr = nullptr;
  int32_t n_fill_dense = 0, n_fill_lr = 0;
  int64_t dense_rows = 0;
  int64_t device_bytes = 0;  // task data of both schedules on the device
  ~SchedBundle() {
    dF.free_all();
    dS.free_all();
    if (d_fill_dense) dev_free(d_fill_dense);
    if (d_fill_lr) dev_free(d_fill_lr);
  }
};

std::mutex g_cache_mu;
std::mutex g_batch_mu;            // serialises batched launches (shared order buffer)
unsigned long long* g_batch_q = nullptr;  // ready queue of batched launches
int64_t g_batch_q_len = 0;
std::vector<std::shared_ptr<SchedBundle>> g_cache;  // most recent last
size_t g_cache_entries = 16;                   // schedules kept (hlu_set_schedule_cache)
int64_t g_cache_bytes = int64_t(24) << 30;    // device bytes of cached schedules

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ULL;
  }
  return h;
}

struct KrylovWS {
  int64_t N = 0;
  int m = 0, nr = 0;
  double *V = nullptr, *Z = nullptr, *W = nullptr, *h1 = nullptr, *h2 = nullptr, *hn = nullptr, *H = nullptr,
         *cs = nullptr, *sn = nullptr, *g = nullptr, *est = nullptr, *y = nullptr, *bn = nullptr, *part = nullptr,
         *tmp = nullptr;
  int* jr = nullptr;
  // on_stream: only work queued on stream s used the buffers (GMRES states),
  // so a caller-supplied allocator gets them back after that stream drains
  // instead of after the whole device does
  void free_all(cudaStream_t s = nullptr, bool on_stream = false) {
    for (void* p : {(void*)V, (void*)Z, (void*)W, (void*)h1, (void*)h2, (void*)hn, (void*)H, (void*)cs, (void*)sn,
                    (void*)g, (void*)est, (void*)y, (void*)bn, (void*)part, (void*)tmp, (void*)jr})
      if (p) {
        if (on_stream)
          dev_free_on(p, s);
        else
          dev_free(p);
      }
    *this = KrylovWS();
  }
};

}  // namespace

namespace {
// The Schulz inverse of A_H (hlu_hinverse): four copies of the factor tree in
// its own arena, the start / iteration / apply schedules, and the iteration's
// record.
struct InvState {
  bool built = false, ready = false;
  int precision = -1;
  ArenaLayout L;
  std::vector<Block> Bx;
  SchedStats st;
  DevSched start, iter, apply;
  FillDesc* d_fill_dense = nullptr;
  FillDesc* d_fill_lr = nullptr;
  int32_t n_fill_dense = 0, n_fill_lr = 0;
  int64_t dense_rows = 0;
  void* d_arena = nullptr;
  int32_t* d_ranks = nullptr;
  int32_t* d_piv = nullptr;
  void* d_scratch = nullptr;
  int64_t scratch_stride = 0;
  int grid = 0;
  int32_t* d_status = nullptr;
  double* d_flops = nullptr;
  double* d_z = nullptr;  // residual-estimate probes (N x 4) and workspace (N x 8)
  double* d_w = nullptr;
  double alpha = 0;
  std::vector<double> res;
  void free_data() {
    for (void* p : {d_arena, (void*)d_ranks, (void*)d_piv, d_scratch, (void*)d_status, (void*)d_flops})
      if (p) dev_free(p);
    d_arena = d_scratch = nullptr;
    d_ranks = d_piv = d_status = nullptr;
    d_flops = nullptr;
    precision = -1;
    ready = false;
  }
  void free_all() {
    free_data();
    start.free_all();
    iter.free_all();
    apply.free_all();
    for (void* p : {(void*)d_fill_dense, (void*)d_fill_lr, (void*)d_z, (void*)d_w})
      if (p) dev_free(p);
    d_fill_dense = d_fill_lr = nullptr;
    d_z = d_w = nullptr;
    built = false;
  }
};
}  // namespace

struct hlu_handle {
  int n = 0, leaf = 0, rank_cap = kRankMax;
  double kappa = 0, eta = 0, eps = 0;
  int64_t eta2 = 0;
  DevMesh mesh;
  DevCSR A;
  int32_t* d_perm = nullptr;
  int32_t* d_iperm = nullptr;
  HostTrees trees;
  std::vector<Cluster> C;
  std::vector<Block> B;   // block tree (as exported)
  int32_t tile = 0;
  std::shared_ptr<SchedBundle> sb;  // factor tree, layout, DAGs (shared by identical trees)
  ArenaLayout L;                    // copy of sb->L
  DevSched dF, dS;                  // views of sb's DAGs with this handle's flags
  // factor state
  int precision = -1;
  void* d_arena = nullptr;
  int64_t arena_elems = 0;
  int32_t* d_ranks = nullptr;
  int32_t cur_nrhs = 0;  // the value last written to the right-hand-side count slot
  int32_t* d_term_p = nullptr;  // solve terms' column counts after the last factorisation
  bool term_p_fresh = false;
  int32_t* d_piv = nullptr;
  void* d_scratch = nullptr;
  int64_t scratch_stride = 0;
  int grid = 0;
  int32_t* d_status = nullptr;
  double* d_flops = nullptr;
  void** d_arenas = nullptr;
  int32_t** d_rankp = nullptr;
  int32_t** d_pivp = nullptr;
  hlu_factor_info info;
  KrylovWS kw;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  unsigned long long* d_prof = nullptr;  // executor profile of the last factorisation
  unsigned long long* d_trace = nullptr; // per-task trace of the next factorisation (debug)
  bool factor_pending = false;           // hlu_factor_async launched, hlu_factor_wait not yet done
  cudaStream_t factor_stream = nullptr;
  InvState inv;                          // Schulz inverse of A_H (hlu_hinverse)
  int32_t precond = HLU_PRECOND_LU;      // preconditioner of gmres_solve / hlu_richardson
};

namespace {

void free_factor(hlu_handle* h) {
  for (void* p : {(void*)h->d_arena, (void*)h->d_ranks, (void*)h->d_piv, (void*)h->d_scratch, (void*)h->d_status,
                  (void*)h->d_flops, (void*)h->d_arenas, (void*)h->d_rankp, (void*)h->d_pivp,
                  (void*)h->d_prof, (void*)h->d_term_p})
    if (p) dev_free(p);
  h->d_prof = nullptr;
  h->d_term_p = nullptr;
  h->term_p_fresh = false;
  h->d_arena = nullptr;
  h->d_ranks = nullptr;
  h->d_piv = nullptr;
  h->d_scratch = nullptr;
  h->d_status = nullptr;
  h->d_flops = nullptr;
  h->d_arenas = nullptr;
  h->d_rankp = nullptr;
  h->d_pivp = nullptr;
  h->precision = -1;
}

int esize(int precision) { return precision == HLU_FP64 ? 8 : 4; }

// per-CTA scratch stride in elements of the factor type
int64_t scratch_stride_elems(const ArenaLayout& L, int es) {
  return trunc_scratch_bytes(std::max(L.max_trunc_rows, 1), es) / es;
}

template <class T>
int blocks_per_sm() {
  return exec_blocks_per_sm<T>();
}

// Column count of each solve term's A (its rank after the factorisation, or
// its fixed width); -1 for a term whose width is the right-hand-side count.
__global__ void k_term_ranks(const Term* terms, int64_t n, const int32_t* ranks, int32_t nrhs_slot, int32_t* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const View& A = terms[q].A;
    out[q] = A.slot < 0 ? A.cols : (A.slot == nrhs_slot ? -1 : ranks[A.slot]);
  }
}

// Before a launch of schedule ds on h: a factorisation makes the resolved
// term widths stale; a solve launch refreshes them (stream-ordered after the
// factorisation that produced the ranks).
int prepare_terms(hlu_handle* h, DevSched& ds, cudaStream_t s) {
  if (&ds == &h->dF) {
    h->term_p_fresh = false;
    return HLU_OK;
  }
  if (&ds != &h->dS || ds.nterms == 0 || !h->d_term_p || h->term_p_fresh) return HLU_OK;
  const int blocks = (int)std::min<int64_t>((ds.nterms + 255) / 256, 1184);
  note_launch();
  k_term_ranks<<<blocks, 256, 0, s>>>(ds.terms, ds.nterms, h->d_ranks, h->L.nrhs_slot, h->d_term_p);
  CKR(cudaGetLastError(), "term widths");
  h->term_p_fresh = true;
  return HLU_OK;
}

ProbSched prob_of(hlu_handle* h, DevSched& ds, int64_t limit) {
  ProbSched p;
  std::memset(&p, 0, sizeof(p));
  p.tasks = ds.tasks;
  p.terms = ds.terms;
  p.pieces = ds.pieces;
  p.succ_ptr = ds.succ_ptr;
  p.succ_idx = ds.succ_idx;
  p.indeg = ds.indeg;
  p.arena = h->d_arena;
  p.ranks = h->d_ranks;
  p.piv = h->d_piv;
  p.eps = h->eps;
  p.ntasks = ds.ntasks;
  p.limit = ds.run_count(limit);
  p.nrhs_slot = h->L.nrhs_slot;
  p.nrhs = h->cur_nrhs;
  p.term_p = (&ds == &h->dS && h->term_p_fresh) ? h->d_term_p : nullptr;
  return p;
}

void fill_common(ExecArgs& a, hlu_handle* scratch_owner, hlu_handle* h0, bool with_flops) {
  a.scratch = scratch_owner->d_scratch;
  a.scratch_stride = scratch_owner->scratch_stride;
  a.trunc_rows = std::max(scratch_owner->L.max_trunc_rows, 1);
  a.status = h0->d_status;
  a.flops = with_flops ? h0->d_flops : nullptr;
  a.wait_limit_ns = (unsigned long long)(g_wait_limit_ms * 1e6);
  a.jacobi_tol = g_jacobi_tol;
  a.compress_at = g_compress_at;
  a.prof = with_flops ? h0->d_prof : nullptr;
  a.tf32 = (with_flops && h0->precision == HLU_TF32) ? 1 : 0;  // factorisations only; solves stay FP32
  a.trace = h0->d_trace;
}

// The executor kernel for a launch: FP64, FP32, or FP32 with TF32 tile
// products (a separate kernel: tensor memory holds it to one CTA per SM, so
// its grid is capped at that occupancy).
cudaError_t launch_exec(int precision, const ExecArgs& a, int g, cudaStream_t s) {
  if (precision == HLU_FP64) return exec_launch<double>(a, g, s);
  if (!a.tf32) return exec_launch<float>(a, g, s);
  static int tc_grid = 0;
  if (tc_grid == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    tc_grid = std::max(1, sms * std::max(tcx::exec_blocks_per_sm<float>(), 1));
  }
  return tcx::exec_launch<float>(a, std::min(g, tc_grid), s);
}

// One launch of the executor over one problem's schedule (or its first
// `limit` tasks): counters reset, queue cleared and seeded with the roots.
int exec_run(hlu_handle* h, DevSched& ds, int grid, cudaStream_t s, bool with_flops, int64_t limit = -1) {
  if (int rc = prepare_terms(h, ds, s)) return rc;
  ExecArgs a;
  std::memset(&a, 0, sizeof(a));
  a.probs[0] = prob_of(h, ds, limit);
  a.nprobs = 1;
  a.ntotal = ds.run_count(limit);
  a.queue = ds.queue;
  a.qctl = ds.qctl;
  fill_common(a, h, h, with_flops);
  if (a.ntotal == 0) return HLU_OK;
  const int64_t nr = ds.root_count(limit);
  int32_t st0[8] = {0, -1, 0, 0, 0, 0, 0, 0};
  unsigned long long q0[2] = {0ULL, (unsigned long long)nr};
  CKR(cudaMemcpyAsync(h->d_status, st0, sizeof(st0), cudaMemcpyHostToDevice, s), "status reset");
  CKR(cudaMemcpyAsync(ds.qctl, q0, sizeof(q0), cudaMemcpyHostToDevice, s), "queue reset");
  CKR(cudaMemcpyAsync(ds.indeg, ds.indeg0, sizeof(int32_t) * ds.ntasks, cudaMemcpyDeviceToDevice, s), "counters");
  CKR(cudaMemcpyAsync(ds.queue, ds.roots, sizeof(unsigned long long) * nr, cudaMemcpyDeviceToDevice, s), "roots");
  if (a.ntotal > nr)
    CKR(cudaMemsetAsync(ds.queue + nr, 0, sizeof(unsigned long long) * (a.ntotal - nr), s), "queue clear");
  int g = (int)std::min<int64_t>(grid, a.ntotal);
  cudaError_t e = launch_exec(h->precision, a, g, s);
  CKR(e, "executor launch");
  return HLU_OK;
}

// Queue seed of a batched launch: the problems' roots interleaved by relative
// position (root j of problem p at key (j + 1/2) / n_p), as queue entries
// ((p << 40) | task) + 1.
std::vector<unsigned long long> batch_roots(const std::vector<const std::vector<int32_t>*>& roots) {
  struct Item {
    double key;
    int32_t p;
    int64_t j;
    bool operator<(const Item& o) const { return key > o.key || (key == o.key && p > o.p); }
  };
  std::vector<unsigned long long> out;
  std::priority_queue<Item> pq;
  for (size_t p = 0; p < roots.size(); ++p)
    if (!roots[p]->empty()) pq.push(Item{0.5 / roots[p]->size(), (int32_t)p, 0});
  while (!pq.empty()) {
    Item it = pq.top();
    pq.pop();
    const std::vector<int32_t>& r = *roots[it.p];
    out.push_back((((unsigned long long)it.p) << 40 | (unsigned long long)r[it.j]) + 1ULL);
    if (it.j + 1 < (int64_t)r.size()) pq.push(Item{(it.j + 1.5) / r.size(), it.p, it.j + 1});
  }
  return out;
}

// One launch over the factor (which = 0) or solve (which = 1) schedules of
// several handles with the same precision.  Handle 0's status, flop counter
// and profile are used; the scratch is that of the handle with the largest
// truncation stacks; the queue (all problems' tasks) lives in *d_q.
int exec_run_batch(hlu_handle* const* hs, int count, int which, cudaStream_t s, unsigned long long** d_q,
                   int64_t* d_q_len) {
  if (count < 1 || count > kMaxBatch) return fail(HLU_ERR_ARG, "batch size");
  ExecArgs a;
  std::memset(&a, 0, sizeof(a));
  hlu_handle* hs0 = hs[0];
  hlu_handle* big = hs0;
  std::vector<const std::vector<int32_t>*> roots(count);
  int64_t total = 0;
  for (int i = 0; i < count; ++i) {
    hlu_handle* h = hs[i];
    if (h->precision != hs0->precision) return fail(HLU_ERR_ARG, "mixed precisions in a batch");
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return fail(HLU_ERR_ARG, "a handle appears twice in a batch");
    DevSched& ds = which == 0 ? h->dF : h->dS;
    if (int rc = prepare_terms(h, ds, s)) return rc;
    a.probs[i] = prob_of(h, ds, -1);
    roots[i] = &ds.h_roots;
    total += ds.ntasks;
    if (h->L.max_trunc_rows > big->L.max_trunc_rows) big = h;
  }
  a.nprobs = count;
  a.ntotal = total;
  if (total == 0) return HLU_OK;
  std::vector<unsigned long long> seed = batch_roots(roots);
  if (*d_q_len < total + 2) {
    if (*d_q) dev_free(*d_q);
    *d_q = nullptr;
    *d_q_len = 0;
    CKR(dev_malloc(d_q, sizeof(unsigned long long) * (total + 2)), "queue");
    *d_q_len = total + 2;
  }
  a.qctl = *d_q;
  a.queue = *d_q + 2;
  fill_common(a, big, hs0, which == 0);
  int32_t st0[8] = {0, -1, 0, 0, 0, 0, 0, 0};
  unsigned long long q0[2] = {0ULL, (unsigned long long)seed.size()};
  CKR(cudaMemcpyAsync(hs0->d_status, st0, sizeof(st0), cudaMemcpyHostToDevice, s), "status reset");
  CKR(cudaMemcpyAsync(a.qctl, q0, sizeof(q0), cudaMemcpyHostToDevice, s), "queue reset");
  for (int i = 0; i < count; ++i) {
    DevSched& ds = which == 0 ? hs[i]->dF : hs[i]->dS;
    CKR(cudaMemcpyAsync(ds.indeg, ds.indeg0, sizeof(int32_t) * ds.ntasks, cudaMemcpyDeviceToDevice, s), "counters");
  }
  CKR(cudaMemcpyAsync(a.queue, seed.data(), sizeof(unsigned long long) * seed.size(), cudaMemcpyHostToDevice, s),
      "seed");
  if (total > (int64_t)seed.size())
    CKR(cudaMemsetAsync(a.queue + seed.size(), 0, sizeof(unsigned long long) * (total - seed.size()), s), "clear");
  int g = (int)std::min<int64_t>(hs0->grid, a.ntotal);
  cudaError_t e = launch_exec(hs0->precision, a, g, s);
  CKR(e, "executor launch");
  // the host seed buffer must outlive the copy
  CKR(cudaStreamSynchronize(s), "sync");
  return HLU_OK;
}

int read_status(hlu_handle* h, cudaStream_t s, int32_t* out4) {
  CKR(cudaMemcpyAsync(out4, h->d_status, sizeof(int32_t) * 8, cudaMemcpyDeviceToHost, s), "status read");
  CKR(cudaStreamSynchronize(s), "sync");
  if (out4[0] == 5) return fail(HLU_ERR_TIMEOUT, "device wait exceeded its limit at task " + std::to_string(out4[1]));
  if (out4[0] == 3) return fail(HLU_ERR_ZERO_PIVOT, "zero pivot in a diagonal leaf");
  if (out4[0] == 7) return fail(HLU_ERR_STATE, "an A_H block exceeds the rank capacity");
  return HLU_OK;
}

template <class T>
int solve_impl(const hlu_handle* hc, const double* b, double* x, int32_t nrhs, int64_t ld, cudaStream_t s) {
  hlu_handle* h = const_cast<hlu_handle*>(hc);
  const int64_t N = h->A.N;
  T* work = reinterpret_cast<T*>(h->d_arena) + h->L.work_off;
  for (int32_t c0 = 0; c0 < nrhs; c0 += h->L.nrhs_max) {
    int32_t nc = std::min(h->L.nrhs_max, nrhs - c0);
    CKR(set_int(h->d_ranks + h->L.nrhs_slot, nc, s), "nrhs slot");
    h->cur_nrhs = nc;
    CKR(gather_cast<T>(N, h->d_perm, b + c0 * ld, ld, work, nc, s), "gather");
    int rc = exec_run(h, h->dS, h->grid, s, false);
    if (rc) return rc;
    CKR(scatter_cast<T>(N, h->d_perm, work, x + c0 * ld, ld, nc, s), "scatter");
  }
  return HLU_OK;
}

// One launch of the executor over a schedule of the Schulz inverse (its own
// arena and rank slots); alpha is the launch scalar of the start, nrhs the
// column count of the apply.
int exec_run_inv(hlu_handle* h, DevSched& ds, double alpha, int32_t nrhs, cudaStream_t s) {
  InvState& iv = h->inv;
  ExecArgs a;
  std::memset(&a, 0, sizeof(a));
  ProbSched& p = a.probs[0];
  p.tasks = ds.tasks;
  p.terms = ds.terms;
  p.pieces = ds.pieces;
  p.succ_ptr = ds.succ_ptr;
  p.succ_idx = ds.succ_idx;
  p.indeg = ds.indeg;
  p.arena = iv.d_arena;
  p.ranks = iv.d_ranks;
  p.piv = iv.d_piv;
  p.eps = h->eps;
  p.ntasks = ds.ntasks;
  p.limit = ds.ntasks;
  p.nrhs_slot = iv.L.nrhs_slot;
  p.nrhs = nrhs;
  p.term_p = nullptr;
  p.alpha = alpha;
  a.nprobs = 1;
  a.ntotal = ds.ntasks;
  a.queue = ds.queue;
  a.qctl = ds.qctl;
  a.scratch = iv.d_scratch;
  a.scratch_stride = iv.scratch_stride;
  a.trunc_rows = std::max(iv.L.max_trunc_rows, 1);
  a.status = iv.d_status;
  a.flops = iv.d_flops;
  a.wait_limit_ns = (unsigned long long)(g_wait_limit_ms * 1e6);
  a.jacobi_tol = g_jacobi_tol;
  a.compress_at = g_compress_at;
  if (a.ntotal == 0) return HLU_OK;
  const int64_t nr = ds.root_count(-1);
  int32_t st0[8] = {0, -1, 0, 0, 0, 0, 0, 0};
  unsigned long long q0[2] = {0ULL, (unsigned long long)nr};
  CKR(cudaMemcpyAsync(iv.d_status, st0, sizeof(st0), cudaMemcpyHostToDevice, s), "status reset");
  CKR(cudaMemcpyAsync(ds.qctl, q0, sizeof(q0), cudaMemcpyHostToDevice, s), "queue reset");
  CKR(cudaMemcpyAsync(ds.indeg, ds.indeg0, sizeof(int32_t) * ds.ntasks, cudaMemcpyDeviceToDevice, s), "counters");
  CKR(cudaMemcpyAsync(ds.queue, ds.roots, sizeof(unsigned long long) * nr, cudaMemcpyDeviceToDevice, s), "roots");
  if (a.ntotal > nr)
    CKR(cudaMemsetAsync(ds.queue + nr, 0, sizeof(unsigned long long) * (a.ntotal - nr), s), "queue clear");
  const int g = (int)std::min<int64_t>(iv.grid, a.ntotal);
  CKR(launch_exec(iv.precision, a, g, s), "executor launch");
  int32_t stf[8];
  CKR(cudaMemcpyAsync(stf, iv.d_status, sizeof(stf), cudaMemcpyDeviceToHost, s), "status read");
  CKR(cudaStreamSynchronize(s), "sync");
  if (stf[0] == 5) return fail(HLU_ERR_TIMEOUT, "device wait exceeded its limit");
  return HLU_OK;
}

// x = B_H b through the apply schedule, nrhs_max columns per launch
template <class T>
int hinv_apply_impl(hlu_handle* h, const double* b, double* x, int32_t nrhs, int64_t ld, cudaStream_t s) {
  InvState& iv = h->inv;
  const int64_t N = h->A.N;
  T* work = reinterpret_cast<T*>(iv.d_arena) + iv.L.work_off;
  T* out = reinterpret_cast<T*>(iv.d_arena) + iv.L.out_off;
  for (int32_t c0 = 0; c0 < nrhs; c0 += iv.L.nrhs_max) {
    const int32_t nc = std::min(iv.L.nrhs_max, nrhs - c0);
    CKR(set_int(iv.d_ranks + iv.L.nrhs_slot, nc, s), "nrhs slot");
    CKR(gather_cast<T>(N, h->d_perm, b + c0 * ld, ld, work, nc, s), "gather");
    int rc = exec_run_inv(h, iv.apply, 0.0, nc, s);
    if (rc) return rc;
    CKR(scatter_cast<T>(N, h->d_perm, out, x + c0 * ld, ld, nc, s), "scatter");
  }
  return HLU_OK;
}
int hinv_apply_any(hlu_handle* h, const double* b, double* x, int32_t nrhs, int64_t ld, cudaStream_t s) {
  return h->inv.precision == HLU_FP64 ? hinv_apply_impl<double>(h, b, x, nrhs, ld, s)
                                      : hinv_apply_impl<float>(h, b, x, nrhs, ld, s);
}

// the preconditioner of the Krylov solvers: the H-LU solve, or B_H x
int solve_any(const hlu_handle* hc, const double* b, double* x, int32_t nrhs, int64_t ld, cudaStream_t s) {
  hlu_handle* h = const_cast<hlu_handle*>(hc);
  if (h->precond == HLU_PRECOND_HINV) return hinv_apply_any(h, b, x, nrhs, ld, s);
  return h->precision == HLU_FP64 ? solve_impl<double>(h, b, x, nrhs, ld, s) : solve_impl<float>(h, b, x, nrhs, ld, s);
}
// whether the selected preconditioner can run
bool precond_ready(const hlu_handle* h) {
  if (h->precond == HLU_PRECOND_HINV) return h->inv.ready;
  return h->precision >= 0 && !h->factor_pending;
}

int ensure_kw(hlu_handle* h, int m, int nr) {
  KrylovWS& k = h->kw;
  if (k.N == h->A.N && k.m >= m && k.nr >= nr) return HLU_OK;
  k.free_all();
  int64_t N = h->A.N;
  // the sizes are recorded only once every buffer exists: a workspace left
  // partial by an allocation failure is freed and rebuilt by the next call
  // instead of passing the size test above with null buffers
  CKR(dev_malloc(&k.V, sizeof(double) * N * (m + 1) * nr), "alloc V");
  CKR(dev_malloc(&k.Z, sizeof(double) * N * (m + 1) * nr), "alloc Z");
  CKR(dev_malloc(&k.W, sizeof(double) * N * nr), "alloc W");
  CKR(dev_malloc(&k.tmp, sizeof(double) * N * nr), "alloc tmp");
  CKR(dev_malloc(&k.h1, sizeof(double) * (m + 1) * nr), "alloc");
  CKR(dev_malloc(&k.h2, sizeof(double) * (m + 1) * nr), "alloc");
  CKR(dev_malloc(&k.hn, sizeof(double) * nr), "alloc");
  CKR(dev_malloc(&k.H, sizeof(double) * (m + 1) * m * nr), "alloc");
  CKR(dev_malloc(&k.cs, sizeof(double) * m * nr), "alloc");
  CKR(dev_malloc(&k.sn, sizeof(double) * m * nr), "alloc");
  CKR(dev_malloc(&k.g, sizeof(double) * (m + 1) * nr), "alloc");
  CKR(dev_malloc(&k.est, sizeof(double) * nr), "alloc");
  CKR(dev_malloc(&k.y, sizeof(double) * m * nr), "alloc");
  CKR(dev_malloc(&k.bn, sizeof(double) * nr), "alloc");
  CKR(dev_malloc(&k.part, sizeof(double) * std::max(multidot_partials(N, m + 1, nr), 1)), "alloc");
  CKR(dev_malloc(&k.jr, sizeof(int) * nr), "alloc");
  k.N = N;
  k.m = m;
  k.nr = nr;
  return HLU_OK;
}

// column norms of X (N x nr, ld) into dev[nr] and host[nr]
int col_norms(hlu_handle* h, const double* X, int64_t ld, int nr, double* dev, double* host, cudaStream_t s) {
  KrylovWS& k = h->kw;
  CKR(multidot(h->A.N, X, ld, 1, X, ld, nr, k.part, dev, 1, s), "norm");
  CKR(sqrt_inplace(dev, nr, s), "sqrt");
  if (host) {
    CKR(cudaMemcpyAsync(host, dev, sizeof(double) * nr, cudaMemcpyDeviceToHost, s), "norm d2h");
    CKR(cudaStreamSynchronize(s), "sync");
  }
  return HLU_OK;
}

int gmres_chunk(hlu_handle* h, const double* b, double* x, int nr, int64_t ld, int m, double tol, int maxit,
                hlu_stats* st, cudaStream_t s) {
  int rc = ensure_kw(h, m, nr);
  if (rc) return rc;
  KrylovWS& k = h->kw;
  const int64_t N = h->A.N;
  const int64_t ldr = N * (m + 1);
  std::vector<double> bn(nr), beta(nr), est(nr);
  std::vector<int> conv(nr, 0), jr(nr, 0);
  for (int r = 0; r < nr; ++r) CKR(cudaMemsetAsync(x + r * ld, 0, sizeof(double) * N, s), "x0");
  rc = col_norms(h, b, ld, nr, k.bn, bn.data(), s);
  if (rc) return rc;
  for (int r = 0; r < nr; ++r)
    if (!std::isfinite(bn[r]))
      return fail(HLU_ERR_ARG, "right-hand side column " + std::to_string(r) + " is not finite (x = 0 written)");
  int iters = 0, restarts = 0;
  double pms = 0;
  bool broke = false;  // a residual turned non-finite: the iteration cannot go on
  for (;;) {
    CKR(residual(h->A.rowptr, h->A.col, h->A.val, N, x, ld, b, ld, k.V, ldr, nr, s), "residual");
    rc = col_norms(h, k.V, ldr, nr, k.hn, beta.data(), s);
    if (rc) return rc;
    bool all = true;
    for (int r = 0; r < nr; ++r) {
      conv[r] = (bn[r] == 0.0) || (beta[r] <= tol * bn[r]);
      all = all && conv[r];
      broke = broke || !std::isfinite(beta[r]);
    }
    if (all || iters >= maxit || broke) break;
    CKR(scale_cols(N, k.V, ldr, k.hn, k.V, ldr, nr, s), "scale");
    CKR(init_g(nr, m, k.hn, k.g, s), "init g");
    std::fill(jr.begin(), jr.end(), 0);
    for (int j = 0; j < m; ++j) {
      CKR(cudaEventRecord(h->ev0, s), "ev");
      rc = solve_any(h, k.V + j * N, k.Z + j * N, nr, ldr, s);
      if (rc) return rc;
      CKR(cudaEventRecord(h->ev1, s), "ev");
      CKR(spmv(h->A.rowptr, h->A.col, h->A.val, N, k.Z + j * N, ldr, k.W, N, nr, s), "spmv");
      CKR(multidot(N, k.V, ldr, j + 1, k.W, N, nr, k.part, k.h1, m + 1, s), "cgs1");
      CKR(multiaxpy(N, k.V, ldr, j + 1, k.h1, m + 1, k.W, N, nr, s), "cgs1 axpy");
      CKR(multidot(N, k.V, ldr, j + 1, k.W, N, nr, k.part, k.h2, m + 1, s), "cgs2");
      CKR(multiaxpy(N, k.V, ldr, j + 1, k.h2, m + 1, k.W, N, nr, s), "cgs2 axpy");
      rc = col_norms(h, k.W, N, nr, k.hn, nullptr, s);
      if (rc) return rc;
      CKR(scale_cols(N, k.W, N, k.hn, k.V + (j + 1) * N, ldr, nr, s), "scale");
      CKR(givens(nr, m, j, k.h1, k.h2, m + 1, k.hn, k.H, k.cs, k.sn, k.g, k.est, s), "givens");
      CKR(cudaMemcpyAsync(est.data(), k.est, sizeof(double) * nr, cudaMemcpyDeviceToHost, s), "est");
      CKR(cudaStreamSynchronize(s), "sync");
      float ms = 0;
      cudaEventElapsedTime(&ms, h->ev0, h->ev1);
      pms += ms;
      if (st) st->precond_applies++;
      ++iters;
      bool done = true;
      for (int r = 0; r < nr; ++r) {
        if (conv[r]) continue;
        if (jr[r] == 0 && est[r] <= tol * bn[r]) jr[r] = j + 1;
        done = done && jr[r] > 0;
      }
      if (done || j == m - 1 || iters >= maxit) {
        for (int r = 0; r < nr; ++r)
          if (!conv[r] && jr[r] == 0) jr[r] = j + 1;
        break;
      }
    }
    for (int r = 0; r < nr; ++r)
      if (conv[r]) jr[r] = 0;
    CKR(cudaMemcpyAsync(k.jr, jr.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, s), "jr");
    CKR(backsub(nr, m, k.jr, k.H, k.g, k.y, s), "backsub");
    // Z columns live with stride ldr (same layout as V)
    CKR(xupdate(N, k.Z, ldr, m, k.y, x, ld, nr, s), "xupdate");
    ++restarts;
  }
  if (st) {
    st->iterations = std::max(st->iterations, iters);
    st->restarts = std::max(st->restarts, restarts);
    double rmax = 0, amax = 0;
    bool all = true;
    for (int r = 0; r < nr; ++r) {
      double rr = bn[r] > 0 ? beta[r] / bn[r] : 0.0;
      rmax = std::max(rmax, rr);
      amax = std::max(amax, beta[r]);
      all = all && conv[r];
    }
    st->relres_max = std::max(st->relres_max, rmax);
    st->abs_res_max = std::max(st->abs_res_max, amax);
    st->converged = st->converged && all;
    st->precond_ms += pms;
  }
  bool all = true;
  for (int r = 0; r < nr; ++r) all = all && conv[r];
  if (broke) return fail(HLU_ERR_NOT_CONVERGED, "GMRES stopped: a residual is not finite");
  return all ? HLU_OK : fail(HLU_ERR_NOT_CONVERGED, "GMRES reached maxit");
}

}  // namespace

extern "C" {

const char* hlu_status_string(int s) {
  switch (s) {
    case HLU_OK: return "HLU_OK";
    case HLU_ERR_ARG: return "HLU_ERR_ARG";
    case HLU_ERR_OOM: return "HLU_ERR_OOM";
    case HLU_ERR_ZERO_PIVOT: return "HLU_ERR_ZERO_PIVOT";
    case HLU_ERR_NOT_CONVERGED: return "HLU_ERR_NOT_CONVERGED";
    case HLU_ERR_TIMEOUT: return "HLU_ERR_TIMEOUT";
    case HLU_ERR_CUDA: return "HLU_ERR_CUDA";
    case HLU_ERR_STATE: return "HLU_ERR_STATE";
    default: return "HLU_ERR_UNKNOWN";
  }
}
const char* hlu_last_error(void) { return g_err.c_str(); }
void hlu_set_wait_limit_ms(double ms) {
  if (ms > 0) g_wait_limit_ms = ms;
}
void hlu_set_tile(int32_t tile) { g_tile = std::max(0, std::min(tile, (int32_t)64)); }


int64_t hlu_n(const hlu_handle* h) { return h ? h->A.N : 0; }
int hlu_mesh_kuhn_cube(int32_t n, hlu_mesh* out) {
  if (!out || n < 1 || n > 200) return fail(HLU_ERR_ARG, "bad argument");
  const int64_t nv = (int64_t)(n + 1) * (n + 1) * (n + 1), nt = (int64_t)6 * n * n * n;
  double* xyz = (double*)std::malloc(sizeof(double) * 3 * nv);
  int32_t* tets = (int32_t*)std::malloc(sizeof(int32_t) * 4 * nt);
  if (!xyz || !tets) {
    std::free(xyz);
    std::free(tets);
    return fail(HLU_ERR_OOM, "host allocation failed");
  }
  for (int64_t v = 0; v < nv; ++v) {
    const int64_t i = v / ((int64_t)(n + 1) * (n + 1)), j = (v / (n + 1)) % (n + 1), k = v % (n + 1);
    xyz[3 * v] = (double)i / n;
    xyz[3 * v + 1] = (double)j / n;
    xyz[3 * v + 2] = (double)k / n;
  }
  // tetrahedron 6 c + p of sub-cube c = (c0 n + c1) n + c2: corners c, c + e_p0,
  // c + e_p0 + e_p1, c + (1, 1, 1) for the axis permutations p in lexicographic order
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int64_t c = 0; c < (int64_t)n * n * n; ++c) {
    const int64_t c0 = c / ((int64_t)n * n), c1 = (c / n) % n, c2 = c % n;
    for (int p = 0; p < 6; ++p) {
      int64_t q[3] = {c0, c1, c2};
      int32_t* t = tets + 4 * (6 * c + p);
      t[0] = (int32_t)((q[0] * (n + 1) + q[1]) * (n + 1) + q[2]);
      for (int s = 0; s < 3; ++s) {
        q[perms[p][s]] += 1;
        t[s + 1] = (int32_t)((q[0] * (n + 1) + q[1]) * (n + 1) + q[2]);
      }
    }
  }
  out->nv = (int32_t)nv;
  out->nt = (int32_t)nt;
  out->xyz = xyz;
  out->tets = tets;
  out->lattice_n = n;
  out->beta = nullptr;
  return HLU_OK;
}

void hlu_mesh_free(hlu_mesh* m) {
  if (!m) return;
  std::free(const_cast<double*>(m->xyz));
  std::free(const_cast<int32_t*>(m->tets));
  m->xyz = nullptr;
  m->tets = nullptr;
  m->nv = m->nt = 0;
  m->lattice_n = 0;
}

int hlu_set_schedule_cache(int32_t entries, int64_t bytes) {
  if (entries < 1 || bytes < 0) return fail(HLU_ERR_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(g_cache_mu);
  g_cache_entries = (size_t)entries;
  g_cache_bytes = bytes;
  return HLU_OK;
}
int64_t hlu_launch_count(void) { return g_launches.load(); }

void hlu_destroy(hlu_handle* h) {
  if (!h) return;
  if (h->factor_pending) cudaEventSynchronize(h->ev1);  // no kernel may still use the memory
  h->inv.free_all();
  free_factor(h);
  h->dF.free_all();
  h->dS.free_all();
  h->kw.free_all();
  h->sb.reset();
  for (void* p : {(void*)h->mesh.dofmap, (void*)h->mesh.edges, (void*)h->mesh.pts, (void*)h->mesh.xyz,
                  (void*)h->mesh.tets, (void*)h->mesh.ekeys, (void*)h->mesh.beta, (void*)h->A.rowptr,
                  (void*)h->A.col, (void*)h->A.val,
                  (void*)h->d_perm, (void*)h->d_iperm})
    if (p) dev_free(p);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

int hlu_build(const hlu_mesh* mesh, double kappa, int32_t leaf, double eta, double eps, int32_t rank_cap,
              void* stream, hlu_handle** out) {
  NvtxRange nvtx_("hlu_build");
  try {
    if (!mesh || !out) return fail(HLU_ERR_ARG, "null argument");
    *out = nullptr;
    const int n = mesh->lattice_n;
    if (n > 200 || n < 0) return fail(HLU_ERR_ARG, "lattice_n out of range");
    if (n == 0) {  // a general mesh: check what the device code relies on
      if (!mesh->xyz || !mesh->tets || mesh->nv < 4 || mesh->nt < 1)
        return fail(HLU_ERR_ARG, "a general mesh needs nv >= 4 vertices, nt >= 1 tetrahedra, xyz and tets");
      if (mesh->nv >= (1 << 21)) return fail(HLU_ERR_ARG, "at most 2^21 - 1 vertices");
      for (int64_t q = 0; q < 4 * (int64_t)mesh->nt; ++q)
        if (mesh->tets[q] < 0 || mesh->tets[q] >= mesh->nv) return fail(HLU_ERR_ARG, "tetrahedron vertex id out of range");
      for (int64_t t = 0; t < mesh->nt; ++t) {
        const int32_t* v = mesh->tets + 4 * t;
        for (int a = 0; a < 4; ++a)
          for (int b = a + 1; b < 4; ++b)
            if (v[a] == v[b]) return fail(HLU_ERR_ARG, "a tetrahedron repeats a vertex");
      }
      for (int64_t q = 0; q < 3 * (int64_t)mesh->nv; ++q)
        if (!std::isfinite(mesh->xyz[q])) return fail(HLU_ERR_ARG, "vertex coordinates must be finite");
    }
    const int64_t n_tets = n > 0 ? (int64_t)6 * n * n * n : (int64_t)mesh->nt;
    if (mesh->beta)
      for (int64_t t = 0; t < n_tets; ++t)
        if (!(std::isfinite(mesh->beta[t]) && mesh->beta[t] > 0))
          return fail(HLU_ERR_ARG, "beta must be finite and positive on every tetrahedron");
    if (leaf < 2 || leaf > 64) return fail(HLU_ERR_ARG, "leaf must be in [2, 64]");
    if (!(eta > 0)) return fail(HLU_ERR_ARG, "eta must be > 0");
    double e2 = eta * eta;
    int64_t eta2 = (int64_t)std::llround(e2);
    if (std::fabs(e2 - (double)eta2) > 1e-12) return fail(HLU_ERR_ARG, "eta^2 must be an integer");
    if (!(eps > 0) || !(kappa > 0)) return fail(HLU_ERR_ARG, "eps and kappa must be > 0");
    if (rank_cap <= 0) rank_cap = kRankMax;
    if (rank_cap > kRankMax) return fail(HLU_ERR_ARG, "rank_cap must be <= " + std::to_string(kRankMax));
    cudaStream_t s = (cudaStream_t)stream;
    hlu_handle* h = new hlu_handle();
    h->n = n;
    h->leaf = leaf;
    h->kappa = kappa;
    h->eta = eta;
    h->eta2 = eta2;
    h->eps = eps;
    h->rank_cap = rank_cap;
    std::memset(&h->info, 0, sizeof(h->info));
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char* w) {
      int rc = cuda_fail(err, w);
      hlu_destroy(h);
      return rc;
    };
    if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return bail(e, "event");
    if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return bail(e, "event");
    if (n > 0)
      e = build_mesh_dofs(n, s, h->mesh);
    else
      e = build_mesh_general(mesh->nv, mesh->nt, mesh->xyz, mesh->tets, s, h->mesh);
    if (e != cudaSuccess) return bail(e, "mesh");
    if (mesh->beta) {
      if ((e = dev_malloc(&h->mesh.beta, sizeof(double) * n_tets)) != cudaSuccess) return bail(e, "beta");
      if ((e = cudaMemcpyAsync(h->mesh.beta, mesh->beta, sizeof(double) * n_tets, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return bail(e, "beta");
    }
    if ((e = assemble_csr(h->mesh, kappa, s, h->A)) != cudaSuccess) return bail(e, "assembly");
    const int64_t N = h->A.N;
    if ((e = dev_malloc(&h->d_perm, sizeof(int32_t) * N)) != cudaSuccess) return bail(e, "perm");
    if ((e = dev_malloc(&h->d_iperm, sizeof(int32_t) * N)) != cudaSuccess) return bail(e, "iperm");
    if ((e = build_trees(h->mesh, leaf, eta2, s, h->trees, h->d_perm)) != cudaSuccess) return bail(e, "trees");
    if ((e = invert_perm((int32_t)N, h->d_perm, h->d_iperm, s)) != cudaSuccess) return bail(e, "iperm");
    trees_from_export(h->trees.nc, h->trees.clusters.data(), h->trees.nb, h->trees.blocks.data(), h->C, h->B);
    h->tile = std::min(g_tile, (int32_t)64);
    const int32_t nrhs_max = 16;
    uint64_t key = 1469598103934665603ULL;
    key = fnv1a(key, h->trees.clusters.data(), sizeof(int32_t) * h->trees.clusters.size());
    key = fnv1a(key, h->trees.blocks.data(), sizeof(int32_t) * h->trees.blocks.size());
    int32_t params[4] = {rank_cap, h->tile, nrhs_max, (int32_t)N};
    key = fnv1a(key, params, sizeof(params));
    bool cache_hit = false;
    {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      for (size_t i = 0; i < g_cache.size(); ++i)
        if (g_cache[i]->key == key) {
          h->sb = g_cache[i];
          cache_hit = true;
          g_cache.erase(g_cache.begin() + i);
          g_cache.push_back(h->sb);
          break;
        }
    }
    if (!h->sb) {
      auto sb = std::make_shared<SchedBundle>();
      sb->key = key;
      Schedule F, S;
      build_schedules(h->C, h->B, rank_cap, nrhs_max, h->tile, sb->L, F, S, sb->st,
                      &sb->FB);
      if ((e = sb->dF.load(F)) != cudaSuccess) return bail(e, "upload factor schedule");
      if ((e = sb->dS.load(S)) != cudaSuccess) return bail(e, "upload solve schedule");
      // A_H fill descriptors
      std::vector<FillDesc> fd, fl;
      int64_t rows = 0;
      for (size_t b = 0; b < sb->FB.size(); ++b) {
        const Block& bk = sb->FB[b];
        if (bk.kind == KIND_SUB) continue;
        FillDesc f;
        std::memset(&f, 0, sizeof(f));
        f.roff = h->C[bk.row].off;
        f.m = h->C[bk.row].size;
        f.coff = h->C[bk.col].off;
        f.n = h->C[bk.col].size;
        if (bk.kind == KIND_DENSE) {
          f.off = sb->L.dense_off[b];
          f.row_prefix = rows;
          rows += f.m;
          fd.push_back(f);
        } else {
          f.off = sb->L.x_off[b];
          f.off2 = sb->L.y_off[b];
          f.slot = sb->L.slot[b];
          f.cap = sb->L.cap[b];
          fl.push_back(f);
        }
      }
      sb->n_fill_dense = (int32_t)fd.size();
      sb->n_fill_lr = (int32_t)fl.size();
      sb->dense_rows = rows;
      if ((e = upload(&sb->d_fill_dense, fd)) != cudaSuccess) return bail(e, "fill desc");
      if ((e = upload(&sb->d_fill_lr, fl)) != cudaSuccess) return bail(e, "fill desc");
      for (const Schedule* sc : {&F, &S})
        sb->device_bytes += (int64_t)(sizeof(Task) * sc->tasks.size() +
                                      sizeof(Term) * sc->terms.size() + sizeof(Piece) * sc->pieces.size() +
                                      2 * sizeof(int64_t) * (sc->tasks.size() + 1) + 2 * sizeof(int32_t) *
                                      sc->pred_idx.size() + 2 * sizeof(int32_t) * sc->tasks.size());
      h->sb = sb;
      std::lock_guard<std::mutex> lk(g_cache_mu);
      g_cache.push_back(sb);
      // bounded by entries and by device bytes (least recently used first;
      // handles still holding an evicted schedule keep it alive)
      auto cached_bytes = [&]() {
        int64_t b = 0;
        for (const auto& e : g_cache) b += e->device_bytes;
        return b;
      };
      while (g_cache.size() > g_cache_entries || (g_cache.size() > 1 && cached_bytes() > g_cache_bytes))
        g_cache.erase(g_cache.begin());
    }
    h->L = h->sb->L;
    h->dF = h->sb->dF.share();
    h->dS = h->sb->dS.share();
    if ((e = h->dF.alloc_state()) != cudaSuccess) return bail(e, "queue");
    if ((e = h->dS.alloc_state()) != cudaSuccess) return bail(e, "queue");
    if (h->dS.nterms > 0 && (e = dev_malloc(&h->d_term_p, sizeof(int32_t) * h->dS.nterms)) != cudaSuccess)
      return bail(e, "term widths");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bail(e, "sync");
    h->info.n_tasks = h->sb->st.n_factor_tasks;
    h->info.n_solve_tasks = h->sb->st.n_solve_tasks;
    h->info.schedule_ms = cache_hit ? 0.0 : h->sb->st.host_ms;
    h->info.n_clusters = h->trees.nc;
    h->info.n_blocks = h->trees.nb;
    for (const Block& bk : h->B) {
      h->info.n_adm += bk.kind == KIND_ADM;
      h->info.n_dense += bk.kind == KIND_DENSE;
    }
    *out = h;
    return HLU_OK;
  } catch (const std::bad_alloc&) {
    return fail(HLU_ERR_OOM, "host allocation failed");
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_export_trees(const hlu_handle* h, int32_t* perm, int32_t* clusters, int32_t* blocks, int64_t* sizes) {
  if (!h || !sizes) return fail(HLU_ERR_ARG, "null argument");
  sizes[0] = h->trees.nc;
  sizes[1] = h->trees.nb;
  if (perm) std::memcpy(perm, h->trees.perm.data(), sizeof(int32_t) * h->trees.perm.size());
  if (clusters) std::memcpy(clusters, h->trees.clusters.data(), sizeof(int32_t) * h->trees.clusters.size());
  if (blocks) std::memcpy(blocks, h->trees.blocks.data(), sizeof(int32_t) * h->trees.blocks.size());
  return HLU_OK;
}

int hlu_export_csr(const hlu_handle* h, int64_t* rowptr, int32_t* col, double* val, int64_t* nnz) {
  if (!h || !nnz) return fail(HLU_ERR_ARG, "null argument");
  *nnz = h->A.nnz;
  if (rowptr) CKR(cudaMemcpy(rowptr, h->A.rowptr, sizeof(int64_t) * (h->A.N + 1), cudaMemcpyDeviceToHost), "csr");
  if (col) CKR(cudaMemcpy(col, h->A.col, sizeof(int32_t) * h->A.nnz, cudaMemcpyDeviceToHost), "csr");
  if (val) CKR(cudaMemcpy(val, h->A.val, sizeof(double) * h->A.nnz, cudaMemcpyDeviceToHost), "csr");
  return HLU_OK;
}

int hlu_rhs_manufactured(const hlu_handle* h, double* b_dev, void* stream) {
  if (!h || !b_dev) return fail(HLU_ERR_ARG, "null argument");
  CKR(manufactured_rhs(h->mesh, h->kappa, b_dev, (cudaStream_t)stream), "rhs");
  return HLU_OK;
}

int hlu_rhs_constant_current(const hlu_handle* h, double jx, double jy, double jz, double* b_dev, void* stream) {
  if (!h || !b_dev) return fail(HLU_ERR_ARG, "null argument");
  if (!std::isfinite(jx) || !std::isfinite(jy) || !std::isfinite(jz)) return fail(HLU_ERR_ARG, "J must be finite");
  const double J[3] = {jx, jy, jz};
  CKR(constant_current_rhs(h->mesh, J, b_dev, (cudaStream_t)stream), "rhs (constant current)");
  return HLU_OK;
}

int hlu_rhs_manufactured_noalloc(const hlu_handle* h, double* b_dev, void* stream) {
  if (!h || !b_dev) return fail(HLU_ERR_ARG, "null argument");
  if (h->n < 1) return fail(HLU_ERR_ARG, "the allocation-free load vector takes Kuhn-cube meshes only");
  const int64_t need = (int64_t)36 * h->n * h->n * h->n;
  if (need > rhs_noalloc_max_entries())
    return fail(HLU_ERR_ARG, "mesh needs " + std::to_string(need) + " element contributions; the fixed scratch holds " +
                                 std::to_string(rhs_noalloc_max_entries()) + " (n <= 24)");
  CKR(manufactured_rhs_noalloc(h->mesh, h->kappa, b_dev, (cudaStream_t)stream), "rhs (no allocation)");
  return HLU_OK;
}

int hlu_spmv(const hlu_handle* h, const double* x, double* y, int32_t nrhs, int64_t ld, void* stream) {
  if (!h || !x || !y || nrhs < 1 || ld < h->A.N) return fail(HLU_ERR_ARG, "bad argument");
  CKR(spmv(h->A.rowptr, h->A.col, h->A.val, h->A.N, x, ld, y, ld, nrhs, (cudaStream_t)stream), "spmv");
  return HLU_OK;
}

int64_t hlu_factor_bytes_estimate(const hlu_handle* h, int32_t precision) {
  if (!h || (precision != HLU_FP64 && precision != HLU_FP32 && precision != HLU_TF32)) return -1;
  int es = esize(precision);
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (int64_t)sms * 2;
  return h->L.total * es + grid * scratch_stride_elems(h->L, es) * es + (int64_t)h->L.n_slots * 4 + h->L.piv_total * 4;
}

static int factor_impl(hlu_handle* h, int32_t precision, void* stream, int64_t limit);
int hlu_factor(hlu_handle* h, int32_t precision, void* stream) {
  NvtxRange nvtx_("hlu_factor");
  return factor_impl(h, precision, stream, -1);
}

// allocation for `precision` (first time), rank/status/flop resets, A_H fill
static int factor_prepare(hlu_handle* h, int32_t precision, cudaStream_t s) {
  const int es = esize(precision);
  if (h->precision < 0 || esize(h->precision) != es) {  // FP32 and TF32 share the FP32 storage
    free_factor(h);
    int dev = 0;
    CKR(cudaGetDevice(&dev), "device");
    int sms = 0;
    CKR(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sms");
    int bps = precision == HLU_FP64 ? blocks_per_sm<double>() : blocks_per_sm<float>();
    if (bps < 1) return fail(HLU_ERR_CUDA, "executor does not fit on an SM");
    h->grid = sms * bps;
    h->scratch_stride = scratch_stride_elems(h->L, es);
    h->arena_elems = h->L.total;
    CKR(dev_malloc(&h->d_arena, (size_t)es * h->L.total), "arena");
    CKR(dev_malloc(&h->d_ranks, sizeof(int32_t) * std::max(h->L.n_slots, 1)), "ranks");
    CKR(dev_malloc(&h->d_piv, sizeof(int32_t) * std::max<int64_t>(h->L.piv_total, 1)), "piv");
    CKR(dev_malloc(&h->d_scratch, (size_t)es * h->scratch_stride * h->grid), "scratch");
    CKR(dev_malloc(&h->d_status, sizeof(int32_t) * 8), "status");
    CKR(dev_malloc(&h->d_flops, sizeof(double)), "flops");
    CKR(dev_malloc(&h->d_prof, sizeof(unsigned long long) * kProfEntries), "prof");
  }
  h->precision = precision;
  CKR(cudaMemsetAsync(h->d_ranks, 0, sizeof(int32_t) * std::max(h->L.n_slots, 1), s), "ranks");
  h->cur_nrhs = 0;
  int32_t st0[8] = {0, -1, 0, 0, 0, 0, 0, 0};
  CKR(cudaMemcpyAsync(h->d_status, st0, sizeof(st0), cudaMemcpyHostToDevice, s), "status");
  cudaError_t e;
  if (precision == HLU_FP64)
    e = fill_ah<double>(h->A, h->d_perm, h->d_iperm, h->sb->d_fill_dense, h->sb->n_fill_dense, h->sb->dense_rows,
                        h->sb->d_fill_lr, h->sb->n_fill_lr, (double*)h->d_arena, h->L.work_off, h->L.ident_off,
                        h->L.ident_n, h->d_ranks, h->d_status, s);
  else
    e = fill_ah<float>(h->A, h->d_perm, h->d_iperm, h->sb->d_fill_dense, h->sb->n_fill_dense, h->sb->dense_rows,
                       h->sb->d_fill_lr, h->sb->n_fill_lr, (float*)h->d_arena, h->L.work_off, h->L.ident_off,
                       h->L.ident_n, h->d_ranks, h->d_status, s);
  CKR(e, "A_H fill");
  int32_t stf[8];
  int rc = read_status(h, s, stf);
  if (rc) return rc;
  CKR(cudaMemsetAsync(h->d_flops, 0, sizeof(double), s), "flops");
  CKR(cudaMemsetAsync(h->d_prof, 0, sizeof(unsigned long long) * kProfEntries, s), "prof");
  return HLU_OK;
}

// statistics after the factorisation ran (status read from `status_of`)
static int factor_finish(hlu_handle* h, hlu_handle* status_of, cudaStream_t s, float ms) {
  int32_t stf[8];
  int rc = read_status(status_of, s, stf);
  h->info.factor_ms = ms;
  h->info.rank_cap_hits = stf[2];
  h->info.rank_wanted_max = stf[4];
  h->info.trunc_dense_fallbacks = stf[5];
  double fl = 0;
  CKR(cudaMemcpy(&fl, status_of->d_flops, sizeof(double), cudaMemcpyDeviceToHost), "flops");
  h->info.flops = fl;
  std::vector<int32_t> rk(std::max(h->L.n_slots, 1));
  CKR(cudaMemcpy(rk.data(), h->d_ranks, sizeof(int32_t) * rk.size(), cudaMemcpyDeviceToHost), "ranks");
  int64_t rsum = 0, nadm = 0, live = 0;
  int32_t rmax = 0;
  for (size_t b = 0; b < h->sb->FB.size(); ++b) {
    const Block& bk = h->sb->FB[b];
    const int64_t m = h->C[bk.row].size, n = h->C[bk.col].size;
    if (bk.kind == KIND_ADM) {
      int32_t r = rk[h->L.slot[b]];
      rmax = std::max(rmax, r);
      rsum += r;
      ++nadm;
      live += (m + n) * r;
    } else if (bk.kind == KIND_DENSE) {
      live += m * n;
    }
  }
  const int es = esize(h->precision);
  h->info.factor_live_bytes = live * es;
  h->info.grid_ctas = h->grid;
  h->info.rank_max = rmax;
  h->info.rank_mean = nadm ? (double)rsum / nadm : 0.0;
  h->info.factor_bytes = h->L.factor_elems * es;
  h->info.workspace_bytes = (h->L.total - h->L.factor_elems) * es + h->scratch_stride * h->grid * es;
  return rc;
}

static int factor_impl(hlu_handle* h, int32_t precision, void* stream, int64_t limit) {
  try {
    if (!h) return fail(HLU_ERR_ARG, "null handle");
    if (h->factor_pending) return fail(HLU_ERR_STATE, "a factorisation of this handle is in flight");
    if (precision != HLU_FP64 && precision != HLU_FP32 && precision != HLU_TF32)
      return fail(HLU_ERR_ARG, "precision");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = factor_prepare(h, precision, s);
    if (rc) return rc;
    CKR(cudaEventRecord(h->ev0, s), "event");
    rc = exec_run(h, h->dF, h->grid, s, true, limit);
    if (rc) return rc;
    CKR(cudaEventRecord(h->ev1, s), "event");
    CKR(cudaEventSynchronize(h->ev1), "sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    return factor_finish(h, h, s, ms);
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_factor_async(hlu_handle* h, int32_t precision, int32_t max_ctas, void* stream) {
  NvtxRange nvtx_("hlu_factor_async");
  try {
    if (!h || max_ctas < 0) return fail(HLU_ERR_ARG, "bad argument");
    if (precision != HLU_FP64 && precision != HLU_FP32 && precision != HLU_TF32)
      return fail(HLU_ERR_ARG, "precision");
    if (h->factor_pending) return fail(HLU_ERR_STATE, "a factorisation of this handle is in flight");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = factor_prepare(h, precision, s);
    if (rc) return rc;
    CKR(cudaEventRecord(h->ev0, s), "event");
    const int grid = max_ctas > 0 ? std::min(h->grid, (int)max_ctas) : h->grid;
    rc = exec_run(h, h->dF, grid, s, true);
    if (rc) return rc;
    CKR(cudaEventRecord(h->ev1, s), "event");
    h->factor_pending = true;
    h->factor_stream = s;
    return HLU_OK;
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_factor_wait(hlu_handle* h, int32_t block, int32_t* done) {
  try {
    if (!h || !done) return fail(HLU_ERR_ARG, "null argument");
    *done = 0;
    if (!h->factor_pending) {
      *done = 1;
      return HLU_OK;
    }
    if (block) {
      CKR(cudaEventSynchronize(h->ev1), "sync");
    } else {
      const cudaError_t e = cudaEventQuery(h->ev1);
      if (e == cudaErrorNotReady) return HLU_OK;
      CKR(e, "event query");
    }
    h->factor_pending = false;
    *done = 1;
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    return factor_finish(h, h, h->factor_stream, ms);
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_factor_profile(const hlu_handle* h, uint64_t* out) {
  if (!h || !out) return fail(HLU_ERR_ARG, "null argument");
  if (!h->d_prof) return fail(HLU_ERR_STATE, "not factored");
  CKR(cudaMemcpy(out, h->d_prof, sizeof(uint64_t) * kProfEntries, cudaMemcpyDeviceToHost), "profile");
  return HLU_OK;
}

int hlu_factor_stats(const hlu_handle* h, hlu_factor_info* info) {
  if (!h || !info) return fail(HLU_ERR_ARG, "null argument");
  *info = h->info;
  return HLU_OK;
}

int hlu_solve(const hlu_handle* h, const double* b, double* x, int32_t nrhs, int64_t ld, void* stream) {
  NvtxRange nvtx_("hlu_solve");
  if (!h || !b || !x || nrhs < 1 || ld < h->A.N) return fail(HLU_ERR_ARG, "bad argument");
  if (h->precision < 0 || h->factor_pending) return fail(HLU_ERR_STATE, "not factored");
  return solve_any(h, b, x, nrhs, ld, (cudaStream_t)stream);
}

int gmres_solve(const hlu_handle* hc, const double* b, double* x, int32_t nrhs, int64_t ld, int32_t restart,
                double tol, int32_t maxit, int32_t flexible, hlu_stats* stats, void* stream) {
  NvtxRange nvtx_("gmres_solve");
  (void)flexible;  // the flexible (stored z_j) form is used in every case
  try {
    hlu_handle* h = const_cast<hlu_handle*>(hc);
    if (!h || !b || !x || nrhs < 1 || ld < h->A.N || restart < 1 || restart > 1000 || !(tol > 0) || maxit < 1)
      return fail(HLU_ERR_ARG, "bad argument");
    if (!precond_ready(h)) return fail(HLU_ERR_STATE, "preconditioner not ready (not factored)");
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->converged = 1;
      stats->nrhs = nrhs;
    }
    int worst = HLU_OK;
    for (int32_t c0 = 0; c0 < nrhs; c0 += h->L.nrhs_max) {
      int nr = std::min(h->L.nrhs_max, nrhs - c0);
      int rc = gmres_chunk(h, b + c0 * ld, x + c0 * ld, nr, ld, restart, tol, maxit, stats, s);
      if (rc == HLU_ERR_NOT_CONVERGED)
        worst = rc;
      else if (rc)
        return rc;
    }
    if (stats)
      stats->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return worst;
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_richardson(const hlu_handle* hc, const double* b, double* x, int32_t nrhs, int64_t ld, double tol,
                   int32_t maxit, hlu_stats* stats, void* stream) {
  NvtxRange nvtx_("hlu_richardson");
  try {
    hlu_handle* h = const_cast<hlu_handle*>(hc);
    if (!h || !b || !x || nrhs < 1 || ld < h->A.N || !(tol > 0) || maxit < 1) return fail(HLU_ERR_ARG, "bad argument");
    if (!precond_ready(h)) return fail(HLU_ERR_STATE, "preconditioner not ready (not factored)");
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    int rc = ensure_kw(h, 1, std::min(nrhs, h->L.nrhs_max));
    if (rc) return rc;
    KrylovWS& k = h->kw;
    const int64_t N = h->A.N;
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->nrhs = nrhs;
      stats->converged = 1;
    }
    bool all_conv = true, broke = false;
    for (int32_t c0 = 0; c0 < nrhs; c0 += h->L.nrhs_max) {
      int nr = std::min(h->L.nrhs_max, nrhs - c0);
      const double* bc = b + c0 * ld;
      double* xc = x + c0 * ld;
      std::vector<double> bn(nr), rn(nr);
      for (int r = 0; r < nr; ++r) CKR(cudaMemsetAsync(xc + r * ld, 0, sizeof(double) * N, s), "x0");
      rc = col_norms(h, bc, ld, nr, k.bn, bn.data(), s);
      if (rc) return rc;
      for (int r = 0; r < nr; ++r)
        if (!std::isfinite(bn[r]))
          return fail(HLU_ERR_ARG,
                      "right-hand side column " + std::to_string(c0 + r) + " is not finite (x = 0 written)");
      int it = 0;
      bool conv = false;
      while (it < maxit) {
        ++it;
        CKR(residual(h->A.rowptr, h->A.col, h->A.val, N, xc, ld, bc, ld, k.W, N, nr, s), "residual");
        rc = col_norms(h, k.W, N, nr, k.hn, rn.data(), s);
        if (rc) return rc;
        for (int r = 0; r < nr; ++r) broke = broke || !std::isfinite(rn[r]);
        if (broke) break;
        rc = solve_any(h, k.W, k.tmp, nr, N, s);
        if (rc) return rc;
        // x += M^-1 r
        std::vector<double> one(nr, -1.0);
        CKR(cudaMemcpyAsync(k.h1, one.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, s), "ones");
        CKR(multiaxpy(N, k.tmp, N, 1, k.h1, 1, xc, ld, nr, s), "update");
        if (stats) stats->precond_applies++;
        conv = true;
        for (int r = 0; r < nr; ++r) conv = conv && (bn[r] == 0 || rn[r] < tol * bn[r]);
        if (conv) break;
      }
      CKR(residual(h->A.rowptr, h->A.col, h->A.val, N, xc, ld, bc, ld, k.W, N, nr, s), "residual");
      rc = col_norms(h, k.W, N, nr, k.hn, rn.data(), s);
      if (rc) return rc;
      if (stats) {
        stats->iterations = std::max(stats->iterations, it);
        for (int r = 0; r < nr; ++r) {
          stats->abs_res_max = std::max(stats->abs_res_max, rn[r]);
          stats->relres_max = std::max(stats->relres_max, bn[r] > 0 ? rn[r] / bn[r] : 0.0);
        }
        stats->converged = stats->converged && conv;
      }
      all_conv = all_conv && conv;
      if (broke) break;
    }
    if (stats)
      stats->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (broke) return fail(HLU_ERR_NOT_CONVERGED, "Richardson stopped: a residual is not finite");
    return all_conv ? HLU_OK : fail(HLU_ERR_NOT_CONVERGED, "Richardson reached maxit");
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_set_preconditioner(hlu_handle* h, int32_t which) {
  if (!h || (which != HLU_PRECOND_LU && which != HLU_PRECOND_HINV)) return fail(HLU_ERR_ARG, "bad argument");
  h->precond = which;
  return HLU_OK;
}

int hlu_hinverse(hlu_handle* h, int32_t precision, double tol, int32_t maxit, hlu_hinv_info* info, void* stream) {
  NvtxRange nvtx_("hlu_hinverse");
  try {
    if (!h || !(tol > 0) || maxit < 0 || maxit > HLU_HINV_MAX_ITERS) return fail(HLU_ERR_ARG, "bad argument");
    if (precision != HLU_FP64 && precision != HLU_FP32) return fail(HLU_ERR_ARG, "precision (FP64 or FP32)");
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    InvState& iv = h->inv;
    const int64_t N = h->A.N;
    if (!iv.built) {
      Schedule S0, S1, S2;
      build_inverse_schedules(h->C, h->sb->FB, h->rank_cap, 16, h->tile, iv.L, iv.Bx, S0, S1, S2, iv.st);
      CKR(iv.start.load(S0), "upload start schedule");
      CKR(iv.iter.load(S1), "upload iteration schedule");
      CKR(iv.apply.load(S2), "upload apply schedule");
      for (DevSched* d : {&iv.start, &iv.iter, &iv.apply}) CKR(d->alloc_state(), "queue");
      // A_H fill descriptors of copy 0
      std::vector<FillDesc> fd, fl;
      int64_t rows = 0;
      const size_t nb = h->sb->FB.size();
      for (size_t b = 0; b < nb; ++b) {
        const Block& bk = iv.Bx[b];
        if (bk.kind == KIND_SUB) continue;
        FillDesc f;
        std::memset(&f, 0, sizeof(f));
        f.roff = h->C[bk.row].off;
        f.m = h->C[bk.row].size;
        f.coff = h->C[bk.col].off;
        f.n = h->C[bk.col].size;
        if (bk.kind == KIND_DENSE) {
          f.off = iv.L.dense_off[b];
          f.row_prefix = rows;
          rows += f.m;
          fd.push_back(f);
        } else {
          f.off = iv.L.x_off[b];
          f.off2 = iv.L.y_off[b];
          f.slot = iv.L.slot[b];
          f.cap = iv.L.cap[b];
          fl.push_back(f);
        }
      }
      iv.n_fill_dense = (int32_t)fd.size();
      iv.n_fill_lr = (int32_t)fl.size();
      iv.dense_rows = rows;
      CKR(upload(&iv.d_fill_dense, fd), "fill desc");
      CKR(upload(&iv.d_fill_lr, fl), "fill desc");
      // residual probes: 4 columns of uniforms in [-1, 1) (SplitMix64)
      std::vector<double> z((size_t)N * 4);
      uint64_t st = 0x5eedULL;
      for (double& v : z) {
        st += 0x9E3779B97F4A7C15ULL;
        uint64_t q = st;
        q = (q ^ (q >> 30)) * 0xBF58476D1CE4E5B9ULL;
        q = (q ^ (q >> 27)) * 0x94D049BB133111EBULL;
        q ^= q >> 31;
        v = 2.0 * ((double)(q >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
      }
      CKR(upload(&iv.d_z, z), "probes");
      CKR(dev_malloc(&iv.d_w, sizeof(double) * N * 8), "probe workspace");
      iv.built = true;
    }
    const int es = esize(precision);
    if (iv.precision != precision) {
      iv.free_data();
      int dev = 0, sms = 0;
      CKR(cudaGetDevice(&dev), "device");
      CKR(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sms");
      const int bps = precision == HLU_FP64 ? blocks_per_sm<double>() : blocks_per_sm<float>();
      if (bps < 1) return fail(HLU_ERR_CUDA, "executor does not fit on an SM");
      iv.grid = sms * bps;
      iv.scratch_stride = scratch_stride_elems(iv.L, es);
      CKR(dev_malloc(&iv.d_arena, (size_t)es * iv.L.total), "inverse arena");
      CKR(dev_malloc(&iv.d_ranks, sizeof(int32_t) * std::max(iv.L.n_slots, 1)), "ranks");
      CKR(dev_malloc(&iv.d_piv, sizeof(int32_t)), "piv");
      CKR(dev_malloc(&iv.d_scratch, (size_t)es * iv.scratch_stride * iv.grid), "scratch");
      CKR(dev_malloc(&iv.d_status, sizeof(int32_t) * 8), "status");
      CKR(dev_malloc(&iv.d_flops, sizeof(double)), "flops");
      iv.precision = precision;
    }
    iv.ready = false;
    CKR(cudaMemsetAsync(iv.d_ranks, 0, sizeof(int32_t) * std::max(iv.L.n_slots, 1), s), "ranks");
    int32_t st0[8] = {0, -1, 0, 0, 0, 0, 0, 0};
    CKR(cudaMemcpyAsync(iv.d_status, st0, sizeof(st0), cudaMemcpyHostToDevice, s), "status");
    cudaError_t e;
    if (precision == HLU_FP64)
      e = fill_ah<double>(h->A, h->d_perm, h->d_iperm, iv.d_fill_dense, iv.n_fill_dense, iv.dense_rows, iv.d_fill_lr,
                          iv.n_fill_lr, (double*)iv.d_arena, iv.L.work_off, iv.L.ident_off, iv.L.ident_n, iv.d_ranks,
                          iv.d_status, s);
    else
      e = fill_ah<float>(h->A, h->d_perm, h->d_iperm, iv.d_fill_dense, iv.n_fill_dense, iv.dense_rows, iv.d_fill_lr,
                         iv.n_fill_lr, (float*)iv.d_arena, iv.L.work_off, iv.L.ident_off, iv.L.ident_n, iv.d_ranks,
                         iv.d_status, s);
    CKR(e, "A_H fill");
    // alpha = 1 / (||A||_1 ||A||_inf) from the CSR
    {
      std::vector<int64_t> rp(N + 1);
      std::vector<int32_t> ci(h->A.nnz);
      std::vector<double> va(h->A.nnz);
      CKR(cudaMemcpy(rp.data(), h->A.rowptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost), "csr");
      CKR(cudaMemcpy(ci.data(), h->A.col, sizeof(int32_t) * h->A.nnz, cudaMemcpyDeviceToHost), "csr");
      CKR(cudaMemcpy(va.data(), h->A.val, sizeof(double) * h->A.nnz, cudaMemcpyDeviceToHost), "csr");
      std::vector<double> colsum(N, 0.0);
      double ninf = 0;
      for (int64_t r = 0; r < N; ++r) {
        double rs = 0;
        for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
          rs += std::fabs(va[q]);
          colsum[ci[q]] += std::fabs(va[q]);
        }
        ninf = std::max(ninf, rs);
      }
      double n1 = 0;
      for (double c : colsum) n1 = std::max(n1, c);
      iv.alpha = 1.0 / (n1 * ninf);
    }
    int rc = exec_run_inv(h, iv.start, iv.alpha, 0, s);
    if (rc) return rc;
    rc = ensure_kw(h, 1, 4);
    if (rc) return rc;
    // ||z - A B z|| / ||z|| over the 4 probes
    std::vector<double> zn(4);
    rc = col_norms(h, iv.d_z, N, 4, h->kw.hn, zn.data(), s);
    if (rc) return rc;
    auto estimate = [&](double* out) -> int {
      int r2 = hinv_apply_any(h, iv.d_z, iv.d_w, 4, N, s);
      if (r2) return r2;
      CKR(residual(h->A.rowptr, h->A.col, h->A.val, N, iv.d_w, N, iv.d_z, N, iv.d_w + 4 * N, N, 4, s), "residual");
      std::vector<double> rn(4);
      r2 = col_norms(h, iv.d_w + 4 * N, N, 4, h->kw.hn, rn.data(), s);
      if (r2) return r2;
      double m = 0;
      for (int j = 0; j < 4; ++j) m = std::max(m, rn[j] / zn[j]);
      *out = m;
      return HLU_OK;
    };
    iv.res.clear();
    double r0 = 0;
    if ((rc = estimate(&r0))) return rc;
    iv.res.push_back(r0);
    bool diverged = false;
    int it = 0;
    while (iv.res.back() > tol && it < maxit) {
      if ((rc = exec_run_inv(h, iv.iter, 0.0, 0, s))) return rc;
      double r = 0;
      if ((rc = estimate(&r))) return rc;
      ++it;
      if (!std::isfinite(r) || r > 10.0) {
        diverged = true;
        iv.res.push_back(r);
        break;
      }
      iv.res.push_back(r);
      // the truncation floor: the estimate rises again after it had fallen a
      // hundredfold (before that, the Schulz residual only falls: the
      // residual matrix squares each step)
      const double prev = iv.res[iv.res.size() - 2];
      if (r > prev && prev < 1e-2 * iv.res[0]) break;
    }
    iv.ready = !diverged;
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iterations = it;
      info->alpha = iv.alpha;
      info->n_residuals = (int32_t)std::min<size_t>(iv.res.size(), HLU_HINV_MAX_ITERS + 1);
      for (int32_t k = 0; k < info->n_residuals; ++k) info->residual[k] = iv.res[k];
      std::vector<int32_t> rk(std::max(iv.L.n_slots, 1));
      CKR(cudaMemcpy(rk.data(), iv.d_ranks, sizeof(int32_t) * rk.size(), cudaMemcpyDeviceToHost), "ranks");
      const size_t nb = h->sb->FB.size();
      int64_t rs = 0, na = 0, live = 0;
      for (size_t b = nb; b < 2 * nb; ++b) {  // copy 1: the inverse
        const Block& bk = iv.Bx[b];
        const int64_t m = h->C[bk.row].size, n = h->C[bk.col].size;
        if (bk.kind == KIND_ADM) {
          const int32_t r = rk[iv.L.slot[b]];
          info->rank_max = std::max(info->rank_max, r);
          rs += r;
          ++na;
          live += (m + n) * r;
        } else if (bk.kind == KIND_DENSE) {
          live += m * n;
        }
      }
      info->rank_mean = na ? (double)rs / na : 0.0;
      info->inverse_live_bytes = live * es;
      info->arena_bytes = iv.L.total * es;
      info->n_iter_tasks = iv.iter.ntasks;
      info->schedule_ms = iv.st.host_ms;
      info->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return diverged ? fail(HLU_ERR_NOT_CONVERGED, "Schulz iteration diverged (truncation too coarse)") : HLU_OK;
  } catch (const std::bad_alloc&) {
    return fail(HLU_ERR_OOM, "host allocation failed");
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_hinverse_apply(const hlu_handle* hc, const double* b, double* x, int32_t nrhs, int64_t ld, void* stream) {
  NvtxRange nvtx_("hlu_hinverse_apply");
  hlu_handle* h = const_cast<hlu_handle*>(hc);
  if (!h || !b || !x || nrhs < 1 || ld < h->A.N) return fail(HLU_ERR_ARG, "bad argument");
  if (!h->inv.ready) return fail(HLU_ERR_STATE, "no inverse (hlu_hinverse)");
  return hinv_apply_any(h, b, x, nrhs, ld, (cudaStream_t)stream);
}

int hlu_factor_batch(hlu_handle** hs, int32_t count, int32_t precision, void* stream) {
  NvtxRange nvtx_("hlu_factor_batch");
  try {
    if (!hs || count < 1 || count > kMaxBatch) return fail(HLU_ERR_ARG, "bad argument");
    if (precision != HLU_FP64 && precision != HLU_FP32 && precision != HLU_TF32)
      return fail(HLU_ERR_ARG, "precision");
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t i = 0; i < count; ++i) {
      if (!hs[i]) return fail(HLU_ERR_ARG, "null handle");
      int rc = factor_prepare(hs[i], precision, s);
      if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    CKR(cudaEventRecord(hs[0]->ev0, s), "event");
    int rc = exec_run_batch(hs, count, 0, s, &g_batch_q, &g_batch_q_len);
    if (rc) return rc;
    CKR(cudaEventRecord(hs[0]->ev1, s), "event");
    CKR(cudaEventSynchronize(hs[0]->ev1), "sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, hs[0]->ev0, hs[0]->ev1);
    int worst = HLU_OK;
    for (int32_t i = 0; i < count; ++i) {
      rc = factor_finish(hs[i], hs[0], s, ms);
      if (rc) worst = rc;
    }
    return worst;
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_solve_batch(hlu_handle* const* hs, int32_t count, const double* const* b, double* const* x,
                    const int32_t* nrhs, void* stream) {
  NvtxRange nvtx_("hlu_solve_batch");
  try {
    if (!hs || !b || !x || !nrhs || count < 1 || count > kMaxBatch) return fail(HLU_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t i = 0; i < count; ++i) {
      hlu_handle* h = hs[i];
      if (!h || !b[i] || !x[i] || nrhs[i] < 1) return fail(HLU_ERR_ARG, "bad argument");
      if (h->precision < 0 || h->factor_pending) return fail(HLU_ERR_STATE, "not factored");
      if (h->precision != hs[0]->precision) return fail(HLU_ERR_ARG, "mixed precisions in a batch");
      if (nrhs[i] > h->L.nrhs_max) return fail(HLU_ERR_ARG, "nrhs above the batched limit (16)");
    }
    for (int32_t i = 0; i < count; ++i) {
      hlu_handle* h = hs[i];
      CKR(set_int(h->d_ranks + h->L.nrhs_slot, nrhs[i], s), "nrhs slot");
      h->cur_nrhs = nrhs[i];
      if (h->precision == HLU_FP64)
        CKR(gather_cast<double>(h->A.N, h->d_perm, b[i], h->A.N, (double*)h->d_arena + h->L.work_off, nrhs[i], s),
            "gather");
      else
        CKR(gather_cast<float>(h->A.N, h->d_perm, b[i], h->A.N, (float*)h->d_arena + h->L.work_off, nrhs[i], s),
            "gather");
    }
    {
      std::lock_guard<std::mutex> lk(g_batch_mu);
      int rc = exec_run_batch(hs, count, 1, s, &g_batch_q, &g_batch_q_len);
      if (rc) return rc;
    }
    for (int32_t i = 0; i < count; ++i) {
      hlu_handle* h = hs[i];
      if (h->precision == HLU_FP64)
        CKR(scatter_cast<double>(h->A.N, h->d_perm, (double*)h->d_arena + h->L.work_off, x[i], h->A.N, nrhs[i], s),
            "scatter");
      else
        CKR(scatter_cast<float>(h->A.N, h->d_perm, (float*)h->d_arena + h->L.work_off, x[i], h->A.N, nrhs[i], s),
            "scatter");
    }
    int32_t st[8];
    return read_status(hs[0], s, st);
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

}  // extern "C"

// Fault injection for the bounded device waits: a two-task schedule in which
// task 0 waits for task 1, run by a single CTA.  Task 1 can only start after
// task 0, so the wait can never be satisfied; it must run out after limit_ms,
// set HLU_ERR_TIMEOUT and let the kernel return.
extern "C" int hlu_set_trunc_params(int32_t compress_at, double jacobi_tol) {
  if (compress_at != 0 && (compress_at < 8 || compress_at > kTruncStack)) return fail(HLU_ERR_ARG, "compress_at");
  if (jacobi_tol < 0 || jacobi_tol >= 1) return fail(HLU_ERR_ARG, "jacobi_tol");
  g_compress_at = compress_at;
  g_jacobi_tol = jacobi_tol;
  return HLU_OK;
}

extern "C" int hlu_debug_wait_timeout(double limit_ms, int32_t* status_out) {
  if (!status_out || !(limit_ms > 0) || limit_ms > 5000) return fail(HLU_ERR_ARG, "bad argument");
  Schedule S;
  Task t;
  std::memset(&t, 0, sizeof(t));
  t.type = TK_NUM;  // no work
  t.out_slot = -1;
  S.tasks = {t, t};
  // task 1 waits for itself: its queue slot is never filled
  S.pred_ptr = {0, 0, 1};
  S.pred_idx = {1};
  hlu_handle h;
  h.precision = HLU_FP32;
  DevSched ds;
  CKR(ds.load(S), "upload");
  CKR(ds.alloc_state(), "queue");
  CKR(dev_malloc(&h.d_status, sizeof(int32_t) * 8), "alloc");
  // valid (unused) per-problem pointers: the two tasks do no work
  CKR(dev_malloc(&h.d_arena, 256), "alloc");
  CKR(dev_malloc(&h.d_arenas, sizeof(void*)), "alloc");
  CKR(dev_malloc(&h.d_rankp, sizeof(int32_t*)), "alloc");
  CKR(dev_malloc(&h.d_pivp, sizeof(int32_t*)), "alloc");
  CKR(cudaMemcpy(h.d_arenas, &h.d_arena, sizeof(void*), cudaMemcpyHostToDevice), "ptr");
  CKR(cudaMemcpy(h.d_rankp, &h.d_arena, sizeof(void*), cudaMemcpyHostToDevice), "ptr");
  CKR(cudaMemcpy(h.d_pivp, &h.d_arena, sizeof(void*), cudaMemcpyHostToDevice), "ptr");
  double saved = g_wait_limit_ms;
  g_wait_limit_ms = limit_ms;
  int rc = exec_run(&h, ds, 1, nullptr, false);
  g_wait_limit_ms = saved;
  int32_t st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (!rc) rc = read_status(&h, nullptr, st);
  status_out[0] = st[0];
  status_out[1] = st[1];
  ds.free_all();
  for (void* p : {(void*)h.d_status, (void*)h.d_arena, (void*)h.d_arenas, (void*)h.d_rankp,
                  (void*)h.d_pivp})
    dev_free(p);
  h.d_status = nullptr;
  h.d_arena = nullptr;
  h.d_arenas = nullptr;
  h.d_rankp = nullptr;
  h.d_pivp = nullptr;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "after timeout test");
  return rc;
}

// Runs A_H fill and the first `limit` tasks of the factorisation DAG, then
// copies the arena (elements, in the factor precision) and the rank slots to
// host buffers; sizes[0] = arena elements, sizes[1] = rank slots, sizes[2] =
// factor tasks.  Query sizes with NULL buffers.
extern "C" int hlu_debug_factor_prefix(hlu_handle* h, int32_t precision, int64_t limit, void* arena_out,
                                       int32_t* ranks_out, int64_t* sizes) {
  if (!h || !sizes) return fail(HLU_ERR_ARG, "null argument");
  sizes[0] = h->L.total;
  sizes[1] = h->L.n_slots;
  sizes[2] = h->dF.ntasks;
  if (!arena_out && !ranks_out) return HLU_OK;
  // allocate (first call), then clear the whole arena so that memory no task
  // wrote compares equal with the host executor's zero-initialised arena
  int rc = factor_impl(h, precision, nullptr, 0);
  if (rc && rc != HLU_ERR_ZERO_PIVOT) return rc;
  CKR(cudaMemset(h->d_arena, 0, (size_t)esize(precision) * h->L.total), "clear");
  rc = factor_impl(h, precision, nullptr, limit);
  if (rc && rc != HLU_ERR_ZERO_PIVOT) return rc;
  if (arena_out)
    CKR(cudaMemcpy(arena_out, h->d_arena, (size_t)esize(precision) * h->L.total, cudaMemcpyDeviceToHost), "arena");
  if (ranks_out) CKR(cudaMemcpy(ranks_out, h->d_ranks, sizeof(int32_t) * h->L.n_slots, cudaMemcpyDeviceToHost), "ranks");
  return HLU_OK;
}

// Factorises with a per-task trace and copies the trace, the DAG and the task
// records out; sizes[0] = tasks, sizes[1] = dependency edges (query with NULL
// buffers).
extern "C" int hlu_debug_factor_trace(hlu_handle* h, int32_t precision, uint64_t* trace_out, int64_t* pred_ptr_out,
                                      int32_t* pred_idx_out, void* tasks_out, int64_t* sizes) {
  if (!h || !sizes) return fail(HLU_ERR_ARG, "null argument");
  const int64_t nt = h->dF.ntasks;
  sizes[0] = nt;
  sizes[1] = 0;
  if (h->dF.pred_ptr && nt > 0)
    CKR(cudaMemcpy(&sizes[1], h->dF.pred_ptr + nt, sizeof(int64_t), cudaMemcpyDeviceToHost), "edges");
  if (!trace_out) return HLU_OK;
  CKR(dev_malloc(&h->d_trace, sizeof(unsigned long long) * 4 * std::max<int64_t>(nt, 1)), "trace");
  CKR(cudaMemset(h->d_trace, 0, sizeof(unsigned long long) * 4 * std::max<int64_t>(nt, 1)), "trace");
  int rc = factor_impl(h, precision, nullptr, -1);
  cudaError_t e = cudaMemcpy(trace_out, h->d_trace, sizeof(uint64_t) * 4 * nt, cudaMemcpyDeviceToHost);
  dev_free(h->d_trace);
  h->d_trace = nullptr;
  if (rc) return rc;
  CKR(e, "trace copy");
  if (pred_ptr_out)
    CKR(cudaMemcpy(pred_ptr_out, h->dF.pred_ptr, sizeof(int64_t) * (nt + 1), cudaMemcpyDeviceToHost), "dag");
  if (pred_idx_out)
    CKR(cudaMemcpy(pred_idx_out, h->dF.pred_idx, sizeof(int32_t) * sizes[1], cudaMemcpyDeviceToHost), "dag");
  if (tasks_out) CKR(cudaMemcpy(tasks_out, h->dF.tasks, sizeof(Task) * nt, cudaMemcpyDeviceToHost), "tasks");
  return HLU_OK;
}

// Runs one triangular solve of a factored handle (nrhs columns of the work
// vector, whatever they hold) with a per-task trace; outputs as
// hlu_debug_factor_trace for the solve DAG.
extern "C" int hlu_debug_solve_trace(hlu_handle* h, int32_t nrhs, uint64_t* trace_out, int64_t* pred_ptr_out,
                                     int32_t* pred_idx_out, void* tasks_out, int64_t* sizes) {
  if (!h || !sizes || nrhs < 1 || nrhs > h->L.nrhs_max) return fail(HLU_ERR_ARG, "bad argument");
  const int64_t nt = h->dS.ntasks;
  sizes[0] = nt;
  sizes[1] = 0;
  if (h->dS.pred_ptr && nt > 0)
    CKR(cudaMemcpy(&sizes[1], h->dS.pred_ptr + nt, sizeof(int64_t), cudaMemcpyDeviceToHost), "edges");
  if (!trace_out) return HLU_OK;
  if (h->precision < 0 || h->factor_pending) return fail(HLU_ERR_STATE, "not factored");
  CKR(dev_malloc(&h->d_trace, sizeof(unsigned long long) * 4 * std::max<int64_t>(nt, 1)), "trace");
  CKR(cudaMemset(h->d_trace, 0, sizeof(unsigned long long) * 4 * std::max<int64_t>(nt, 1)), "trace");
  CKR(set_int(h->d_ranks + h->L.nrhs_slot, nrhs, nullptr), "nrhs slot");
  h->cur_nrhs = nrhs;
  int rc = exec_run(h, h->dS, h->grid, nullptr, false);
  if (!rc) {
    int32_t st[8];
    rc = read_status(h, nullptr, st);
  }
  cudaError_t e = cudaMemcpy(trace_out, h->d_trace, sizeof(uint64_t) * 4 * nt, cudaMemcpyDeviceToHost);
  dev_free(h->d_trace);
  h->d_trace = nullptr;
  if (rc) return rc;
  CKR(e, "trace copy");
  if (pred_ptr_out)
    CKR(cudaMemcpy(pred_ptr_out, h->dS.pred_ptr, sizeof(int64_t) * (nt + 1), cudaMemcpyDeviceToHost), "dag");
  if (pred_idx_out)
    CKR(cudaMemcpy(pred_idx_out, h->dS.pred_idx, sizeof(int32_t) * sizes[1], cudaMemcpyDeviceToHost), "dag");
  if (tasks_out) CKR(cudaMemcpy(tasks_out, h->dS.tasks, sizeof(Task) * nt, cudaMemcpyDeviceToHost), "tasks");
  return HLU_OK;
}

// Zeroes row and column `dof` of A (columns are ascending within a row).
__global__ void k_zero_dof(int64_t N, const int64_t* rowptr, const int32_t* col, double* val, int32_t dof) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rowptr[r], e = rowptr[r + 1];
    if (r == dof) {
      for (int64_t q = b; q < e; ++q) val[q] = 0.0;
      continue;
    }
    int64_t lo = b, hi = e;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (col[mid] < dof)
        lo = mid + 1;
      else
        hi = mid;
    }
    if (lo < e && col[lo] == dof) val[lo] = 0.0;
  }
}

extern "C" int hlu_debug_tf32_tile(const float* A, const float* B, float* D, int32_t K, int32_t* status_out) {
  if (!A || !B || !D || K < 1 || K > 4096) return fail(HLU_ERR_ARG, "bad argument");
  int32_t* st = nullptr;
  CKR(dev_malloc(&st, sizeof(int32_t) * 4), "status");
  int32_t z[4] = {0, -1, 0, 0};
  cudaError_t e = cudaMemcpy(st, z, sizeof(z), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = tcx::tc_tile_product(A, B, D, K, st, (unsigned long long)(g_wait_limit_ms * 1e6), nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int32_t hs[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hs, st, sizeof(hs), cudaMemcpyDeviceToHost);
  dev_free(st);
  CKR(e, "tf32 tile");
  if (status_out) *status_out = hs[0];
  return hs[0] == 5 ? fail(HLU_ERR_TIMEOUT, "tensor-core completion wait ran out") : HLU_OK;
}

// One truncation task (TK_TRUNC) run by the device executor on its own: the
// stack X Y^T (m x w and n x w, host column-major FP64) goes in as pieces of
// at most piece_cols columns; the kept factors come back.
template <class T>
static int debug_truncate(int32_t precision, int32_t m, int32_t n, int32_t w, int32_t piece_cols, int32_t flags,
                          const double* X, const double* Y, double eps, int32_t cap, double* Xo, double* Yo,
                          int32_t* rank, int32_t* status_out) {
  auto al = [](int64_t e) { return (e + 31) & ~int64_t(31); };
  const int64_t xo = 0, yo = al((int64_t)m * w), oxo = yo + al((int64_t)n * w), oyo = oxo + al((int64_t)m * cap);
  const int64_t total = oyo + al((int64_t)n * cap);
  std::vector<T> harena((size_t)total, T(0));
  const bool ytrans = (flags & 2) != 0, quad = (flags & 4) != 0, alias = (flags & 1) != 0;
  const int32_t pw = piece_cols > 0 ? piece_cols : std::max(w, 1);
  for (int64_t i = 0; i < (int64_t)m * w; ++i) harena[xo + i] = T(X[i]);
  if (!ytrans) {
    for (int64_t i = 0; i < (int64_t)n * w; ++i) harena[yo + i] = T(Y[i]);
  } else {  // each piece's Y block stored row-major (rows x its columns)
    for (int32_t c0 = 0; c0 < w; c0 += pw) {
      const int32_t wc = std::min(pw, w - c0);
      for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < wc; ++j) harena[yo + (int64_t)c0 * n + (int64_t)i * wc + j] = T(Y[i + (int64_t)(c0 + j) * n]);
    }
  }
  Schedule S;
  Task t;
  std::memset(&t, 0, sizeof(t));
  t.type = TK_TRUNC;
  t.a = View{oxo, 1, m, m, cap, 0, 0};
  t.b = View{oyo, 1, n, n, cap, 0, 0};
  t.c.slot = -1;
  t.out_slot = 0;
  t.cap = cap;
  t.piv_off = -1;
  t.sign = 1.0f;
  const int32_t mh = m / 2, nh = n / 2;
  int32_t q_index = 0;
  for (int32_t c0 = 0; c0 < w; c0 += pw, ++q_index) {
    Piece q;
    std::memset(&q, 0, sizeof(q));
    const int32_t wc = std::min(pw, w - c0);
    int32_t xr0 = 0, xr = m, yr0 = 0, yr = n;
    if (quad) {  // piece q covers quadrant ((q mod 4) / 2, q mod 2)
      const int32_t qi = (q_index % 4) / 2, qj = q_index % 2;
      xr0 = qi ? mh : 0;
      xr = qi ? m - mh : mh;
      yr0 = qj ? nh : 0;
      yr = qj ? n - nh : nh;
    }
    q.X = View{xo + (int64_t)c0 * m + xr0, 1, m, xr, wc, -1, 0};
    if (!ytrans)
      q.Y = View{yo + (int64_t)c0 * n + yr0, 1, n, yr, wc, -1, 0};
    else
      q.Y = View{yo + (int64_t)c0 * n + (int64_t)yr0 * wc, wc, 1, yr, wc, -1, 0};
    q.xoff = xr0;
    q.yoff = yr0;
    q.sign = 1.0f;
    if (alias && q_index == 0 && !quad && !ytrans && wc <= cap) {
      // the target's current factors are the first piece (an update X += ...)
      for (int32_t j = 0; j < wc; ++j) {
        for (int32_t i = 0; i < m; ++i) harena[oxo + i + (int64_t)j * m] = harena[xo + i + (int64_t)j * m];
        for (int32_t i = 0; i < n; ++i) harena[oyo + i + (int64_t)j * n] = harena[yo + i + (int64_t)j * n];
      }
      q.X = View{oxo, 1, m, m, cap, 0, 0};
      q.Y = View{oyo, 1, n, n, cap, 0, 0};
    }
    S.pieces.push_back(q);
  }
  const int32_t rank0 = (alias && !quad && !ytrans && std::min(pw, w) <= cap) ? std::min(pw, w) : 0;
  t.list_begin = 0;
  t.list_count = (int32_t)S.pieces.size();
  S.tasks.push_back(t);
  S.pred_ptr = {0, 0};
  DevSched ds;
  T* d_arena = nullptr;
  int32_t *d_ranks = nullptr, *d_piv = nullptr, *d_status = nullptr;
  void* d_scratch = nullptr;
  const int64_t rows = std::max(std::max(m, n), 1);
  const int64_t sbytes = trunc_scratch_bytes(rows, (int)sizeof(T));
  cudaError_t e = ds.load(S);
  if (e == cudaSuccess) e = ds.alloc_state();
  if (e == cudaSuccess) e = upload(&d_arena, harena);
  if (e == cudaSuccess) e = upload(&d_ranks, std::vector<int32_t>{rank0, 1});
  if (e == cudaSuccess) e = upload(&d_piv, std::vector<int32_t>{0});
  if (e == cudaSuccess) e = upload(&d_status, std::vector<int32_t>{0, -1, 0, 0, 0, 0, 0, 0});
  if (e == cudaSuccess) e = dev_malloc(&d_scratch, (size_t)sbytes);
  if (e == cudaSuccess) {
    ExecArgs a;
    std::memset(&a, 0, sizeof(a));
    ProbSched& p = a.probs[0];
    p.tasks = ds.tasks;
    p.terms = ds.terms;
    p.pieces = ds.pieces;
    p.succ_ptr = ds.succ_ptr;
    p.succ_idx = ds.succ_idx;
    p.indeg = ds.indeg;
    p.arena = d_arena;
    p.ranks = d_ranks;
    p.piv = d_piv;
    p.eps = eps;
    p.ntasks = 1;
    p.limit = 1;
    p.nrhs_slot = 1;
    p.nrhs = 1;
    a.nprobs = 1;
    a.ntotal = 1;
    a.queue = ds.queue;
    a.qctl = ds.qctl;
    a.scratch = d_scratch;
    a.scratch_stride = sbytes / (int64_t)sizeof(T);
    a.trunc_rows = rows;
    a.status = d_status;
    a.wait_limit_ns = (unsigned long long)(g_wait_limit_ms * 1e6);
    a.jacobi_tol = g_jacobi_tol;
    a.compress_at = g_compress_at;
    unsigned long long q0[2] = {0ULL, 1ULL};
    e = cudaMemcpy(ds.qctl, q0, sizeof(q0), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ds.indeg, ds.indeg0, sizeof(int32_t), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ds.queue, ds.roots, sizeof(unsigned long long), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = launch_exec(precision, a, 1, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  int32_t hs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int32_t hr[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(hs, d_status, sizeof(hs), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hr, d_ranks, sizeof(hr), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(harena.data(), d_arena, sizeof(T) * total, cudaMemcpyDeviceToHost);
  ds.free_all();
  for (void* q : {(void*)d_arena, (void*)d_ranks, (void*)d_piv, (void*)d_status, d_scratch})
    if (q) dev_free(q);
  CKR(e, "truncation");
  *rank = hr[0];
  for (int64_t i = 0; i < (int64_t)m * cap; ++i) Xo[i] = (double)harena[oxo + i];
  for (int64_t i = 0; i < (int64_t)n * cap; ++i) Yo[i] = (double)harena[oyo + i];
  if (status_out)
    for (int k = 0; k < 8; ++k) status_out[k] = hs[k];
  return hs[0] == 5 ? fail(HLU_ERR_TIMEOUT, "device wait ran out") : HLU_OK;
}

extern "C" int hlu_debug_truncate(int32_t precision, int32_t m, int32_t n, int32_t w, int32_t piece_cols,
                                  int32_t flags, const double* X, const double* Y, double eps, int32_t cap, double* Xo,
                                  double* Yo, int32_t* rank, int32_t* status_out) {
  if (!X || !Y || !Xo || !Yo || !rank || m < 1 || n < 1 || w < 0 || piece_cols < 0 || eps <= 0 || cap < 1 ||
      cap > kRankMax || cap > std::min(m, n) || (flags & ~7) != 0 ||
      (precision != HLU_FP64 && precision != HLU_FP32))
    return fail(HLU_ERR_ARG, "bad argument");
  if ((int64_t)std::max(m, n) > (int64_t)1 << 20 || w > (1 << 16)) return fail(HLU_ERR_ARG, "too large");
  return precision == HLU_FP64 ? debug_truncate<double>(precision, m, n, w, piece_cols, flags, X, Y, eps, cap, Xo, Yo,
                                                        rank, status_out)
                               : debug_truncate<float>(precision, m, n, w, piece_cols, flags, X, Y, eps, cap, Xo, Yo,
                                                       rank, status_out);
}

extern "C" int hlu_debug_zero_dof(hlu_handle* h, int64_t dof) {
  if (!h || dof < 0 || dof >= h->A.N) return fail(HLU_ERR_ARG, "bad argument");
  note_launch();
  k_zero_dof<<<(int)std::min<int64_t>((h->A.N + 255) / 256, 4096), 256>>>(h->A.N, h->A.rowptr, h->A.col, h->A.val,
                                                                          (int32_t)dof);
  CKR(cudaGetLastError(), "zero dof");
  CKR(cudaDeviceSynchronize(), "zero dof");
  return HLU_OK;
}

// Copies factorisation task `idx` (its raw 128-byte record) to `out`.
extern "C" int hlu_debug_task_record(const hlu_handle* h, int64_t idx, void* out) {
  if (!h || !out || idx < 0 || idx >= h->dF.ntasks) return fail(HLU_ERR_ARG, "bad argument");
  CKR(cudaMemcpy(out, h->dF.tasks + idx, sizeof(Task), cudaMemcpyDeviceToHost), "task");
  return HLU_OK;
}

// ---------------------------------------------------------------------------
// Continuous batching: GMRES states that advance together.  Each step runs
// the preconditioner of every active state in ONE persistent launch (states
// that share a factor have their columns placed side by side in that
// factor's work vector), then each state's SpMV, CGS2 and Givens update.
// ---------------------------------------------------------------------------
namespace {

int alloc_ws(KrylovWS& k, int64_t N, int m, int nr) {
  k.free_all();
  k.N = N;
  k.m = m;
  k.nr = nr;
  CKR(dev_malloc(&k.V, sizeof(double) * N * (m + 1) * nr), "alloc V");
  CKR(dev_malloc(&k.Z, sizeof(double) * N * (m + 1) * nr), "alloc Z");
  CKR(dev_malloc(&k.W, sizeof(double) * N * nr), "alloc W");
  CKR(dev_malloc(&k.h1, sizeof(double) * (m + 1) * nr), "alloc");
  CKR(dev_malloc(&k.h2, sizeof(double) * (m + 1) * nr), "alloc");
  CKR(dev_malloc(&k.hn, sizeof(double) * nr), "alloc");
  CKR(dev_malloc(&k.H, sizeof(double) * (m + 1) * m * nr), "alloc");
  CKR(dev_malloc(&k.cs, sizeof(double) * m * nr), "alloc");
  CKR(dev_malloc(&k.sn, sizeof(double) * m * nr), "alloc");
  CKR(dev_malloc(&k.g, sizeof(double) * (m + 1) * nr), "alloc");
  CKR(dev_malloc(&k.est, sizeof(double) * nr), "alloc");
  CKR(dev_malloc(&k.y, sizeof(double) * m * nr), "alloc");
  CKR(dev_malloc(&k.bn, sizeof(double) * nr), "alloc");
  CKR(dev_malloc(&k.part, sizeof(double) * std::max(multidot_partials(N, m + 1, nr), 1)), "alloc");
  CKR(dev_malloc(&k.jr, sizeof(int) * nr), "alloc");
  return HLU_OK;
}

int norms_ws(KrylovWS& k, const double* X, int64_t ld, int nr, double* dev, cudaStream_t s) {
  CKR(multidot(k.N, X, ld, 1, X, ld, nr, k.part, dev, 1, s), "norm");
  CKR(sqrt_inplace(dev, nr, s), "sqrt");
  return HLU_OK;
}

struct SolveSeg {
  const double* b;
  double* x;
  int64_t ld;
  int nr;
};

// x = (LU)^-1 b for segments grouped by handle, one launch for all handles
int solve_segments(std::vector<hlu_handle*>& hs, std::vector<std::vector<SolveSeg>>& segs, cudaStream_t s) {
  for (size_t i = 0; i < hs.size(); ++i) {
    hlu_handle* h = hs[i];
    int off = 0;
    for (const SolveSeg& g : segs[i]) {
      if (h->precision == HLU_FP64)
        CKR(gather_cast<double>(h->A.N, h->d_perm, g.b, g.ld, (double*)h->d_arena + h->L.work_off + off * h->A.N,
                                g.nr, s), "gather");
      else
        CKR(gather_cast<float>(h->A.N, h->d_perm, g.b, g.ld, (float*)h->d_arena + h->L.work_off + off * h->A.N,
                               g.nr, s), "gather");
      off += g.nr;
    }
    CKR(set_int(h->d_ranks + h->L.nrhs_slot, off, s), "nrhs slot");
    h->cur_nrhs = off;
  }
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    int rc = exec_run_batch(hs.data(), (int)hs.size(), 1, s, &g_batch_q, &g_batch_q_len);
    if (rc) return rc;
  }
  for (size_t i = 0; i < hs.size(); ++i) {
    hlu_handle* h = hs[i];
    int off = 0;
    for (const SolveSeg& g : segs[i]) {
      if (h->precision == HLU_FP64)
        CKR(scatter_cast<double>(h->A.N, h->d_perm, (double*)h->d_arena + h->L.work_off + off * h->A.N, g.x, g.ld,
                                 g.nr, s), "scatter");
      else
        CKR(scatter_cast<float>(h->A.N, h->d_perm, (float*)h->d_arena + h->L.work_off + off * h->A.N, g.x, g.ld,
                                g.nr, s), "scatter");
      off += g.nr;
    }
  }
  return HLU_OK;
}

}  // namespace

struct hlu_gmres {
  hlu_handle* h = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int nr = 0;
  int64_t ld = 0;
  int m = 0;
  double tol = 0;
  int maxit = 0;
  KrylovWS k;
  std::vector<double> bn, beta, est;
  std::vector<int> conv, jr;
  int j = -1;  // inner step of the running cycle, -1: next step starts a cycle
  int iters = 0, restarts = 0;
  bool done = false;
  int status = HLU_OK;
  double precond_ms = 0;
  int applies = 0;
  cudaStream_t s = nullptr;  // the stream of hlu_gmres_begin
};

extern "C" {

int hlu_gmres_begin(const hlu_handle* hc, const double* b, double* x, int32_t nrhs, int64_t ld, int32_t restart,
                    double tol, int32_t maxit, void* stream, hlu_gmres** out) {
  NvtxRange nvtx_("hlu_gmres_begin");
  try {
    hlu_handle* h = const_cast<hlu_handle*>(hc);
    if (!out || !h || !b || !x || nrhs < 1 || ld < h->A.N || restart < 1 || restart > 1000 || !(tol > 0) || maxit < 1)
      return fail(HLU_ERR_ARG, "bad argument");
    if (nrhs > h->L.nrhs_max) return fail(HLU_ERR_ARG, "nrhs above 16 per GMRES state");
    if (h->precision < 0 || h->factor_pending) return fail(HLU_ERR_STATE, "not factored");
    cudaStream_t s = (cudaStream_t)stream;
    hlu_gmres* g = new hlu_gmres();
    g->h = h;
    g->s = s;
    g->b = b;
    g->x = x;
    g->nr = nrhs;
    g->ld = ld;
    g->m = restart;
    g->tol = tol;
    g->maxit = maxit;
    // every failure below frees the state and its workspace: the caller
    // gets no handle to end
    auto start = [&]() -> int {
      int rc = alloc_ws(g->k, h->A.N, restart, nrhs);
      if (rc) return rc;
      g->bn.assign(nrhs, 0);
      g->beta.assign(nrhs, 0);
      g->est.assign(nrhs, 0);
      g->conv.assign(nrhs, 0);
      g->jr.assign(nrhs, 0);
      for (int r = 0; r < nrhs; ++r) CKR(cudaMemsetAsync(x + r * ld, 0, sizeof(double) * h->A.N, s), "x0");
      rc = norms_ws(g->k, b, ld, nrhs, g->k.bn, s);
      if (rc) return rc;
      CKR(cudaMemcpyAsync(g->bn.data(), g->k.bn, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s), "d2h");
      CKR(cudaStreamSynchronize(s), "sync");
      return HLU_OK;
    };
    int rc;
    try {
      rc = start();
    } catch (const std::bad_alloc&) {  // the host vectors of the state
      rc = fail(HLU_ERR_OOM, "host allocation");
    }
    if (rc) {
      cudaStreamSynchronize(s);  // the memset / norm work queued so far
      g->k.free_all();
      delete g;
      return rc;
    }
    *out = g;
    return HLU_OK;
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_gmres_step_batch(hlu_gmres* const* gs, int32_t count, void* stream) {
  NvtxRange nvtx_("hlu_gmres_step_batch");
  try {
    if (!gs || count < 1) return fail(HLU_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    // phase A: states that start a cycle compute their residual and its norm
    std::vector<hlu_gmres*> act;
    for (int i = 0; i < count; ++i) {
      hlu_gmres* g = gs[i];
      if (!g || g->done) continue;
      if (g->j < 0) {
        const int64_t N = g->h->A.N, ldr = N * (g->m + 1);
        CKR(residual(g->h->A.rowptr, g->h->A.col, g->h->A.val, N, g->x, g->ld, g->b, g->ld, g->k.V, ldr, g->nr, s),
            "residual");
        int rc = norms_ws(g->k, g->k.V, ldr, g->nr, g->k.hn, s);
        if (rc) return rc;
        CKR(cudaMemcpyAsync(g->beta.data(), g->k.hn, sizeof(double) * g->nr, cudaMemcpyDeviceToHost, s), "d2h");
      }
      act.push_back(g);
    }
    CKR(cudaStreamSynchronize(s), "sync");
    std::vector<hlu_gmres*> run;
    for (hlu_gmres* g : act) {
      if (g->j < 0) {
        bool all = true;
        for (int r = 0; r < g->nr; ++r) {
          g->conv[r] = (g->bn[r] == 0.0) || (g->beta[r] <= g->tol * g->bn[r]);
          all = all && g->conv[r];
        }
        if (all || g->iters >= g->maxit) {
          g->done = true;
          g->status = all ? HLU_OK : HLU_ERR_NOT_CONVERGED;
          continue;
        }
        const int64_t N = g->h->A.N, ldr = N * (g->m + 1);
        CKR(scale_cols(N, g->k.V, ldr, g->k.hn, g->k.V, ldr, g->nr, s), "scale");
        CKR(init_g(g->nr, g->m, g->k.hn, g->k.g, s), "init g");
        std::fill(g->jr.begin(), g->jr.end(), 0);
        g->j = 0;
      }
      run.push_back(g);
    }
    if (run.empty()) return HLU_OK;
    // phase B: one launch for every preconditioner application
    std::vector<hlu_handle*> hs;
    std::vector<std::vector<SolveSeg>> segs;
    for (hlu_gmres* g : run) {
      const int64_t N = g->h->A.N, ldr = N * (g->m + 1);
      SolveSeg sg{g->k.V + g->j * N, g->k.Z + g->j * N, ldr, g->nr};
      size_t i = 0;
      while (i < hs.size() && hs[i] != g->h) ++i;
      int used = 0;
      if (i < hs.size())
        for (const SolveSeg& q : segs[i]) used += q.nr;
      if (i == hs.size() || used + g->nr > g->h->L.nrhs_max) {
        if (i < hs.size()) {
          // the factor's work vector is full: finish this group first
          int rc = solve_segments(hs, segs, s);
          if (rc) return rc;
          hs.clear();
          segs.clear();
        }
        if ((int)hs.size() == kMaxBatch) {
          int rc = solve_segments(hs, segs, s);
          if (rc) return rc;
          hs.clear();
          segs.clear();
        }
        hs.push_back(g->h);
        segs.push_back({sg});
      } else {
        segs[i].push_back(sg);
      }
    }
    CKR(cudaEventRecord(run[0]->h->ev0, s), "event");
    if (!hs.empty()) {
      int rc = solve_segments(hs, segs, s);
      if (rc) return rc;
    }
    CKR(cudaEventRecord(run[0]->h->ev1, s), "event");
    // phase C: Arnoldi step of every running state
    for (hlu_gmres* g : run) {
      KrylovWS& k = g->k;
      const int64_t N = g->h->A.N, ldr = N * (g->m + 1);
      const int j = g->j, m = g->m, nr = g->nr;
      CKR(spmv(g->h->A.rowptr, g->h->A.col, g->h->A.val, N, k.Z + j * N, ldr, k.W, N, nr, s), "spmv");
      CKR(multidot(N, k.V, ldr, j + 1, k.W, N, nr, k.part, k.h1, m + 1, s), "cgs1");
      CKR(multiaxpy(N, k.V, ldr, j + 1, k.h1, m + 1, k.W, N, nr, s), "cgs1 axpy");
      CKR(multidot(N, k.V, ldr, j + 1, k.W, N, nr, k.part, k.h2, m + 1, s), "cgs2");
      CKR(multiaxpy(N, k.V, ldr, j + 1, k.h2, m + 1, k.W, N, nr, s), "cgs2 axpy");
      int rc = norms_ws(k, k.W, N, nr, k.hn, s);
      if (rc) return rc;
      CKR(scale_cols(N, k.W, N, k.hn, k.V + (j + 1) * N, ldr, nr, s), "scale");
      CKR(givens(nr, m, j, k.h1, k.h2, m + 1, k.hn, k.H, k.cs, k.sn, k.g, k.est, s), "givens");
      CKR(cudaMemcpyAsync(g->est.data(), k.est, sizeof(double) * nr, cudaMemcpyDeviceToHost, s), "est");
    }
    CKR(cudaStreamSynchronize(s), "sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, run[0]->h->ev0, run[0]->h->ev1);
    for (hlu_gmres* g : run) {
      KrylovWS& k = g->k;
      g->precond_ms += ms / run.size();
      g->applies++;
      g->iters++;
      bool end = true;
      for (int r = 0; r < g->nr; ++r) {
        if (g->conv[r]) continue;
        if (g->jr[r] == 0 && g->est[r] <= g->tol * g->bn[r]) g->jr[r] = g->j + 1;
        end = end && g->jr[r] > 0;
      }
      if (end || g->j == g->m - 1 || g->iters >= g->maxit) {
        for (int r = 0; r < g->nr; ++r) {
          if (g->conv[r])
            g->jr[r] = 0;
          else if (g->jr[r] == 0)
            g->jr[r] = g->j + 1;
        }
        CKR(cudaMemcpyAsync(k.jr, g->jr.data(), sizeof(int) * g->nr, cudaMemcpyHostToDevice, s), "jr");
        CKR(backsub(g->nr, g->m, k.jr, k.H, k.g, k.y, s), "backsub");
        CKR(xupdate(g->h->A.N, k.Z, g->h->A.N * (g->m + 1), g->m, k.y, g->x, g->ld, g->nr, s), "xupdate");
        g->restarts++;
        g->j = -1;
      } else {
        g->j++;
      }
    }
    CKR(cudaStreamSynchronize(s), "sync");
    return HLU_OK;
  } catch (const std::exception& ex) {
    return fail(HLU_ERR_CUDA, ex.what());
  }
}

int hlu_gmres_status(const hlu_gmres* g, int32_t* done, hlu_stats* st) {
  if (!g) return fail(HLU_ERR_ARG, "null state");
  if (done) *done = g->done ? 1 : 0;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->iterations = g->iters;
    st->restarts = g->restarts;
    st->converged = g->done && g->status == HLU_OK;
    st->nrhs = g->nr;
    double rmax = 0, amax = 0;
    for (int r = 0; r < g->nr; ++r) {
      rmax = std::max(rmax, g->bn[r] > 0 ? g->beta[r] / g->bn[r] : 0.0);
      amax = std::max(amax, g->beta[r]);
    }
    st->relres_max = rmax;
    st->abs_res_max = amax;
    st->precond_ms = g->precond_ms;
    st->precond_applies = g->applies;
  }
  return g->done ? g->status : HLU_OK;
}

void hlu_gmres_end(hlu_gmres* g) {
  if (!g) return;
  g->k.free_all(g->s, true);
  delete g;
}

}  // extern "C"

namespace hlu {
}  // namespace hlu
