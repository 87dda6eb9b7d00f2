// Static race check of the task DAGs (host only, no GPU).
//
// The scheduler derives its edges from an abstract model of the data: accesses
// to (buffer, leaf-cluster segment) pairs, plus fences where temporary memory
// is re-used.  This check does not use that model.  It reads only the emitted
// tasks (operand views, ROWMV / RSOLVE terms, TRUNC pieces, pivot offsets,
// rank slots) and expands every operand to the elements it may touch: a view
// at its full capacity, whatever rank a run produces.  It then replays the DAG
// in program order.  An access that conflicts with an earlier one (write after
// write, read after write, write after read) must come from a task that the
// DAG's edges, taken transitively, order after the earlier task; otherwise two
// tasks of one launch may run in either order, or at the same time, on the
// device.  The factor arena, the pivot vectors and the rank slots are separate
// address spaces, and every access must stay inside its space.
//
// Rank slots are read where the device kernels take a live column count
// (TRSM, PROJ, ROWMV, DADD, RSOLVE operands and the terms' and pieces' left
// factors; the solve's right-hand-side count is a launch parameter, not a
// slot read).  ROWMV writes its output's slot with a copy of its input's
// count and TRUNC with the rank it computes.  Two writes of the same copied
// value (the same source slot, unchanged in between, or the same constant)
// leave the slot as it was, so they need no order between them: the
// scheduler splits one product's output rows over several ROWMV tasks that
// all do this.  A read then needs one of those writers before it.
#include <algorithm>
#include <cstring>
#include <exception>
#include <stdexcept>
#include <vector>

#include "../../include/hlu_debug.h"
#include "hlu_internal.h"

namespace hlu {
void trees_from_export(int32_t nc, const int32_t* cl, int32_t nb, const int32_t* bl,
                       std::vector<Cluster>& C, std::vector<Block>& B);
}

using namespace hlu;

namespace {

enum Space { SP_ARENA = 0, SP_PIV = 1, SP_SLOT = 2 };

class HazardCheck {
 public:
  HazardCheck(const Schedule& S, int64_t arena, int64_t piv, int64_t slots, int32_t nrhs_slot)
      : S_(S), nrhs_slot_(nrhs_slot) {
    size_[SP_ARENA] = arena;
    size_[SP_PIV] = std::max<int64_t>(piv, 1);
    size_[SP_SLOT] = std::max<int64_t>(slots, 1);
    for (int s = 0; s < 2; ++s) {
      lw_[s].assign((size_t)size_[s], -1);
      rhead_[s].assign((size_t)size_[s], -1);
    }
    slot_.assign((size_t)size_[SP_SLOT], SlotState());
    T_ = (int64_t)S.tasks.size();
    W_ = (T_ + 63) / 64;
    anc_.assign((size_t)(T_ * W_), 0);
    seen_.assign((size_t)T_, -1);
  }

  // report: see hlu_debug_check_hazards
  void run(int64_t* rep) {
    for (int64_t t = 0; t < T_; ++t) {
      uint64_t* row = anc_.data() + t * W_;
      for (int64_t e = S_.pred_ptr[t]; e < S_.pred_ptr[t + 1]; ++e) {
        const int64_t p = S_.pred_idx[e];
        if (p < 0 || p >= t) throw std::logic_error("a predecessor does not precede its task");
        const uint64_t* pr = anc_.data() + p * W_;
        for (int64_t w = 0; w <= p / 64; ++w) row[w] |= pr[w];
        row[p / 64] |= uint64_t(1) << (p % 64);
      }
      cur_ = (int32_t)t;
      task(S_.tasks[t]);
    }
    rep[0] = T_;
    rep[1] = accesses_;
    rep[2] = checks_;
    rep[3] = violations_;
    rep[4] = first_[0];
    rep[5] = first_[1];
    rep[6] = first_[2];
    rep[7] = first_[3];
    rep[8] = out_of_range_;
    rep[9] = S_.n_edges;
  }
  // whether task t is ordered after task p by the edges
  bool ordered(int64_t p, int64_t t) const { return (anc_[(size_t)(t * W_ + p / 64)] >> (p % 64)) & 1; }

 private:
  // value a slot write stores: a copy of slot `src` at `version`, a constant
  // (src -1, version = the value), or a computed rank (src -2, version = task)
  struct Value {
    int64_t src = -3, version = 0;
    bool operator==(const Value& o) const { return src == o.src && version == o.version; }
  };
  struct SlotState {
    std::vector<int32_t> writers;  // writers of the current value
    std::vector<int32_t> readers;  // readers since the value was set
    Value value;
    int64_t version = 0;           // bumped whenever the value changes
  };
  const Schedule& S_;
  const int32_t nrhs_slot_;
  int64_t size_[3];
  std::vector<int32_t> lw_[2], rhead_[2];  // last writer; head of the readers since it
  std::vector<SlotState> slot_;
  std::vector<int32_t> pool_task_, pool_next_;
  std::vector<uint64_t> anc_;  // ancestors of each task, T x W bits
  std::vector<int32_t> seen_;  // seen_[u] == cur_: the pair (u, cur_) is already checked
  int64_t T_ = 0, W_ = 0;
  int32_t cur_ = -1;
  bool writing_ = false;
  int64_t accesses_ = 0, checks_ = 0, violations_ = 0, out_of_range_ = 0;
  int64_t first_[4] = {-1, -1, -1, -1};

  bool ancestor(int32_t u) const {
    return (anc_[(size_t)(cur_ * W_ + u / 64)] >> (u % 64)) & 1;
  }
  void require(int32_t u, int space, int64_t e) {
    if (u < 0 || u == cur_ || seen_[u] == cur_) return;
    seen_[u] = cur_;
    ++checks_;
    if (!ancestor(u)) {
      if (violations_ == 0) {
        first_[0] = u;
        first_[1] = cur_;
        first_[2] = space;
        first_[3] = e;
      }
      ++violations_;
    }
  }
  void touch(int space, int64_t e) {
    ++accesses_;
    if (e < 0 || e >= size_[space]) {
      if (out_of_range_ == 0 && violations_ == 0) {
        first_[0] = -1;
        first_[1] = cur_;
        first_[2] = space;
        first_[3] = e;
      }
      ++out_of_range_;
      return;
    }
    std::vector<int32_t>& lw = lw_[space];
    std::vector<int32_t>& rh = rhead_[space];
    require(lw[e], space, e);
    if (!writing_) {
      if (rh[e] >= 0 && pool_task_[rh[e]] == cur_) return;
      if (pool_task_.size() >= (size_t)1 << 31) throw std::length_error("too many reads to track");
      pool_task_.push_back(cur_);
      pool_next_.push_back(rh[e]);
      rh[e] = (int32_t)pool_task_.size() - 1;
      return;
    }
    for (int32_t r = rh[e]; r >= 0; r = pool_next_[r]) require(pool_task_[r], space, e);
    rh[e] = -1;
    lw[e] = cur_;
  }
  void range(int space, int64_t lo, int64_t n) {
    for (int64_t i = 0; i < n; ++i) touch(space, lo + i);
  }
  bool slot_ok(int64_t sl) {
    ++accesses_;
    if (sl >= 0 && sl < size_[SP_SLOT]) return true;
    if (out_of_range_ == 0 && violations_ == 0) {
      first_[0] = -1;
      first_[1] = cur_;
      first_[2] = SP_SLOT;
      first_[3] = sl;
    }
    ++out_of_range_;
    return false;
  }
  // the live column count of v, where a kernel reads it
  void count(const View& v) {
    if (v.slot < 0 || v.slot == nrhs_slot_ || !slot_ok(v.slot)) return;
    SlotState& st = slot_[v.slot];
    if (!st.writers.empty()) {
      bool after_one = false;
      for (int32_t w : st.writers) after_one = after_one || w == cur_ || ancestor(w);
      if (!after_one) require(st.writers[0], SP_SLOT, v.slot);
    }
    if (st.readers.empty() || st.readers.back() != cur_) st.readers.push_back(cur_);
  }
  Value value_of(const View& v) const {  // what a copy of v's count stores
    Value x;
    if (v.slot < 0) {
      x.src = -1;
      x.version = v.cols;
    } else if (v.slot == nrhs_slot_) {
      x.src = -1;
      x.version = -1;  // the launch's right-hand-side count
    } else {
      x.src = v.slot;
      x.version = (v.slot < size_[SP_SLOT]) ? slot_[v.slot].version : 0;
    }
    return x;
  }
  void slot_write(int32_t sl, const Value& x) {
    if (!slot_ok(sl)) return;
    SlotState& st = slot_[sl];
    if (!st.writers.empty() && st.value == x) {  // the same value again
      st.writers.push_back(cur_);
      return;
    }
    for (int32_t w : st.writers) require(w, SP_SLOT, sl);
    for (int32_t r : st.readers) require(r, SP_SLOT, sl);
    st.writers.assign(1, cur_);
    st.readers.clear();
    st.value = x;
    ++st.version;
  }
  // every element a view may address: rows x cols (cols is the capacity when
  // the count comes from a rank slot)
  void view(const View& v) {
    for (int64_t j = 0; j < v.cols; ++j)
      for (int64_t i = 0; i < v.rows; ++i) touch(SP_ARENA, v.off + i * v.rs + j * v.cs);
  }
  // a task's term or piece list must lie inside the schedule's list
  bool list_ok(const Task& t, size_t n) {
    if (t.list_count == 0 || (t.list_begin >= 0 && t.list_count > 0 &&
                              (size_t)t.list_begin + (size_t)t.list_count <= n))
      return true;
    if (out_of_range_ == 0 && violations_ == 0) {
      first_[0] = -1;
      first_[1] = cur_;
      first_[2] = SP_ARENA;
      first_[3] = t.list_begin;
    }
    ++out_of_range_;
    return false;
  }
  void terms(const Task& t) {
    if (!list_ok(t, S_.terms.size())) return;
    for (int32_t q = 0; q < t.list_count; ++q) {
      const Term& m = S_.terms[t.list_begin + q];
      count(m.A);
      view(m.A);
      view(m.B);
    }
  }
  void pieces(const Task& t) {
    if (!list_ok(t, S_.pieces.size())) return;
    for (int32_t q = 0; q < t.list_count; ++q) {
      const Piece& p = S_.pieces[t.list_begin + q];
      count(p.X);
      view(p.X);
      view(p.Y);
    }
  }

  // reads first, then writes; an operand both read and written is in both
  void task(const Task& t) {
    writing_ = false;
    switch (t.type) {
      case TK_GETRF: view(t.a); break;
      case TK_TRSM_L: count(t.b); view(t.a); range(SP_PIV, t.piv_off, t.a.rows); view(t.b); break;
      case TK_TRSM_UT:
      case TK_TRSM_U: count(t.b); view(t.a); view(t.b); break;
      case TK_PROJ: count(t.a); count(t.b); view(t.a); view(t.b); break;
      case TK_ROWMV: count(t.b); terms(t); if (!(t.flags & TF_OVERWRITE)) view(t.c); break;
      case TK_TRUNC: pieces(t); break;
      case TK_DADD: count(t.c); count(t.a); view(t.a); view(t.b); if (!(t.flags & TF_OVERWRITE)) view(t.c); break;
      case TK_RSOLVE:
        count(t.b);
        count(t.c);
        terms(t);
        view(t.a);
        if (!(t.flags & TF_UPPER)) range(SP_PIV, t.piv_off, t.a.rows);
        view(t.c);
        break;
      case TK_FENCE: break;
      default: throw std::logic_error("task type");
    }
    writing_ = true;
    switch (t.type) {
      case TK_GETRF: view(t.a); range(SP_PIV, t.piv_off, t.a.rows); break;
      case TK_TRSM_L:
      case TK_TRSM_UT:
      case TK_TRSM_U: view(t.b); break;
      case TK_PROJ: view(t.c); break;
      case TK_ROWMV: view(t.c); break;
      case TK_TRUNC: view(t.a); view(t.b); break;
      case TK_DADD: view(t.c); break;
      case TK_RSOLVE: view(t.c); break;
      default: break;
    }
    writing_ = false;
    if (t.out_slot >= 0) {
      if (t.type == TK_ROWMV) {
        slot_write(t.out_slot, value_of(t.b));
      } else {
        Value x;
        x.src = -2;
        x.version = cur_;
        slot_write(t.out_slot, x);
      }
    }
  }
};

}  // namespace

extern "C" int hlu_debug_check_hazards(int32_t nc, const int32_t* clusters, int32_t nb, const int32_t* blocks,
                                       int32_t rank_cap, int32_t tile, int32_t nrhs_max, int32_t which,
                                       int64_t drop_edge, int64_t* report) {
  try {
    if (!clusters || !blocks || !report || nc < 1 || nb < 1 || nrhs_max < 1 || nrhs_max > 16 || which < 0 ||
        which > 4 || rank_cap < 0 || rank_cap > kRankMax)
      return 1;
    std::memset(report, 0, sizeof(int64_t) * 11);
    std::vector<Cluster> C;
    std::vector<Block> B;
    trees_from_export(nc, clusters, nb, blocks, C, B);
    const int32_t cap = rank_cap > 0 ? rank_cap : kRankMax;
    ArenaLayout L;
    SchedStats st;
    Schedule F, S, S0, S1, S2;
    Schedule* pick = nullptr;
    if (which <= 1) {
      build_schedules(C, B, cap, nrhs_max, tile, L, F, S, st, nullptr);
      pick = which == 0 ? &F : &S;
    } else {
      std::vector<Block> FB = factor_tree(C, B, tile), Bx;
      build_inverse_schedules(C, FB, cap, nrhs_max, tile, L, Bx, S0, S1, S2, st);
      pick = which == 2 ? &S0 : which == 3 ? &S1 : &S2;
    }
    if (drop_edge >= (int64_t)pick->pred_idx.size()) return 1;
    int64_t drop_from = -1, drop_to = -1;
    if (drop_edge >= 0) {  // a planted mistake, to test the check itself
      drop_from = pick->pred_idx[drop_edge];
      drop_to = std::upper_bound(pick->pred_ptr.begin(), pick->pred_ptr.end(), drop_edge) - pick->pred_ptr.begin() - 1;
      pick->pred_idx.erase(pick->pred_idx.begin() + drop_edge);
      for (size_t t = 1; t < pick->pred_ptr.size(); ++t)
        if (pick->pred_ptr[t] > drop_edge) --pick->pred_ptr[t];
      --pick->n_edges;
    }
    const int64_t T = (int64_t)pick->tasks.size();
    if (T > 40000 || L.total > (int64_t)1 << 27) return 6;  // bitsets and element states stay in host memory
    HazardCheck hc(*pick, L.total, L.piv_total, L.n_slots, L.nrhs_slot);
    hc.run(report);
    report[10] = drop_edge >= 0 ? (int64_t)hc.ordered(drop_from, drop_to) : -1;
    return (report[3] || report[8]) ? 9 : 0;
  } catch (const std::exception&) {
    return 6;
  }
}
