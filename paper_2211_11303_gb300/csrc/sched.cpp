// Host task scheduler: turns the recursive H-LU of Algorithm 1 step II (block
// form: LU(A11); A12 <- L11^-1 P A12; A21 <- A21 U11^-1; A22 <- A22 - A21 A12
// truncated; LU(A22), as in the H-LU source the paper cites) and the
// preconditioner application U^-1 (L^-1 r) of step III into task DAGs.
//
// The recursion is walked once on the host.  Every leaf-level operation becomes
// a task of one of the kinds in hlu_internal.h; the data it touches is
// recorded per (buffer, leaf-cluster segment), which yields read-after-write,
// write-after-read and write-after-write edges.  The emission order is the
// sequential program order, hence a topological order: the device executor
// hands out tasks in that order and each task only waits on earlier ones.
//
// Ranks of low-rank blocks are data dependent.  The schedule only uses rank
// capacities; kernels read the live rank from a rank slot when they run.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <stdexcept>

#include "hlu_internal.h"

namespace hlu {
namespace {

// The schedule's vectors reach gigabytes (n = 24: 2.2 GB of tasks, 1.2 GB of
// terms, 0.9 GB of predecessor indices), and every reallocation writes its
// new block once.  Growing by 4 instead of 2 writes about 4/3 of the final
// size instead of about 2x, which took a quarter off the n = 24 build (most
// of it page faults); the unused capacity is address space only.
template <class V>
inline void grow4(V& v, size_t extra = 1) {
  if (v.size() + extra > v.capacity())
    v.reserve(std::max<size_t>(v.size() + extra, std::max<size_t>(4096, v.capacity() * 4)));
}

struct MV {
  int32_t buf;   // dependency buffer (-1: read-only, untracked)
  int32_t clus;  // cluster whose index range the rows cover
  View v;
};
struct LR {
  MV X, Y;
};
struct PieceMV {
  LR p;
  int32_t xoff, yoff;
  float sign;
};

struct Buf {
  int32_t base_leaf;
  int32_t nseg;
  int64_t seg0;
};

// Targets of a subdivided x subdivided product up to this size on both sides
// are agglomerated in one truncation (the executor's dense route handles them
// whole); larger ones quadrant by quadrant first.
constexpr int32_t kOneStepAgglomeration = 128;

class Sched {
 public:
  Sched(const std::vector<Cluster>& C, const std::vector<Block>& B, int32_t kcap, ArenaLayout& L,
        Schedule* S, std::vector<int32_t>& dbuf, std::vector<int32_t>& xbuf,
        std::vector<int32_t>& ybuf, bool make_buffers, int32_t segsz, int64_t ring_off,
        int64_t ring_size)
      : C_(C), B_(B), kcap_(kcap), L_(L), S_(S), dbuf_(dbuf), xbuf_(xbuf), ybuf_(ybuf),
        ring_off_(ring_off), ring_size_(ring_size) {
    S_->pred_ptr.assign(1, 0);
    // dependency segments: clusters of at most `segsz` DOFs whose parent is
    // larger (the tile level, or the leaves); every cluster covers a range of them
    seg_begin_.assign(C_.size(), 0);
    seg_end_.assign(C_.size(), 0);
    seg_cluster_.clear();
    segsz_ = segsz;
    assign_segments(0, false, segsz);
    chunk_occ_.assign((size_t)((ring_size_ + kChunk - 1) / kChunk) + 1, std::vector<int32_t>());
    chunk_fence_task_.assign(chunk_occ_.size(), -1);
    chunk_pass_.assign(chunk_occ_.size(), 0);
    if (make_buffers) {
      dbuf_.assign(B_.size(), -1);
      xbuf_.assign(B_.size(), -1);
      ybuf_.assign(B_.size(), -1);
    }
    // each schedule tracks its own buffer states from scratch
    for (size_t b = 0; b < B_.size(); ++b) {
      if (B_[b].kind == KIND_DENSE) dbuf_[b] = new_buf_single();
      if (B_[b].kind == KIND_ADM) {
        xbuf_[b] = new_buf_leaves(B_[b].row);
        ybuf_[b] = new_buf_leaves(B_[b].col);
      }
    }
  }

  // ---------------------------------------------------------------- segments
  void assign_segments(int32_t c, bool inside, int32_t segsz) {
    const Cluster& cl = C_[c];
    bool is_seg = !inside && (cl.size <= segsz || cl.son[0] < 0);
    if (is_seg || inside) {
      if (is_seg) seg_cluster_.push_back(c);
      int32_t sidx = (int32_t)seg_cluster_.size() - 1;
      seg_begin_[c] = sidx;
      seg_end_[c] = sidx + 1;
      if (cl.son[0] >= 0) {
        assign_segments(cl.son[0], true, segsz);
        assign_segments(cl.son[1], true, segsz);
      }
      return;
    }
    seg_begin_[c] = (int32_t)seg_cluster_.size();
    assign_segments(cl.son[0], false, segsz);
    assign_segments(cl.son[1], false, segsz);
    seg_end_[c] = (int32_t)seg_cluster_.size();
  }

  // ---------------------------------------------------------------- arena
  // Temporaries live in a ring region.  Re-using ring memory orders the new
  // occupant's writers after every task that touched the memory before.
  static constexpr int64_t kChunk = 1 << 14;
  int64_t alloc(int64_t n) {
    n = (n + 31) & ~int64_t(31);
    temp_elems_ += n;
    if (n > ring_size_) throw std::runtime_error("temporary larger than the ring");
    if (cursor_ + n > ring_size_) {
      cursor_ = 0;
      ++pass_;
      ++wraps_;
    }
    int64_t o = cursor_;
    cursor_ += n;
    pending_fence_.clear();
    for (int64_t ch = o / kChunk; ch <= (o + n - 1) / kChunk; ++ch) {
      if (chunk_pass_[ch] != pass_) {
        // first use of this chunk in this pass: a no-work fence task waits for
        // every task that touched the chunk's previous occupants
        chunk_fence_task_[ch] = -1;
        if (!chunk_occ_[ch].empty()) {
          Task f = make(TK_FENCE);
          int32_t saved_cur = cur_;
          std::vector<int32_t> saved_deps;
          saved_deps.swap(deps_);
          begin(f);
          for (int32_t old : chunk_occ_[ch])
            for (int64_t r = acc_head_[old]; r >= 0; r = acc_next_[r]) dep(acc_task_[r]);
          end();
          chunk_fence_task_[ch] = cur_;
          deps_.swap(saved_deps);
          cur_ = saved_cur;
        }
        chunk_occ_[ch].clear();
        chunk_pass_[ch] = pass_;
      }
      if (chunk_fence_task_[ch] >= 0) pending_fence_.push_back(chunk_fence_task_[ch]);
    }
    last_alloc_lo_ = o / kChunk;
    last_alloc_hi_ = (o + n - 1) / kChunk;
    return ring_off_ + o;
  }
  // attach the fence of the last allocation to buffer `b` and record it as
  // the occupant of that ring range
  void bind_alloc(int32_t b) {
    if (!pending_fence_.empty()) {
      std::sort(pending_fence_.begin(), pending_fence_.end());
      pending_fence_.erase(std::unique(pending_fence_.begin(), pending_fence_.end()), pending_fence_.end());
      fence_begin_[b] = (int64_t)fence_pool_.size();
      fence_pool_.insert(fence_pool_.end(), pending_fence_.begin(), pending_fence_.end());
      fence_end_[b] = (int64_t)fence_pool_.size();
      pending_fence_.clear();
    }
    for (int64_t ch = last_alloc_lo_; ch <= last_alloc_hi_; ++ch) chunk_occ_[ch].push_back(b);
  }
  int32_t new_slot() { return L_.n_slots++; }
  int64_t temp_elems_ = 0;
  int64_t peak_ = 0;

  // ---------------------------------------------------------------- buffers
  int32_t push_buf(const Buf& b) {
    bufs_.push_back(b);
    acc_head_.push_back(-1);
    acc_last_.push_back(-1);
    fence_begin_.push_back(0);
    fence_end_.push_back(0);
    return (int32_t)bufs_.size() - 1;
  }
  int32_t new_buf_leaves(int32_t clus) {
    Buf b;
    b.base_leaf = seg_begin_[clus];
    b.nseg = seg_end_[clus] - seg_begin_[clus];
    b.seg0 = (int64_t)seg_writer_.size();
    seg_writer_.resize(seg_writer_.size() + b.nseg, -1);
    seg_rhead_.resize(seg_rhead_.size() + b.nseg, -1);
    seg_buf_.resize(seg_buf_.size() + b.nseg, (int32_t)bufs_.size());
    return push_buf(b);
  }
  int32_t new_buf_single() {
    Buf b;
    b.base_leaf = -1;
    b.nseg = 1;
    b.seg0 = (int64_t)seg_writer_.size();
    seg_writer_.push_back(-1);
    seg_rhead_.push_back(-1);
    seg_buf_.push_back((int32_t)bufs_.size());
    return push_buf(b);
  }

  // ---------------------------------------------------------------- views
  int32_t rowc(int32_t b) const { return B_[b].row; }
  int32_t colc(int32_t b) const { return B_[b].col; }
  int32_t sz(int32_t c) const { return C_[c].size; }
  int32_t kind(int32_t b) const { return B_[b].kind; }
  int32_t son(int32_t b, int i, int j) const { return B_[b].son[2 * i + j]; }

  MV mvD(int32_t b) const {
    MV m;
    m.buf = dbuf_[b];
    m.clus = rowc(b);
    m.v = View{L_.dense_off[b], 1, sz(rowc(b)), sz(rowc(b)), sz(colc(b)), -1, 0};
    return m;
  }
  MV mvDT(int32_t b) const {
    MV m;
    m.buf = dbuf_[b];
    m.clus = colc(b);
    m.v = View{L_.dense_off[b], sz(rowc(b)), 1, sz(colc(b)), sz(rowc(b)), -1, 0};
    return m;
  }
  MV mvX(int32_t b) const {
    MV m;
    m.buf = xbuf_[b];
    m.clus = rowc(b);
    m.v = View{L_.x_off[b], 1, sz(rowc(b)), sz(rowc(b)), L_.cap[b], L_.slot[b], 0};
    return m;
  }
  MV mvY(int32_t b) const {
    MV m;
    m.buf = ybuf_[b];
    m.clus = colc(b);
    m.v = View{L_.y_off[b], 1, sz(colc(b)), sz(colc(b)), L_.cap[b], L_.slot[b], 0};
    return m;
  }
  MV mvIdent(int32_t clus) const {
    if (sz(clus) > L_.ident_n) throw std::logic_error("identity too small");
    MV m;
    m.buf = -1;
    m.clus = clus;
    m.v = View{L_.ident_off, 1, L_.ident_n, sz(clus), sz(clus), -1, 0};
    return m;
  }
  MV sub(const MV& m, int32_t s) const {
    int32_t d = C_[s].off - C_[m.clus].off;
    if (d < 0 || d + C_[s].size > C_[m.clus].size) throw std::logic_error("sub view outside");
    MV r = m;
    r.clus = s;
    r.v.off += (int64_t)d * m.v.rs;
    r.v.rows = C_[s].size;
    return r;
  }
  // fresh temporary with per-leaf dependency segments; column count via a slot
  MV new_temp(int32_t clus, int32_t cols_cap) {
    MV m;
    m.clus = clus;
    int32_t rows = sz(clus);
    int64_t off = alloc((int64_t)rows * std::max(cols_cap, 1));
    m.buf = new_buf_leaves(clus);
    bind_alloc(m.buf);
    m.v = View{off, 1, rows, rows, cols_cap, new_slot(), 0};
    return m;
  }
  MV new_dense_temp(int32_t clus, int32_t cols) {
    MV m;
    m.clus = clus;
    int32_t rows = sz(clus);
    int64_t off = alloc((int64_t)rows * cols);
    m.buf = new_buf_single();
    bind_alloc(m.buf);
    m.v = View{off, 1, rows, rows, cols, -1, 0};
    return m;
  }
  int32_t cols_cap(const View& v) const { return v.cols; }

  // ---------------------------------------------------------------- tasks
  int32_t begin(const Task& t) {
    int32_t id = (int32_t)S_->tasks.size();
    grow4(S_->tasks);
    S_->tasks.push_back(t);
    stamp_.push_back(-1);
    cur_ = id;
    deps_.clear();
    return id;
  }
  void dep(int32_t p) {
    if (p < 0 || p == cur_) return;
    if (stamp_[p] == cur_) return;
    stamp_[p] = cur_;
    deps_.push_back(p);
  }
  void note_access(int32_t b) {
    if (acc_last_[b] == cur_) return;
    acc_last_[b] = cur_;
    grow4(acc_task_);
    grow4(acc_next_);
    acc_task_.push_back(cur_);
    acc_next_.push_back(acc_head_[b]);
    acc_head_[b] = (int64_t)acc_task_.size() - 1;
  }
  void touch(int64_t seg, bool w) {
    const int32_t b = seg_buf_[seg];
    if (seg_writer_[seg] < 0)
      for (int64_t f = fence_begin_[b]; f < fence_end_[b]; ++f) dep(fence_pool_[f]);
    note_access(b);
    dep(seg_writer_[seg]);
    if (w) {
      for (int64_t r = seg_rhead_[seg]; r >= 0; r = rnext_[r]) dep(rtask_[r]);
      seg_rhead_[seg] = -1;
      seg_writer_[seg] = cur_;
    } else {
      grow4(rtask_);
      grow4(rnext_);
      rtask_.push_back(cur_);
      rnext_.push_back(seg_rhead_[seg]);
      seg_rhead_[seg] = (int64_t)rtask_.size() - 1;
    }
  }
  void acc(const MV& m, bool w) {
    if (m.buf < 0) return;
    const Buf& b = bufs_[m.buf];
    if (b.nseg == 1 && b.base_leaf < 0) {
      touch(b.seg0, w);
      return;
    }
    for (int32_t l = seg_begin_[m.clus]; l < seg_end_[m.clus]; ++l) {
      int64_t s = b.seg0 + (l - b.base_leaf);
      touch(s, w);
    }
  }
  // read of one segment: enough to order the task after any writer of the
  // buffer's rank slot (rank writers write every segment).  The right-hand
  // side count of a solve or apply is a launch parameter that no task
  // writes, so a count taken from it orders nothing: without this, every
  // update of the backward solve waited for the first segment of its input,
  // which is solved last
  void acc_rank(const MV& m) {
    if (m.buf < 0 || m.v.slot < 0 || m.v.slot == L_.nrhs_slot) return;
    const Buf& b = bufs_[m.buf];
    touch(b.seg0, false);
  }
  void end() {
    std::sort(deps_.begin(), deps_.end());
    grow4(S_->pred_idx, deps_.size());
    grow4(S_->pred_ptr);
    S_->pred_idx.insert(S_->pred_idx.end(), deps_.begin(), deps_.end());
    S_->pred_ptr.push_back((int64_t)S_->pred_idx.size());
  }

  static Task make(int32_t type) {
    Task t;
    std::memset(&t, 0, sizeof(t));
    t.type = type;
    t.out_slot = -1;
    t.piv_off = -1;
    t.sign = 1.0f;
    t.a.slot = t.b.slot = t.c.slot = -1;
    return t;
  }

  // ---------------------------------------------------------------- leaf ops
  void getrf(int32_t d) {
    Task t = make(TK_GETRF);
    t.a = mvD(d).v;
    t.piv_off = L_.piv_off[d];
    begin(t);
    acc(mvD(d), true);
    end();
  }
  void trsm_leaf(int32_t type, int32_t d, const MV& V) {
    const int32_t sg = seg_begin_[rowc(d)];
    if ((type == TK_TRSM_L || type == TK_TRSM_U) && seg_end_[rowc(d)] - sg == 1 && sg < (int32_t)pending_.size() &&
        pending_[sg].active && seg_cluster_[sg] == rowc(d)) {
      // the late update of this segment and its triangular solve in one task
      Pending& pd = pending_[sg];
      Task k = make(TK_RSOLVE);
      k.flags = type == TK_TRSM_U ? TF_UPPER : 0;
      k.a = mvD(d).v;
      k.b = pd.Vin.v;  // column count source
      k.c = V.v;
      k.piv_off = L_.piv_off[d];
      k.sign = pd.sign;
      k.list_begin = (int32_t)S_->terms.size();
      k.list_count = (int32_t)pd.list.size();
      begin(k);
      push_terms(pd.lv, pd.T, pd.list, pd.Vin, rowc(d), pd.trans);
      acc_rank(pd.Vin);
      acc(mvD(d), false);
      acc(V, true);
      end();
      pd = Pending();
      return;
    }
    Task t = make(type);
    t.a = mvD(d).v;
    t.b = V.v;
    t.piv_off = L_.piv_off[d];
    begin(t);
    acc(mvD(d), false);
    acc(V, true);
    end();
  }

  // ---------------------------------------------------------------- H x multivector
  void leaves_of(int32_t b, std::vector<int32_t>& out) const {
    if (kind(b) != KIND_SUB) {
      out.push_back(b);
      return;
    }
    for (int k = 0; k < 4; ++k) leaves_of(B_[b].son[k], out);
  }

  // Vout (+)= sign * op(b) Vin, op = transpose when trans.  Vin covers the
  // in-cluster of b, Vout its out-cluster.  overwrite: Vout starts from zero
  // and out_slot receives Vin's column count.
  // late_seg >= 0 (solves, accumulating): the terms of every output unit are
  // split into two ROWMV tasks, those whose input does not cover segment
  // late_seg (the input's last segment to be solved) first, so that only the
  // few terms reading it wait for the end of the preceding solve.
  // fuse_seg >= 0 (solve schedule): the late task of the unit that is
  // segment fuse_seg is not emitted here but merged into that segment's next
  // triangular leaf solve (one RSOLVE task instead of a ROWMV and a TRSM).
  void hmul(int32_t b, const MV& Vin, const MV& Vout, float sign, bool trans, bool overwrite,
            int32_t out_slot, int32_t late_seg = -1, int32_t fuse_seg = -1) {
    std::vector<int32_t> lv;
    leaves_of(b, lv);
    int32_t oc = trans ? colc(b) : rowc(b);
    if (Vout.clus != oc || Vin.clus != (trans ? rowc(b) : colc(b)))
      throw std::logic_error("hmul cluster mismatch");
    std::vector<MV> T(lv.size());
    for (size_t i = 0; i < lv.size(); ++i) {
      int32_t be = lv[i];
      if (kind(be) != KIND_ADM) continue;
      MV A = trans ? mvX(be) : mvY(be);
      int32_t ic = trans ? rowc(be) : colc(be);
      MV vin = sub(Vin, ic);
      MV t;
      t.clus = -1;
      int32_t cap = L_.cap[be];
      int64_t toff = alloc((int64_t)cap * std::max(vin.v.cols, 1));
      t.buf = new_buf_single();
      bind_alloc(t.buf);
      t.v = View{toff, 1, cap, cap, vin.v.cols, vin.v.slot, 0};
      Task k = make(TK_PROJ);
      k.a = A.v;
      k.b = vin.v;
      k.c = t.v;
      begin(k);
      acc(A, false);
      acc(vin, false);
      touch(bufs_[t.buf].seg0, true);
      end();
      T[i] = t;
    }
    // output units: the segment clusters under the out-cluster (or the
    // out-cluster itself when it lies inside one segment)
    std::vector<int32_t> units;
    if (seg_end_[oc] - seg_begin_[oc] <= 1) {
      units.push_back(oc);
    } else {
      for (int32_t q = seg_begin_[oc]; q < seg_end_[oc]; ++q) units.push_back(seg_cluster_[q]);
    }
    const int32_t nu = (int32_t)units.size();
    const int32_t u0 = seg_begin_[oc];
    auto unit_of = [&](int32_t segidx) { return nu == 1 ? 0 : segidx - u0; };
    std::vector<int32_t> cnt(nu + 1, 0);
    for (size_t i = 0; i < lv.size(); ++i) {
      int32_t obc = trans ? colc(lv[i]) : rowc(lv[i]);
      for (int32_t q = seg_begin_[obc]; q < seg_end_[obc]; ++q) cnt[unit_of(q) + 1]++;
    }
    for (int32_t l = 0; l < nu; ++l) cnt[l + 1] += cnt[l];
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1), items(cnt[nu]);
    for (size_t i = 0; i < lv.size(); ++i) {
      int32_t obc = trans ? colc(lv[i]) : rowc(lv[i]);
      for (int32_t q = seg_begin_[obc]; q < seg_end_[obc]; ++q) items[fill[unit_of(q)]++] = (int32_t)i;
    }
    MV kview = Vin;
    for (int32_t l = 0; l < nu; ++l) {
      if (cnt[l] == cnt[l + 1] && !overwrite) continue;
      const int32_t lc = units[l];
      // terms grouped by how long before late_seg their input is final: group
      // g >= 1 holds the terms whose last-solved input segment lies between
      // 2^(g-1) and 2^g - 1 segments before late_seg, group 0 those reading
      // late_seg itself; the groups run in that order, so each one waits only
      // for inputs solved well before it and the last ones are small
      constexpr int kGroups = 33;
      std::vector<int32_t> parts[kGroups];
      for (int32_t q = cnt[l]; q < cnt[l + 1]; ++q) {
        const int32_t i = items[q];
        int g = 0;
        if (late_seg >= 0 && !overwrite) {
          const int32_t ic = trans ? rowc(lv[i]) : colc(lv[i]);
          int32_t dist = 0;
          if (late_seg >= seg_end_[ic])
            dist = late_seg - (seg_end_[ic] - 1);
          else if (late_seg < seg_begin_[ic])
            dist = seg_begin_[ic] - late_seg;
          while (dist > 0) {
            ++g;
            dist >>= 1;
          }
        }
        parts[g].push_back(i);
      }
      for (int part = kGroups - 1; part >= 0; --part) {
        if (parts[part].empty() && (part != 0 || !overwrite)) continue;
        if (part == 0 && late_seg >= 0 && fuse_seg >= 0 && fuse_seg < (int32_t)pending_.size() &&
            lc == seg_cluster_[fuse_seg] && !pending_[fuse_seg].active) {
          Pending& pd = pending_[fuse_seg];
          pd.active = true;
          pd.lv = lv;
          pd.T = T;
          pd.list = parts[part];
          pd.Vin = Vin;
          pd.sign = sign;
          pd.trans = trans;
          continue;
        }
        emit_rowmv(lv, T, parts[part], Vin, Vout, lc, sign, trans, overwrite, out_slot, kview);
      }
    }
  }
  // the terms of a ROWMV (or RSOLVE) task for unit lc, with their reads
  void push_terms(const std::vector<int32_t>& lv, const std::vector<MV>& T, const std::vector<int32_t>& list,
                  const MV& Vin, int32_t lc, bool trans) {
    for (int32_t i : list) {
      int32_t be = lv[i];
      int32_t obc = trans ? colc(be) : rowc(be);
      // the term covers rows (obc intersect lc) of the unit
      int32_t rc = C_[obc].size <= C_[lc].size ? obc : lc;
      Term tm;
      std::memset(&tm, 0, sizeof(tm));
      tm.roff = C_[rc].off - C_[lc].off;
      if (kind(be) == KIND_DENSE) {
        MV A = sub(trans ? mvDT(be) : mvD(be), rc);
        MV Bv = sub(Vin, trans ? rowc(be) : colc(be));
        tm.A = A.v;
        tm.B = Bv.v;
        acc(A, false);
        acc(Bv, false);
      } else {
        MV A = sub(trans ? mvY(be) : mvX(be), rc);
        tm.A = A.v;
        tm.B = T[i].v;
        acc(A, false);
        touch(bufs_[T[i].buf].seg0, false);
      }
      grow4(S_->terms);
      S_->terms.push_back(tm);
    }
  }
  // one ROWMV task: unit lc of Vout (+)= sign * sum over the listed leaves
  void emit_rowmv(const std::vector<int32_t>& lv, const std::vector<MV>& T, const std::vector<int32_t>& list,
                  const MV& Vin, const MV& Vout, int32_t lc, float sign, bool trans, bool overwrite,
                  int32_t out_slot, const MV& kview) {
    {
      Task k = make(TK_ROWMV);
      k.flags = overwrite ? TF_OVERWRITE : 0;
      k.sign = sign;
      k.c = sub(Vout, lc).v;
      k.b = Vin.v;  // column count source
      k.out_slot = out_slot;
      k.list_begin = (int32_t)S_->terms.size();
      k.list_count = (int32_t)list.size();
      begin(k);
      push_terms(lv, T, list, Vin, lc, trans);
      acc_rank(kview);
      acc(sub(Vout, lc), true);
      end();
    }
  }
  MV hmul_new(int32_t b, const MV& Vin, bool trans) {
    int32_t oc = trans ? colc(b) : rowc(b);
    MV out = new_temp(oc, Vin.v.cols);
    hmul(b, Vin, out, 1.0f, trans, true, out.v.slot);
    return out;
  }

  // ---------------------------------------------------------------- triangular
  void solve_lower(int32_t d, const MV& V) {
    if (kind(d) == KIND_DENSE) {
      trsm_leaf(TK_TRSM_L, d, V);
      return;
    }
    const Cluster& c = C_[rowc(d)];
    MV V0 = sub(V, c.son[0]), V1 = sub(V, c.son[1]);
    solve_lower(son(d, 0, 0), V0);
    hmul(son(d, 1, 0), V0, V1, -1.0f, false, false, -1, seg_end_[c.son[0]] - 1, seg_begin_[c.son[1]]);
    solve_lower(son(d, 1, 1), V1);
  }
  void solve_upperT(int32_t d, const MV& W) {
    if (kind(d) == KIND_DENSE) {
      trsm_leaf(TK_TRSM_UT, d, W);
      return;
    }
    const Cluster& c = C_[rowc(d)];
    MV W0 = sub(W, c.son[0]), W1 = sub(W, c.son[1]);
    solve_upperT(son(d, 0, 0), W0);
    hmul(son(d, 0, 1), W0, W1, -1.0f, true, false, -1);
    solve_upperT(son(d, 1, 1), W1);
  }
  void solve_upper(int32_t d, const MV& V) {
    if (kind(d) == KIND_DENSE) {
      trsm_leaf(TK_TRSM_U, d, V);
      return;
    }
    const Cluster& c = C_[rowc(d)];
    MV V0 = sub(V, c.son[0]), V1 = sub(V, c.son[1]);
    solve_upper(son(d, 1, 1), V1);
    hmul(son(d, 0, 1), V1, V0, -1.0f, false, false, -1, seg_begin_[c.son[1]], seg_end_[c.son[0]] - 1);
    solve_upper(son(d, 0, 0), V0);
  }

  // ---------------------------------------------------------------- truncation
  void emit_trunc(const MV& X, const MV& Y, int32_t slot, int32_t cap,
                  const std::vector<PieceMV>& ps, bool alpha = false) {
    Task t = make(TK_TRUNC);
    t.a = X.v;
    t.b = Y.v;
    t.out_slot = slot;
    t.cap = cap;
    t.list_begin = (int32_t)S_->pieces.size();
    t.list_count = (int32_t)ps.size();
    int32_t W = 0;
    begin(t);
    for (const PieceMV& p : ps) {
      Piece q;
      std::memset(&q, 0, sizeof(q));
      q.X = p.p.X.v;
      q.Y = p.p.Y.v;
      q.xoff = p.xoff;
      q.yoff = p.yoff;
      q.sign = p.sign;
      q.pad = alpha ? PF_ALPHA : 0;
      grow4(S_->pieces);
      S_->pieces.push_back(q);
      acc(p.p.X, false);
      acc(p.p.Y, false);
      W += p.p.X.v.cols;
    }
    acc(X, true);
    acc(Y, true);
    end();
    L_.wmax = std::max(L_.wmax, W);
    L_.max_trunc_rows = std::max(L_.max_trunc_rows, std::max(X.v.rows, Y.v.rows));
  }
  LR trunc_new(int32_t rc, int32_t cc, const std::vector<PieceMV>& ps) {
    int32_t cap = std::min(kcap_, std::min(sz(rc), sz(cc)));
    int32_t slot = new_slot();
    LR r;
    r.X.clus = rc;
    int64_t xo = alloc((int64_t)sz(rc) * cap);
    r.X.buf = new_buf_leaves(rc);
    bind_alloc(r.X.buf);
    r.X.v = View{xo, 1, sz(rc), sz(rc), cap, slot, 0};
    r.Y.clus = cc;
    int64_t yo = alloc((int64_t)sz(cc) * cap);
    r.Y.buf = new_buf_leaves(cc);
    bind_alloc(r.Y.buf);
    r.Y.v = View{yo, 1, sz(cc), sz(cc), cap, slot, 0};
    emit_trunc(r.X, r.Y, slot, cap, ps);
    return r;
  }

  // ---------------------------------------------------------------- H-gemm
  LR product(int32_t a, int32_t b) {
    int32_t ka = kind(a), kb = kind(b);
    int32_t tau = rowc(a), sig = colc(a), rho = colc(b);
    if (ka == KIND_ADM) return LR{mvX(a), hmul_new(b, mvY(a), true)};
    if (kb == KIND_ADM) return LR{hmul_new(a, mvX(b), false), mvY(b)};
    if (ka == KIND_DENSE && kb == KIND_DENSE) {
      // exact factors of the narrowest width among |sigma|, |tau|, |rho|
      int32_t ws = sz(sig), wt = sz(tau), wr = sz(rho);
      if (ws <= kcap_ || (ws <= wt && ws <= wr)) return LR{mvD(a), mvDT(b)};
      MV P = new_dense_temp(tau, sz(rho));
      Task t = make(TK_DADD);
      t.flags = TF_OVERWRITE;
      t.c = P.v;
      t.a = mvD(a).v;
      t.b = mvDT(b).v;
      begin(t);
      acc(mvD(a), false);
      acc(mvDT(b), false);
      acc(P, true);
      end();
      if (wr <= wt) return LR{P, mvIdent(rho)};
      // P^T as the Y factor: rows rho, columns |tau|
      MV PT = P;
      PT.clus = rho;
      PT.v = View{P.v.off, sz(tau), 1, sz(rho), sz(tau), -1, 0};
      return LR{mvIdent(tau), PT};
    }
    if (ka == KIND_DENSE) return LR{mvIdent(tau), hmul_new(b, mvDT(a), true)};
    if (kb == KIND_DENSE) return LR{hmul_new(a, mvD(b), false), mvIdent(rho)};
    // both subdivided (formatted agglomeration)
    const Cluster& T = C_[tau];
    const Cluster& R = C_[rho];
    if (T.size <= kOneStepAgglomeration && R.size <= kOneStepAgglomeration) {
      // small target: the eight son products, placed at their son offsets,
      // are truncated in one task (the executor forms the dense sum)
      std::vector<PieceMV> ps;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int k = 0; k < 2; ++k) {
            LR sp = product(son(a, i, k), son(b, k, j));
            ps.push_back(PieceMV{sp, C_[T.son[i]].off - T.off, C_[R.son[j]].off - R.off, 1.0f});
          }
      return trunc_new(tau, rho, ps);
    }
    // larger target: the two son products of each quadrant are summed and
    // truncated (four independent tasks), then the four quadrants, placed at
    // their son offsets, are truncated together
    std::vector<PieceMV> quads;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        std::vector<PieceMV> ps;
        for (int k = 0; k < 2; ++k) ps.push_back(PieceMV{product(son(a, i, k), son(b, k, j)), 0, 0, 1.0f});
        LR q = trunc_new(T.son[i], R.son[j], ps);
        quads.push_back(PieceMV{q, C_[T.son[i]].off - T.off, C_[R.son[j]].off - R.off, 1.0f});
      }
    return trunc_new(tau, rho, quads);
  }

  // c <- c + sign * sum_p X_p Y_p^T in the format of c: one DADD per product
  // for a dense c, one truncation of all products for a low-rank c
  void add_multi(int32_t c, const std::vector<LR>& ps, float sign) {
    if (ps.empty()) return;
    for (const LR& p : ps)
      if (p.X.clus != rowc(c) || p.Y.clus != colc(c)) throw std::logic_error("add shape");
    int32_t k = kind(c);
    if (k == KIND_DENSE) {
      for (const LR& p : ps) {
        Task t = make(TK_DADD);
        t.c = mvD(c).v;
        t.a = p.X.v;
        t.b = p.Y.v;
        t.sign = sign;
        begin(t);
        acc(p.X, false);
        acc(p.Y, false);
        acc(mvD(c), true);
        end();
      }
    } else if (k == KIND_ADM) {
      std::vector<PieceMV> pieces;
      pieces.push_back(PieceMV{LR{mvX(c), mvY(c)}, 0, 0, 1.0f});
      for (const LR& p : ps) pieces.push_back(PieceMV{p, 0, 0, sign});
      emit_trunc(mvX(c), mvY(c), L_.slot[c], L_.cap[c], pieces);
    } else {
      const Cluster& R = C_[rowc(c)];
      const Cluster& Q = C_[colc(c)];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          std::vector<LR> sub_ps;
          for (const LR& p : ps) sub_ps.push_back(LR{sub(p.X, R.son[i]), sub(p.Y, Q.son[j])});
          add_multi(son(c, i, j), sub_ps, sign);
        }
    }
  }

  // c <- c + sign * a b in the format of c (formatted H-product: son
  // products where all three are subdivided, agglomeration otherwise); the
  // H-LU's Schur complement update is sign = -1
  void gemm(int32_t c, int32_t a, int32_t b, float sign = -1.0f) {
    if (kind(c) == KIND_SUB && kind(a) == KIND_SUB && kind(b) == KIND_SUB) {
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          // the two son products into c_ij that are not themselves subdivided
          // products are added together
          std::vector<LR> ps;
          for (int k = 0; k < 2; ++k) {
            int32_t cc = son(c, i, j), aa = son(a, i, k), bb = son(b, k, j);
            if (kind(cc) == KIND_SUB && kind(aa) == KIND_SUB && kind(bb) == KIND_SUB)
              gemm(cc, aa, bb, sign);
            else
              ps.push_back(product(aa, bb));
          }
          add_multi(son(c, i, j), ps, sign);
        }
      return;
    }
    add_multi(c, {product(a, b)}, sign);
  }

  // ---------------------------------------------------------------- whole H-matrices
  // dst <- sign * src (times the launch's alpha when `alpha`), leaf by leaf;
  // dst and src have the same block structure.  Dense leaves: one DADD of
  // src against the identity; admissible leaves: a truncation of the one
  // piece (exact: the rank does not change).
  void copy_scaled(int32_t dst, int32_t src, float sign, bool alpha) {
    if (kind(dst) == KIND_SUB) {
      for (int k = 0; k < 4; ++k) copy_scaled(B_[dst].son[k], B_[src].son[k], sign, alpha);
      return;
    }
    if (kind(dst) == KIND_DENSE) {
      // dense blocks have one side of at most the identity's size: D I or I D
      Task t = make(TK_DADD);
      t.flags = TF_OVERWRITE | (alpha ? TF_ALPHA : 0);
      t.sign = sign;
      t.c = mvD(dst).v;
      if (sz(colc(dst)) <= L_.ident_n) {
        t.a = mvD(src).v;
        t.b = mvIdent(colc(dst)).v;
      } else {
        t.a = mvIdent(rowc(dst)).v;
        t.b = mvDT(src).v;
      }
      begin(t);
      acc(mvD(src), false);
      acc(mvD(dst), true);
      end();
      return;
    }
    PieceMV p{LR{mvX(src), mvY(src)}, 0, 0, sign};
    std::vector<PieceMV> ps{p};
    emit_trunc(mvX(dst), mvY(dst), L_.slot[dst], L_.cap[dst], ps, alpha);
  }
  // dst <- 0: dense leaves overwritten with an empty product, admissible
  // leaves truncated from no pieces (rank 0)
  void zero(int32_t dst) {
    if (kind(dst) == KIND_SUB) {
      for (int k = 0; k < 4; ++k) zero(B_[dst].son[k]);
      return;
    }
    if (kind(dst) == KIND_DENSE) {
      Task t = make(TK_DADD);
      t.flags = TF_OVERWRITE;
      t.c = mvD(dst).v;
      t.a = mvD(dst).v;
      t.a.cols = 0;  // no columns: the product is zero
      t.b = mvDT(dst).v;
      t.b.cols = 0;
      begin(t);
      acc(mvD(dst), true);
      end();
      return;
    }
    emit_trunc(mvX(dst), mvY(dst), L_.slot[dst], L_.cap[dst], {});
  }
  // Vout <- H(b) Vin for a whole H-matrix b (its row cluster is the root)
  void apply(int32_t b, const MV& Vin, const MV& Vout) { hmul(b, Vin, Vout, 1.0f, false, true, Vout.v.slot); }

  // ---------------------------------------------------------------- H-trsm, H-LU
  void trsm_left(int32_t d, int32_t b) {
    int32_t k = kind(b);
    if (k == KIND_ADM) {
      solve_lower(d, mvX(b));
    } else if (k == KIND_DENSE) {
      solve_lower(d, mvD(b));
    } else {
      for (int j = 0; j < 2; ++j) {
        trsm_left(son(d, 0, 0), son(b, 0, j));
        gemm(son(b, 1, j), son(d, 1, 0), son(b, 0, j));
        trsm_left(son(d, 1, 1), son(b, 1, j));
      }
    }
  }
  void trsm_right(int32_t b, int32_t d) {
    int32_t k = kind(b);
    if (k == KIND_ADM) {
      solve_upperT(d, mvY(b));
    } else if (k == KIND_DENSE) {
      solve_upperT(d, mvDT(b));
    } else {
      for (int i = 0; i < 2; ++i) {
        trsm_right(son(b, i, 0), son(d, 0, 0));
        gemm(son(b, i, 1), son(b, i, 0), son(d, 0, 1));
        trsm_right(son(b, i, 1), son(d, 1, 1));
      }
    }
  }
  void lu(int32_t d) {
    if (kind(d) == KIND_DENSE) {
      getrf(d);
      return;
    }
    int32_t d00 = son(d, 0, 0), d01 = son(d, 0, 1), d10 = son(d, 1, 0), d11 = son(d, 1, 1);
    lu(d00);
    trsm_left(d00, d01);
    trsm_right(d10, d00);
    gemm(d11, d10, d01);
    lu(d11);
  }

  void solve_all(int32_t nrhs_max) {
    pending_.assign(seg_cluster_.size(), Pending());
    MV W;
    W.buf = new_buf_leaves(0);  // per-segment tracking over the whole vector
    W.clus = 0;
    int32_t N = sz(0);
    W.v = View{L_.work_off, 1, N, N, nrhs_max, L_.nrhs_slot, 0};
    solve_lower(0, W);
    solve_upper(0, W);
  }

 private:
  const std::vector<Cluster>& C_;
  const std::vector<Block>& B_;
  int32_t kcap_;
  ArenaLayout& L_;
  Schedule* S_;
  std::vector<int32_t>& dbuf_;
  std::vector<int32_t>& xbuf_;
  std::vector<int32_t>& ybuf_;
  int32_t seg_size_of(int32_t) const { return segsz_; }
  int32_t segsz_ = 0;
  int64_t ring_off_ = 0, ring_size_ = 0, cursor_ = 0;
  std::vector<int32_t> seg_begin_, seg_end_, seg_cluster_;
  std::vector<std::vector<int32_t>> chunk_occ_;
  std::vector<int32_t> chunk_fence_task_;
  std::vector<int32_t> chunk_pass_;
  int32_t pass_ = 0;
 public:
  int64_t wraps_ = 0;
 private:
  std::vector<int32_t> pending_fence_;
  int64_t last_alloc_lo_ = 0, last_alloc_hi_ = -1;
  int32_t fence_stamp_ = 0;
  std::vector<int32_t> buf_fence_mark_;
  std::vector<int64_t> fence_begin_, fence_end_;
  std::vector<int32_t> fence_pool_;
  std::vector<int64_t> acc_head_;
  std::vector<int32_t> acc_last_;
  std::vector<int32_t> acc_task_;
  std::vector<int64_t> acc_next_;
  std::vector<int32_t> seg_buf_;
  std::vector<Buf> bufs_;
  std::vector<int32_t> seg_writer_;
  std::vector<int64_t> seg_rhead_;
  std::vector<int32_t> rtask_;
  std::vector<int64_t> rnext_;
  std::vector<int32_t> stamp_;
  std::vector<int32_t> deps_;
  int32_t cur_ = -1;
  // late updates waiting to be merged into a segment's leaf solve
  struct Pending {
    bool active = false;
    std::vector<int32_t> lv, list;
    std::vector<MV> T;
    MV Vin;
    float sign = 0;
    bool trans = false;
  };
  std::vector<Pending> pending_;
};

}  // namespace

std::vector<Block> factor_tree(const std::vector<Cluster>& C, const std::vector<Block>& B, int32_t tile) {
  std::vector<Block> out;
  out.reserve(B.size());
  // DFS over the block tree; a node whose row and column clusters both hold at
  // most `tile` DOFs becomes one dense tile (its sub-blocks merged exactly)
  struct Rec {
    static int32_t go(const std::vector<Cluster>& C, const std::vector<Block>& B, int32_t tile, int32_t b,
                      int32_t parent, std::vector<Block>& out) {
      const Block& src = B[b];
      int32_t id = (int32_t)out.size();
      out.push_back(src);
      Block& nb = out.back();
      nb.parent = parent;
      for (int k = 0; k < 4; ++k) nb.son[k] = -1;
      int32_t big = std::max(C[src.row].size, C[src.col].size);
      int32_t small = std::min(C[src.row].size, C[src.col].size);
      // a subdivided node turns dense as soon as one of its clusters is a tile,
      // so a dense diagonal tile never meets a subdivided block in its block
      // row or column; an admissible node turns dense when both clusters are
      if ((src.kind == KIND_SUB && small <= tile) || (src.kind == KIND_ADM && big <= tile)) {
        out[id].kind = KIND_DENSE;
        return id;
      }
      if (src.kind == KIND_SUB) {
        int32_t sons[4];
        for (int k = 0; k < 4; ++k) sons[k] = go(C, B, tile, src.son[k], id, out);
        for (int k = 0; k < 4; ++k) out[id].son[k] = sons[k];
      }
      return id;
    }
  };
  Rec::go(C, B, tile, 0, -1, out);
  return out;
}

void build_schedules(const std::vector<Cluster>& C, const std::vector<Block>& Bfull, int32_t rank_cap,
                     int32_t nrhs_max, int32_t tile, ArenaLayout& L,
                     Schedule& factor, Schedule& solve,
                     SchedStats& st, std::vector<Block>* factor_blocks) {
  std::vector<Block> Bt = factor_tree(C, Bfull, tile);
  const std::vector<Block>& B = Bt;
  if (factor_blocks) *factor_blocks = Bt;
  auto t0 = std::chrono::steady_clock::now();
  const size_t nb = B.size();
  L = ArenaLayout();
  L.dense_off.assign(nb, -1);
  L.x_off.assign(nb, -1);
  L.y_off.assign(nb, -1);
  L.cap.assign(nb, 0);
  L.slot.assign(nb, -1);
  L.piv_off.assign(nb, -1);
  int32_t leafmax = 0;
  for (const Cluster& c : C)
    if (c.son[0] < 0) leafmax = std::max(leafmax, c.size);
  auto alloc = [&](int64_t n) {
    int64_t o = L.total;
    L.total += (n + 31) & ~int64_t(31);
    return o;
  };
  L.ident_n = std::max(std::max(leafmax, tile), 1);
  L.ident_off = alloc((int64_t)L.ident_n * L.ident_n);
  int64_t fe = 0;
  for (size_t b = 0; b < nb; ++b) {
    int32_t m = C[B[b].row].size, n = C[B[b].col].size;
    if (B[b].kind == KIND_DENSE) {
      L.dense_off[b] = alloc((int64_t)m * n);
      fe += (int64_t)m * n;
      if (B[b].row == B[b].col) {
        L.piv_off[b] = L.piv_total;
        L.piv_total += m;
      }
    } else if (B[b].kind == KIND_ADM) {
      int32_t cap = std::min(rank_cap, std::min(m, n));
      L.cap[b] = cap;
      L.slot[b] = L.n_slots++;
      L.x_off[b] = alloc((int64_t)m * cap);
      L.y_off[b] = alloc((int64_t)n * cap);
      fe += (int64_t)(m + n) * cap;
    }
  }
  L.factor_elems = fe;
  L.nrhs_max = nrhs_max;
  L.nrhs_slot = L.n_slots++;
  L.work_off = alloc((int64_t)C[0].size * nrhs_max);
  L.wmax = 0;
  // ring region for temporaries (both schedules; they never run concurrently).
  // Every wrap of the ring orders the new occupants of a chunk after all
  // users of its previous ones (FENCE tasks); at rank capacity 64 the
  // temporaries are twice those of capacity 32, and a 2^31-element bound
  // keeps the number of wraps (and fences) of the larger workloads at what a
  // 2^30 bound gave at capacity 32.
  const int64_t ring = std::min<int64_t>(std::max<int64_t>(8 * fe, int64_t(1) << 22), int64_t(1) << 31);
  const int64_t ring_off = alloc(ring);
  L.ring_off = ring_off;
  L.ring_size = ring;
  const int32_t segsz = std::max(leafmax, tile);
  factor = Schedule();
  solve = Schedule();
  std::vector<int32_t> dbuf, xbuf, ybuf;
  {
    Sched s(C, B, rank_cap, L, &factor, dbuf, xbuf, ybuf, true, segsz, ring_off, ring);
    s.lu(0);
    st.temp_elems = s.temp_elems_;
    st.ring_wraps = s.wraps_;
  }
  {
    Sched s(C, B, rank_cap, L, &solve, dbuf, xbuf, ybuf, true, segsz, ring_off, ring);
    s.solve_all(nrhs_max);
    st.temp_elems += s.temp_elems_;
  }
  factor.n_edges = (int64_t)factor.pred_idx.size();
  solve.n_edges = (int64_t)solve.pred_idx.size();
  st.n_factor_tasks = (int64_t)factor.tasks.size();
  st.n_solve_tasks = (int64_t)solve.tasks.size();
  st.host_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void build_inverse_schedules(const std::vector<Cluster>& C, const std::vector<Block>& FB, int32_t rank_cap,
                             int32_t nrhs_max, int32_t tile, ArenaLayout& L, std::vector<Block>& Bx,
                             Schedule& start, Schedule& iter, Schedule& apply, SchedStats& st) {
  auto t0 = std::chrono::steady_clock::now();
  const int32_t nb = (int32_t)FB.size();
  Bx.assign((size_t)4 * nb, Block());
  for (int32_t q = 0; q < 4; ++q)
    for (int32_t b = 0; b < nb; ++b) {
      Block k = FB[b];
      for (int s = 0; s < 4; ++s)
        if (k.son[s] >= 0) k.son[s] += q * nb;
      if (k.parent >= 0) k.parent += q * nb;
      Bx[(size_t)q * nb + b] = k;
    }
  const size_t nx = Bx.size();
  L = ArenaLayout();
  L.dense_off.assign(nx, -1);
  L.x_off.assign(nx, -1);
  L.y_off.assign(nx, -1);
  L.cap.assign(nx, 0);
  L.slot.assign(nx, -1);
  L.piv_off.assign(nx, -1);
  int32_t leafmax = 0;
  for (const Cluster& c : C)
    if (c.son[0] < 0) leafmax = std::max(leafmax, c.size);
  auto alloc = [&](int64_t n) {
    int64_t o = L.total;
    L.total += (n + 31) & ~int64_t(31);
    return o;
  };
  L.ident_n = std::max(std::max(leafmax, tile), 1);
  L.ident_off = alloc((int64_t)L.ident_n * L.ident_n);
  int64_t fe = 0;
  for (size_t b = 0; b < nx; ++b) {
    const int32_t m = C[Bx[b].row].size, n = C[Bx[b].col].size;
    if (Bx[b].kind == KIND_DENSE) {
      L.dense_off[b] = alloc((int64_t)m * n);
      fe += (int64_t)m * n;
    } else if (Bx[b].kind == KIND_ADM) {
      const int32_t cap = std::min(rank_cap, std::min(m, n));
      L.cap[b] = cap;
      L.slot[b] = L.n_slots++;
      L.x_off[b] = alloc((int64_t)m * cap);
      L.y_off[b] = alloc((int64_t)n * cap);
      fe += (int64_t)(m + n) * cap;
    }
  }
  L.factor_elems = fe;
  L.nrhs_max = nrhs_max;
  L.nrhs_slot = L.n_slots++;
  L.work_off = alloc((int64_t)C[0].size * nrhs_max);
  L.out_off = alloc((int64_t)C[0].size * nrhs_max);
  const int64_t ring = std::min<int64_t>(std::max<int64_t>(8 * fe, int64_t(1) << 22), int64_t(1) << 31);
  L.ring_off = alloc(ring);
  L.ring_size = ring;
  const int32_t segsz = std::max(leafmax, tile);
  start = Schedule();
  iter = Schedule();
  apply = Schedule();
  std::vector<int32_t> dbuf, xbuf, ybuf;
  const int32_t A0 = 0, X0 = nb, T0 = 2 * nb, Y0 = 3 * nb;
  {
    Sched s(C, Bx, rank_cap, L, &start, dbuf, xbuf, ybuf, true, segsz, L.ring_off, ring);
    s.copy_scaled(X0, A0, 1.0f, true);
  }
  {
    Sched s(C, Bx, rank_cap, L, &iter, dbuf, xbuf, ybuf, true, segsz, L.ring_off, ring);
    s.zero(T0);
    s.gemm(T0, A0, X0, -1.0f);  // T = -A X
    s.copy_scaled(Y0, X0, 2.0f, false);
    s.gemm(Y0, X0, T0, 1.0f);   // Y = 2 X - X A X
    s.copy_scaled(X0, Y0, 1.0f, false);
    st.temp_elems = s.temp_elems_;
    st.ring_wraps = s.wraps_;
  }
  {
    Sched s(C, Bx, rank_cap, L, &apply, dbuf, xbuf, ybuf, true, segsz, L.ring_off, ring);
    const int32_t N = C[0].size;
    MV Win, Wout;
    Win.buf = -1;  // read-only here
    Win.clus = 0;
    Win.v = View{L.work_off, 1, N, N, nrhs_max, L.nrhs_slot, 0};
    Wout.buf = s.new_buf_leaves(0);
    Wout.clus = 0;
    Wout.v = View{L.out_off, 1, N, N, nrhs_max, L.nrhs_slot, 0};
    s.apply(X0, Win, Wout);
  }
  for (Schedule* sc : {&start, &iter, &apply}) sc->n_edges = (int64_t)sc->pred_idx.size();
  st.n_factor_tasks = (int64_t)iter.tasks.size();
  st.n_solve_tasks = (int64_t)apply.tasks.size();
  st.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace hlu
