// Internal data structures shared by the host task scheduler and the device
// task executor.  Everything here is plain old data: it is built on the host,
// copied to the device once per block tree, and interpreted by the persistent
// executor kernel (exec.cu).
#pragma once
#include <cstdint>
#include <vector>

namespace hlu {

// ---- trees (host copies, DFS pre-order ids) ---------------------------------
struct Cluster {
  int32_t off, size, lo[3], hi[3], son[2], level, parent;
  int32_t leaf_begin, leaf_end;  // range of leaf clusters covered (leaf order)
};
struct Block {
  int32_t row, col, kind, son[4], parent;
};
enum { KIND_ADM = 0, KIND_DENSE = 1, KIND_SUB = 2 };

// Largest (and default) rank capacity of an admissible block.
constexpr int32_t kRankMax = 64;

// ---- strided matrix view into a problem's arena ----------------------------
// Element (i, j) lives at arena[off + i*rs + j*cs].  The column count is `cols`
// when slot < 0, otherwise ranks[slot] read on the device at execution time.
struct View {
  int64_t off;
  int32_t rs, cs;
  int32_t rows;
  int32_t cols;
  int32_t slot;
  int32_t pad;
};

// ---- task kinds of the H-LU / H-solve DAG -----------------------------------
enum TaskType : int32_t {
  TK_GETRF = 0,   // a: dense diagonal leaf (n x n) in place, partial pivoting
  TK_TRSM_L = 1,  // b <- L_a^-1 P_a b   (a: factored leaf, b: n x k view)
  TK_TRSM_UT = 2, // b <- U_a^-T b
  TK_TRSM_U = 3,  // b <- U_a^-1 b
  TK_PROJ = 4,    // c (r x k) <- a^T b  (a: m x r, b: m x k)
  TK_ROWMV = 5,   // c (n x k) <- [c] + sign * sum_terms A_t B_t
  TK_TRUNC = 6,   // (a, b) <- truncate(sum_pieces sign X Y^T) to eps, rank -> out_slot
  TK_DADD = 7,    // c (m x n) <- [c] + sign * a b^T  (a: m x k, b: n x k)
  TK_RSOLVE = 8,  // c <- tri(a)^-1 (c - sum_terms A_t B_t): one tile of a triangular solve;
                  // flags & TF_UPPER: U^-1, else L^-1 P (pivots at piv_off)
  TK_NUM = 9,
  TK_FENCE = 9    // no work: orders re-use of temporary memory after its readers
};
// TF_ALPHA (DADD) and PF_ALPHA (a TRUNC piece): the sign is multiplied by the
// launch's scalar alpha (the Schulz start X_0 = alpha A)
enum : int32_t { TF_OVERWRITE = 1, TF_UPPER = 2, TF_ALPHA = 4 };
enum : int32_t { PF_ALPHA = 1 };

struct Task {
  int32_t type;
  int32_t flags;
  int32_t list_begin, list_count;  // ROWMV / RSOLVE terms or TRUNC pieces
  View a, b, c;
  int64_t piv_off;   // pivot vector offset (int32 elements) for leaf tasks
  int32_t out_slot;  // rank slot written by the task (-1: none)
  int32_t cap;       // TRUNC: rank capacity of the target
  float sign;
  int32_t prob;      // problem index (batched launches)
};

// ROWMV term: A (A.rows x p) times B (p x k) added to output rows
// [roff, roff + A.rows); p = A's column count.
struct Term {
  View A, B;
  int32_t roff;
  int32_t pad;
};
// TRUNC piece: sign * X Y^T placed at rows [xoff, xoff + X.rows) of the target
// and columns [yoff, yoff + Y.rows); pad holds PF_ flags.
struct Piece {
  View X, Y;
  int32_t xoff, yoff;
  float sign;
  int32_t pad;
};

// ---- a complete schedule -----------------------------------------------------
struct Schedule {
  std::vector<Task> tasks;
  std::vector<Term> terms;
  std::vector<Piece> pieces;
  std::vector<int64_t> pred_ptr;  // CSR of predecessors (all with smaller index)
  std::vector<int32_t> pred_idx;
  int64_t n_edges = 0;
};

// Layout of one problem's factor arena (element offsets).
struct ArenaLayout {
  int64_t total = 0;       // elements
  int64_t ident_off = 0;   // identity matrix (ident_n x ident_n, column-major)
  int32_t ident_n = 0;
  int64_t work_off = 0;    // H-solve work vector (N x nrhs_max, column-major)
  int32_t nrhs_max = 0;
  int32_t nrhs_slot = -1;  // rank slot holding the current nrhs of a solve
  std::vector<int64_t> dense_off;  // per block (-1 if not dense)
  std::vector<int64_t> x_off, y_off;  // per block (-1 if not admissible)
  std::vector<int32_t> cap;        // per block rank capacity
  std::vector<int32_t> slot;       // per block rank slot (-1 if not admissible)
  std::vector<int64_t> piv_off;    // per block pivot offset (diagonal dense leaves)
  int64_t piv_total = 0;
  int32_t n_slots = 0;
  int64_t factor_elems = 0;        // dense + low-rank capacity elements
  int32_t max_trunc_rows = 0;      // largest TRUNC target dimension
  int32_t wmax = 0;                // largest stacked width of a TRUNC
  int64_t ring_off = 0, ring_size = 0;  // region for temporaries
  int64_t out_off = -1;            // H-matrix apply: output vector (N x nrhs_max), -1 if none
};

struct SchedStats {
  int64_t n_factor_tasks = 0, n_solve_tasks = 0;
  int64_t temp_elems = 0;
  int64_t ring_wraps = 0;
  double host_ms = 0;
};

// Build the factorisation schedule and the triangular-solve schedule for the
// given trees.  Fills the arena layout (factor storage, temporaries, work
// vector).  rank_cap: capacity of admissible blocks.
// `tile`: every block-tree node whose row and column clusters both hold at most
// `tile` DOFs is factored as one dense tile (tile <= leaf keeps the block tree
// as it is).  factor_blocks (optional) receives the factor tree the schedules
// and the arena layout refer to.
void build_schedules(const std::vector<Cluster>& C, const std::vector<Block>& B, int32_t rank_cap,
                     int32_t nrhs_max, int32_t tile, ArenaLayout& L,
                     Schedule& factor, Schedule& solve, SchedStats& st, std::vector<Block>* factor_blocks);
std::vector<Block> factor_tree(const std::vector<Cluster>& C, const std::vector<Block>& B, int32_t tile);

// The Schulz iteration for the inverse of A_H (Sec. 3, Sec. 4) over four
// copies of the factor tree FB in one arena: copy 0 holds A_H, 1 the iterate
// X, 2 the product T, 3 the next iterate Y (block b of copy q is block
// q * |FB| + b of Bx).  start: X <- alpha A_H (alpha from the launch);
// iter: T <- -A_H X, Y <- 2 X, Y <- Y + X T, X <- Y (formatted H-products
// truncated to eps); apply: out <- X in for nrhs_max columns (work_off ->
// out_off).
void build_inverse_schedules(const std::vector<Cluster>& C, const std::vector<Block>& FB, int32_t rank_cap,
                             int32_t nrhs_max, int32_t tile, ArenaLayout& L, std::vector<Block>& Bx,
                             Schedule& start, Schedule& iter, Schedule& apply, SchedStats& st);

}  // namespace hlu
