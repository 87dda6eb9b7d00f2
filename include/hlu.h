/*
 * hlu.h - C ABI of the GB300 H-LU preconditioned Maxwell solver.
 *
 * Method: Parvizi, Khodadadian, Beuchler, Wick, "Hierarchical LU
 * preconditioning for the time-harmonic Maxwell equations" (arXiv 2211.11303).
 * The library assembles the lowest-order Nedelec edge-element matrix of
 * curl curl E - kappa^2 E = J with E x n = 0 (Sec. 2, Eq. 4-7), builds the
 * geometric cluster tree and the eta-admissible block tree (Sec. 3, Sec. 4),
 * computes the H-matrix approximation A_H and its H-LU factorisation
 * (Algorithm 1, steps I-II) on the GPU, and applies U^-1 L^-1 inside
 * restarted flexible GMRES (Sec. 4, Example 1) or the Richardson loop
 * (Algorithm 1, steps III-IV).
 *
 * Conventions shared by every call:
 *  - Status: every call returns an int status, HLU_OK (0) on success.  No
 *    exception or longjmp crosses the ABI.  hlu_status_string() names a code;
 *    hlu_last_error() returns a thread-local message for the last failure.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Device-pointer arguments are read/written in stream
 *    order; calls documented as "synchronous" return after the stream has
 *    drained.
 *  - Memory: the library allocates the device memory of the handle's
 *    matrices, trees, factors, workspaces and build temporaries through the
 *    allocator set by hlu_set_allocator() (default cudaMalloc/cudaFree) and
 *    frees it in hlu_destroy() (temporaries before the call returns).
 *    Vectors passed in are caller-owned.
 *  - Vectors: column-major, `nrhs` columns of length N with leading
 *    dimension `ld` >= N, FP64, in the original interior-edge DOF order.
 *  - DOF order: interior edges (lo, hi) of the Kuhn mesh sorted by (lo, hi),
 *    vertex id (i (n+1) + j)(n+1) + k; an edge is oriented lo -> hi.
 */
#ifndef HLU_H
#define HLU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HLU_OK 0
#define HLU_ERR_ARG 1           /* invalid argument (NULL, size, range)        */
#define HLU_ERR_OOM 2           /* device or host allocation failed            */
#define HLU_ERR_ZERO_PIVOT 3    /* exact zero pivot inside a diagonal leaf     */
#define HLU_ERR_NOT_CONVERGED 4 /* Krylov iteration hit maxit; x still written  */
#define HLU_ERR_TIMEOUT 5       /* a bounded device-side wait gave up          */
#define HLU_ERR_CUDA 6          /* a CUDA runtime call failed                  */
#define HLU_ERR_STATE 7         /* call out of order (e.g. solve before factor)*/

/* ---- precisions of the factor ------------------------------------------ */
#define HLU_FP64 0 /* factor and triangular solves in FP64 ("plain" path) */
#define HLU_FP32 1 /* factor and triangular solves in FP32, FP32 accumulate */
#define HLU_TF32 2 /* FP32 factor whose tile products (dense and low-rank GEMM
                      contractions: projections, H x multivector updates, dense
                      updates, dense-route sums) run as TF32 MMAs on the tensor
                      cores (tcgen05, FP32 accumulation in tensor memory), each
                      operand split into a TF32 part and the TF32 rounding of
                      its remainder so that the products keep FP32 accuracy;
                      LU, QR, SVD and the triangular solves in FP32 */

/* ---- preconditioners of gmres_solve / hlu_richardson ------------------- */
#define HLU_PRECOND_LU 0   /* (LU)_H^-1 of hlu_factor (Alg. 1 step III), the default */
#define HLU_PRECOND_HINV 1 /* B_H ~ A_H^-1 of hlu_hinverse (Sec. 3: Schulz iteration) */

/* ---- block kinds in the exported block tree ------------------------------ */
#define HLU_BLOCK_ADM 0   /* admissible: low-rank X Y^T (Definition 1)       */
#define HLU_BLOCK_DENSE 1 /* inadmissible with a leaf cluster: dense         */
#define HLU_BLOCK_SUB 2   /* subdivided into four sons                       */

typedef struct hlu_handle hlu_handle;

/* Mesh: a conforming tetrahedral mesh of the domain (Sec. 2.1), given as
 * nv vertex coordinates xyz (double[nv * 3], host) and nt tetrahedra tets
 * (int32[nt * 4] vertex ids, host), or, with lattice_n > 0, the unit cube cut
 * into lattice_n^3 sub-cubes, each split into the 6 Kuhn tetrahedra along
 * the axis permutations (Sec. 4, Example 1: the cube cut into 6 tetrahedra
 * and refined); lattice_n > 0 takes precedence (xyz and tets may then be
 * NULL; hlu_mesh_kuhn_cube fills them for inspection).
 * General meshes: a face that belongs to one tetrahedron is a boundary face;
 * edges on boundary faces carry E x n = 0 and are eliminated; the remaining
 * (interior) edges, oriented from the lower to the higher vertex id, are the
 * DOFs in increasing (lo, hi) order.  The cluster tree's points are the edge
 * midpoints on an integer grid, p = rint((x_lo + x_hi - 2 b) s), b the lower
 * corner of the vertices' bounding box and s the largest power of two with
 * 2 extent s <= 2^21.  beta (may be NULL: beta = 1 everywhere): the
 * material coefficient of the curl-curl term (Sec. 2: the operator
 * curl(beta^-1 curl E) - kappa E), one positive value per tetrahedron, in the
 * order of tets (for lattice_n > 0: in the order hlu_mesh_kuhn_cube lists
 * them); Example 3's magnet is beta = 10 inside, 1 in the air.  The caller
 * keeps xyz, tets and beta; hlu_build copies them. */
typedef struct {
  int32_t nv, nt;
  const double* xyz;
  const int32_t* tets;
  int32_t lattice_n;
  const double* beta;
} hlu_mesh;

/* hlu_mesh_kuhn_cube - the Kuhn cube with n^3 sub-cubes as a mesh: vertex
 * id (i (n+1) + j)(n+1) + k at (i, j, k) / n, tetrahedron 6 c + p of sub-cube
 * c = (c0 n + c1) n + c2 with corners c, c + e_p0, c + e_p0 + e_p1, c + (1,1,1)
 * for the axis permutations p in lexicographic order; lattice_n = n.  The
 * arrays are allocated by the library (host memory) and released by
 * hlu_mesh_free.  HLU_ERR_ARG for n outside [1, 200]; HLU_ERR_OOM. */
int hlu_mesh_kuhn_cube(int32_t n, hlu_mesh* out);
void hlu_mesh_free(hlu_mesh* m);

/* Per-solve statistics (host struct filled by gmres_solve / hlu_richardson;
 * valid when the call returns). */
typedef struct {
  int32_t iterations;      /* inner Krylov steps (max over columns)             */
  int32_t restarts;        /* restart cycles (max over columns)                 */
  int32_t converged;       /* 1 if every column met tol                         */
  int32_t nrhs;            /* columns solved                                    */
  double relres_max;       /* max over columns of ||b - A x|| / ||b|| at exit    */
  double abs_res_max;      /* max over columns of ||A x - b||_2 (Alg. 1 step IV) */
  double precond_ms;       /* device time in preconditioner applications        */
  double total_ms;         /* wall time of the call                             */
  int32_t precond_applies; /* number of U^-1 L^-1 applications                  */
  int32_t reserved;
} hlu_stats;

/* Factor statistics (hlu_factor_stats). */
typedef struct {
  int64_t n_tasks;          /* tasks in the factorisation DAG                    */
  int64_t n_solve_tasks;    /* tasks in one triangular-solve pass (L then U)     */
  int64_t factor_bytes;     /* device bytes of dense + low-rank factor storage   */
  int64_t workspace_bytes;  /* device bytes of temporaries and scratch           */
  double flops;             /* algorithmic flops of the factorisation (counted)  */
  double factor_ms;         /* device time of the last hlu_factor                */
  double schedule_ms;       /* host time spent building the task DAG             */
  int32_t rank_max;         /* max rank of an admissible block after factoring   */
  int32_t rank_cap_hits;    /* truncations clipped at the rank capacity          */
  double rank_mean;         /* mean rank over admissible blocks                  */
  int32_t n_clusters, n_blocks, n_adm, n_dense;
  int32_t rank_wanted_max;  /* largest rank a truncation asked for (s_i > eps s_1);
                               rank capacity + 1 when it asked for more          */
  int32_t trunc_dense_fallbacks; /* dense-route truncations redone by the stack route */
  int64_t factor_live_bytes; /* bytes of the factor at its live ranks: dense words plus
                                (rows + cols) x rank per admissible block; what one
                                triangular-solve pass (L then U) reads            */
  int32_t grid_ctas;        /* CTAs of the factorisation launch (persistent)       */
  int32_t reserved_;
} hlu_factor_info;

/* hlu_build - Algorithm 1 step I and the structures it needs.
 * Builds, on the GPU: the mesh's interior-edge numbering (Sec. 2.1: one DOF
 * per interior edge, sigma(Phi_i, e_j) = delta_ij), the CSR matrix
 * A = K - kappa^2 M of a(E, Phi) = <beta^-1 curl E, curl Phi> - kappa^2 <E, Phi>
 * (Sec. 2.1 weak form, with the mesh's beta; the paper's kappa is kappa^2
 * here), the geometric
 * cluster tree on the edge midpoints (doubled lattice coordinates on the Kuhn
 * cube, the integer grid of hlu_mesh otherwise; Sec. 4, geometrically balanced
 * bisection, leaf size `leaf`), the block tree with admissibility
 * min(diam tau, diam sigma) <= eta dist(tau, sigma) (Sec. 3-4, eta = 2 in the
 * paper; eta^2 must be an integer), and the exact A_H (dense leaves from A,
 * admissible blocks as X Y^T of their nonzero rows).
 * kappa: wave number (> 0).  eps: relative truncation tolerance used by
 * hlu_factor (Sec. 4 truncated SVD; keep s_i > eps s_1).  rank_cap: maximum
 * stored rank of an admissible block (0 = the default and largest value,
 * 64); a truncation that asks for more keeps the first rank_cap singular
 * triplets and counts a rank-capacity hit (hlu_factor_info).
 * The build is synchronous (trees are copied to the host for scheduling).
 * Errors: HLU_ERR_ARG for lattice_n outside [0, 200], a general mesh with
 * fewer than 4 vertices, no tetrahedra, 2^21 or more vertices, a vertex id
 * out of range, a repeated vertex in a tetrahedron or a non-finite
 * coordinate, a beta value that is not finite and positive, leaf < 2,
 * eta <= 0 or non-integer eta^2, eps <= 0; HLU_ERR_OOM; HLU_ERR_CUDA. */
int hlu_build(const hlu_mesh* mesh, double kappa, int32_t leaf, double eta, double eps,
              int32_t rank_cap, void* stream, hlu_handle** out);

/* hlu_set_schedule_cache - size of the process-wide cache of task DAGs
 * (default 16 schedules, 24 GiB of device memory): hlu_build reuses the
 * DAGs of an identical block tree, so a server that keeps its mesh catalogue
 * cached builds a new mesh's DAG on the host once.  The least recently used
 * schedule beyond either bound is dropped (handles holding it keep it).
 * HLU_ERR_ARG for entries < 1 or bytes < 0. */
int hlu_set_schedule_cache(int32_t entries, int64_t bytes);

/* Number of interior-edge DOFs N of a built handle (0 for NULL). */
int64_t hlu_n(const hlu_handle* h);

/* hlu_export_trees - copy the trees to caller host buffers (Sec. 3-4).
 * perm: int32[N], perm[i] = original DOF at permuted position i.
 * clusters: int32[nc*12] rows (offset, size, lo[3], hi[3], son0, son1, level,
 *   parent), ids in DFS pre-order, boxes in doubled lattice units.
 * blocks: int32[nb*8] rows (row cluster, col cluster, kind, son0..son3,
 *   parent), DFS pre-order.
 * sizes: int64[2] receives (nc, nb); any array pointer may be NULL to query
 * sizes only.  Synchronous.  HLU_ERR_ARG on NULL handle/sizes. */
int hlu_export_trees(const hlu_handle* h, int32_t* perm, int32_t* clusters, int32_t* blocks,
                     int64_t* sizes);

/* hlu_export_csr - copy the assembled CSR matrix A (Sec. 2.1,
 * stiffness-matrix equation) to host buffers: rowptr int64[N+1], col
 * int32[nnz], val double[nnz]; columns ascending within a row, every pair of
 * interior edges sharing a tetrahedron present (explicit zeros kept).
 * nnz: int64 out, may be queried with NULL arrays.  Synchronous. */
int hlu_export_csr(const hlu_handle* h, int64_t* rowptr, int32_t* col, double* val, int64_t* nnz);

/* hlu_rhs_manufactured - load vector b_j = <J, Phi_j> (Sec. 2.1) for the
 * manufactured field E = (sin pi y sin pi z, sin pi z sin pi x, sin pi x sin pi y),
 * J = (2 pi^2 - kappa^2) E, by a 4-point degree-2 rule.  b_dev: device
 * double[N].  Synchronous: its element-contribution scratch comes from the
 * library's allocator and is freed before the call returns. */
int hlu_rhs_manufactured(const hlu_handle* h, double* b_dev, void* stream);

/* hlu_rhs_constant_current - load vector b_j = <J_S, Phi_j> (Sec. 2.1) of a
 * constant current density J_S = (jx, jy, jz); Sec. 4, Example 1 uses
 * J_S = [0, 0, 1]^T.  The basis functions are linear on each tetrahedron, so
 * the integral is exact: b_e = |T|/4 J_S . (grad lam_b - grad lam_a) summed
 * over the tetrahedra of edge e = (a, b).  b_dev: device double[N].
 * Synchronous (scratch from the library's allocator).  HLU_ERR_ARG for a
 * non-finite J_S. */
int hlu_rhs_constant_current(const hlu_handle* h, double jx, double jy, double jz, double* b_dev, void* stream);

/* hlu_rhs_manufactured_noalloc - the same load vector as hlu_rhs_manufactured,
 * computed without allocating any memory.  The paper has no counterpart: this
 * entry serves callers that must not allocate, such as a serving loop that
 * admits work against a fixed HBM budget (an allocation behind its back can
 * push the device over the budget or fail under memory pressure) and
 * latency-critical loops (cudaMalloc synchronises the device).
 * hlu_rhs_manufactured allocates its element-contribution scratch and the
 * sort's temporaries on every call; this variant keeps the 6 contributions
 * per tetrahedron in a fixed device array of 524,288 entries (6 MiB) and
 * adds them into b with atomics, so the result equals hlu_rhs_manufactured's
 * up to the order of the floating-point additions (relative differences of
 * order 1e-16 per entry).  Limit: 36 n^3 <= 524,288, i.e. Kuhn meshes with
 * n <= 24; larger meshes return HLU_ERR_ARG with a message and write nothing.
 * Nothing needs to start at zero: every scratch entry is written before it is
 * read, and b_dev is cleared by the call.  The first call on each device looks
 * up the scratch's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The scratch is
 * shared by all calls on a device: calls that overlap in time (other streams
 * or host threads) race on it and must be serialised by the caller.
 * b_dev: device double[N].  Asynchronous on stream. */
int hlu_rhs_manufactured_noalloc(const hlu_handle* h, double* b_dev, void* stream);

/* hlu_spmv - y = A x for nrhs columns (FP64 CSR), device pointers, ld >= N.
 * Asynchronous.  Used by the Krylov solvers and exposed for tests. */
int hlu_spmv(const hlu_handle* h, const double* x_dev, double* y_dev, int32_t nrhs, int64_t ld,
             void* stream);

/* hlu_factor - Algorithm 1 step II: H-LU of A_H in H-arithmetic.
 * Recursive block LU (LU(A11); A12 <- L11^-1 P A12; A21 <- A21 U11^-1;
 * A22 <- A22 - A21 A12 truncated to eps; LU(A22)), partial pivoting inside
 * dense diagonal leaves only.  precision: HLU_FP64 or HLU_FP32.  May be
 * called again (e.g. with another precision): A_H is re-filled first.
 * Synchronous (returns after the device finished; factor_ms recorded).
 * Errors: HLU_ERR_ZERO_PIVOT (factor unusable), HLU_ERR_TIMEOUT, HLU_ERR_OOM. */
int hlu_factor(hlu_handle* h, int32_t precision, void* stream);

/* hlu_factor_async - hlu_factor without waiting for the device: the A_H
 * fill runs (the call returns after it, with its status), then the
 * factorisation is queued on `stream` and the call returns.  max_ctas > 0
 * caps the persistent launch at that many CTAs (0: the full grid), which
 * leaves SM slots for other work on other streams: a server factors a newly
 * admitted request's matrix while the running requests' GMRES steps go on
 * (Alg. 1 step II beside step III of other problems).  Until
 * hlu_factor_wait reports it done, the handle's solves return HLU_ERR_STATE
 * and a second factorisation is refused.  Same errors as hlu_factor, the
 * device-side ones (zero pivot, timeout) from hlu_factor_wait. */
int hlu_factor_async(hlu_handle* h, int32_t precision, int32_t max_ctas, void* stream);

/* hlu_factor_wait - completion of hlu_factor_async: *done = 1 once the
 * factorisation finished (statistics filled, status returned as hlu_factor
 * would), *done = 0 if it is still running and block == 0; block != 0 waits.
 * *done = 1 at once when nothing is in flight. */
int hlu_factor_wait(hlu_handle* h, int32_t block, int32_t* done);

/* hlu_factor_stats - fill *info for the last factorisation. */
int hlu_factor_stats(const hlu_handle* h, hlu_factor_info* info);

/* hlu_factor_profile - per task kind of the last factorisation's task DAG:
 * out[3*k + 0] tasks run, out[3*k + 1] SM clock cycles spent waiting for a
 * ready task, out[3*k + 2] cycles spent running, summed over CTAs; kinds
 * k = 0..8 are GETRF, TRSM_L, TRSM_UT, TRSM_U, PROJ, ROWMV, TRUNC, DADD,
 * RSOLVE and k = 9 the no-work fences; then the truncation phases summed
 * over all compressions: out[30] stacking (shared-memory route) or dense
 * sum, out[31] QR cycles, out[32] core product, out[33] Jacobi SVD, out[34]
 * selection and Q application, out[35] compressions, out[36] Jacobi sweeps,
 * out[37] summed stack widths.  out: uint64[38] host buffer. */
int hlu_factor_profile(const hlu_handle* h, uint64_t* out);

/* hlu_solve - x = (LU)_H^-1 b, the preconditioner of Algorithm 1 step III
 * (U^-1 (L^-1 r), leaf pivots applied in the forward pass).  b_dev, x_dev:
 * device FP64, nrhs >= 1 columns, ld >= N; b and x may alias.  Runs in the
 * factor's precision (FP64 vectors are cast at entry and exit).
 * Asynchronous.  HLU_ERR_STATE if not factored. */
int hlu_solve(const hlu_handle* h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
              void* stream);

/* gmres_solve - restarted GMRES(restart) with right preconditioner
 * (LU)_H^-1 (Sec. 4, Example 1; flexible form when `flexible` != 0, which is
 * required for exactness when the factor is FP32), x0 = 0, CGS2
 * orthogonalisation and Givens rotations in FP64, stop when
 * ||b - A x||_2 <= tol ||b||_2 (true residual checked at exit), at most maxit
 * inner steps.  All nrhs columns iterate together; their preconditioner
 * applications are batched.  Synchronous; *stats filled if non-NULL.
 * Returns HLU_ERR_NOT_CONVERGED (x written) if a column missed tol. */
int gmres_solve(const hlu_handle* h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                int32_t restart, double tol, int32_t maxit, int32_t flexible, hlu_stats* stats,
                void* stream);

/* hlu_set_trunc_params - tuning of the recompression (Sec. 3: QR of both
 * stacked factors, SVD of the small core, keep s_i > eps s_1).  A target's
 * pieces are stacked and compressed whenever the stack would grow past
 * compress_at columns (8..96; 0 restores the default 48).  jacobi_tol is the
 * orthogonality tolerance |a^T b| <= tol ||a|| ||b|| at which the one-sided
 * Jacobi SVD of the core stops (0 restores the default: 1e-6 for FP32
 * factors, 1e-14 for FP64).  The truncation error is the norm of the
 * discarded columns whatever the tolerance; a looser one can only raise the
 * kept rank.  Process-wide; applies to factorisations started afterwards.
 * Returns HLU_ERR_ARG for values out of range. */
int hlu_set_trunc_params(int32_t compress_at, double jacobi_tol);

/* Continuous batching of GMRES solves (serving).  A hlu_gmres state holds
 * one request's restarted flexible GMRES (same method as gmres_solve; at most
 * 16 columns).  hlu_gmres_step_batch advances every unfinished state of the
 * list by one inner step (a new cycle starts with the true residual, as in
 * gmres_solve); the preconditioner applications of all states run in ONE
 * persistent launch (states sharing a factor share its work vector, up to 16
 * columns per launch).  States may join or leave between steps; a state's
 * result does not depend on which states it was batched with.
 * hlu_gmres_begin: x = 0, column norms of b; synchronous.  b, x stay owned by
 * the caller and must stay valid until hlu_gmres_end.  Its workspace is
 * 2 (restart + 1) N nrhs + O(N nrhs) doubles of device memory; when it cannot
 * be had (HLU_ERR_OOM) or any later step fails, nothing stays allocated and
 * *out is not written, so the call may be retried once memory is freed.
 * hlu_gmres_status: *done = 1 once finished; stats as in gmres_solve; returns
 * HLU_ERR_NOT_CONVERGED for a finished state that missed tol.
 * All calls on one stream; step_batch is synchronous. */
typedef struct hlu_gmres hlu_gmres;
int hlu_gmres_begin(const hlu_handle* h, const double* b_dev, double* x_dev, int32_t nrhs, int64_t ld,
                    int32_t restart, double tol, int32_t maxit, void* stream, hlu_gmres** out);
int hlu_gmres_step_batch(hlu_gmres* const* states, int32_t count, void* stream);
int hlu_gmres_status(const hlu_gmres* g, int32_t* done, hlu_stats* stats);
void hlu_gmres_end(hlu_gmres* g);

/* hlu_richardson - Algorithm 1 steps III-IV: r = b - A x, err = ||r||/||b||,
 * x <- x + U^-1 (L^-1 r), stop when err < tol or after maxit; then
 * error = ||A x - b||_2 into stats->abs_res_max.  Same vector conventions as
 * gmres_solve.  Synchronous. */
int hlu_richardson(const hlu_handle* h, const double* b_dev, double* x_dev, int32_t nrhs,
                   int64_t ld, double tol, int32_t maxit, hlu_stats* stats, void* stream);

/* Record of hlu_hinverse. */
#define HLU_HINV_MAX_ITERS 64
typedef struct {
  int32_t iterations;          /* Schulz steps taken                                 */
  int32_t n_residuals;         /* entries of residual[] (iterations + 1)             */
  double residual[HLU_HINV_MAX_ITERS + 1]; /* max over 4 probes z of ||z - A B z|| / ||z||,
                                               for X_0, X_1, ...                      */
  double alpha;                /* X_0 = alpha A_H, alpha = 1 / (||A||_1 ||A||_inf)    */
  int32_t rank_max;            /* largest rank of an admissible block of B_H          */
  int32_t reserved;
  double rank_mean;
  int64_t inverse_live_bytes;  /* B_H's words at live ranks (what an apply reads)     */
  int64_t arena_bytes;         /* device bytes of the iteration's four H-matrices,
                                  ring and vectors                                    */
  int64_t n_iter_tasks;        /* tasks of one Schulz step                            */
  double schedule_ms;          /* host time of the first build of the schedules       */
  double total_ms;             /* wall time of the call                               */
} hlu_hinv_info;

/* hlu_hinverse - B_H ~ A_H^-1 by the Schulz iteration (Sec. 3, "the inverse
 * ... by the iterative method of Schulz"; Sec. 4 truncated SVDs of the
 * admissible blocks; Example 2): X_0 = alpha A_H, then per step T = A_H (.) X,
 * X <- 2 X - X (.) T, the formatted H-products of the factorisation (son
 * products, agglomeration, truncation to s_i > eps s_1 at rank capacity
 * `rank_cap` of hlu_build), all tasks of a step in one persistent launch, in
 * FP32 or FP64.  After every step the residual ||I - A B|| is estimated by 4
 * fixed probe vectors; the iteration stops when it is <= tol, after maxit
 * steps, at the floor the truncation leaves (the estimate rises again after
 * falling a hundredfold), or on divergence (above 10: HLU_ERR_NOT_CONVERGED,
 * no inverse).  *info (may be NULL) is filled.  The first call builds the four
 * H-matrix copies' schedules on the host.  Synchronous.  HLU_ERR_ARG for
 * tol <= 0, maxit outside [0, HLU_HINV_MAX_ITERS] or HLU_TF32. */
int hlu_hinverse(hlu_handle* h, int32_t precision, double tol, int32_t maxit, hlu_hinv_info* info, void* stream);

/* hlu_hinverse_apply - x = B_H b (H-matrix times nrhs vectors; same vector
 * conventions as hlu_solve).  Synchronous.  HLU_ERR_STATE without an inverse. */
int hlu_hinverse_apply(const hlu_handle* h, const double* b, double* x, int32_t nrhs, int64_t ld, void* stream);

/* hlu_set_preconditioner - preconditioner of gmres_solve and hlu_richardson on
 * this handle: HLU_PRECOND_LU (default; needs hlu_factor) or HLU_PRECOND_HINV
 * (the inverse B_H used "as a preconditioner to solve the linear system",
 * Sec. 4, Example 2; needs hlu_hinverse).  The serving calls (hlu_gmres_*)
 * use the H-LU.  HLU_ERR_ARG for another value. */
int hlu_set_preconditioner(hlu_handle* h, int32_t which);

/* hlu_factor_batch - factor `count` built handles in ONE persistent launch
 * (their task DAGs interleaved), sharing the device.  Same semantics as
 * hlu_factor per handle.  Synchronous. */
int hlu_factor_batch(hlu_handle** hs, int32_t count, int32_t precision, void* stream);

/* hlu_solve_batch - x_i = (LU)_H,i^-1 b_i for `count` factored handles in one
 * persistent launch (cross-request batching of the triangular solves).
 * b[i], x[i]: device FP64 pointers with nrhs[i] columns, leading dimension
 * N_i.  Asynchronous. */
int hlu_solve_batch(hlu_handle* const* hs, int32_t count, const double* const* b,
                    double* const* x, const int32_t* nrhs, void* stream);

/* hlu_factor_bytes_estimate - device bytes hlu_factor will hold for this
 * handle at `precision` (factor storage + workspaces), for admission
 * control; -1 on error. */
int64_t hlu_factor_bytes_estimate(const hlu_handle* h, int32_t precision);

/* hlu_set_wait_limit_ms - bound (milliseconds, default 20000) of every
 * device-side dependency wait; a wait that runs out sets HLU_ERR_TIMEOUT and
 * the kernel returns.  Process-wide. */
void hlu_set_wait_limit_ms(double ms);

/* hlu_set_tile - factorisation granularity for subsequent hlu_build calls
 * (process-wide, default 64).  Every block-tree node whose row and column
 * clusters both hold at most `tile` DOFs is stored and factored as one dense
 * tile: its A_H entries and all fill inside it are kept exactly (no
 * truncation), so the factor is at least as accurate as the leaf-level H-LU.
 * Admissible blocks above the tile size stay low rank.  The exported trees
 * are not affected.  tile <= leaf keeps the block tree's own leaves; values
 * above 64 are clamped to 64. */
void hlu_set_tile(int32_t tile);


/* Device allocator of the library (process-wide).  alloc(bytes, ctx) returns
 * device memory of the current device, or NULL when it cannot (the library
 * call then fails with HLU_ERR_OOM); free(ptr, bytes, ctx) takes back a block
 * alloc returned.  Every block is freed by the allocator that returned it,
 * even after the allocator changed.  The library synchronises the device
 * before it hands a block to free, so the allocator may reuse it at once.
 * Both NULL restores cudaMalloc/cudaFree.  The Python binding uses this to
 * put the library's memory in PyTorch's caching allocator.  Returns
 * HLU_ERR_ARG when only one of the two is NULL. */
typedef void* (*hlu_alloc_fn)(size_t bytes, void* ctx);
typedef void (*hlu_free_fn)(void* ptr, size_t bytes, void* ctx);
int hlu_set_allocator(hlu_alloc_fn alloc, hlu_free_fn free, void* ctx);

/* hlu_set_device_memory_limit - cap (bytes, process-wide; 0 = none) on the
 * device memory the library holds through its allocator.  An allocation
 * that would pass it is refused and the call fails with HLU_ERR_OOM, leaving
 * the device and the library usable (for admission control, and to test the
 * out-of-memory path on the host).  HLU_ERR_ARG for a negative value. */
int hlu_set_device_memory_limit(int64_t bytes);

/* Device bytes the library holds through its allocator right now. */
int64_t hlu_device_bytes_in_use(void);

/* hlu_launch_count - number of this library's own CUDA kernel launches so far
 * in this process (kernels from CUDA's bundled sort/scan templates are not
 * counted).  Lets a caller count the launches inside a timed region. */
int64_t hlu_launch_count(void);

void hlu_destroy(hlu_handle* h);
const char* hlu_status_string(int status);
const char* hlu_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HLU_H */
