/*
 * kkt.h — C interface of the GB300 (sm_103a) solver for symmetric
 * positive-definite block-tridiagonal-arrow KKT systems
 *
 *        Psi x = b,   Psi = [ D_1  E_1^T                 G_1^T ]
 *                           [ E_1  D_2   E_2^T           G_2^T ]
 *                           [       .     .     .          .   ]
 *                           [             E_{N-1} D_N    G_N^T ]
 *                           [ G_1  G_2   ...      G_N    R     ]
 *
 * (Eq. (3) of "Parallel KKT Solver in PIQP for Multistage Optimization",
 * arXiv 2511.00946), by the partitioned block Cholesky factorization of
 * Algorithm 1 and the forward/backward substitutions of Algorithms 2 and 3.
 *
 * Conventions shared by every call:
 *  - All matrices are FP64, row-major, natural stage order j = 0..N-1,
 *    stage block size n, arrow (global-variable) width m >= 0:
 *        D [N][n][n]    D[j] = Psi_{j,j}      (lower triangle is read)
 *        E [N-1][n][n]  E[j] = Psi_{j+1,j}
 *        G [N][m][n]    G[j] = Psi_{g,j}      (ignored when m = 0)
 *        R [m][m]       Psi_{g,g}             (lower triangle is read)
 *        b [N*n+m][ldb] right-hand sides in the first nrhs columns
 *  - Matrix and vector pointers passed to kkt_factor/kkt_solve* are DEVICE
 *    pointers owned by the caller; the library only reads them (b is
 *    overwritten with the solution). kkt_factor_solve_host alone takes HOST
 *    pointers (see there). The factor and all scratch space are
 *    device memory owned by the handle, allocated by kkt_create* and freed
 *    by kkt_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). kkt_factor and kkt_solve* only enqueue work: they never
 *    synchronize, never allocate and are safe inside CUDA-graph capture.
 *  - Numerical breakdown (a pivot block that is not positive definite,
 *    including NaN input) never traps: the kernels record the first failure
 *    in a device-side record read by kkt_get_info after the stream is
 *    synchronized. The results of a failed factorization are undefined.
 *  - Every call returns a kkt_status; no call aborts the process.
 *
 * Batches: kkt_batch_create describes `count` independent systems of
 * possibly different (N, n, m, P). Their inputs are packed back to back in
 * system order: system s's D starts count_D(s) = sum_{t<s} N_t n_t^2
 * elements after the D base pointer, E after sum (N_t-1) n_t^2, G after
 * sum N_t m_t n_t, R after sum m_t^2 and b after sum (N_t n_t + m_t) rows.
 * kkt_batch_offsets returns these offsets.
 */
#ifndef KKT_H_
#define KKT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KKT_OK = 0,
  KKT_ERR_ARG = 1,        /* a size, pointer or option is invalid              */
  KKT_ERR_PARTITION = 2,  /* no partition: P < 1 or P > floor((N+1)/2)          */
  KKT_ERR_NOT_SPD = 3,    /* a pivot block was not positive definite            */
  KKT_ERR_CUDA = 4,       /* a CUDA runtime call failed (allocation, launch)   */
  KKT_ERR_TIMEOUT = 5,    /* a bounded wait inside a kernel ran out (reported by
                             kkt_get_info; the results of that call are invalid) */
  KKT_ERR_STATE = 6,      /* call out of order (solve before factor)           */
  KKT_ERR_CAPACITY = 7,   /* problem larger than a fixed-size buffer allows     */
  KKT_ERR_BOUNDS = 8      /* an index check of the debug build (KKT_DEBUG) failed:
                             a task's geometry or shared-memory layout did not fit;
                             the task was skipped, nothing trapped              */
} kkt_status;

/* Arithmetic of the factorization.
 *  KKT_FP64            every operation in FP64.
 *  KKT_MIXED_FP32      level-1 segments (the stage blocks of Psi): FP64 pivot
 *                      blocks (the diagonal-block Cholesky) and FP64 Schur
 *                      accumulators, FP32 panel triangular solves and FP32
 *                      Schur-complement dot products, and an FP32 copy of the
 *                      factor for the substitutions; the reduced separator
 *                      systems (levels >= 2) and the corner stay FP64.
 *                      kkt_solve then returns an unrefined solution;
 *                      kkt_solve_refined recovers FP64 accuracy by iterative
 *                      refinement on the FP64 residual.
 *  KKT_MIXED_FP32_ALL  the same arithmetic on every level.
 *  KKT_MIXED_TF32      KKT_MIXED_FP32 with the Schur-complement products of
 *                      level-1 blocks n >= 32 (the stacked panel's Z Z^T of
 *                      Algorithm 1, Eqs. (8a)-(8b)) on the tensor cores:
 *                      operands rounded to TF32, products accumulated in
 *                      FP32 and subtracted from the FP64 Schur accumulator;
 *                      pivots, trsm and smaller blocks as KKT_MIXED_FP32.
 *  KKT_MIXED_BF16      the same with BF16 operands (FP32 accumulation).
 *  The lower-precision products need more refinement sweeps for the same
 *  accuracy (kkt_solve_refined). */
typedef enum {
  KKT_FP64 = 0,
  KKT_MIXED_FP32 = 1,
  KKT_MIXED_FP32_ALL = 2,
  KKT_MIXED_TF32 = 3,
  KKT_MIXED_BF16 = 4
} kkt_precision;

/* How a level's N stages are split into P segments.
 *  KKT_PARTITION_PAPER     Eq. (13): N_1 and P-1 equal lengths N_k, with the
 *                          balance ratio 19/7 (Sec. 3.3). The rounding slack
 *                          all goes to the first segment, which is harmless
 *                          for a few threads and costly for hundreds of CTAs.
 *  KKT_PARTITION_BALANCED  the same cost model with the kernel's per-stage
 *                          flop counts, stage by stage to the cheapest
 *                          segment: lengths N_1 and N_k or N_k + 1. On a
 *                          level whose factor tasks run as CTA pairs (see
 *                          kkt_set_pairing) the fill-in rows are off the
 *                          critical path and every segment's stages cost
 *                          about the same, so the lengths come out nearly
 *                          equal. A handle pairs a level when the second
 *                          CTA has work (some segment has fill-in, or it is
 *                          the top level of a plan with lower levels, whose
 *                          corner partials it sums) and two CTAs per task
 *                          fit on the device's SMs (2 x tasks <= SMs). */
typedef enum { KKT_PARTITION_PAPER = 0, KKT_PARTITION_BALANCED = 1 } kkt_partition_mode;

typedef struct kkt_handle kkt_handle;

/* First breakdown recorded by the device since the last kkt_factor. */
typedef struct {
  int status;  /* KKT_OK, KKT_ERR_NOT_SPD, KKT_ERR_TIMEOUT or KKT_ERR_BOUNDS     */
  int system;  /* system index in the batch                                     */
  int stage;   /* natural stage of the failing pivot block; N for the corner R */
  int level;   /* 1 = stage blocks of Psi, 2.. = reduced (separator) systems    */
} kkt_info;

/* Create a solver for one system with N >= 1 stage blocks of size
 * 1 <= n <= 48 and arrow width 0 <= m <= 16, split into P segments by the
 * partition rule of Eq. (13) (Sec. 3.3, balance ratio 19/7). The reduced
 * separator system of Eq. (7) is factored sequentially by one CTA, which is
 * the paper's two-phase method. Returns KKT_ERR_PARTITION when
 * P > floor((N+1)/2). On success *out owns device memory for the factor,
 * including the fill-in blocks. */
kkt_status kkt_create(int N, int n, int m, int P, int precision, kkt_handle** out);

/* Like kkt_create but the reduced system is itself partitioned again
 * (recursively): level 1 splits the N stages into P_levels[0] segments; the
 * P_levels[0]-1 separators form the level-2 block-tridiagonal-arrow system
 * (Eqs. (7), (8)), which is split into P_levels[1] segments, and so on.
 * The last entry must be 1 (that level is factored sequentially). nlevels
 * >= 1; nlevels = 2 with P_levels = {P, 1} is kkt_create. The solution is
 * the same up to rounding; the factor is the Cholesky factor of the
 * correspondingly nested permutation. */
kkt_status kkt_create_levels(int N, int n, int m, int nlevels, const int* P_levels,
                             int precision, kkt_handle** out);

/* kkt_create_levels with a choice of partition rule for every level
 * (kkt_partition_mode). */
kkt_status kkt_create_plan(int N, int n, int m, int nlevels, const int* P_levels, int partition,
                           int precision, kkt_handle** out);

/* Batch of `count` independent systems; system s has N[s], n[s], m[s] and
 * P[s] segments (the two-phase method of kkt_create; P[s] = 1 is the
 * sequential method). P = NULL lets the autotuner pick every system's level
 * plan: the call is then kkt_batch_create_tuned (it blocks while the
 * candidates are timed and must be made outside any graph capture).
 * Limits per system as for kkt_create. */
kkt_status kkt_batch_create(int count, const int* N, const int* n, const int* m, const int* P,
                            int precision, kkt_handle** out);

/* Batch of `count` independent systems whose level plans (segments per
 * level, KKT_PARTITION_BALANCED partitions) are picked by an autotuner: it
 * times one factor + one single-RHS solve of every candidate on the current
 * device, with synthetic inputs of the batch's shapes (identity pivot blocks;
 * the kernels' run time does not depend on the values), and keeps the
 * fastest. Candidates: every system sequential (P = 1, no fill-in; best when
 * the systems alone fill the GPU), and level-1 segment totals of 1/2, 1, 2,
 * 4, 8, 16, 32 and 64 per SM spread over the systems in proportion to their
 * stage counts, with 4x or 8x fewer segments on each level above, down to a
 * sequential top level. levels_out (optional, length count) receives the
 * number of levels chosen per system; kkt_partition reads the plan. Blocks
 * until the tuning runs finish and allocates scratch memory for them
 * (freed before returning): call it outside any graph capture. Errors as
 * for kkt_batch_create, KKT_ERR_CUDA when the tuning runs fail. */
kkt_status kkt_batch_create_tuned(int count, const int* N, const int* n, const int* m, int precision,
                                  int* levels_out, kkt_handle** out);

/* Free the handle and its device memory (NULL is accepted). */
kkt_status kkt_destroy(kkt_handle* h);

/* Segment lengths of system `system` at level `level` (1-based):
 * seg_len[0..P-1] = (N_1, N_k, ..., N_k). `P_out` receives P. seg_len may
 * be NULL to query P only. */
kkt_status kkt_partition(const kkt_handle* h, int system, int level, int* P_out, int* seg_len);

/* Host-side partition rule of Eq. (13) without a handle: writes P lengths.
 * Returns KKT_ERR_PARTITION when infeasible. */
kkt_status kkt_partition_rule(int N, int P, int* seg_len);

/* Segment lengths of the balanced partition (KKT_PARTITION_BALANCED) of N
 * stages of size n with arrow m into P segments, for an unpaired (paired =
 * 0) or a paired (paired = 1) level. */
kkt_status kkt_partition_balanced(int N, int n, int m, int P, int paired, int* seg_len);

/* Element offsets of every system's inputs in the packed batch layout
 * (arrays of length count+1; any pointer may be NULL). off_b counts rows. */
kkt_status kkt_batch_offsets(const kkt_handle* h, size_t* off_D, size_t* off_E, size_t* off_G,
                             size_t* off_R, size_t* off_b);

/* Factor Psi (Algorithm 1). D, E, G, R: device pointers in the layout above
 * (E may be NULL when every N = 1; G and R may be NULL when every m = 0).
 * Enqueued on `stream`; asynchronous. */
kkt_status kkt_factor(kkt_handle* h, const double* D, const double* E, const double* G,
                      const double* R, void* stream);

/* Solve Psi x = b with the current factor (Algorithms 2 and 3): b is a
 * device pointer to (N*n+m) rows of ldb >= nrhs doubles (for batches the
 * packed rows of every system), overwritten with x in its first nrhs
 * columns. nrhs >= 1. Asynchronous on `stream`.
 * Systems planned as one level (P = 1) are solved with one right-hand side
 * by one warp each (forward sweep, corner and backward sweep, the stage
 * blocks streamed by bulk copies; their waits are bounded as described at
 * kkt_set_wait_limit and a timeout is reported through kkt_get_info); with
 * several right-hand sides, for odd n, or for other plans by the segment
 * kernels, whose panel products sum in another order: a column solved alone
 * and in a chunk of several then agree to rounding, not bit for bit. */
kkt_status kkt_solve(kkt_handle* h, double* b, int nrhs, int ldb, void* stream);

/* Factor Psi and solve Psi x = b in one pass (kkt_factor followed by
 * kkt_solve, with the same result up to rounding): the right-hand side is
 * bordered onto the arrow, i.e. the matrix [[Psi, b], [b^T, .]] is factored,
 * so the forward substitution (Algorithm 2) is carried by the factorization
 * (its extra arrow row is y = L-hat^{-1} b, stage by stage and across the
 * levels through the same slots) and only the corner and the backward
 * substitution (Algorithm 3) follow. b (device, ldb >= nrhs) is overwritten
 * with x. Used for FP64 handles with nrhs = 1 and an arrow of at most 15 rows
 * (room for the bordered row); otherwise it runs kkt_factor and kkt_solve.
 * The factor stays usable for kkt_solve, kkt_solve_refined and
 * kkt_solve_adjoint; kkt_get_factor then reports KKT_ERR_STATE. Launches
 * recorded by kkt_set_launch_events: the copy of the bordered arrow, the
 * factor launches, then the backward launches. With blocks n > 16 the top
 * level's factor launch also runs the corner solve x_g = R-hat^{-T} y_g and
 * the top level's backward sweep (when the top level has at most one task
 * per SM); otherwise a launch of their own follows the factor launches. */
kkt_status kkt_factor_solve(kkt_handle* h, const double* D, const double* E, const double* G,
                            const double* R, double* b, int nrhs, int ldb, void* stream);

/* kkt_factor_solve from HOST buffers: D, E, G, R and b are host pointers in
 * the layout above; x is written back to b (ldb >= nrhs) when the stream
 * reaches the end of the call. The handle keeps device buffers: a copy of b
 * (allocated by the first call, and again by a call with more right-hand
 * sides than any before) and copies of D, E, G, R (allocated by the first
 * call that copies them). A call that allocates must not run inside a stream
 * capture and invalidates graphs captured before it; the others may be
 * captured. Three ways, by the memory the inputs live in:
 *  - D, E, G and R all page-locked and addressable by the device
 *    (cudaHostAlloc or cudaHostRegister; torch pin_memory): the factor
 *    launches read them in place over the host link, each element once, and
 *    only b is copied in and x out. The host arrays must stay alive and
 *    unchanged until the stream has passed the call (for a captured call:
 *    every replay reads them again).
 *  - Otherwise, for one system with the bordered pass (FP64, nrhs = 1,
 *    P >= 2 level-1 segments): the copy of the stage rows of D, E, G and b is
 *    split at separator stages into up to eight chunks on an internal
 *    stream, and each chunk's bordered arrow copy and level-1 segments start
 *    on a stream of their own as soon as its rows have arrived (the segments
 *    of Algorithm 1 are independent), so the transfer overlaps the level-1
 *    factorization; the corner and the g-rows of b travel with the first
 *    chunk.
 *  - Otherwise the inputs are copied on `stream` and kkt_factor_solve runs on
 *    the device copies.
 * The result is that of kkt_factor_solve on the same inputs, bit for bit.
 * Launch events are not recorded. */
kkt_status kkt_factor_solve_host(kkt_handle* h, const double* D, const double* E, const double* G,
                                 const double* R, double* b, int nrhs, int ldb, void* stream);

/* Mixed-precision iterative refinement: x = Psi^{-1} b by x_0 = 0,
 * c <- b; then `sweeps` times: c <- (L-hat L-hat^T)^{-1} c with the current
 * factor (FP32 substitutions on mixed levels), x <- x + c, c <- b - Psi x in
 * FP64 with the blocks of Eq. (3), eta = ||c||_inf / (||Psi||_inf ||x||_inf +
 * ||b||_inf) over the system's right-hand sides together. A system stops
 * when its eta is <= tol, or when its eta is at the rounding level of the
 * FP64 residual (<= 4 u, u = 2^-53) and a sweep cuts it by less than 10 %
 * (refinement has reached its floor); its remaining sweeps return at once on the device (no host
 * synchronization, capturable in a CUDA graph). With tol = 0 every system
 * refines until its eta stops falling; with tol < 0 every sweep runs. A relative residual within a small
 * factor of the FP64 factorization's needs eta at that level (about 1e-16
 * on barrier-scaled systems), i.e. tol <= 1e-16; a looser tol stops earlier
 * at a correspondingly larger residual. D, E, G, R must be the
 * matrix that was factored; b (read-only) and x (written) are device
 * pointers with leading dimensions ldb, ldx >= nrhs. 1 <= sweeps <= 16.
 * Works with any precision (with KKT_FP64 one sweep is a plain solve plus a
 * residual check). */
kkt_status kkt_solve_refined(kkt_handle* h, const double* D, const double* E, const double* G,
                             const double* R, const double* b, int ldb, double* x, int ldx, int nrhs,
                             int sweeps, double tol, void* stream);

/* Adjoint of the solve, for a loss L(x) with x = Psi^{-1} b: given x (the
 * solution, ldx) and xbar = dL/dx (ldxb), writes bbar = dL/db = Psi^{-1} xbar
 * (ldbb) with the current factor (refined with `sweeps` sweeps of
 * kkt_solve_refined when the factor is mixed; D, E, G, R are then required)
 * and the gradients with respect to the stored blocks, in the layout of the
 * inputs (dPsi = -bbar x^T restricted to the blocks, summed over the nrhs
 * columns; a symmetric pair of entries is one parameter):
 *   dD_j[r][c] = -(bbar_r x_c + bbar_c x_r) for r > c, -bbar_r x_r for r = c,
 *                0 above the diagonal (the upper triangle is not read)
 *   dE_j = -(bbar_{j+1} x_j^T + x_{j+1} bbar_j^T)
 *   dG_j = -(bbar_g x_j^T + x_g bbar_j^T)
 *   dR   like dD on the g rows.
 * All pointers are device pointers; dE may be NULL when every N = 1, dG and
 * dR when every m = 0. Asynchronous on `stream`. */
kkt_status kkt_solve_adjoint(kkt_handle* h, const double* D, const double* E, const double* G,
                             const double* R, const double* x, int ldx, const double* xbar, int ldxb,
                             double* bbar, int ldbb, int nrhs, double* dD, double* dE, double* dG,
                             double* dR, int sweeps, void* stream);

/* Refinement tolerance of kkt_solve_adjoint on a mixed factor (its tol
 * argument to kkt_solve_refined; same meaning): 0, the default, refines each
 * system until its eta stops falling; a value such as 1e-16 stops a system
 * as soon as its eta is at or below it, which saves the sweep that only
 * confirms the floor. NaN gives KKT_ERR_ARG. */
kkt_status kkt_set_refine_tol(kkt_handle* h, double tol);

/* Fallback of kkt_solve_refined for systems whose refinement stalls:
 * cg_iters > 0 enables it. A system whose eta, still above the rounding
 * level, is not at least halved by a sweep is taken out of the classic sweeps
 * and, after them, together with any system that did not converge within
 * `sweeps`, runs cg_iters iterations of preconditioned conjugate gradients
 * on Psi x = b (Psi is SPD) from its refined x, preconditioned by the same
 * (mixed) factor: the conjugate-gradient form of refinement with a
 * low-precision preconditioner (Carson and Higham, 2018), which converges
 * where the stationary iteration stalls because its rate depends on the
 * spread of the preconditioned spectrum rather than on its distance from 1.
 * FP64 vectors and products, the factor's substitutions, per-system scalars
 * on the device: no host synchronization, capturable. kkt_refine_eta of the
 * last sweep then reports the eta after the fallback. cg_iters = 0 (the
 * default) disables it; the first call with cg_iters > 0 allocates its
 * vectors (3 x rows x 16 doubles; call it outside any graph capture). */
kkt_status kkt_set_refine_fallback(kkt_handle* h, int cg_iters);

/* eta of every system after sweep `sweep` (0-based) of the last
 * kkt_solve_refined (last right-hand-side chunk); eta[count]. Synchronizes.
 * Values after a system converged are those of its converging sweep. */
kkt_status kkt_refine_eta(kkt_handle* h, int sweep, double* eta);

/* Copy the first recorded breakdown to *info. Synchronizes with the device
 * (call it after the stream that ran kkt_factor is synchronized). Clears the
 * record when `clear` != 0. */
kkt_status kkt_get_info(kkt_handle* h, kkt_info* info, int clear);

/* Copy the blocks of the factor of system `system` to HOST buffers in the
 * natural-order layout of the two-level method (Algorithm 1):
 *   Ld [N][n][n]  D-hat at segment stages, A-hat_k at separator s_k
 *   Le [N-1][n][n] E-hat inside a segment, F-hat_k at the last stage of
 *                 segment k, zero at the separators
 *   Lw [N][n][n]  fill-in W = L-hat(s_k, j) (the paper's B-hat^T) at the
 *                 stages j of segments k >= 2, zero elsewhere
 *   Lh [N][n][n]  fill-in H_k = L-hat(s_{k+1}, s_k) at j = s_k, zero elsewhere
 *   Lg [N][m][n]  G-hat at segment stages, Q-hat_k at separator s_k
 *   Lr [m][m]     R-hat
 * Row-major, lower triangles of the diagonal blocks (upper parts zero).
 * Only for handles with at most two levels; any pointer may be NULL.
 * Synchronizes with the device. */
kkt_status kkt_get_factor(kkt_handle* h, int system, double* Ld, double* Le, double* Lw,
                          double* Lh, double* Lg, double* Lr);

/* Attach `count` cudaEvent_t handles (passed as void*) that kkt_factor and
 * kkt_solve record on their stream right after each of their kernel
 * launches, in launch order (event i after launch i of the call; launches
 * beyond `count` record nothing). Lets a caller time each launch with no
 * extra work on the device. count = 0 or events = NULL detaches. The events
 * stay owned by the caller and must outlive their use. When the stream is
 * being captured into a CUDA graph, the records are captured as external
 * event-record nodes and happen on every replay of the graph. */
kkt_status kkt_set_launch_events(kkt_handle* h, void* const* events, int count);

/* Layout of the factor kernel's segment tasks. With pairing, a segment runs
 * on a cluster of two CTAs on separate SMs: one carries the chain of
 * Algorithm 1 (pivot factorization, E- and G-rows, their Schur updates), the
 * other the fill-in rows W of segments k >= 2 and their updates of A~, Q~
 * and the next W, fed through distributed shared memory; on the top level
 * the second CTA sums the lower levels' corner partials while the first
 * runs the stages. This gives a task two SMs' FP64 units and pays off on
 * levels with fewer tasks than SM pairs. KKT_PAIR_AUTO (the default) pairs exactly those levels;
 * Systems with blocks n <= 16 run one warp per segment task (several tasks
 * per CTA) in every case and never pair: at that size what counts is how
 * many independent stage chains an SM interleaves.
 * On FP64 levels whose segments are all single stages with fill-in rows
 * (the deep levels of a recursive plan), KKT_PAIR_AUTO runs each task on a
 * cluster of 2, 4 or 8 CTAs instead (the largest size whose clusters all
 * fit on the device at once, at most two CTAs per SM): every CTA factors
 * the pivot block, solves a band of the panel rows and applies the Schur
 * update (Alg. 1) to a band of about 1/C of its elements, the bands
 * exchanged through distributed shared memory. KKT_PAIR_AUTO_PAIRS is the
 * automatic choice without these clusters.
 * KKT_PAIR_OFF and KKT_PAIR_ON force one layout on every level (the
 * partition chosen at creation is kept). The layouts give bitwise identical
 * results: each element is computed by the same operations in the same
 * order; only the assignment to threads differs. Returns KKT_ERR_ARG for a
 * NULL handle or an unknown policy. Takes effect at the next kkt_factor. */
typedef enum {
  KKT_PAIR_AUTO = 0,
  KKT_PAIR_OFF = 1,
  KKT_PAIR_ON = 2,
  KKT_PAIR_AUTO_PAIRS = 3
} kkt_pair_policy;
kkt_status kkt_set_pairing(kkt_handle* h, int policy);

/* Schedule of kkt_factor. on = 0 (the default): one launch per level and
 * block-size class. on = 1: ONE persistent launch for the whole
 * factorization of every system at every level (Algorithm 1's parallel phase
 * and, level by level, the reduced systems of Eq. (7)). Its CTAs take work
 * items by ticket from a queue in topological order (level by level; within
 * a level the most expensive segment tasks first, i.e. longest processing
 * time first, so long systems start first and short ones fill the tail;
 * tasks with blocks n <= 16 in bundles of up to eight, one per warp). A
 * reduced-system task starts as soon as the lower-level tasks whose slots it
 * reads have released their per-task ready counters, instead of at a level
 * boundary; each wait is bounded (kkt_set_wait_limit) and reports
 * KKT_ERR_TIMEOUT through kkt_get_info instead of hanging. Segment tasks never
 * run as CTA pairs in this schedule, and mixed levels use FP32 CUDA-core
 * Schur products. Results are bitwise those of the per-level launches (the
 * same operations per element). Requires every level of the handle to have
 * the same arithmetic (KKT_FP64, KKT_MIXED_FP32_ALL, or single-level plans
 * of any precision), else KKT_ERR_ARG. The first call with on = 1 builds the
 * work list and allocates a small device buffer (call it outside any graph
 * capture); kkt_factor then enqueues one memset and one kernel (capturable).
 * kkt_factor_solve and kkt_factor_solve_host keep the per-level launches. */
kkt_status kkt_set_persistent(kkt_handle* h, int on);

/* The backward substitution of the levels below the top (Algorithm 3,
 * parallel phase of each level) as ONE launch (on = 1, the default where it
 * applies) or one launch per level and block-size class (on = 0). It applies
 * to solves of one right-hand side (kkt_factor_solve, single-column
 * kkt_solve and the refinement's correction solves) on handles with at
 * least three levels whose backward tasks all have blocks n > 16 and whose
 * levels below the top share one precision; elsewhere, and for chunks of
 * several right-hand sides, the per-level launches run whatever `on` says. In the single launch CTAs take
 * (task, column group) items by ticket, top level first; an item requests
 * its stage's factor blocks at once, then waits until every item of the
 * level above has released its counter (a bounded wait, see
 * kkt_set_wait_limit), solves, and releases its own level's counter.
 * Results are bitwise those of the per-level launches (the same operations
 * per element). kkt_launch_counts reflects the setting for one right-hand
 * side. Returns KKT_ERR_ARG for a NULL handle. Takes effect at the next
 * solve. */
kkt_status kkt_set_backward_chain(kkt_handle* h, int on);

/* Instruction warm-up of kkt_factor_solve's bordered pass (on = 1; default
 * off). After an L2 flush, or when other work has evicted them, the code of
 * the kernels that run once per call (the cluster kernel of the deep levels,
 * the top level's corner factorization and corner solve, the single-launch
 * backward substitution) is fetched from device memory the first time each
 * runs, a cost of several microseconds per kernel on a latency-bound
 * critical path. With the warm-up, each kkt_factor_solve first forks a side
 * stream on which a companion system (7 stages with the handle's largest
 * block sizes, identity blocks, plan [4, 2, 1]) runs its own bordered pass,
 * concurrently with this call's border copy and first level, so that those
 * kernels' code is in L2 when the call reaches them; the call joins the
 * side stream before it returns (graph capture sees a fork and a join). The
 * companion's results are discarded and do not touch this handle's factor,
 * info record or events. Applies to FP64 handles with room for the bordered
 * row; a no-op elsewhere. on = 1 allocates the companion (a few hundred KB)
 * and a stream: call it outside any graph capture. Returns KKT_ERR_ARG for a
 * NULL handle. */
kkt_status kkt_set_code_warmup(kkt_handle* h, int on);

/* Bounded waits of the persistent schedule, of the single-launch backward
 * substitution and of the one-warp substitution
 * of sequential systems (one level, P = 1, one right-hand side), whose stage
 * blocks arrive by bulk copies counted on an mbarrier: a task gives up
 * waiting for its feeders (or its copies) after `cycles` SM clock cycles
 * (default 2^31, about a second), records KKT_ERR_TIMEOUT (system, natural
 * stage and level of the waiting task) and carries on without its own work,
 * so nothing hangs; the substitution first waits, with the same bound, for
 * its copies still in flight. unmet != 0 adds one unsatisfiable dependency
 * to every waiting task (a counter no task ever releases) and makes every
 * stage of the substitution expect 16 bytes more than its copies deliver,
 * which makes every wait run out: a test of the timeout path on the device;
 * unmet = 0 restores the real counts. */
kkt_status kkt_set_wait_limit(kkt_handle* h, long long cycles, int unmet);

/* Number of kernel launches one kkt_factor / one kkt_solve (per chunk of up
 * to 16 right-hand sides) enqueues for this handle. The solve count is that
 * of a chunk with one right-hand side; where the backward levels run as one
 * launch (kkt_set_backward_chain), a chunk of several right-hand sides runs
 * them one launch per level and block-size class instead. */
kkt_status kkt_launch_counts(const kkt_handle* h, int* factor_launches, int* solve_launches);

/* CTAs per segment task in the per-level factor launches of level `level`
 * (0-based) under the current pairing policy: 1 (one CTA per task, or one
 * warp per task for blocks n <= 16), 2 (CTA pairs, or clusters of two), 4 or
 * 8 (clusters of one-stage segments); the largest over the level's launch
 * groups. *ctas is written on success; KKT_ERR_ARG for a NULL handle or
 * pointer or a level outside [0, number of levels). */
kkt_status kkt_factor_ctas_per_task(const kkt_handle* h, int level, int* ctas);

/* Algorithmic FP64 flops of one kkt_factor and of one kkt_solve with one
 * right-hand side for this handle, in the standard counting convention
 * (potrf n^3/3+n^2/2+n/6, trsm r n^2, syrk r(r+1)k, gemm 2rck, trsv n^2,
 * gemv 2rc), as executed by the partitioned method (fill-in included), and
 * the flops of the sequential method on the same systems. */
kkt_status kkt_flops(const kkt_handle* h, double* factor_flops, double* solve_flops,
                     double* sequential_factor_flops);

/* Same counts as kkt_flops for one system planned like kkt_create_plan on a
 * device with `sms` SMs (which decides the paired levels of a balanced
 * partition; 0 = no level paired), computed on the host without a handle
 * or a GPU. */
kkt_status kkt_plan_flops(int N, int n, int m, int nlevels, const int* P_levels, int partition, int sms,
                          double* factor_flops, double* solve_flops,
                          double* sequential_factor_flops);

/* Factor and solve ONE system without allocating any memory (the paper has
 * no counterpart: this serves callers that cannot allocate device memory
 * where they solve, e.g. a real-time control loop that must not touch an
 * allocator, a plugin whose host framework owns every allocation, or a
 * process whose memory pool is exhausted). Same method as
 * kkt_create(N, n, m, P, KKT_FP64) followed by kkt_factor and kkt_solve,
 * with the same results.
 *  - D, E, G, R, b: device pointers as for kkt_factor / kkt_solve; b is
 *    overwritten with the solution. `info`: optional device pointer to 4
 *    ints that receive the kkt_info record of a breakdown (zeroed first by
 *    this call; status KKT_ERR_NOT_SPD = 3 on breakdown), NULL to skip.
 *  - The factor and every scratch table live in one library-owned,
 *    statically sized device array of 16 MiB that each GPU loading the
 *    library holds until the process exits. A shape whose factor and tables
 *    need more (roughly 6 n^2 + 2 m n doubles per stage; for example
 *    N = 256, n = 32, m = 8 fits, N = 1024, n = 32 does not), or N > 16384
 *    or P > 1024, returns KKT_ERR_CAPACITY before any work is enqueued.
 *  - The first call on a device (with that device current) looks up the
 *    array's device address with cudaGetSymbolAddress; make that first call
 *    before any stream capture. Every call stages its small tables
 *    (descriptors, tasks, index maps) from host memory into the array with
 *    cudaMemcpyAsync from a pageable buffer, which may block the host until
 *    the data is staged, and clears the breakdown record with
 *    cudaMemsetAsync.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind. Calls whose work overlaps on the GPU (other streams, other
 *    host threads) race on it and give undefined results: serialize them,
 *    e.g. on one stream.
 * Returns KKT_ERR_ARG for invalid sizes or pointers, KKT_ERR_PARTITION when
 * P > floor((N+1)/2). */
kkt_status kkt_solve_noalloc(int N, int n, int m, int P, const double* D, const double* E,
                             const double* G, const double* R, double* b, int nrhs, int ldb,
                             int* info, void* stream);

/* Human-readable name of a status code (static string). */
const char* kkt_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* KKT_H_ */
