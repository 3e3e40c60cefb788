// Internal structures shared by the host plan (kkt_api.cu) and the kernels
// (kkt_kernels.cu). Not part of the public interface.
//
// Hierarchy. A system is solved level by level. Level 1 is Psi itself: its
// N stages are split into P segments (Sec. 3.1, Eq. (13)). The P-1 separator
// stages form the level-2 system, which has the same block-tridiagonal-arrow
// form (Eqs. (7)-(8)): diagonal A~_k, sub-diagonal H~_k, arrow Q~_k and the
// running corner R~. The last level of a system has P = 1 and is factored
// sequentially by one CTA, which also factors the corner R-hat. Two levels
// are exactly the paper's two-phase method (parallel phase over segments,
// sequential phase over the reduced system).
//
// Stacked panel. Within a segment, stage i carries the panel
//   Z_i = [ E-rows ; G-rows ; W-rows ]   ((2n+m) x n, rows [0,n), [n,n+m), [n+m,2n+m))
// holding E_i (or F_k at the last stage), G_i and the fill-in W_i (the
// paper's B-hat^T). One stage is: D-hat_i = chol(D_i) (potrf), Z_i <- Z_i
// D-hat_i^{-T} (one trsm, Alg. 1 lines for E-hat, G-hat, B-hat and F-hat) and
// T -= Z_i Z_i^T on the lower triangle, where the blocks of T are
//   T_EE = D_{i+1}   T_GE = G_{i+1}   T_GG = R~_k partial
//   T_WE = W_{i+1}   T_WG = Q~_k^T    T_WW = A~_k
// i.e. every Schur update of Algorithm 1 (Eqs. (8a)-(8b)) in one syrk. At the
// last stage the E-rows hold F_k, so T_EE, T_GE, T_WE collect -F^ F^T,
// -G^ F^T (the cross-segment terms of Eq. (8c), owned by this segment in a
// slot of its own) and H~_k^T.
#pragma once
#include <cstddef>

namespace kkt {

#ifndef KKT_FACTOR_THREADS
#define KKT_FACTOR_THREADS 256
#endif
#ifndef KKT_SOLVE_THREADS
#define KKT_SOLVE_THREADS 256
#endif
constexpr int kFactorThreads = KKT_FACTOR_THREADS;  // threads per factor CTA
constexpr int kSolveThreads = KKT_SOLVE_THREADS;    // threads per solve CTA
constexpr int kMaxN = 48;        // largest stage block supported
constexpr int kMaxM = 16;        // largest arrow width supported
constexpr int kRhsChunk = 16;    // right-hand sides per solve launch sequence

struct LevelDesc {
  // shape of this level of this system; segment k covers stages
  // seg[k] .. seg[k+1]-2, its separator is stage seg[k]-1 (k >= 1), and
  // seg[P] = N + 1
  int N, n, m, P;
  const int* seg;
  int level;      // 1-based
  int is_top;     // P == 1 and no deeper level: also factors/solves the corner
  int sys;        // system index in the batch
  int precision;  // kkt_precision
  // right-hand sides bordered onto the arrow (0, or 1 in a fused factor-and-solve
  // pass): the last mr of the m arrow rows then hold b, the factorization carries
  // the forward substitution, and the real arrow has m - mr rows
  int mr;
  long long offGu, offRu;  // bordered level 1: the caller's G and R (offG, offR index the bordered copies)
  // inputs: level 1 reads the caller's arrays at these element offsets;
  // deeper levels read the slots the level above wrote (D = Dw + D2w, etc.)
  long long offD, offE, offG, offR, offB;
  long long rowG;  // row of the system's first global-variable entry in b (level-1 N*n + offB)
  int Nnat;        // level-1 stage count of the system (stage reported for the corner)
  const double* Dw;
  const double* D2w;
  const double* Ew;
  const double* Gw;
  const double* G2w;
  const int* nat;  // natural (level-1) stage index of every stage of this level
  // factor of this level: D-hat [N][n][n], 1/diag [N][n], panel [N][R][n],
  // and D-hat with its columns divided by their diagonal ([N][n][n], strict
  // lower part), which the substitutions use
  double* Ld;
  double* Lri;
  double* Lp;
  double* LdM;
  double* LdR;  // D-hat with its rows divided by their diagonal (backward substitution)
  // mixed precision: the factor in FP32 for the correction solves, and
  // whether this level's segments run their panel trsm/syrk in FP32
  int mixed;
  float* LdMf;
  float* LdRf;
  float* Lrif;
  float* Lpf;
  // slots for the next level (null at the top), indexed by next-level stage
  double* DA;  // [P-1][n][n]  A~_{k}   written by segment k   (index k-1)
  double* DB;  // [P-1][n][n]  -F^_k F^_k^T  by segment k       (index k)
  double* EN;  // [P-2][n][n]  H~_k          by segment k       (index k-1)
  double* GA;  // [P-1][m][n]  Q~_k          by segment k       (index k-1)
  double* GB;  // [P-1][m][n]  -G^_l F^_k^T  by segment k       (index k)
  double* Rpart;  // [P][m][m] this level's R~_k partials
  // solve: this level's vectors [N][n][kRhsChunk] (level 1 uses the caller's b)
  double* X;
  const double* RA;  // right-hand side of this level (levels >= 2): RA + RB
  const double* RB;
  double* YA;     // [P-1][n][chunk] next level's rhs part written by segment k (index k-1)
  double* YB;     // [P-1][n][chunk] next level's rhs part written by segment k (index k)
  double* ygpart; // [P][m][chunk]
  double* Xnext;  // next level's X (solutions at this level's separators)
  // system-wide, used by the top level
  double* Rhat;       // [m][m] corner factor
  double* Rri;        // [m]
  double* Rpart_all;  // every level's partials (levels 1..L-1), contiguous
  int nRpart_all;
  double* yg_all;     // every level's yg partials, contiguous [..][m][chunk]
  int nyg_all;
};

struct Task {
  int desc;  // index into the LevelDesc array
  int seg;   // segment index k (0-based)
};

// Persistent factorization (one launch for every level of every system):
// work items in topological order (level by level; within a level the most
// expensive first), each one segment task run by a whole CTA or a bundle of
// up to eight small-block tasks run one per warp. An item that reads the
// slots of lower-level tasks starts once its counter in `ready` reaches
// `need`; a finished item adds `weight` to the counter of each consumer.
struct PItem {
  int first;  // first task in the persistent task array
  int cnt;    // tasks (1 for a CTA item, <= 8 for a warp bundle)
  int warp;   // 1: one warp per task (blocks n <= kWarpMaxN)
  int need;   // feeder tasks to wait for
  int cons0;  // first consumer edge
  int ncons;  // consumer edges
};
struct PCons {
  int item;    // consumer item
  int weight;  // feeder tasks of the consumer in this item
};

// Device-side breakdown record (kkt_info layout).
struct Info {
  int status, system, stage, level;
};

// Shared-memory layouts, byte offsets, identical on host and device. Square
// FP64 buffers are sized for q = max(n, m) because the corner (m x m) reuses
// them. zb = bytes per panel element (8: FP64 path, 4: mixed). Odd leading
// dimensions keep row- and column-wise accesses free of bank conflicts.
// `fill`: the level has fill-in rows (P > 1). A level without them (P = 1,
// the last level of its systems) keeps only the E- and G-rows of the panel
// and of T in shared memory (Rs = n + m instead of R = 2n + m rows), which
// lets more CTAs share an SM; R stays the panel height of the factor in
// global memory.
struct FacLayout {
  int q, R, Rs, ldD, ldZ, ldT, oDfac, oM, oRinv, oRinvZ, oZ, oT, oTab, oDfac2, oRinv2, oCorner, total;
};
__host__ __device__ inline int kkt_align16(int b) { return (b + 15) & ~15; }
// `dbl`: a second pivot buffer (and rinv) so that warp 4 can write the
// previous stage's pivot blocks while the next ones are being factored; a
// launch goes without it when that lets more CTAs share an SM.
__host__ __device__ inline FacLayout fac_layout(int n, int m, int zb, bool fill = true, bool dbl = true) {
  FacLayout L;
  L.q = n > m ? n : m;
  L.R = 2 * n + m;
  L.Rs = fill ? L.R : n + m;
  L.ldD = L.q | 1;
  L.ldZ = n | 1;
  L.ldT = L.Rs | 1;
  L.oDfac = 0;
  L.oM = L.oDfac + kkt_align16(8 * L.q * L.ldD);
  L.oRinv = L.oM + kkt_align16(zb * n * L.ldD);
  L.oRinvZ = L.oRinv + kkt_align16(8 * L.q);
  L.oZ = L.oRinvZ + kkt_align16(zb * L.q);
  L.oT = L.oZ + kkt_align16(zb * L.Rs * L.ldZ);
  L.oTab = L.oT + kkt_align16(8 * L.Rs * L.ldT);  // potrf element table, q(q-1)/2 ints
  // second pivot block and rinv: the next stage's pivot factorization runs
  // while the current stage's factor blocks are still being written
  L.oDfac2 = L.oTab + kkt_align16(4 * (L.q * (L.q - 1) / 2 + 1));
  L.oRinv2 = L.oDfac2 + (dbl ? kkt_align16(8 * L.q * L.ldD) : 0);
  // sum of the lower levels' corner partials (m x m), formed before the corner
  L.oCorner = L.oRinv2 + (dbl ? kkt_align16(8 * L.q) : 0);
  L.total = L.oCorner + kkt_align16(8 * kMaxM * kMaxM);
  return L;
}
// One warp's slice for a small-block segment task (k_factor_w): the same
// blocks without the second pivot buffer, and an m x m corner sum.
__host__ __device__ inline FacLayout fac_layout_w(int n, int m, int zb, bool fill = true) {
  FacLayout L = fac_layout(n, m, zb, fill);
  L.oDfac2 = L.oRinv2 = 0;
  L.oCorner = L.oTab + kkt_align16(4 * (L.q * (L.q - 1) / 2 + 1));
  L.total = L.oCorner + kkt_align16(8 * (m * m > 0 ? m * m : 1));
  return L;
}
constexpr int kWarpMaxN = 16;  // largest stage block of the warp-per-task kernels
// The substitution kernels double-buffer the factor blocks (L, rinv, Z) so
// that the next stage's blocks stream in while the current stage is solved.
struct SolLayout {
  int q, R, ldL, ldZ, ldV, oL[2], oRinv[2], oZ[2], oV, oT, total;
};
// (fill: as for fac_layout; a level with P = 1 keeps only the E- and G-rows of
// the panel and of V)
__host__ __device__ inline SolLayout sol_layout(int n, int m, int sb, bool fill = true) {
  SolLayout L;
  L.q = n > m ? n : m;
  L.R = fill ? 2 * n + m : n + m;
  L.ldL = L.q | 1;
  L.ldZ = n | 1;
  L.ldV = kRhsChunk | 1;
  int o = 0;
  for (int b = 0; b < 2; ++b) {
    L.oL[b] = o;
    o += kkt_align16(sb * L.q * L.ldL);
    L.oRinv[b] = o;
    o += kkt_align16(sb * L.q);
    L.oZ[b] = o;
    o += kkt_align16(sb * L.R * L.ldZ);
  }
  L.oV = o;
  L.oT = L.oV + kkt_align16(sb * L.R * L.ldV);
  L.total = L.oT + kkt_align16(sb * L.q * L.ldV);
  return L;
}

// Substitution of a system whose plan is one level with P = 1, one
// right-hand side, one warp per system (k_seq_solve): up to kSeqMaxBuf
// mbarriers, then `nbuf` buffers each holding one stage's n x n multipliers
// (unpadded; the forward ones transposed) and its n + m panel rows, both
// filled by bulk copies. sb = bytes per element (8 FP64, 4 FP32).
constexpr int kSeqMaxBuf = 4;
constexpr int kSeqHeader = 8 * kSeqMaxBuf;
constexpr int kSeqRing = 4;  // slots of right-hand-side rows (64 doubles each) after the buffers
__host__ __device__ inline int seq_zoff_bytes(int n, int sb) { return kkt_align16(sb * n * n); }
__host__ __device__ inline int seq_buf_bytes(int n, int m, int sb) {
  return seq_zoff_bytes(n, sb) + kkt_align16(sb * (n + m) * n);
}
__host__ __device__ inline int seq_slice_bytes(int n, int m, int sb, int nbuf) {
  return kSeqHeader + nbuf * seq_buf_bytes(n, m, sb) + kSeqRing * 64 * 8;
}
// Copies in flight: the deepest pipeline (up to kSeqMaxBuf buffers) with
// which every task of the launch still finds a place in the first wave
// (about 228 KB of shared memory per SM, one warp per CTA, at most 32 CTAs
// per SM), at least double buffering.
__host__ __device__ inline int seq_nbuf(int n, int m, int sb, int ntasks, int sms) {
  const int per_sm = (ntasks + (sms > 0 ? sms : 1) - 1) / (sms > 0 ? sms : 1);
  const int want = per_sm < 32 ? per_sm : 32;
  if ((228 * 1024) / (seq_slice_bytes(n, m, sb, kSeqMaxBuf) + 1024) >= want) return kSeqMaxBuf;
  return 2;  // (a power of two: buffer = visit & (nbuf - 1))
}
// Bulk copies move whole 16-byte units from 16-byte aligned addresses: every
// block a stage copies starts and ends on such a boundary when n is even and,
// for FP32 blocks, m n is a multiple of 4 (the panel of stage j starts at
// element j (2n + m) n).
__host__ __device__ inline bool seq_shape_ok(int n, int m, int sb) {
  return n >= 2 && n % 2 == 0 && n <= kMaxN && m <= kMaxM && (sb == 8 || (m * n) % 4 == 0);
}

// Residual kernel: stages per pass, as many (up to kResChunk) as fill the
// most lanes with up to three rows each (an FP64 instruction costs its issue
// slot with or without a row in the lane), and the x rows it stages per warp
// (the pass and one stage on either side).
constexpr int kResChunkStages = 8;  // (= kResChunk, defined below)
__host__ __device__ inline int res_spw(int n) {
  int best = 1, bn = 0, bd = 1;  // utilisation bn / bd of the best count so far
  for (int s = 1; s <= kResChunkStages && s * n <= 96; ++s) {
    const int rows = s * n, cap = 32 * ((rows + 31) / 32);
    if (rows * bd > bn * cap) { best = s; bn = rows; bd = cap; }
  }
  return best;
}
__host__ __device__ inline int res_xs_doubles(int n) { return (res_spw(n) + 2) * n; }

// Residual pass of iterative refinement: one CTA per chunk of kResChunk
// stages of one system.
constexpr int kResChunk = kResChunkStages;
struct ResTask {
  int desc;   // level-1 descriptor of the system
  int j0;     // first stage of the chunk
  int part;   // index of this chunk's partial-result slot within the system
  int nparts; // chunks of the system
};
// per-chunk partial results: g-rows (m x chunk) then max|r|, max|x|, max|b|,
// max row sum of |Psi| (chunk columns each)
constexpr int kResPartDoubles = kMaxM * kRhsChunk + 4 * kRhsChunk;

// Kernel launchers (kkt_kernels.cu). Each returns the cudaError_t of the launch.
// `mixed`: FP32 panel arithmetic in the factor; `pair`: every factor task runs
// on a cluster of two CTAs (chain and fill-in rows on separate SMs);
// `single`: FP32 substitution
// with the FP32 factor copy (mixed levels only); `skip`: per-system flags
// (null = never skip), a set flag makes the system's CTAs return at once.
// one warp per task (blocks n <= kWarpMaxN), several tasks per CTA
// (b, ldb: where the forward solution y of a bordered pass is written; unused otherwise)
// (fill: some task of the launch has fill-in rows; 0 sizes shared memory for
// the compact layout of levels with P = 1)
int launch_factor_w(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int mixed,
                    const double* D, const double* E, const double* G, const double* R, Info* info,
                    void* stream, double* b = nullptr, int ldb = 1, int fill = 1);
// (top_solve: on a bordered pass the top level's tasks also run their corner
// solve and backward sweep at the end of the factor kernel)
// (tc: Schur products of a mixed launch on the tensor cores, 1 = TF32, 2 = BF16
// operands, FP32 accumulation; used for blocks n >= 32 where the layout allows)
int launch_factor(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int mixed, int pair,
                  const double* D, const double* E, const double* G, const double* R, Info* info,
                  void* stream, double* b = nullptr, int ldb = 1, int fill = 1, int top_solve = 0, int tc = 0);
// The backward levels below the top in one launch (k_backward_chain): chain
// level li (0 = the level below the top, then down to level 1) holds the
// tasks [off[li], off[li] + its count) of the task array, each split into
// split[li] column groups; end[li] is the cumulative item count. ctr: nlev +
// 1 device ints (zeroed by the launcher); sms: the device's SM count (the
// grid is at most the CTAs resident at once).
constexpr int kChainMax = 32;
struct ChainPlan {
  int nlev;
  int off[kChainMax];
  int end[kChainMax];
  int split[kChainMax];
};
int launch_backward_chain(const LevelDesc* d, const Task* t, const ChainPlan& cp, int* ctr, int maxn, int maxm,
                          int single, double* b, int ldb, int nrhs, const int* skip, Info* info, long long wait,
                          int unmet, int sms, void* stream);
// One-stage segment tasks (FP64, fill-in rows) on clusters of C CTAs, 2 <= C
// <= 8 (k_factor_clus): bitwise the results of launch_factor.
// factor_clus_size: the largest C of 8, 4, 2 for which every cluster of the
// launch is resident at once (at most two CTAs per SM), 0 if none.
int factor_clus_size(int ntasks, int maxn, int maxm, int sms);
int launch_factor_clus(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int C, const double* D,
                       const double* E, const double* G, Info* info, void* stream, double* b = nullptr,
                       int ldb = 1);
// (split: CTAs per task, each on its own group of right-hand-side columns)
// (fill: some task's level has P > 1; 0 sizes shared memory for the compact
// layout of levels with P = 1)
int launch_forward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single,
                   double* b, int ldb, int nrhs, const int* skip, void* stream, int fwd_done = 0, int split = 1,
                   int fill = 1);
int launch_backward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single,
                    double* b, int ldb, int nrhs, const int* skip, void* stream, int split = 1, int fill = 1);
// one warp per task (blocks n <= kWarpMaxN), forward or backward substitution
int launch_solve_w(bool backward, const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single,
                   double* b, int ldb, int nrhs, const int* skip, void* stream, int fwd_done = 0, int fill = 1);
// whole substitution (Algorithms 2 and 3, corner of Eq. (7)) of systems
// whose level plan is one level with P = 1, one right-hand side, one warp per
// system; every system of the launch satisfies seq_shape_ok. A bulk copy
// that has not arrived within `wait` clock cycles records KKT_ERR_TIMEOUT in
// `info` and ends the system's task (`unmet`: every stage expects 16 bytes
// more than its copies deliver, so that every wait runs out).
// (sms: the device's SM count, for the pipeline depth; uniform: every system
// of the launch has n = maxn)
int launch_seq_solve(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single, double* b,
                     int ldb, const int* skip, Info* info, long long wait, int unmet, int sms, int uniform,
                     void* stream);
// bordered inputs of a fused factor-and-solve pass, for every system: Gb_j =
// [G_j; b_j^T] ((m+1) x n per stage), Rb = [[R, b_g], [b_g^T, 0]] ((m+1)^2)
// (stages [j0, j1) of every system's arrow, and with `corner` the bordered corners)
int launch_border(const LevelDesc* db, const int* sys_desc, int count, long long max_elems, const double* G,
                  const double* R, const double* b, int ldb, double* Gb, double* Rb, void* stream, int j0 = 0,
                  int j1 = 1 << 30, int corner = 1);
// x += c (stage rows per residual task, g rows by each system's first task)
int launch_axpy(const LevelDesc* d, const ResTask* t, int ntasks, double* x, int ldx, const double* c,
                int nr, const int* skip, void* stream);
// c = b - Psi x over the stage rows of each task (+ partials for the g rows
// and the max norms; the row sums of |Psi| only when `norms`, otherwise the
// values of an earlier call stay in `parts`); c has leading dimension kRhsChunk
// (xs_doubles: the largest res_xs_doubles over the systems, per warp; maxm:
// the largest m over the systems)
int launch_residual(const LevelDesc* d, const ResTask* t, int ntasks, const double* D, const double* E,
                    const double* G, const double* b, int ldb, const double* x, int ldx, double* c, int nr,
                    double* parts, const int* skip, int norms, void* stream, int xs_doubles,
                    int maxm = kMaxM);
// g rows of c, eta per system, converged[s] = (eta <= tol); a system that had
// converged before copies its eta from eta_prev (the previous sweep's; may be null)
// (stall: mark systems whose refinement stalls with flag 3 for the fallback)
int launch_residual_final(const LevelDesc* d, const int* sys_desc, const int* part0, int count,
                          const double* G, const double* R, const double* b, int ldb, const double* x,
                          int ldx, double* c, int nr, const double* parts, double tol, double* eta_out,
                          const double* eta_prev, int* converged, void* stream, int stall = 0);
// refinement fallback (preconditioned conjugate gradients): per-system dot
// products of vectors with leading dimension kRhsChunk (systems outside the
// fallback skipped), the x/r (mode 0) and p (mode 1) updates with per-system
// scalars num/den, and the skip mask of the fallback's solves and products
int launch_sys_dot(const LevelDesc* d, const int* sys_desc, const int* conv, int count, const double* u,
                   const double* v, int nr, double* out, void* stream);
int launch_pcg_update(const LevelDesc* d, const ResTask* t, int ntasks, const int* conv, int mode, int nr,
                      double* x, int ldx, double* r, const double* qn, double* p, const double* z,
                      const double* num, const double* den, void* stream);
int launch_pcg_mask(const int* conv, int* skip, int count, void* stream);
// adjoint block gradients (symmetric-entry convention) per residual task
int launch_adjoint_grad(const LevelDesc* d, const ResTask* t, int ntasks, const double* x, int ldx,
                        const double* xb, int ldxb, int nr, double* dD, double* dE, double* dG,
                        double* dR, void* stream);
// D (every system's stage blocks) <- identity blocks, R <- identity corners
int launch_fill_identity(const LevelDesc* d, const int* sys_desc, int count, double* D, double* R,
                         void* stream);
// Persistent factorization of a handle whose levels share one precision:
// items [0, nitems) over `grid` CTAs with `smem` bytes of shared memory;
// ready[0..nitems) and the ticket counter ready[nitems] must be zero; a
// dependency wait gives up after wait_cycles clock cycles (KKT_ERR_TIMEOUT).
// `slice`: shared memory of one warp task; `dbl`: the CTA tasks keep the
// second pivot buffer.
int launch_factor_persist(const LevelDesc* d, const Task* t, const PItem* items, int nitems, const PCons* cons,
                          int* ready, int mixed, const double* D, const double* E, const double* G,
                          const double* R, Info* info, int grid, size_t smem, int slice, int dbl,
                          long long wait_cycles, void* stream);
// the debug build's index-check record (status 8 on a failed check; zero in
// the normal build); `clear` resets it
int debug_info(Info* out, int clear);
// occupancy (CTAs per SM) of the persistent kernel with `smem` bytes
int persist_occupancy(int mixed, size_t smem);
size_t factor_smem_bytes(int maxn, int maxm, int mixed, int fill = 1, int dbl = 1);
size_t factor_w_slice_bytes(int maxn, int maxm, int mixed, int fill = 1);
size_t solve_smem_bytes(int maxn, int maxm, int single, int fill = 1);

}  // namespace kkt
