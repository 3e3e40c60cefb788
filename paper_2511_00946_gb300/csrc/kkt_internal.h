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
  // mixed precision: FP32 copies of the factor used by the refinement solve
  float* Lp32;
};

struct Task {
  int desc;  // index into the LevelDesc array
  int seg;   // segment index k (0-based)
};

// Device-side breakdown record (kkt_info layout).
struct Info {
  int status, system, stage, level;
};

// Shared-memory layouts (in doubles), identical on host and device. Square
// buffers are sized for q = max(n, m) because the corner (m x m) reuses them.
// Odd leading dimensions keep row- and column-wise FP64 accesses conflict-free.
struct FacLayout {
  int q, R, ldD, ldZ, ldT, oDfac, oM, oRinv, oZ, oT, total;
};
__host__ __device__ inline FacLayout fac_layout(int n, int m) {
  FacLayout L;
  L.q = n > m ? n : m;
  L.R = 2 * n + m;
  L.ldD = L.q | 1;
  L.ldZ = n | 1;
  L.ldT = L.R | 1;
  L.oDfac = 0;
  L.oM = L.oDfac + L.q * L.ldD;
  L.oRinv = L.oM + n * L.ldD;
  L.oZ = L.oRinv + ((L.q + 1) & ~1);
  L.oT = L.oZ + L.R * L.ldZ;
  L.total = L.oT + L.R * L.ldT;
  return L;
}
struct SolLayout {
  int q, R, ldL, ldZ, ldV, oL, oRinv, oZ, oV, oT, total;
};
__host__ __device__ inline SolLayout sol_layout(int n, int m) {
  SolLayout L;
  L.q = n > m ? n : m;
  L.R = 2 * n + m;
  L.ldL = L.q | 1;
  L.ldZ = n | 1;
  L.ldV = kRhsChunk | 1;
  L.oL = 0;
  L.oRinv = L.oL + L.q * L.ldL;
  L.oZ = L.oRinv + ((L.q + 1) & ~1);
  L.oV = L.oZ + L.R * L.ldZ;
  L.oT = L.oV + L.R * L.ldV;
  L.total = L.oT + L.q * L.ldV;
  return L;
}

// Kernel launchers (kkt_kernels.cu). Each returns the cudaError_t of the launch.
int launch_factor(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm,
                  const double* D, const double* E, const double* G, const double* R, Info* info,
                  void* stream);
int launch_forward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, double* b,
                   int ldb, int nrhs, const double* R, void* stream);
int launch_backward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, double* b,
                    int ldb, int nrhs, void* stream);
size_t factor_smem_bytes(int maxn, int maxm);
size_t solve_smem_bytes(int maxn, int maxm);

}  // namespace kkt
