// Kernels of the partitioned block Cholesky factorization and solve of an SPD
// block-tridiagonal-arrow KKT matrix (arXiv 2511.00946, Algorithms 1-3).
//
// One CTA per segment task (kFactorThreads / kSolveThreads threads). Per stage the CTA keeps the pivot
// block, the stacked panel Z = [E; G; W] and the Schur accumulator T in
// shared memory (row-major, odd leading dimensions so that row- and
// column-wise accesses of FP64 words are free of bank conflicts) and runs
//   potrf(D)  ->  Z <- Z D-hat^{-T}  ->  T -= Z Z^T (lower triangle)
// with every thread on the element loops. FP64 is the scarce resource on this
// part (about 1/70 of the FP32 rate), so the loops are laid out to issue FP64
// instructions from full warps only: lower triangles are enumerated linearly
// instead of with a masked square.
#include <cuda_runtime.h>

#include "kkt_internal.h"

namespace kkt {
namespace {

__device__ __forceinline__ int odd(int c) { return c | 1; }

// Row-by-row enumeration of a lower triangle (diagonal included):
// e -> (a, b) with 0 <= b <= a, e = a(a+1)/2 + b.
__device__ __forceinline__ void tri_rc(int e, int& a, int& b) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > e) --r;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  a = r;
  b = e - r * (r + 1) / 2;
}

__device__ void record_breakdown(Info* info, int sys, int stage, int level) {
  if (atomicCAS(&info->status, 0, -1) == 0) {
    info->system = sys;
    info->stage = stage;
    info->level = level;
    __threadfence();
    atomicExch(&info->status, 3 /* KKT_ERR_NOT_SPD */);
  }
}

// dst (rows x cols, smem, ld) <- A (+ B) from global row-major [rows][cols],
// or the transpose of A (+ B) given as [cols][rows] when `trans`. A null A
// loads zeros. Coalesced over the global array.
__device__ void load_blk(double* dst, int ld, const double* A, const double* B, int rows, int cols,
                         bool trans) {
  const int tot = rows * cols;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int r, c;
    if (trans) { c = e / rows; r = e - c * rows; }
    else { r = e / cols; c = e - r * cols; }
    double v = 0.0;
    if (A) v = A[e];
    if (B) v += B[e];
    dst[r * ld + c] = v;
  }
}

// global row-major [rows][cols] <- src (smem), or the transpose when `trans`
// (dst is then [cols][rows]). `lower` writes zeros above the diagonal.
__device__ void store_blk(double* dst, const double* src, int ld, int rows, int cols, bool trans,
                          bool lower) {
  const int tot = rows * cols;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int r, c;
    if (trans) { c = e / rows; r = e - c * rows; }
    else { r = e / cols; c = e - r * cols; }
    double v = src[r * ld + c];
    if (lower && c > r) v = 0.0;
    dst[e] = v;
  }
}

// smem -> smem copy of a rows x cols block (lower triangle only when `lower`).
__device__ void copy_blk(double* dst, int ldd, const double* src, int lds, int rows, int cols) {
  for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
    const int r = e / cols, c = e - r * cols;
    dst[r * ldd + c] = src[r * lds + c];
  }
}

// 1/sqrt(d) for a pivot d > 0 in about five dependent FP64 operations instead
// of a square root and a division (each several hundred cycles on this part).
// The exponent is split off with integer operations so that d' = d 4^-k lies
// in [1, 4); a single-precision hardware estimate r ~ 1/sqrt(d') (relative
// error below 2^-21) is refined by one step of Halley's method for
// f(r) = r^-2 - d': with e = 1 - d' r^2, r <- r (1 + e/2 + 3 e^2 / 8), which
// leaves an error of order e^3 (below 2^-62), so the result is within a few
// units in the last place; finally r 2^-k. Returns NaN when d is not a
// positive finite normal number.
__device__ __forceinline__ double pivot_rsqrt(double d) {
  const long long bits = __double_as_longlong(d);
  const int ex = (int)((bits >> 52) & 0x7ff) - 1023;
  if (!(d > 0.0) || ex <= -1022 || ex >= 1023) return (d > 0.0 && d < 1e300) ? 1.0 / sqrt(d) : __longlong_as_double(0x7ff8000000000000LL);
  const int k = ex >> 1;  // floor(ex / 2)
  const double dp = __longlong_as_double(bits - ((long long)(2 * k) << 52));
  double r = (double)rsqrtf((float)dp);
  const double e = fma(-dp * r, r, 1.0);
  r = fma(r * e, fma(0.375, e, 0.5), r);
  return __longlong_as_double(__double_as_longlong(r) - ((long long)k << 52));
}

// In-place lower Cholesky of A (n x n). Writes rinv[j] = 1 / L_jj; on a pivot
// that is not positive, sets *bad (first column + 1) and carries on (NaNs
// propagate; no trap). Right-looking: per column a scalar pivot, a column
// scaling and a rank-1 update of the trailing lower triangle.
__device__ void potrf_sm(double* A, int ld, int n, double* rinv, int* bad) {
  const int tid = threadIdx.x;
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = A[j * ld + j];
      if (!(d > 0.0) && *bad == 0) *bad = j + 1;
      const double r = pivot_rsqrt(d);
      A[j * ld + j] = d * r;
      rinv[j] = r;
    }
    __syncthreads();
    const double r = rinv[j];
    const int w = n - 1 - j;
    for (int e = tid; e < w; e += blockDim.x) A[(j + 1 + e) * ld + j] *= r;
    __syncthreads();
    const int ntri = w * (w + 1) / 2;
    for (int e = tid; e < ntri; e += blockDim.x) {
      int a, b;
      tri_rc(e, a, b);
      const int i = j + 1 + a, k = j + 1 + b;
      A[i * ld + k] = fma(-A[i * ld + j], A[k * ld + j], A[i * ld + k]);
    }
    __syncthreads();
  }
}

// M[c][j] = L[c][j] / L[j][j] for c > j (strict lower triangle).
__device__ void scaled_cols(double* M, const double* L, int ld, int n, const double* rinv) {
  const int ntri = (n - 1) * n / 2;
  for (int e = threadIdx.x; e < ntri; e += blockDim.x) {
    int a, b;
    tri_rc(e, a, b);
    const int c = a + 1, j = b;
    M[c * ld + j] = L[c * ld + j] * rinv[j];
  }
}

// Z[r0:r1) <- Z[r0:r1) L^{-T}: column sweep with the pre-scaled columns M
// (x_j = b_j / L_jj; b_c -= x_j L_cj = b_j M_cj), then the diagonal scaling.
__device__ void trsm_panel(double* Z, int ldz, int r0, int r1, const double* M, int ldm, int n,
                           const double* rinv) {
  const int rows = r1 - r0;
  for (int j = 0; j < n - 1; ++j) {
    const int w = n - 1 - j, tot = rows * w;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int rr = e / w, c = j + 1 + (e - rr * w);
      double* zr = Z + (r0 + rr) * ldz;
      zr[c] = fma(-zr[j], M[c * ldm + j], zr[c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int rr = e / n, c = e - rr * n;
    Z[(r0 + rr) * ldz + c] *= rinv[c];
  }
  __syncthreads();
}

// T[i][j] -= sum_t Z[i][t] Z[j][t] for r0 <= j <= i < r1.
__device__ void syrk_panel(double* T, int ldt, const double* Z, int ldz, int r0, int r1, int n) {
  const int w = r1 - r0, ntri = w * (w + 1) / 2;
  for (int e = threadIdx.x; e < ntri; e += blockDim.x) {
    int a, b;
    tri_rc(e, a, b);
    const double* zi = Z + (r0 + a) * ldz;
    const double* zj = Z + (r0 + b) * ldz;
    double s0 = 0.0, s1 = 0.0;
    int t = 0;
    for (; t + 1 < n; t += 2) {
      s0 = fma(zi[t], zj[t], s0);
      s1 = fma(zi[t + 1], zj[t + 1], s1);
    }
    if (t < n) s0 = fma(zi[t], zj[t], s0);
    T[(r0 + a) * ldt + (r0 + b)] -= s0 + s1;
  }
  __syncthreads();
}

struct SegGeom {
  int f, len, hasW, hasF;
};

__device__ __forceinline__ SegGeom seg_geom(const LevelDesc& d, int k) {
  SegGeom g;
  g.f = d.seg[k];
  g.len = d.seg[k + 1] - d.seg[k] - 1;
  g.hasW = (k >= 1);
  g.hasF = (k < d.P - 1);
  return g;
}

// ---------------------------------------------------------------------------
// Factorization: Algorithm 1 for one segment (parallel phase); the top level
// (P = 1) is the sequential phase on the reduced system and also factors the
// corner R-hat = chol(R + sum of every R~_k partial).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFactorThreads) k_factor(const LevelDesc* __restrict__ descs,
                                                     const Task* __restrict__ tasks,
                                                     const double* __restrict__ uD,
                                                     const double* __restrict__ uE,
                                                     const double* __restrict__ uG,
                                                     const double* __restrict__ uR, Info* info) {
  extern __shared__ double sm[];
  __shared__ int bad;
  const Task tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  const int n = d.n, m = d.m, R = 2 * n + m;
  const FacLayout lay = fac_layout(n, m);
  const int ldD = odd(n), ldZ = lay.ldZ, ldT = lay.ldT;
  double* Dfac = sm + lay.oDfac;
  double* M = sm + lay.oM;
  double* rinv = sm + lay.oRinv;
  double* Z = sm + lay.oZ;
  double* T = sm + lay.oT;
  const int oG = n, oW = n + m;  // panel row offsets
  const SegGeom g = seg_geom(d, tk.seg);
  const int s = g.f - 1;  // separator of this segment (k >= 1)
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;

  // level inputs: the caller's arrays at level 1, the slots of the level above otherwise
  const double* Din = d.level == 1 ? uD + d.offD : d.Dw;
  const double* D2 = d.level == 1 ? nullptr : d.D2w;
  const double* Ein = d.level == 1 ? uE + d.offE : d.Ew;
  const double* Gin = d.level == 1 ? (m ? uG + d.offG : nullptr) : d.Gw;
  const double* G2 = d.level == 1 ? nullptr : d.G2w;
  auto Dp = [&](const double* b, int j) { return b ? b + (size_t)j * nn : nullptr; };
  auto Gp = [&](const double* b, int j) { return b ? b + (size_t)j * mn : nullptr; };

  if (threadIdx.x == 0) bad = 0;
  // zero T (accumulators start at zero unless initialised below)
  for (int e = threadIdx.x; e < R * ldT; e += blockDim.x) T[e] = 0.0;
  __syncthreads();
  load_blk(Dfac, ldD, Dp(Din, g.f), Dp(D2, g.f), n, n, false);
  if (g.len > 1 || g.hasF) load_blk(Z, ldZ, Dp(Ein, g.f), nullptr, n, n, false);
  if (m) load_blk(Z + oG * ldZ, ldZ, Gp(Gin, g.f), Gp(G2, g.f), m, n, false);
  if (g.hasW) {
    load_blk(Z + oW * ldZ, ldZ, Dp(Ein, s), nullptr, n, n, true);              // W_1 = B_k = E[s]^T
    load_blk(T + oW * ldT + oW, ldT, Dp(Din, s), Dp(D2, s), n, n, false);       // A_k
    if (m) load_blk(T + oW * ldT + oG, ldT, Gp(Gin, s), Gp(G2, s), n, m, true);  // Q_k^T
  }
  if (g.len > 1) {
    load_blk(T, ldT, Dp(Din, g.f + 1), Dp(D2, g.f + 1), n, n, false);          // D_{2}
    if (m) load_blk(T + oG * ldT, ldT, Gp(Gin, g.f + 1), Gp(G2, g.f + 1), m, n, false);
  }
  __syncthreads();

  for (int i = 0; i < g.len; ++i) {
    const int j = g.f + i;
    const bool eRows = (i < g.len - 1) || g.hasF;
    const int r0 = eRows ? 0 : n;
    const int r1 = n + m + (g.hasW ? n : 0);
    potrf_sm(Dfac, ldD, n, rinv, &bad);
    if (bad && threadIdx.x == 0) { record_breakdown(info, d.sys, d.nat[j], d.level); bad = 0; }
    scaled_cols(M, Dfac, ldD, n, rinv);
    __syncthreads();
    trsm_panel(Z, ldZ, r0, r1, M, ldD, n, rinv);
    // factor blocks of this stage
    store_blk(d.Ld + (size_t)j * nn, Dfac, ldD, n, n, false, true);
    store_blk(d.LdM + (size_t)j * nn, M, ldD, n, n, false, true);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {  // rows divided by their diagonal
      const int r = e / n, c = e - r * n;
      d.LdR[(size_t)j * nn + e] = c < r ? Dfac[r * ldD + c] * rinv[r] : 0.0;
    }
    for (int e = threadIdx.x; e < n; e += blockDim.x) d.Lri[(size_t)j * n + e] = rinv[e];
    {
      double* P = d.Lp + (size_t)j * R * n;
      for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        P[e] = (r >= r0 && r < r1) ? Z[r * ldZ + c] : 0.0;
      }
    }
    syrk_panel(T, ldT, Z, ldZ, r0, r1, n);
    if (i + 1 < g.len) {
      // rotate: the updated blocks become the next stage's inputs
      copy_blk(Dfac, ldD, T, ldT, n, n);                                       // D_{i+1}
      if (m) copy_blk(Z + oG * ldZ, ldZ, T + oG * ldT, ldT, m, n);             // G_{i+1}
      if (g.hasW) copy_blk(Z + oW * ldZ, ldZ, T + oW * ldT, ldT, n, n);        // W_{i+1}
      __syncthreads();
      if ((i + 1 < g.len - 1) || g.hasF) load_blk(Z, ldZ, Dp(Ein, j + 1), nullptr, n, n, false);
      if (i + 2 < g.len) {
        load_blk(T, ldT, Dp(Din, j + 2), Dp(D2, j + 2), n, n, false);
        if (m) load_blk(T + oG * ldT, ldT, Gp(Gin, j + 2), Gp(G2, j + 2), m, n, false);
      } else {
        load_blk(T, ldT, nullptr, nullptr, n, n, false);
        if (m) load_blk(T + oG * ldT, ldT, nullptr, nullptr, m, n, false);
      }
      if (g.hasW) load_blk(T + oW * ldT, ldT, nullptr, nullptr, n, n, false);  // W_{i+2} <- 0
      __syncthreads();
    }
  }

  if (!d.is_top) {
    const int k = tk.seg;
    if (g.hasF) {
      store_blk(d.DB + (size_t)k * nn, T, ldT, n, n, false, true);             // -F^ F^T
      if (m) store_blk(d.GB + (size_t)k * mn, T + oG * ldT, ldT, m, n, false, false);  // -G^ F^T
    }
    if (g.hasW) {
      store_blk(d.DA + (size_t)(k - 1) * nn, T + oW * ldT + oW, ldT, n, n, false, true);  // A~_k
      if (m) store_blk(d.GA + (size_t)(k - 1) * mn, T + oW * ldT + oG, ldT, n, m, true, false);  // Q~_k
      if (g.hasF) store_blk(d.EN + (size_t)(k - 1) * nn, T + oW * ldT, ldT, n, n, true, false);  // H~_k
    }
    if (m) store_blk(d.Rpart + (size_t)k * m * m, T + oG * ldT + oG, ldT, m, m, false, true);
  } else if (m) {
    // corner: R-hat = chol(R + sum_k R~_k over every level), in a fixed order
    double* Rs = Dfac;  // reuse
    const int ldR = odd(m);
    const double* Ru = uR + d.offR;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = e / m, c = e - r * m;
      double v = Ru[e];
      for (int p = 0; p < d.nRpart_all; ++p) v += d.Rpart_all[(size_t)p * m * m + e];
      v += T[(oG + r) * ldT + oG + c];
      Rs[r * ldR + c] = v;
    }
    __syncthreads();
    potrf_sm(Rs, ldR, m, rinv, &bad);
    if (bad && threadIdx.x == 0) record_breakdown(info, d.sys, d.Nnat, d.level);
    store_blk(d.Rhat, Rs, ldR, m, m, false, true);
    for (int e = threadIdx.x; e < m; e += blockDim.x) d.Rri[e] = rinv[e];
  }
}

// ---------------------------------------------------------------------------
// Solve
// ---------------------------------------------------------------------------

// rhs / solution rows of stage j at this level: the caller's b at level 1
// (rows offB + j n, stride ldb), this level's X array otherwise.
struct VecView {
  double* p;
  int ld;
};

__device__ __forceinline__ VecView level_vec(const LevelDesc& d, double* b, int ldb, int j) {
  VecView v;
  if (d.level == 1) { v.p = b + (size_t)(d.offB + (long long)j * d.n) * ldb; v.ld = ldb; }
  else { v.p = d.X + (size_t)j * d.n * kRhsChunk; v.ld = kRhsChunk; }
  return v;
}

// dst (rows x nr, smem ld) <- src rows (global, stride lds) (+ src2, stride kRhsChunk)
__device__ void load_vec(double* dst, int ldd, const double* src, int lds, const double* src2,
                         int rows, int nr) {
  for (int e = threadIdx.x; e < rows * nr; e += blockDim.x) {
    const int r = e / nr, c = e - r * nr;
    double v = src ? src[(size_t)r * lds + c] : 0.0;
    if (src2) v += src2[(size_t)r * kRhsChunk + c];
    dst[r * ldd + c] = v;
  }
}

__device__ void store_vec(double* dst, int ldd, const double* src, int lds, int rows, int nr) {
  for (int e = threadIdx.x; e < rows * nr; e += blockDim.x) {
    const int r = e / nr, c = e - r * nr;
    dst[(size_t)r * ldd + c] = src[r * lds + c];
  }
}

// t <- L^{-1} t for L = M diag(1/rinv) (M: the columns of L divided by their
// diagonal, strict lower part used), nr columns: t_i -= M_ij t_j for the
// unscaled t_j, then t_j *= rinv_j.
__device__ void trsv_lower(double* t, int ldt, const double* M, int ldl, const double* rinv, int n,
                           int nr) {
  for (int j = 0; j < n - 1; ++j) {
    const int w = n - 1 - j, tot = w * nr;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int a = e / nr, c = e - a * nr, i = j + 1 + a;
      t[i * ldt + c] = fma(-M[i * ldl + j], t[j * ldt + c], t[i * ldt + c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
    const int r = e / nr, c = e - r * nr;
    t[r * ldt + c] *= rinv[r];
  }
  __syncthreads();
}

// t <- L^{-T} t with MR, the rows of L divided by their diagonal: x_j =
// t_j rinv_j once t_j is final, and t_i -= L_ji x_j = MR_ji t_j (unscaled t_j)
// for i < j.
__device__ void trsv_upper(double* t, int ldt, const double* M, int ldl, const double* rinv, int n,
                           int nr) {
  for (int j = n - 1; j > 0; --j) {
    for (int e = threadIdx.x; e < j * nr; e += blockDim.x) {
      const int i = e / nr, c = e - i * nr;
      t[i * ldt + c] = fma(-M[j * ldl + i], t[j * ldt + c], t[i * ldt + c]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
    const int r = e / nr, c = e - r * nr;
    t[r * ldt + c] *= rinv[r];
  }
  __syncthreads();
}

struct SolveSmem {
  double *L, *rinv, *Z, *V, *t;
  int ldL, ldZ, ldV;
};

__device__ __forceinline__ SolveSmem solve_smem(double* sm, int n, int m) {
  SolveSmem S;
  const SolLayout L = sol_layout(n, m);
  S.ldL = odd(n);
  S.ldZ = L.ldZ;
  S.ldV = L.ldV;
  S.L = sm + L.oL;
  S.rinv = sm + L.oRinv;
  S.Z = sm + L.oZ;
  S.V = sm + L.oV;
  S.t = sm + L.oT;
  return S;
}

// load the factor blocks of stage j (D-hat with its columns (forward) or rows
// (backward) divided by the diagonal, 1/diag, panel rows [r0, r1))
__device__ void load_stage_factor(const SolveSmem& S, const LevelDesc& d, int j, int r0, int r1,
                                  bool backward) {
  const int n = d.n, R = 2 * n + d.m;
  const double* Lg = (backward ? d.LdR : d.LdM) + (size_t)j * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    S.L[r * S.ldL + c] = Lg[e];
  }
  for (int e = threadIdx.x; e < n; e += blockDim.x) S.rinv[e] = d.Lri[(size_t)j * n + e];
  const double* P = d.Lp + (size_t)j * R * n;
  for (int e = threadIdx.x + r0 * n; e < r1 * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    S.Z[r * S.ldZ + c] = P[e];
  }
}

// Backward substitution over the stages of one segment (Algorithm 3,
// parallel phase; for the top level the whole sequential sweep). On entry
// S.V holds [x_next (E rows); x_g (G rows); x_sep (W rows)].
__device__ void backward_segment(const SolveSmem& S, const LevelDesc& d, const SegGeom& g,
                                 double* b, int ldb, int nr) {
  const int n = d.n, m = d.m;
  for (int i = g.len - 1; i >= 0; --i) {
    const int j = g.f + i;
    const bool eRows = (i < g.len - 1) || g.hasF;
    const int r0 = eRows ? 0 : n, r1 = n + m + (g.hasW ? n : 0);
    load_stage_factor(S, d, j, r0, r1, true);
    const VecView y = level_vec(d, b, ldb, j);
    __syncthreads();
    // t = y_j - Z^T v over the active panel rows
    for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
      const int c2 = e / nr, c = e - c2 * nr;
      double acc = y.p[(size_t)c2 * y.ld + c];
      for (int r = r0; r < r1; ++r) acc = fma(-S.Z[r * S.ldZ + c2], S.V[r * S.ldV + c], acc);
      S.t[c2 * S.ldV + c] = acc;
    }
    __syncthreads();
    trsv_upper(S.t, S.ldV, S.L, S.ldL, S.rinv, n, nr);
    store_vec(y.p, y.ld, S.t, S.ldV, n, nr);
    for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
      const int r = e / nr, c = e - r * nr;
      S.V[r * S.ldV + c] = S.t[r * S.ldV + c];
    }
    __syncthreads();
  }
}

// Forward substitution (Algorithm 2) for one segment; the top level (P = 1)
// also solves the corner and runs its own backward sweep (Algorithm 3,
// sequential phase).
__global__ void __launch_bounds__(kSolveThreads) k_forward(const LevelDesc* __restrict__ descs,
                                                      const Task* __restrict__ tasks, double* b,
                                                      int ldb, int nr) {
  extern __shared__ double sm[];
  const Task tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  const int n = d.n, m = d.m;
  const SolveSmem S = solve_smem(sm, n, m);
  const int oG = n, oW = n + m;
  const SegGeom g = seg_geom(d, tk.seg);
  const int k = tk.seg;
  auto rhs = [&](int j, double* dst) {  // this level's right-hand side of stage j
    if (d.level == 1) {
      const VecView v = level_vec(d, b, ldb, j);
      load_vec(dst, S.ldV, v.p, v.ld, nullptr, n, nr);
    } else {
      load_vec(dst, S.ldV, d.RA + (size_t)j * n * kRhsChunk, kRhsChunk,
               d.RB + (size_t)j * n * kRhsChunk, n, nr);
    }
  };
  // V_G <- 0, V_W <- rhs of the separator, t <- rhs of the first stage
  for (int e = threadIdx.x; e < (2 * n + m) * S.ldV; e += blockDim.x) S.V[e] = 0.0;
  __syncthreads();
  if (g.hasW) rhs(g.f - 1, S.V + oW * S.ldV);
  rhs(g.f, S.t);
  __syncthreads();
  for (int i = 0; i < g.len; ++i) {
    const int j = g.f + i;
    const bool eRows = (i < g.len - 1) || g.hasF;
    const int r0 = eRows ? 0 : n, r1 = n + m + (g.hasW ? n : 0);
    load_stage_factor(S, d, j, r0, r1, false);
    if (i + 1 < g.len) rhs(j + 1, S.V);  // V_E <- next stage's rhs (else 0: F-hat term)
    __syncthreads();
    trsv_lower(S.t, S.ldV, S.L, S.ldL, S.rinv, n, nr);
    const VecView y = level_vec(d, b, ldb, j);
    store_vec(y.p, y.ld, S.t, S.ldV, n, nr);
    // [V_E; V_G; V_W] -= Z y over the active panel rows
    for (int e = threadIdx.x; e < (r1 - r0) * nr; e += blockDim.x) {
      const int r = r0 + e / nr, c = e - (e / nr) * nr;
      double acc = 0.0;
      for (int t2 = 0; t2 < n; ++t2) acc = fma(S.Z[r * S.ldZ + t2], S.t[t2 * S.ldV + c], acc);
      S.V[r * S.ldV + c] -= acc;
    }
    __syncthreads();
    if (i + 1 < g.len) {
      for (int e = threadIdx.x; e < n * nr; e += blockDim.x) {
        const int r = e / nr, c = e - r * nr;
        S.t[r * S.ldV + c] = S.V[r * S.ldV + c];
        S.V[r * S.ldV + c] = 0.0;
      }
      __syncthreads();
    }
  }
  if (!d.is_top) {
    if (g.hasF) store_vec(d.YB + (size_t)k * n * kRhsChunk, kRhsChunk, S.V, S.ldV, n, nr);
    if (g.hasW) store_vec(d.YA + (size_t)(k - 1) * n * kRhsChunk, kRhsChunk, S.V + oW * S.ldV, S.ldV, n, nr);
    if (m) store_vec(d.ygpart + (size_t)k * m * kRhsChunk, kRhsChunk, S.V + oG * S.ldV, S.ldV, m, nr);
    return;
  }
  // top level: corner y_g = R-hat^{-1} (r_g + sum of every yg partial + own),
  // x_g = R-hat^{-T} y_g, written to the caller's b; then the backward sweep.
  if (m) {
    double* bg = b + (size_t)d.rowG * ldb;
    double* gv = S.t;
    const int ldR = odd(m);
    for (int e = threadIdx.x; e < m * nr; e += blockDim.x) {
      const int r = e / nr, c = e - r * nr;
      double v = bg[(size_t)r * ldb + c];
      for (int p = 0; p < d.nyg_all; ++p) v += d.yg_all[((size_t)p * m + r) * kRhsChunk + c];
      v += S.V[(oG + r) * S.ldV + c];
      gv[r * S.ldV + c] = v;
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {  // R-hat, columns scaled
      const int r = e / m, c = e - r * m;
      S.L[r * ldR + c] = d.Rhat[e] * d.Rri[c];
    }
    for (int e = threadIdx.x; e < m; e += blockDim.x) S.rinv[e] = d.Rri[e];
    __syncthreads();
    trsv_lower(gv, S.ldV, S.L, ldR, S.rinv, m, nr);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {  // R-hat, rows scaled
      const int r = e / m, c = e - r * m;
      S.L[r * ldR + c] = d.Rhat[e] * d.Rri[r];
    }
    __syncthreads();
    trsv_upper(gv, S.ldV, S.L, ldR, S.rinv, m, nr);
    store_vec(bg, ldb, gv, S.ldV, m, nr);
  }
  // V <- [0; x_g; -] for the backward sweep of the top level
  for (int e = threadIdx.x; e < (2 * n + m) * S.ldV; e += blockDim.x) {
    const int r = e / S.ldV;
    if (r < oG || r >= oW) S.V[e] = 0.0;
    else S.V[e] = S.t[(r - oG) * S.ldV + (e - r * S.ldV)];
  }
  __syncthreads();
  backward_segment(S, d, g, b, ldb, nr);
}

// Backward substitution (Algorithm 3, parallel phase) for one segment below
// the top level: needs x_g (already in b), the separator solutions of the
// next level (x at s_k and s_{k+1}), and this level's y.
__global__ void __launch_bounds__(kSolveThreads) k_backward(const LevelDesc* __restrict__ descs,
                                                       const Task* __restrict__ tasks, double* b,
                                                       int ldb, int nr) {
  extern __shared__ double sm[];
  const Task tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  const int n = d.n, m = d.m;
  const SolveSmem S = solve_smem(sm, n, m);
  const int oG = n, oW = n + m;
  const SegGeom g = seg_geom(d, tk.seg);
  const int k = tk.seg;
  for (int e = threadIdx.x; e < (2 * n + m) * S.ldV; e += blockDim.x) S.V[e] = 0.0;
  __syncthreads();
  if (g.hasF) load_vec(S.V, S.ldV, d.Xnext + (size_t)k * n * kRhsChunk, kRhsChunk, nullptr, n, nr);
  if (m) load_vec(S.V + oG * S.ldV, S.ldV, b + (size_t)d.rowG * ldb, ldb, nullptr, m, nr);
  if (g.hasW) {
    load_vec(S.V + oW * S.ldV, S.ldV, d.Xnext + (size_t)(k - 1) * n * kRhsChunk, kRhsChunk, nullptr,
             n, nr);
    __syncthreads();
    const VecView xs = level_vec(d, b, ldb, g.f - 1);  // this level's copy of x at s_k
    store_vec(xs.p, xs.ld, S.V + oW * S.ldV, S.ldV, n, nr);
  }
  __syncthreads();
  backward_segment(S, d, g, b, ldb, nr);
}

}  // namespace

size_t factor_smem_bytes(int n, int m) { return (size_t)fac_layout(n, m).total * sizeof(double); }

size_t solve_smem_bytes(int n, int m) { return (size_t)sol_layout(n, m).total * sizeof(double); }

static int set_smem(const void* fn, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return (int)e;
}

int launch_factor(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm,
                  const double* D, const double* E, const double* G, const double* R, Info* info,
                  void* stream) {
  if (ntasks <= 0) return 0;
  const size_t sm = factor_smem_bytes(maxn, maxm);
  int e = set_smem((const void*)k_factor, sm);
  if (e) return e;
  k_factor<<<ntasks, kFactorThreads, sm, (cudaStream_t)stream>>>(d, t, D, E, G, R, info);
  return (int)cudaGetLastError();
}

int launch_forward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, double* b,
                   int ldb, int nrhs, const double* R, void* stream) {
  (void)R;
  if (ntasks <= 0) return 0;
  const size_t sm = solve_smem_bytes(maxn, maxm);
  int e = set_smem((const void*)k_forward, sm);
  if (e) return e;
  k_forward<<<ntasks, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, b, ldb, nrhs);
  return (int)cudaGetLastError();
}

int launch_backward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, double* b,
                    int ldb, int nrhs, void* stream) {
  if (ntasks <= 0) return 0;
  const size_t sm = solve_smem_bytes(maxn, maxm);
  int e = set_smem((const void*)k_backward, sm);
  if (e) return e;
  k_backward<<<ntasks, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, b, ldb, nrhs);
  return (int)cudaGetLastError();
}

}  // namespace kkt
