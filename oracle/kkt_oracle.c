/*
 * FP64 CPU oracle for the block-tridiagonal-arrow KKT solve of
 * "Parallel KKT Solver in PIQP for Multistage Optimization" (arXiv 2511.00946).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU baseline
 * use it. It shares no code, header, table or constant with the CUDA library.
 *
 * Plain, slow, obviously-correct loops in double precision. No BLAS, no LAPACK,
 * no blocking, no reordering beyond what the paper's algorithms state.
 *
 * Three parts:
 *   O1  dense Cholesky and dense triangular solves of the assembled matrix
 *       (the textbook definition; for tiny systems).
 *   O2  sequential block factorization and solve in natural stage order: the
 *       block equations of Psi = L L^T for the block-bidiagonal-arrow L
 *       (the sequential method the paper compares against, Sec. 3.3).
 *   O3  the partitioned method: Algorithm 1 (parallel + sequential phase of the
 *       factorization), Algorithm 2 (forward substitution) and Algorithm 3
 *       (backward substitution), with the readings listed in the design notes
 *       (hatted quantities are in-place buffers; R-hat starts at Psi_gg; the
 *       g-partials accumulate; the F-hat terms pair F-hat_k with separator k+1).
 *
 * Layout (all row-major, natural stage order j = 0..N-1, stage block size n,
 * arrow width m >= 0):
 *   D [N][n][n]   Psi_{j,j}      (lower triangle read)
 *   E [N-1][n][n] Psi_{j+1,j}
 *   G [N][m][n]   Psi_{g,j}
 *   R [m][m]      Psi_{g,g}      (lower triangle read)
 *   b [N*n+m][nrhs]
 *
 * Flop counters: every primitive adds its count in two conventions, the
 * paper's (Algorithm 1-3 comments and Table 1: potrf b^3/3, trsm rows*b^2,
 * syrk rows^2*k, gemm 2rck, trsv b^2/2, gemv 2rc) and the standard one
 * (potrf n^3/3+n^2/2+n/6, trsm rows*n^2, syrk n(n+1)k, gemm 2rck, trsv n^2,
 * gemv 2rc). Counters are thread-local.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------------ */
/* flop counters                                                             */
/* ------------------------------------------------------------------------ */
static _Thread_local double fl_paper = 0.0, fl_std = 0.0;

void orc_flops_reset(void) { fl_paper = 0.0; fl_std = 0.0; }
void orc_flops_get(double* paper, double* standard) { *paper = fl_paper; *standard = fl_std; }

/* ------------------------------------------------------------------------ */
/* small dense primitives on row-major blocks with explicit leading dims     */
/* ------------------------------------------------------------------------ */

/* In-place lower Cholesky of the n x n block A (lower triangle read and
 * written, strictly-upper part set to zero). Returns 0, or j+1 when the pivot
 * of column j is not positive (or not finite). Column-by-column (Crout) form. */
static int potrf(int n, double* A, int lda) {
  double dn = n;
  fl_paper += dn * dn * dn / 3.0;
  fl_std += dn * dn * dn / 3.0 + dn * dn / 2.0 + dn / 6.0;
  for (int j = 0; j < n; ++j) {
    double d = A[j * lda + j];
    for (int k = 0; k < j; ++k) d -= A[j * lda + k] * A[j * lda + k];
    if (!(d > 0.0) || !isfinite(d)) return j + 1;
    d = sqrt(d);
    A[j * lda + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * lda + j];
      for (int k = 0; k < j; ++k) s -= A[i * lda + k] * A[j * lda + k];
      A[i * lda + j] = s / d;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A[i * lda + j] = 0.0;
  return 0;
}

/* B <- B L^{-T} for B (rows x n) and lower-triangular L (n x n):
 * each row x of the result solves L x^T = b^T by forward substitution. */
static void trsm_rlt(int rows, int n, const double* L, int ldl, double* B, int ldb) {
  fl_paper += (double)rows * n * n;
  fl_std += (double)rows * n * n;
  for (int r = 0; r < rows; ++r) {
    double* x = B + (size_t)r * ldb;
    for (int j = 0; j < n; ++j) {
      double s = x[j];
      for (int k = 0; k < j; ++k) s -= L[j * ldl + k] * x[k];
      x[j] = s / L[j * ldl + j];
    }
  }
}

/* C (r x r, lower triangle) <- C + alpha * A A^T for A (r x k). */
static void syrk_ln(int r, int k, double alpha, const double* A, int lda, double* C, int ldc) {
  fl_paper += (double)r * r * k;
  fl_std += (double)r * (r + 1) * k;
  for (int i = 0; i < r; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += A[i * lda + t] * A[j * lda + t];
      C[i * ldc + j] += alpha * s;
    }
}

/* C (r x c) <- C + alpha * A B^T for A (r x k), B (c x k). */
static void gemm_nt(int r, int c, int k, double alpha, const double* A, int lda,
                    const double* B, int ldb, double* C, int ldc) {
  fl_paper += 2.0 * r * c * k;
  fl_std += 2.0 * r * c * k;
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += A[i * lda + t] * B[j * ldb + t];
      C[i * ldc + j] += alpha * s;
    }
}

/* x <- L^{-1} x (forward substitution), L lower n x n. */
static void trsv_ln(int n, const double* L, int ldl, double* x) {
  fl_paper += (double)n * n / 2.0;
  fl_std += (double)n * n;
  for (int i = 0; i < n; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * ldl + k] * x[k];
    x[i] = s / L[i * ldl + i];
  }
}

/* x <- L^{-T} x (backward substitution), L lower n x n. */
static void trsv_lt(int n, const double* L, int ldl, double* x) {
  fl_paper += (double)n * n / 2.0;
  fl_std += (double)n * n;
  for (int i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * ldl + i] * x[k];
    x[i] = s / L[i * ldl + i];
  }
}

/* y (r) <- y + alpha * A x for A (r x c). */
static void gemv_n(int r, int c, double alpha, const double* A, int lda, const double* x, double* y) {
  fl_paper += 2.0 * r * c;
  fl_std += 2.0 * r * c;
  for (int i = 0; i < r; ++i) {
    double s = 0.0;
    for (int t = 0; t < c; ++t) s += A[i * lda + t] * x[t];
    y[i] += alpha * s;
  }
}

/* y (c) <- y + alpha * A^T x for A (r x c). */
static void gemv_t(int r, int c, double alpha, const double* A, int lda, const double* x, double* y) {
  fl_paper += 2.0 * r * c;
  fl_std += 2.0 * r * c;
  for (int j = 0; j < c; ++j) {
    double s = 0.0;
    for (int t = 0; t < r; ++t) s += A[t * lda + j] * x[t];
    y[j] += alpha * s;
  }
}

/* ------------------------------------------------------------------------ */
/* O1: dense Cholesky of the assembled matrix (textbook definition)          */
/* ------------------------------------------------------------------------ */

/* L (dim x dim) <- chol(A): L[j][j] = sqrt(A[j][j] - sum_k L[j][k]^2),
 * L[i][j] = (A[i][j] - sum_k L[i][k] L[j][k]) / L[j][j]. Returns 0 or j+1. */
int orc_dense_chol(int dim, const double* A, double* L) {
  memset(L, 0, sizeof(double) * (size_t)dim * dim);
  for (int j = 0; j < dim; ++j) {
    double d = A[(size_t)j * dim + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * dim + k] * L[(size_t)j * dim + k];
    if (!(d > 0.0) || !isfinite(d)) return j + 1;
    d = sqrt(d);
    L[(size_t)j * dim + j] = d;
    for (int i = j + 1; i < dim; ++i) {
      double s = A[(size_t)i * dim + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * dim + k] * L[(size_t)j * dim + k];
      L[(size_t)i * dim + j] = s / d;
    }
  }
  return 0;
}

/* x <- (L L^T)^{-1} x for a dense lower L, one right-hand side. */
void orc_dense_solve(int dim, const double* L, double* x) {
  for (int i = 0; i < dim; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * dim + k] * x[k];
    x[i] = s / L[(size_t)i * dim + i];
  }
  for (int i = dim - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < dim; ++k) s -= L[(size_t)k * dim + i] * x[k];
    x[i] = s / L[(size_t)i * dim + i];
  }
}

/* ------------------------------------------------------------------------ */
/* Partition rule, Sec. 3.3, Eq. (13)                                        */
/* ------------------------------------------------------------------------ */

/* Segment lengths for N stage blocks over P segments. The balance ratio
 * sigma = N_1/N_k = 19/7 equates the first segment's (7/3 N_1) and the other
 * segments' (19/3 N_k) leading flop terms (Table 1). The constraint
 * N_1 + (P-1) N_k + P - 1 = N gives the ideal N_k = (N-P+1)/(P-1+sigma); the
 * rounding (floor or ceil) with the smaller max(7/3 N_1, 19/3 N_k) wins, the
 * floor on a tie. Returns 0, or -1 when P < 1 or P > floor((N+1)/2) (no
 * partition with every N_k >= 1 and N_1 >= 1 exists), or -2 when N < 1. */
int orc_partition(int N, int P, int* seg_len) {
  if (N < 1) return -2;
  if (P < 1) return -1;
  if (P > 1 && P > (N + 1) / 2) return -1;
  if (P == 1) { seg_len[0] = N; return 0; }
  const double sigma = 19.0 / 7.0;
  double nbar = (double)(N - P + 1) / ((double)(P - 1) + sigma);
  int cand[2] = {(int)floor(nbar), (int)ceil(nbar)};
  int best_nk = -1;
  double best_cost = 0.0;
  for (int c = 0; c < 2; ++c) {
    int nk = cand[c];
    if (nk < 1) continue;
    int n1 = N - (P - 1) * (nk + 1);
    if (n1 < 1) continue;
    double cost = fmax(7.0 / 3.0 * n1, 19.0 / 3.0 * nk);
    if (best_nk < 0 || cost < best_cost) { best_nk = nk; best_cost = cost; }
  }
  if (best_nk < 0) return -1;
  seg_len[0] = N - (P - 1) * (best_nk + 1);
  for (int k = 1; k < P; ++k) seg_len[k] = best_nk;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* O2: sequential block factorization in natural order                       */
/* ------------------------------------------------------------------------ */

/* Block equations of Psi = L L^T for L block-bidiagonal-arrow:
 *   L_jj L_jj^T = D_j - L_{j,j-1} L_{j,j-1}^T
 *   L_{j+1,j}   = E_j L_jj^{-T}
 *   L_{g,j}     = (G_j - L_{g,j-1} L_{j,j-1}^T) L_jj^{-T}
 *   L_gg L_gg^T = R - sum_j L_{g,j} L_{g,j}^T
 * Outputs Ld [N][n][n], Le [N-1][n][n], Lg [N][m][n], Lr [m][m].
 * Returns 0, or a breakdown code: -(j+1) when the pivot block of stage j is not
 * positive definite, -(N+1) for the corner block. */
int orc_seq_factor(int N, int n, int m, const double* D, const double* E, const double* G,
                   const double* R, double* Ld, double* Le, double* Lg, double* Lr) {
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  for (int j = 0; j < N; ++j) {
    double* Lj = Ld + j * nn;
    memcpy(Lj, D + j * nn, sizeof(double) * nn);
    if (j > 0) syrk_ln(n, n, -1.0, Le + (j - 1) * nn, n, Lj, n);
    if (potrf(n, Lj, n)) return -(j + 1);
    if (j < N - 1) {
      memcpy(Le + j * nn, E + j * nn, sizeof(double) * nn);
      trsm_rlt(n, n, Lj, n, Le + j * nn, n);
    }
    if (m > 0) {
      memcpy(Lg + j * mn, G + j * mn, sizeof(double) * mn);
      if (j > 0) gemm_nt(m, n, n, -1.0, Lg + (j - 1) * mn, n, Le + (j - 1) * nn, n, Lg + j * mn, n);
      trsm_rlt(m, n, Lj, n, Lg + j * mn, n);
    }
  }
  if (m > 0) {
    memcpy(Lr, R, sizeof(double) * (size_t)m * m);
    for (int j = 0; j < N; ++j) syrk_ln(m, n, -1.0, Lg + j * mn, n, Lr, m);
    if (potrf(m, Lr, m)) return -(N + 1);
  }
  return 0;
}

/* b [(N n + m)][nrhs] <- Psi^{-1} b using the O2 factor: block forward
 * substitution L y = b, then block backward substitution L^T x = y. */
void orc_seq_solve(int N, int n, int m, const double* Ld, const double* Le, const double* Lg,
                   const double* Lr, double* b, int nrhs) {
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  const int dim = N * n + m;
  double* v = (double*)malloc(sizeof(double) * (size_t)dim);
  for (int c = 0; c < nrhs; ++c) {
    for (int i = 0; i < dim; ++i) v[i] = b[(size_t)i * nrhs + c];
    double* vg = v + (size_t)N * n;
    for (int j = 0; j < N; ++j) {
      double* vj = v + (size_t)j * n;
      if (j > 0) gemv_n(n, n, -1.0, Le + (j - 1) * nn, n, vj - n, vj);
      trsv_ln(n, Ld + j * nn, n, vj);
      if (m > 0) gemv_n(m, n, -1.0, Lg + j * mn, n, vj, vg);
    }
    if (m > 0) { trsv_ln(m, Lr, m, vg); trsv_lt(m, Lr, m, vg); }
    for (int j = N - 1; j >= 0; --j) {
      double* vj = v + (size_t)j * n;
      if (m > 0) gemv_t(m, n, -1.0, Lg + j * mn, n, vg, vj);
      if (j < N - 1) gemv_t(n, n, -1.0, Le + j * nn, n, vj + n, vj);
      trsv_lt(n, Ld + j * nn, n, vj);
    }
    for (int i = 0; i < dim; ++i) b[(size_t)i * nrhs + c] = v[i];
  }
  free(v);
}

/* ------------------------------------------------------------------------ */
/* O3: partitioned method, Algorithms 1-3                                    */
/* ------------------------------------------------------------------------ */

/* Stage index map of a partition: segment k (0-based) covers stages
 * f[k] .. f[k]+len[k]-1; for k >= 1 its separator is stage f[k]-1. */
static void seg_map(int P, const int* len, int* f) {
  f[0] = 0;
  for (int k = 1; k < P; ++k) f[k] = f[k - 1] + len[k - 1] + 1;
}

/* Factor storage in natural stage order (sizes as for O2 plus two extra
 * stage-indexed arrays):
 *   Ld[j]  D-hat at segment stages, A-hat_k at separator s_k
 *   Le[j]  E-hat (j, j+1 in one segment); F-hat_k at j = last stage of
 *          segment k (it couples separator k+1 to that stage)
 *   Lw[j]  fill-in W = L-hat(s_k, j) (the paper's B-hat^T) at the stages j of
 *          segments k >= 1; zero elsewhere
 *   Lh[j]  fill-in H_k = L-hat(s_{k+1}, s_k) stored at j = s_k, 1 <= k <= P-2
 *   Lg[j]  G-hat at segment stages, Q-hat_k at separator s_k
 *   Lr     R-hat
 * flops (optional, length 2*(P+1)): [paper, standard] per segment k, then for
 * the sequential phase. Returns 0 or a breakdown code: -(j+1) for natural
 * stage j, -(N+1) for the corner. */
int orc_par_factor(int N, int n, int m, int P, const int* len, const double* D,
                   const double* E, const double* G, const double* R, double* Ld, double* Le,
                   double* Lw, double* Lh, double* Lg, double* Lr, double* flops) {
  const size_t nn = (size_t)n * n, mn = (size_t)m * n, mm = (size_t)m * m;
  int* f = (int*)malloc(sizeof(int) * (size_t)P);
  double* Rk = (double*)calloc((size_t)P * (mm > 0 ? mm : 1), sizeof(double));
  seg_map(P, len, f);
  /* Hatted quantities are in-place working buffers: start from Psi. */
  memcpy(Ld, D, sizeof(double) * nn * N);
  if (N > 1) memcpy(Le, E, sizeof(double) * nn * (N - 1));
  if (m > 0) memcpy(Lg, G, sizeof(double) * mn * N);
  memset(Lw, 0, sizeof(double) * nn * N);
  memset(Lh, 0, sizeof(double) * nn * N);
  /* Psi(s_k+1, s_k) belongs to B_k (read below from E); it is no block of
   * L-hat, so its slot in Le is cleared. */
  for (int k = 1; k < P; ++k) memset(Le + (size_t)(f[k] - 1) * nn, 0, sizeof(double) * nn);
  int status = 0;

  /* Algorithm 1, parallel phase: each segment touches only its own stages,
   * its own separator's A/Q/H slots and its own R partial (Eqs. (4)-(5),
   * (8a)-(8b)). */
  for (int k = 0; k < P && !status; ++k) {
    double p0, s0;
    orc_flops_get(&p0, &s0);
    const int fk = f[k], nk = len[k], lk = fk + nk - 1;
    const int sk = fk - 1; /* separator of segment k >= 1 */
    double* Rp = Rk + (size_t)k * mm;
    /* W_1k <- B_k = Psi(s_k, f_k) = E[s_k]^T; W_ik = 0 for i > 1. */
    if (k >= 1)
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Lw[(size_t)fk * nn + r * n + c] = E[(size_t)sk * nn + c * n + r];
    for (int i = 0; i < nk; ++i) {
      const int j = fk + i;
      double* Dj = Ld + j * nn;
      if (potrf(n, Dj, n)) { status = -(j + 1); break; }                     /* D-hat_ik */
      if (i < nk - 1) trsm_rlt(n, n, Dj, n, Le + j * nn, n);                  /* E-hat_ik */
      if (m > 0) {
        trsm_rlt(m, n, Dj, n, Lg + j * mn, n);                               /* G-hat_ik */
        syrk_ln(m, n, -1.0, Lg + j * mn, n, Rp, m);                          /* R_k -= G G^T */
      }
      if (i < nk - 1) {
        syrk_ln(n, n, -1.0, Le + j * nn, n, Ld + (j + 1) * nn, n);          /* D_{i+1} -= E E^T */
        if (m > 0) gemm_nt(m, n, n, -1.0, Lg + j * mn, n, Le + j * nn, n, Lg + (j + 1) * mn, n);
      }
      if (k >= 1) {
        double* Wj = Lw + j * nn;
        trsm_rlt(n, n, Dj, n, Wj, n);                                        /* W_ik */
        syrk_ln(n, n, -1.0, Wj, n, Ld + (size_t)sk * nn, n);                /* A_k -= W W^T */
        if (i < nk - 1) gemm_nt(n, n, n, -1.0, Wj, n, Le + j * nn, n, Wj + nn, n); /* W_{i+1} */
        if (m > 0) gemm_nt(m, n, n, -1.0, Lg + j * mn, n, Wj, n, Lg + (size_t)sk * mn, n); /* Q_k */
      }
    }
    if (!status && k < P - 1) trsm_rlt(n, n, Ld + (size_t)lk * nn, n, Le + (size_t)lk * nn, n); /* F-hat_k */
    if (!status && k >= 1 && k < P - 1)                                      /* H_k = -F W^T */
      gemm_nt(n, n, n, -1.0, Le + (size_t)lk * nn, n, Lw + (size_t)lk * nn, n, Lh + (size_t)sk * nn, n);
    if (flops) {
      double p1, s1;
      orc_flops_get(&p1, &s1);
      flops[2 * k] = p1 - p0;
      flops[2 * k + 1] = s1 - s0;
    }
  }

  /* Algorithm 1, sequential phase: the reduced system of Eq. (7) plus the
   * cross-segment updates of Eqs. (8c)-(8d). */
  double p0, s0;
  orc_flops_get(&p0, &s0);
  if (!status && m > 0) memcpy(Lr, R, sizeof(double) * mm);                 /* R-hat <- Psi_gg */
  for (int k = 1; k < P && !status; ++k) {
    const int sk = f[k] - 1, lprev = f[k] - 2; /* last stage of segment k-1 */
    double* Ak = Ld + (size_t)sk * nn;
    syrk_ln(n, n, -1.0, Le + (size_t)lprev * nn, n, Ak, n);                 /* A_k -= F F^T */
    if (potrf(n, Ak, n)) { status = -(sk + 1); break; }                      /* A-hat_k */
    if (k < P - 1) trsm_rlt(n, n, Ak, n, Lh + (size_t)sk * nn, n);          /* H_k */
    if (m > 0) {
      double* Qk = Lg + (size_t)sk * mn;
      gemm_nt(m, n, n, -1.0, Lg + (size_t)lprev * mn, n, Le + (size_t)lprev * nn, n, Qk, n);
      trsm_rlt(m, n, Ak, n, Qk, n);                                          /* Q-hat_k */
    }
    if (k < P - 1) {
      const int snext = f[k + 1] - 1;
      syrk_ln(n, n, -1.0, Lh + (size_t)sk * nn, n, Ld + (size_t)snext * nn, n); /* A_{k+1} -= H H^T */
      if (m > 0)
        gemm_nt(m, n, n, -1.0, Lg + (size_t)sk * mn, n, Lh + (size_t)sk * nn, n,
                Lg + (size_t)snext * mn, n);                                 /* Q_{k+1} -= Q H^T */
    }
    if (m > 0) syrk_ln(m, n, -1.0, Lg + (size_t)sk * mn, n, Lr, m);         /* R -= Q Q^T */
  }
  if (!status && m > 0) {
    for (int k = 0; k < P; ++k)                                              /* R += sum_k R_k */
      for (size_t t = 0; t < mm; ++t) Lr[t] += Rk[(size_t)k * mm + t];
    if (potrf(m, Lr, m)) status = -(N + 1);
  }
  if (flops) {
    double p1, s1;
    orc_flops_get(&p1, &s1);
    flops[2 * P] = p1 - p0;
    flops[2 * P + 1] = s1 - s0;
  }
  free(Rk);
  free(f);
  return status;
}

/* b [(N n + m)][nrhs] <- Psi^{-1} b with the O3 factor: Algorithm 2 then
 * Algorithm 3, one right-hand side at a time, in natural order (the
 * permutation is an index map). flops (optional, 2*(P+1)) as for the factor,
 * forward and backward together. */
void orc_par_solve(int N, int n, int m, int P, const int* len, const double* Ld,
                   const double* Le, const double* Lw, const double* Lh, const double* Lg,
                   const double* Lr, double* b, int nrhs, double* flops) {
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  const int dim = N * n + m;
  int* f = (int*)malloc(sizeof(int) * (size_t)P);
  double* v = (double*)malloc(sizeof(double) * (size_t)dim);
  double* ygk = (double*)calloc((size_t)P * (m > 0 ? m : 1), sizeof(double));
  seg_map(P, len, f);
  if (flops) memset(flops, 0, sizeof(double) * 2 * (P + 1));
  for (int c = 0; c < nrhs; ++c) {
    for (int i = 0; i < dim; ++i) v[i] = b[(size_t)i * nrhs + c];
    double* vg = v + (size_t)N * n;
    double p0, s0, p1, s1;
    memset(ygk, 0, sizeof(double) * (size_t)P * (m > 0 ? m : 1));
    /* Algorithm 2, parallel phase (Eqs. (9a)-(9c)). */
    for (int k = 0; k < P; ++k) {
      orc_flops_get(&p0, &s0);
      const int fk = f[k], nk = len[k], sk = fk - 1;
      for (int i = 0; i < nk; ++i) {
        const int j = fk + i;
        double* vj = v + (size_t)j * n;
        trsv_ln(n, Ld + j * nn, n, vj);                                     /* y_ik */
        if (i < nk - 1) gemv_n(n, n, -1.0, Le + j * nn, n, vj, vj + n);     /* t_{i+1} */
        if (k >= 1) gemv_n(n, n, -1.0, Lw + j * nn, n, vj, v + (size_t)sk * n); /* y~_k */
        if (m > 0) gemv_n(m, n, -1.0, Lg + j * mn, n, vj, ygk + (size_t)k * m); /* y~_g,k */
      }
      orc_flops_get(&p1, &s1);
      if (flops) { flops[2 * k] += p1 - p0; flops[2 * k + 1] += s1 - s0; }
    }
    /* Algorithm 2, sequential phase (Eqs. (9d)-(9e), (10)). */
    orc_flops_get(&p0, &s0);
    for (int k = 1; k < P; ++k) {
      const int sk = f[k] - 1, lprev = f[k] - 2;
      double* vk = v + (size_t)sk * n;
      gemv_n(n, n, -1.0, Le + (size_t)lprev * nn, n, v + (size_t)lprev * n, vk); /* F-hat term */
      trsv_ln(n, Ld + (size_t)sk * nn, n, vk);
      if (k < P - 1) gemv_n(n, n, -1.0, Lh + (size_t)sk * nn, n, vk, v + (size_t)(f[k + 1] - 1) * n);
      if (m > 0) gemv_n(m, n, -1.0, Lg + (size_t)sk * mn, n, vk, vg);
    }
    if (m > 0) {
      for (int k = 0; k < P; ++k)
        for (int t = 0; t < m; ++t) vg[t] += ygk[(size_t)k * m + t];
      trsv_ln(m, Lr, m, vg);
      /* Algorithm 3, sequential phase (Eq. (11)). */
      trsv_lt(m, Lr, m, vg);
    }
    for (int k = P - 1; k >= 1; --k) {
      const int sk = f[k] - 1;
      double* vk = v + (size_t)sk * n;
      if (m > 0) gemv_t(m, n, -1.0, Lg + (size_t)sk * mn, n, vg, vk);
      if (k < P - 1) gemv_t(n, n, -1.0, Lh + (size_t)sk * nn, n, v + (size_t)(f[k + 1] - 1) * n, vk);
      trsv_lt(n, Ld + (size_t)sk * nn, n, vk);
    }
    orc_flops_get(&p1, &s1);
    if (flops) { flops[2 * P] += p1 - p0; flops[2 * P + 1] += s1 - s0; }
    /* Algorithm 3, parallel phase (Eqs. (12a)-(12c)). */
    for (int k = 0; k < P; ++k) {
      orc_flops_get(&p0, &s0);
      const int fk = f[k], nk = len[k], lk = fk + nk - 1, sk = fk - 1;
      if (k < P - 1) gemv_t(n, n, -1.0, Le + (size_t)lk * nn, n, v + (size_t)(lk + 1) * n, v + (size_t)lk * n);
      for (int i = nk - 1; i >= 0; --i) {
        const int j = fk + i;
        double* vj = v + (size_t)j * n;
        if (m > 0) gemv_t(m, n, -1.0, Lg + j * mn, n, vg, vj);
        if (k >= 1) gemv_t(n, n, -1.0, Lw + j * nn, n, v + (size_t)sk * n, vj);
        trsv_lt(n, Ld + j * nn, n, vj);
        if (i > 0) gemv_t(n, n, -1.0, Le + (size_t)(j - 1) * nn, n, vj, vj - n);
      }
      orc_flops_get(&p1, &s1);
      if (flops) { flops[2 * k] += p1 - p0; flops[2 * k + 1] += s1 - s0; }
    }
    for (int i = 0; i < dim; ++i) b[(size_t)i * nrhs + c] = v[i];
  }
  free(ygk);
  free(v);
  free(f);
}

/* ------------------------------------------------------------------------ */
/* Batch helper: O2 factor+solve of independent systems spread over threads  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int count, N, n, m, nrhs, stride, nthreads, tid;
  const double *D, *E, *G, *R;
  double* b;
  int* status;
} batch_arg;

static void* batch_worker(void* p) {
  batch_arg* a = (batch_arg*)p;
  const size_t nn = (size_t)a->n * a->n, mn = (size_t)a->m * a->n, mm = (size_t)a->m * a->m;
  const size_t dim = (size_t)a->N * a->n + a->m;
  double* Ld = (double*)malloc(sizeof(double) * nn * a->N);
  double* Le = (double*)malloc(sizeof(double) * nn * (a->N > 1 ? a->N - 1 : 1));
  double* Lg = (double*)malloc(sizeof(double) * (mn ? mn : 1) * a->N);
  double* Lr = (double*)malloc(sizeof(double) * (mm ? mm : 1));
  for (int s = a->tid; s < a->count; s += a->nthreads) {
    const size_t is = (size_t)(a->stride ? s : 0);
    int st = orc_seq_factor(a->N, a->n, a->m, a->D + is * nn * a->N,
                            a->E + is * nn * (a->N > 1 ? a->N - 1 : 0), a->G + is * mn * a->N,
                            a->R + is * mm, Ld, Le, Lg, Lr);
    a->status[s] = st;
    if (!st) orc_seq_solve(a->N, a->n, a->m, Ld, Le, Lg, Lr, a->b + (size_t)s * dim * a->nrhs, a->nrhs);
  }
  free(Ld); free(Le); free(Lg); free(Lr);
  return NULL;
}

/* Factor and solve `count` systems of one shape with O2, systems spread over
 * `nthreads` POSIX threads (system s goes to thread s mod nthreads). With
 * stride = 0 every system reads the same D/E/G/R; b holds count right-hand
 * side blocks of (N n + m) x nrhs. status[count] receives each O2 code. */
int orc_seq_batch(int count, int N, int n, int m, int nrhs, int stride, int nthreads,
                  const double* D, const double* E, const double* G, const double* R,
                  double* b, int* status) {
  if (nthreads < 1) nthreads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  batch_arg* args = (batch_arg*)malloc(sizeof(batch_arg) * (size_t)nthreads);
  for (int t = 0; t < nthreads; ++t) {
    batch_arg a = {count, N, n, m, nrhs, stride, nthreads, t, D, E, G, R, b, status};
    args[t] = a;
    pthread_create(&th[t], NULL, batch_worker, &args[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(args);
  for (int s = 0; s < count; ++s)
    if (status[s]) return status[s];
  return 0;
}
