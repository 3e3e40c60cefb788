// Kernels of the partitioned block Cholesky factorization and solve of an SPD
// block-tridiagonal-arrow KKT matrix (arXiv 2511.00946, Algorithms 1-3), and
// of the FP64 residual used by mixed-precision iterative refinement.
//
// One CTA per segment task. Per stage the CTA keeps the pivot block, the
// stacked panel Z = [E; G; W] and the Schur accumulator T in shared memory
// (row-major, odd leading dimensions: row- and column-wise accesses are free
// of bank conflicts) and runs
//   potrf(D)  ->  Z <- Z D-hat^{-T}  ->  T -= Z Z^T (lower triangle)
// with every thread on the element loops. FP64 is the scarce resource on this
// part: one FP64 warp-instruction occupies a sub-partition's FP64 pipe for
// about 64-76 cycles whether 1 or 32 lanes are active, and FP32 runs about
// 70x faster. So the loops issue FP64 instructions from full warps only
// (lower triangles are enumerated linearly instead of masked squares), and
// the mixed variant (TZ = float) keeps only the pivot Cholesky and the
// Schur accumulator in FP64: the panel trsm and the dot products of the
// syrk run in FP32 and each dot product is subtracted from the FP64
// accumulator once.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "kkt_internal.h"
#include "kkt_bulk.cuh"
#include "kkt_numerics.cuh"
#include "kkt_tc.cuh"

namespace kkt {
namespace {

constexpr int kMaxDevices = 64;  // devices whose kernel attributes are recorded

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

__device__ void record_status(Info* info, int status, int sys, int stage, int level) {
  if (atomicCAS(&info->status, 0, -1) == 0) {
    info->system = sys;
    info->stage = stage;
    info->level = level;
    __threadfence();
    atomicExch(&info->status, status);
  }
}
__device__ void record_breakdown(Info* info, int sys, int stage, int level) {
  record_status(info, 3 /* KKT_ERR_NOT_SPD */, sys, stage, level);
}
// a bounded device wait ran out (the kernel carries on; its results are invalid)
__device__ void record_timeout(Info* info, int sys, int stage, int level) {
  record_status(info, 5 /* KKT_ERR_TIMEOUT */, sys, stage, level);
}

// Debug build (compiled with -DKKT_DEBUG): index checks on entry to every
// segment task and residual task. A task whose geometry does not fit its
// system (segment index, stage range, separator, block sizes) or whose
// shared-memory layout does not fit the launch's dynamic shared memory is
// skipped, and the first such failure is recorded (status 8,
// KKT_ERR_BOUNDS) in a device record that kkt_get_info reports. Nothing
// traps. In the normal build the checks compile to nothing.
#ifdef KKT_DEBUG
__device__ Info g_debug_info;
#endif
extern __shared__ __align__(16) unsigned char kkt_dyn_smem[];
__device__ __forceinline__ bool dbg_ok(bool cond, const LevelDesc& d) {
#ifdef KKT_DEBUG
  if (!cond) record_status(&g_debug_info, 8, d.sys, -1, d.level);
  return cond;
#else
  (void)d;
  return cond || true;
#endif
}
__device__ __forceinline__ bool task_geometry_ok(const LevelDesc& d, int seg, const void* sm, int bytes) {
#ifdef KKT_DEBUG
  unsigned dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const long long off = (long long)__cvta_generic_to_shared(sm) - (long long)__cvta_generic_to_shared(kkt_dyn_smem);
  bool ok = d.n >= 1 && d.n <= kMaxN && d.m >= 0 && d.m <= kMaxM && d.N >= 1 && d.P >= 1 && seg >= 0 &&
            seg < d.P && d.mr >= 0 && d.mr <= d.m;
  if (ok) {
    const int f = d.seg[seg], e = d.seg[seg + 1] - 2;  // first and last stage of the segment
    ok = f >= (seg ? 1 : 0) && e >= f && e < d.N && d.seg[d.P] == d.N + 1;
    if (ok) ok = d.nat[f] >= 0 && d.nat[e] < d.Nnat && (seg == 0 || d.nat[f - 1] >= 0);
  }
  ok = ok && off >= 0 && off + bytes <= (long long)dyn;
  return dbg_ok(ok, d);
#else
  (void)d; (void)seg; (void)sm; (void)bytes;
  return true;
#endif
}

// A group of threads working on one role of a CTA: thread index within the
// group, group size and the named barrier that synchronizes it (0 = the whole
// CTA, __syncthreads; -1 = a single warp, __syncwarp).
struct Grp {
  int tid, nt, bar;
};
__device__ __forceinline__ Grp cta_grp() { return Grp{(int)threadIdx.x, (int)blockDim.x, 0}; }

__device__ __forceinline__ void group_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void group_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void gsync(const Grp& g) {
  if (g.bar == 0) __syncthreads();
  else if (g.bar < 0) __syncwarp();
  else group_bar(g.bar, g.nt);
}

// dst (rows x cols, smem, ld) <- A (+ B) from global row-major [rows][cols],
// or the transpose of A (+ B) given as [cols][rows] when `trans`. A null A
// loads zeros. Coalesced over the global array.
// The three source cases are separate loops: a predicated-off FP64 add still
// holds the FP64 pipe on this part.
// U > 1: every thread issues U loads before their stores. The stores go to
// shared memory, which the compiler cannot prove disjoint from A and B, so
// with U = 1 each load's latency is waited out in turn (U = 1 keeps the
// register footprint of the warp kernels).
template <int U = 1, typename T>
__device__ void load_blk(T* dst, int ld, const double* A, const double* B, int rows, int cols,
                         bool trans, Grp g = cta_grp()) {
  const int tot = rows * cols;
  auto at = [&](int e) {
    int r, c;
    if (trans) { c = e / rows; r = e - c * rows; }
    else { r = e / cols; c = e - r * cols; }
    return r * ld + c;
  };
  auto batched = [&](auto get) {
    for (int e0 = g.tid; e0 < tot; e0 += U * g.nt) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * g.nt;
        v[u] = e < tot ? get(e) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * g.nt;
        if (e < tot) dst[at(e)] = (T)v[u];
      }
    }
  };
  if (A && B) {
    if constexpr (U > 1) batched([&](int e) { return A[e] + B[e]; });
    else for (int e = g.tid; e < tot; e += g.nt) dst[at(e)] = (T)(A[e] + B[e]);
  } else if (A) {
    if constexpr (U > 1) batched([&](int e) { return A[e]; });
    else for (int e = g.tid; e < tot; e += g.nt) dst[at(e)] = (T)A[e];
  } else {
    for (int e = g.tid; e < tot; e += g.nt) dst[at(e)] = T(0);
  }
}

// global row-major [rows][cols] <- src (smem), or the transpose when `trans`
// (dst is then [cols][rows]). `lower` writes zeros above the diagonal.
template <typename TD, typename TS>
__device__ void store_blk(TD* dst, const TS* src, int ld, int rows, int cols, bool trans,
                          bool lower, Grp g = cta_grp()) {
  const int tot = rows * cols;
  for (int e = g.tid; e < tot; e += g.nt) {
    int r, c;
    if (trans) { c = e / rows; r = e - c * rows; }
    else { r = e / cols; c = e - r * cols; }
    TS v = src[r * ld + c];
    if (lower && c > r) v = TS(0);
    dst[e] = (TD)v;
  }
}

// smem -> smem copy of a rows x cols block (with conversion)
template <typename TD, typename TS>
__device__ void copy_blk(TD* dst, int ldd, const TS* src, int lds, int rows, int cols,
                         Grp g = cta_grp()) {
  for (int e = g.tid; e < rows * cols; e += g.nt) {
    const int r = e / cols, c = e - r * cols;
    dst[r * ldd + c] = (TD)src[r * lds + c];
  }
}

// Element table of the trailing updates of an n x n Cholesky: the pairs
// (i, k) with 2 <= k <= i < n ordered by k descending (packed i << 16 | k),
// so that the updates applied by column j form the prefix of length
// (n-2-j)(n-1-j)/2. Built once per CTA (it depends on n only).
__device__ void potrf_table(int* tab, int n) {
  const int np = (n - 2) * (n - 1) / 2;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    int a, b;
    tri_rc(e, a, b);
    const int k = n - 1 - a;
    tab[e] = (k + b) << 16 | k;
  }
}

// Column steps of the in-place lower Cholesky of A (n x n, FP64, n <= 64),
// right-looking with a one-column look-ahead: in the phase of column j
// (final and scaled), warp 0 alone updates column j+1, computes its pivot
// from the register holding the diagonal and scales it, so the serial pivot
// chain runs on a sub-pipe of its own, while warps 1-3 walk the prefix of the
// element table `tab` for the trailing columns. Every loop has a runtime trip
// count: on this part a predicated-off FP64 instruction still holds the FP64
// pipe, so no FP64 work is issued for inactive elements. On a pivot that is
// not positive *bad is set (first column + 1) and the factorization carries
// on (NaNs propagate; no trap). rinv[j] = 1 / L_jj.
__device__ __forceinline__ void potrf_col0(double* A, int ld, int n, double* rinv, int* bad, int lane) {
  const double d = A[0];
  const double r = pivot_rsqrt(d);
  if (lane == 0) {
    if (not_positive(d) && *bad == 0) *bad = 1;
    rinv[0] = r;
  }
  // (lane 0 scales the diagonal: L_00 = d r)
  for (int i = lane; i < n; i += 32) A[i * ld] *= r;
}

// warp 0 in the phase of column j: column j+1 updated, pivoted and scaled
__device__ __forceinline__ void potrf_lookahead(double* A, int ld, int n, double* rinv, int* bad, int j,
                                                int lane) {
  const double lj = A[(j + 1) * ld + j];
  const int i0 = j + 1 + lane, i1 = i0 + 32;
  const bool two = j + 33 < n;  // warp-uniform: a second row per lane
  double v0 = 0.0, v1 = 0.0;
  if (i0 < n) v0 = fma(-A[i0 * ld + j], lj, A[i0 * ld + j + 1]);
  if (two) {
    if (i1 < n) v1 = fma(-A[i1 * ld + j], lj, A[i1 * ld + j + 1]);
  }
  double r = 0.0;
  if (lane == 0) {  // v0 is the diagonal element (j+1, j+1)
    if (not_positive(v0) && *bad == 0) *bad = j + 2;
    r = pivot_rsqrt(v0);
    rinv[j + 1] = r;
  }
  r = __shfl_sync(0xffffffffu, r, 0);
  // one FP64 multiply for the whole column, the diagonal L_{j+1,j+1} = v0 r on lane 0
  if (i0 < n) A[i0 * ld + j + 1] = v0 * r;
  if (two) {
    if (i1 < n) A[i1 * ld + j + 1] = v1 * r;
  }
}

// warps 1-3 in the phase of column j: the updates of columns j+2.. by column j
__device__ __forceinline__ void potrf_trailing(double* A, int ld, int n, const int* tab, int j, int t,
                                               int nt) {
  const int cnt = (n - 2 - j) * (n - 1 - j) / 2;
  for (int e = t; e < cnt; e += nt) {
    const int p = tab[e], i = p >> 16, k = p & 0xffff;
    A[i * ld + k] = fma(-A[i * ld + j], A[k * ld + j], A[i * ld + k]);
  }
}

// In-place lower Cholesky by the first four warps (one per FP64 sub-pipe).
// With `whole`, the CTA's other threads wait at the closing __syncthreads;
// otherwise only warps 0-3 call it and it closes with their own barrier.
constexpr int kPotrfThreads = 128;
constexpr int kPotrfUpd = kPotrfThreads - 32;  // threads of warps 1-3

__device__ void potrf_sm(double* A, int ld, int n, double* rinv, const int* tab, int* bad,
                         bool whole = true) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) potrf_col0(A, ld, n, rinv, bad, lane);
  if (tid < kPotrfThreads) {
    group_bar(1, kPotrfThreads);
    for (int j = 0; j + 1 < n; ++j) {
      if (tid < 32) potrf_lookahead(A, ld, n, rinv, bad, j, lane);
      else potrf_trailing(A, ld, n, tab, j, tid - 32, kPotrfUpd);
      group_bar(1, kPotrfThreads);
    }
  }
  if (whole) __syncthreads();
}

// Fused pivot factorization (FP64) and panel solve (in the panel type TZ:
// FP64, or FP32 in the mixed variant): the Cholesky above and
// Z[r0, r1) <- Z[r0, r1) L^{-T} in the division-free form of trsm_panel (the
// same operations in the same order, so the results are bitwise those of
// potrf_sm + panel_operand + trsm_panel). Warp 0 runs the pivot chain; in the
// phase of column j the workers (warps 1-3 and 5-7) run, each as a tight
// strided loop,
//   - the trailing updates of columns j+2.. by column j,
//   - the panel operand column M[c][j] = L[c][j] / L[j][j] (c > j),
//   - the panel updates z_c -= z_{j-1} M[c][j-1] (c >= j) of every row,
// so the panel lags the factorization by two columns and runs beside the
// pivot chain instead of after it. x_c = z_c / L_cc closes the sweep. Warp 4 does not take part: it
// returns at once and may run other work, touching neither A, rinv, M nor
// panel rows [r0, r1). One named barrier (id 1, 224 threads) per phase; the
// caller synchronizes the CTA before the results are read.
constexpr int kFusedThreads = 224;
constexpr int kFusedWorkers = 192;  // warps 1-3 and 5-7

// all7: warp 4 works too (seven worker warps, a barrier over the whole CTA).
// A warp's FP64 instructions issue on sub-partition (warp % 4): with warps
// 1-3 and 5-7 the workers' FP64 work (trailing updates, panel solve) runs on
// three of the four FP64 pipes while the pivot chain leaves sub-partition 0's
// nearly idle; with warp 4 on board all four take a share.
template <typename TZ>
__device__ void potrf_trsm_sm(double* A, int ld, int n, double* rinv, TZ* M, const int* tab, int* bad,
                              TZ* Z, int ldz, int r0, int r1, bool all7 = false) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (!all7 && tid >= kPotrfThreads && tid < kPotrfThreads + 32) return;  // warp 4
  const int w = all7 ? tid - 32 : (tid < kPotrfThreads ? tid - 32 : tid - 64);  // worker index
  const int nwk = all7 ? kFactorThreads - 32 : kFusedWorkers;
  const int nbar = all7 ? kFactorThreads : kFusedThreads;
  const int rows = r1 - r0;
  // panel mapping: `per` workers on a row, each on every per-th column
  const int per = rows > 0 ? max(1, nwk / rows) : 0;
  const bool pact = tid >= 32 && w < rows * per;
  const int pr = pact ? w % rows : 0, pc = pact ? w / rows : 0;
  TZ* zr = Z + (r0 + pr) * ldz;
  if (tid < 32) potrf_col0(A, ld, n, rinv, bad, lane);
  group_bar(1, nbar);
  for (int j = 0; j < n; ++j) {
    if (tid < 32) {
      if (j + 1 < n) potrf_lookahead(A, ld, n, rinv, bad, j, lane);
    } else {
      potrf_trailing(A, ld, n, tab, j, w, nwk);
      for (int c = j + 1 + w; c < n; c += nwk) M[c * ld + j] = (TZ)(A[c * ld + j] * rinv[j]);
      if (pact && j >= 1) {
        const TZ zj = zr[j - 1];
        for (int c = j + pc; c < n; c += per) zr[c] = fma(-zj, M[c * ld + j - 1], zr[c]);
      }
    }
    group_bar(1, nbar);
  }
  if (tid >= 32)
    for (int e = w; e < rows * n; e += nwk) {
      const int r = e / n, c = e - r * n;
      Z[(r0 + r) * ldz + c] *= (TZ)rinv[c];
    }
}

// Panel operand of the division-free trsm: M[c][j] = L[c][j] / L[j][j]
// (strict lower triangle, computed as L[c][j] * rinv[j]), rounded to TM.
template <typename TM>
__device__ void panel_operand(TM* M, const double* L, int ld, int n, const double* rinv, Grp g) {
  const int ntri = (n - 1) * n / 2;
  for (int e = g.tid; e < ntri; e += g.nt) {
    int a, b;
    tri_rc(e, a, b);
    const int c = a + 1, j = b;
    M[c * ld + j] = (TM)(L[c * ld + j] * rinv[j]);
  }
}

// Z[r0:r1) <- Z[r0:r1) L^{-T} with the pre-scaled columns M (M_cj = L_cj /
// L_jj), in the panel type TZ: for each row, u_c = z_c - sum_{k<c} u_k M_ck
// (in k order) and x_c = u_c / L_cc (times rinv). Column sweep: every thread
// works on every column (FP64 from full warps), thread t owning row
// r0 + t % rows and every (nt/rows)-th column. The group needs at least as
// many threads as rows (true for every panel: rows <= kMaxN + kMaxM per
// role of a split CTA, 2 kMaxN + kMaxM otherwise).
template <typename TZ>
__device__ void trsm_panel(TZ* Z, int ldz, int r0, int r1, const TZ* M, int ldm, int n, const TZ* rinv,
                           Grp g) {
  const int rows = r1 - r0;
  if (rows <= 0) return;
  const int per = g.nt / rows;  // threads per row (>= 1)
  const int rr = g.tid % rows, cc = g.tid / rows;
  const bool act = cc < per;
  TZ* zr = Z + (r0 + rr) * ldz;
  for (int j = 0; j < n - 1; ++j) {
    if (act) {
      const TZ zj = zr[j];
      for (int c = j + 1 + cc; c < n; c += per) zr[c] = fma(-zj, M[c * ldm + j], zr[c]);
    }
    gsync(g);
  }
  if (act)
    for (int c = cc; c < n; c += per) zr[c] *= rinv[c];
  gsync(g);
}

// T[a][b] -= sum_t Z[a][t] Z[b][t] for ra0 <= a < ra1, cb0 <= b <= a (cb0 <=
// ra0: a rectangle of full rows beside a lower triangle; ra0 = cb0 is a plain
// lower triangle). Panel rows below `zsplit` are read from Zlo, the others
// from Z (same leading dimension and row numbering). FP64 panels: T_ab takes
// the rank-1 updates of the columns t = 0, 1, .. in turn, each one fma. FP32
// panels (mixed variant): the dot product is formed in FP32 and subtracted
// from the FP64 accumulator once.
template <typename TZ>
__device__ void syrk_trap(double* T, int ldt, const TZ* Zlo, const TZ* Z, int zsplit, int ldz, int ra0,
                          int ra1, int cb0, int n, Grp g) {
  const int w0 = ra0 - cb0, h = ra1 - ra0;
  const int tot = h * w0 + h * (h + 1) / 2;  // row a holds a - cb0 + 1 elements
  // (a, b) of element g.tid, then advanced by g.nt along the rows
  int a = ra0, b = cb0 + g.tid;
  while (a < ra1 && b > a) { b -= a - cb0 + 1; ++a; }
  for (int e = g.tid; e < tot; e += g.nt) {
    if (e != g.tid) {
      b += g.nt;
      while (b > a) { b -= a - cb0 + 1; ++a; }
    }
    const TZ* zi = (a < zsplit ? Zlo : Z) + a * ldz;
    const TZ* zj = (b < zsplit ? Zlo : Z) + b * ldz;
    if (sizeof(TZ) == 8) {
      // FP64: rank-1 updates in column order, T_ab = fma(-z_at, z_bt, T_ab): no
      // partial sums to combine, and one dependent chain per element already
      // keeps an FP64 pipe busy on this part
      double acc = T[a * ldt + b];
      for (int t = 0; t < n; ++t) acc = fma(-(double)zi[t], (double)zj[t], acc);
      T[a * ldt + b] = acc;
    } else {
      TZ s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      int t = 0;
      for (; t + 3 < n; t += 4) {
        s0 = fma(zi[t], zj[t], s0);
        s1 = fma(zi[t + 1], zj[t + 1], s1);
        s2 = fma(zi[t + 2], zj[t + 2], s2);
        s3 = fma(zi[t + 3], zj[t + 3], s3);
      }
      for (; t < n; ++t) s0 = fma(zi[t], zj[t], s0);
      T[a * ldt + b] -= (double)((s0 + s1) + (s2 + s3));
    }
  }
  gsync(g);
}

// Tensor-core form of the mixed Schur update (whole-CTA layout, eight warps):
// T[a][b] -= (Z Z^T)[a][b] for r0 <= b <= a < pr1, with Z (FP32, ld ldz)
// rounded to TF32 or BF16 and the products accumulated in FP32 by tcgen05
// MMAs (M = 128 rows, N = pr1 rounded up to 16, K = n padded to the
// instruction's 8 or 16), then subtracted from the FP64 accumulator once per
// element, in the element order of syrk_trap. `buf` (shared memory, 16-byte
// aligned) holds the operand, pr1 rows of K, and afterwards the FP32
// products as a packed lower triangle; the tensor core reads 128 rows of
// operand address range from it (rows from pr1 on are arbitrary data inside
// the CTA's shared memory and feed only accumulator rows that are never
// read). `tmem`: the accumulator's tensor-memory address; `bar`: the
// completion mbarrier, waited on with `parity` (its completions so far, mod
// 2); mode 1 = TF32, 2 = BF16. Returns false when the MMAs did not complete
// within the bounded wait (T is then left without the update).
// (out of line: inlined into the stage loop it enlarges the loop's code past
// what the instruction cache holds, and every mixed launch slowed down)
__device__ __noinline__ bool syrk_tc(double* T, int ldt, const float* Z, int ldz, int r0, int pr1, int n,
                                     unsigned char* buf, uint32_t tmem, uint64_t* bar, uint32_t parity, int mode) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool bf = mode == 2;
  const int kin = bf ? 16 : 8, epc = bf ? 8 : 4, eb = bf ? 2 : 4;
  const int Kp = (n + kin - 1) / kin * kin;
  const uint32_t LBO = 128, SBO = (uint32_t)(Kp / epc) * 128;
  __syncthreads();  // earlier readers of the buffer (the pivot blocks) are done
  for (int e = tid; e < pr1 * Kp; e += nt) {
    const int r = e / Kp, k = e - r * Kp;
    const float v = k < n ? Z[r * ldz + k] : 0.0f;
    const uint32_t off = (uint32_t)(r >> 3) * SBO + (uint32_t)(k / epc) * LBO + (uint32_t)(r & 7) * 16 +
                         (uint32_t)(k % epc) * eb;
    if (bf) *(__nv_bfloat16*)(buf + off) = __float2bfloat16_rn(v);
    else *(uint32_t*)(buf + off) = tc::to_tf32(v);
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (tid == 0) {
    const int N = (pr1 + 15) & ~15;
    const uint32_t idesc = tc::instr_desc(bf ? 1u : 2u, 128, N);
    const uint32_t a0 = tc::smem_u32(buf);
    for (int ks = 0; ks < Kp / kin; ++ks) {
      const uint64_t d = tc::smem_desc(a0 + (uint32_t)ks * 2 * LBO, LBO, SBO);
      tc::mma(bf, tmem, d, d, idesc, ks > 0);
    }
    tc::commit(bar);
  }
  const bool ok = tc::wait(bar, parity);
  tc::fence_after();
  // products -> packed lower triangle S[a (a + 1) / 2 + b]: warp w reads the
  // TMEM lanes (rows) 32 (w % 4) .. + 31, warps w and w + 4 take alternate
  // 8-column chunks
  float* S = (float*)buf;
  const int warp = tid >> 5, lane = tid & 31, row0 = 32 * (warp & 3);
  if (ok && row0 < pr1 && row0 + 31 >= r0) {
    const int a = row0 + lane;
    for (int c0 = 8 * (warp >> 2); c0 < pr1 && c0 <= row0 + 31; c0 += 16) {
      float v[8];
      tc::ld8(tmem + ((uint32_t)row0 << 16) + (uint32_t)c0, v);
      if (a < pr1 && a >= r0) {
        float* Sa = S + a * (a + 1) / 2;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (c0 + i >= r0 && c0 + i <= a) Sa[c0 + i] = v[i];
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (ok) {
    // the subtraction, enumerated like syrk_trap (a rectangle of width 0
    // beside the triangle of rows and columns [r0, pr1))
    const int h = pr1 - r0, tot = h * (h + 1) / 2;
    int a = r0, b = r0 + tid;
    while (a < pr1 && b > a) { b -= a - r0 + 1; ++a; }
    for (int e = tid; e < tot; e += nt) {
      if (e != tid) {
        b += nt;
        while (b > a) { b -= a - r0 + 1; ++a; }
      }
      T[a * ldt + b] -= (double)S[a * (a + 1) / 2 + b];
    }
  }
  __syncthreads();
  return ok;
}

// Thread-block-cluster primitives (a factor task may run as a pair of CTAs).
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// split-phase hardware barrier over every thread of the cluster; arrive
// releases this thread's earlier writes (local and remote shared memory),
// wait acquires the other CTAs'
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of this CTA's shared-memory location p in CTA `rank`
__device__ __forceinline__ unsigned cluster_addr(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(unsigned addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// sum_{p < np} part(p, o) for every output o < nout, by the whole CTA, in a
// fixed order that depends only on (nout, np, group size): `sp` adjacent lanes
// (a power of two, at most 32) per output each add every sp-th partial into
// two accumulators, then a shuffle tree combines the lanes; out(o, sum) is
// called once per output. Many partials (one per segment of every lower
// level) are summed with all FP64 sub-pipes instead of one dependent chain
// per output.
// The partials live in L2 (written by earlier launches); the loads of four
// steps are issued before their adds, which keep the order above, so a lane
// waits for one L2 round trip per four steps instead of one per step.
template <typename Fpart, typename Fout>
__device__ void sum_partials(Grp G, int nout, int np, Fpart part, Fout out) {
  int sp = 1;
  while (sp < 32 && sp * 2 * nout <= G.nt) sp *= 2;
  const int groups = G.nt / sp, sub = G.tid & (sp - 1);
  for (int o0 = 0; o0 < nout; o0 += groups) {
    const int o = o0 + G.tid / sp;
    double a0 = 0.0, a1 = 0.0;
    if (o < nout) {
      int p = sub;
      for (; p + 7 * sp < np; p += 8 * sp) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = part(p + u * sp, o);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          a0 += v[u];
          a1 += v[u + 1];
        }
      }
      for (; p + sp < np; p += 2 * sp) {
        a0 += part(p, o);
        a1 += part(p + sp, o);
      }
      if (p < np) a0 += part(p, o);
    }
    double a = a0 + a1;
    for (int s = sp >> 1; s > 0; s >>= 1) a += __shfl_xor_sync(0xffffffffu, a, s);
    if (o < nout && sub == 0) out(o, a);
  }
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
// TZ = double: every operation in FP64. TZ = float: FP64 pivots and Schur
// accumulator, FP32 panel (trsm and dot products), FP32 factor copy written
// for the correction solves.
//
// Roles. The panel rows of a segment with fill-in (k >= 1) fall into two
// groups. The producer runs the chain of Algorithm 1 proper: potrf(D_i), the
// E- and G-rows, and their Schur updates D_{i+1}, G_{i+1}, R~_k. The consumer
// runs the fill-in rows: W_i D-hat_i^{-T} and the updates A~_k, Q~_k^T and
// W_{i+1}, which read the producer's D-hat_i, E-hat_i and G-hat_i but feed
// nothing back into the chain, so the consumer may lag a stage behind. Three
// layouts (`mode`):
//   kWhole  one CTA runs both (segment 1, the top level, and mixed levels
//           that are not paired);
//   kSplit  one CTA, warps 0-3 producer and warps 4-7 consumer (FP64 levels
//           with more segments than SM pairs): the producer factors D_{i+1}
//           while the consumer is still on stage i. Hand-offs are named
//           barriers, each used once per stage by both roles:
//             kBarFullM  M_i, rinv_i ready       kBarFreeM  M_i read
//             kBarFullZ  E-hat_i, G-hat_i ready  kBarFreeZ  E-hat_i, G-hat_i read
//   kPair   a cluster of two CTAs (levels with few segments): CTA 0 is the
//           producer, CTA 1 the consumer, each on an SM of its own, so a
//           segment gets two SMs' FP64 pipes. After its trsm of stage i the
//           producer stores M_i, rinv_i, E-hat_i, G-hat_i into buffer i % 2
//           of the consumer's shared memory and arrives at cluster barrier
//           phase i; the consumer arrives at phase i when it is done with
//           stage i-1 and waits for it before stage i; the producer waits for
//           phase i-1 before it overwrites buffer i % 2 (double buffering).
//           A last phase, after every remote store, ends the task.
// ---------------------------------------------------------------------------
static_assert(kFactorThreads == 256, "the factor roles assume 8 warps per CTA");
constexpr int kWhole = 0, kSplit = 1, kPair = 2;
constexpr int kBarProd = 2, kBarCons = 3, kBarFullM = 4, kBarFreeM = 5, kBarFullZ = 6, kBarFreeZ = 7;
constexpr int kRoleThreads = 128;

// Pairs (i, k) with 1 <= k <= i < n ordered by k descending (packed
// i << 16 | k): the updates by column j are the prefix of length
// (n-1-j)(n-j)/2.
__device__ void pair_table_w(int* tab, int n, int lane) {
  const int np = (n - 1) * n / 2;
  for (int e = lane; e < np; e += 32) {
    int a, b;
    tri_rc(e, a, b);
    const int k = n - 1 - a;
    tab[e] = (k + b) << 16 | k;
  }
  __syncwarp();
}

// In-place lower Cholesky of A (n x n, FP64, n <= kWarpMaxN) by one warp,
// right-looking: pivot by lane 0, column scaled by the lanes, then the
// trailing update by column j over the pair table. Returns the first bad
// column + 1 (0 if every pivot was positive) in lane 0.
__device__ int potrf_w(double* A, int ld, int n, double* rinv, const int* tab, int lane) {
  int bad = 0;
  for (int j = 0; j < n; ++j) {
    double r = 0.0;
    if (lane == 0) {
      const double dj = A[j * ld + j];
      if (not_positive(dj) && bad == 0) bad = j + 1;
      r = pivot_rsqrt(dj);
      A[j * ld + j] = dj * r;
      rinv[j] = r;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    for (int i = j + 1 + lane; i < n; i += 32) A[i * ld + j] *= r;
    __syncwarp();
    const int cnt = (n - 1 - j) * (n - j) / 2;
    for (int e = lane; e < cnt; e += 32) {
      const int p = tab[e], i = p >> 16, k = p & 0xffff;
      A[i * ld + k] = fma(-A[i * ld + j], A[k * ld + j], A[i * ld + k]);
    }
    __syncwarp();
  }
  return bad;
}

// Corner of the top level: R-hat = chol(Rs) on the leading m - mr rows (Rs, ld
// ldR, m x m, in shared memory, already summed); the last mr rows hold
// bordered right-hand sides, which are solved against it instead of pivoted
// (their diagonal is never formed): row r gets (Rs[r][k] - sum_{t<k}
// Rs[r][t] R-hat[k][t]) / R-hat[k][k], the forward solution y_g of the
// corner. Writes R-hat (m x m, upper part zero) and 1/diag; group G; the
// pivot factorization uses warps 0-3 (potrf_sm) or one warp (potrf_w).
template <bool WARP>
__device__ void corner_factor(double* Rs, int ldR, int m, int mr, double* rinv, int* tab, const LevelDesc& d,
                              Info* info, int* bad, Grp G) {
  const int mk = m - mr;
  if (WARP) {
    pair_table_w(tab, mk, G.tid);
    const int bd = potrf_w(Rs, ldR, mk, rinv, tab, G.tid);
    if (G.tid == 0 && bd) record_breakdown(info, d.sys, d.Nnat, d.level);
  } else if (mk > 0) {
    potrf_table(tab, mk);
    __syncthreads();
    potrf_sm(Rs, ldR, mk, rinv, tab, bad);
    if (*bad && threadIdx.x == 0) record_breakdown(info, d.sys, d.Nnat, d.level);
  }
  // bordered rows: a forward substitution with the corner factor, one row per thread
  for (int r = mk + G.tid; r < m; r += G.nt) {
    double* z = Rs + r * ldR;
    for (int k = 0; k < mk; ++k) {
      double a = z[k];
      for (int t = 0; t < k; ++t) a = fma(-z[t], Rs[k * ldR + t], a);
      z[k] = a * rinv[k];
    }
    for (int k = mk; k < m; ++k) z[k] = 0.0;
  }
  gsync(G);
  store_blk(d.Rhat, Rs, ldR, m, m, false, true, G);
  for (int e = G.tid; e < m; e += G.nt) d.Rri[e] = e < mk ? rinv[e] : 0.0;
}

// Shared-memory view and per-stage bookkeeping of one segment task of
// Algorithm 1: where the stage's blocks live, the loads of its inputs (the
// caller's arrays at level 1, the slots of the level below otherwise), the
// stores of its factor blocks and the next level's slots. Used by the CTA
// kernel (k_factor) and the warp kernel (k_factor_w) alike.
template <typename TZ, int LU>
struct FacCtx {
  static constexpr bool mixed = sizeof(TZ) == 4;
  const LevelDesc* d;
  int n, m, R, ldD, ldZ, ldT, oG, oW, s;
  size_t nn, mn;
  SegGeom g;
  double *Dfac, *rinv, *T;
  TZ *M, *rinvZ, *Z;
  int* tab;
  const double *Din, *D2, *Ein, *Gin, *G2;

  __device__ FacCtx(const LevelDesc& dd, int seg, unsigned char* sm, const FacLayout& lay, const double* uD,
                    const double* uE, const double* uG) {
    d = &dd;
    n = dd.n; m = dd.m; R = 2 * n + m;
    ldD = odd(n); ldZ = lay.ldZ; ldT = lay.ldT;
    oG = n; oW = n + m;  // panel row offsets
    g = seg_geom(dd, seg);
    s = g.f - 1;         // separator of this segment (k >= 1)
    nn = (size_t)n * n; mn = (size_t)m * n;
    Dfac = (double*)(sm + lay.oDfac);
    M = (TZ*)(sm + lay.oM);
    rinv = (double*)(sm + lay.oRinv);
    rinvZ = (TZ*)(sm + lay.oRinvZ);
    Z = (TZ*)(sm + lay.oZ);
    T = (double*)(sm + lay.oT);
    tab = (int*)(sm + lay.oTab);
    Din = dd.level == 1 ? uD + dd.offD : dd.Dw;
    D2 = dd.level == 1 ? nullptr : dd.D2w;
    Ein = dd.level == 1 ? uE + dd.offE : dd.Ew;
    Gin = dd.level == 1 ? (m ? uG + dd.offG : nullptr) : dd.Gw;
    G2 = dd.level == 1 ? nullptr : dd.G2w;
  }
  __device__ const double* Dp(const double* b, int j) const { return b ? b + (size_t)j * nn : nullptr; }
  __device__ const double* Gp(const double* b, int j) const { return b ? b + (size_t)j * mn : nullptr; }

  // the pivot block D_j (on levels >= 2 the sum of its two slots) into dst (ld ldD)
  __device__ void load_D(double* dst, int j, Grp G) const {
    load_blk<LU>(dst, ldD, Dp(Din, j), Dp(D2, j), n, n, false, G);
  }

  // the first stage's inputs: pivot block, E- and G-rows and the next D, G
  // (eg); the fill-in rows W_1 = E[s]^T, A_k and Q_k^T (wr)
  __device__ void load_first(bool eg, bool wr, Grp G) const {
    const double* none = nullptr;
    if (eg) {
      load_blk<LU>(Dfac, ldD, Dp(Din, g.f), Dp(D2, g.f), n, n, false, G);
      if (g.len > 1 || g.hasF) load_blk<LU>(Z, ldZ, Dp(Ein, g.f), none, n, n, false, G);
      if (m) load_blk<LU>(Z + oG * ldZ, ldZ, Gp(Gin, g.f), Gp(G2, g.f), m, n, false, G);
      if (g.len > 1) {
        load_blk<LU>(T, ldT, Dp(Din, g.f + 1), Dp(D2, g.f + 1), n, n, false, G);          // D_{2}
        if (m) load_blk<LU>(T + oG * ldT, ldT, Gp(Gin, g.f + 1), Gp(G2, g.f + 1), m, n, false, G);
      }
    }
    if (wr) {
      load_blk<LU>(Z + oW * ldZ, ldZ, Dp(Ein, s), none, n, n, true, G);                 // W_1 = B_k = E[s]^T
      load_blk<LU>(T + oW * ldT + oW, ldT, Dp(Din, s), Dp(D2, s), n, n, false, G);       // A_k
      if (m) load_blk<LU>(T + oW * ldT + oG, ldT, Gp(Gin, s), Gp(G2, s), n, m, true, G);  // Q_k^T
    }
  }

  // factor blocks of stage j from the pivot factor L (Dp_, ld ldD) and
  // rv = 1/diag: Ld = L, LdR = L with its rows divided by their diagonal
  // (backward substitution, row-major), LdM = L with its columns divided by
  // their diagonal (forward substitution: the panel operand Ms when given,
  // else formed here with the same rounding), stored transposed so that
  // column c of L is the contiguous row c of LdM, Lri = rv. Strict lower
  // triangles are computed (no FP64 multiply for an upper half), the
  // diagonals of LdR and LdM hold rv (a substitution reads the reciprocal
  // from the block it streams in) and the rest is zero.
  __device__ void store_pivot(int j, const double* Dp_, const double* rv, const TZ* Ms, Grp G) const {
    store_blk(d->Ld + (size_t)j * nn, Dp_, ldD, n, n, false, true, G);
    TZ* LdRj = mixed ? (TZ*)(d->LdRf + (size_t)j * nn) : (TZ*)(d->LdR + (size_t)j * nn);
    TZ* LdMj = mixed ? (TZ*)(d->LdMf + (size_t)j * nn) : (TZ*)(d->LdM + (size_t)j * nn);
    for (int e = G.tid; e < n * n; e += G.nt) LdRj[e] = TZ(0);
    if (Ms) store_blk(LdMj, Ms, ldD, n, n, true, true, G);
    else
      for (int e = G.tid; e < n * n; e += G.nt) LdMj[e] = TZ(0);
    gsync(G);
    for (int e = G.tid; e < (n - 1) * n / 2; e += G.nt) {
      int a, b;
      tri_rc(e, a, b);
      const int r = a + 1, c = b;
      LdRj[r * n + c] = (TZ)(Dp_[r * ldD + c] * rv[r]);
      if (!Ms) LdMj[c * n + r] = (TZ)(Dp_[r * ldD + c] * rv[c]);
    }
    for (int e = G.tid; e < n; e += G.nt) {
      LdRj[e * n + e] = (TZ)rv[e];
      LdMj[e * n + e] = (TZ)rv[e];
    }
    if (mixed)
      for (int e = G.tid; e < n; e += G.nt) d->Lrif[(size_t)j * n + e] = (float)rv[e];
    for (int e = G.tid; e < n; e += G.nt) d->Lri[(size_t)j * n + e] = rv[e];
  }

  // bordered pass: the last arrow row of the solved panel is y_j^T (the
  // forward substitution of stage j), written where the solve keeps it
  // (the caller's b at level 1, this level's X otherwise)
  __device__ void store_y(int j, double* b, int ldb, Grp G) const {
    const TZ* yr = Z + (oG + m - d->mr) * ldZ;
    double* dst;
    long long ld;
    if (d->level == 1) { dst = b + (size_t)(d->offB + (long long)j * n) * ldb; ld = ldb; }
    else { dst = d->X + (size_t)j * n * kRhsChunk; ld = kRhsChunk; }
    for (int e = G.tid; e < n; e += G.nt) dst[(size_t)e * ld] = (double)yr[e];
  }

  // panel rows [0, rows) of Lp for stage j: rows outside [r0, r1) are zero
  // (a consumer writes the W-rows of a split or paired segment)
  __device__ void store_panel(int j, int r0, int r1, int rows, Grp G) const {
    double* Pd = d->Lp + (size_t)j * R * n;
    float* Pf = mixed ? d->Lpf + (size_t)j * R * n : nullptr;
    for (int e = G.tid; e < rows * n; e += G.nt) {
      const int r = e / n, c = e - r * n;
      const TZ v = (r >= r0 && r < r1) ? Z[r * ldZ + c] : TZ(0);
      Pd[e] = (double)v;
      if (mixed) Pf[e] = (float)v;
    }
  }

  // rotate the panel after the Schur update of stage i: the updated blocks
  // become stage i+1's inputs, the next ones are loaded
  __device__ void rotate(int i, int j, bool withW, Grp G) const {
    const double* none = nullptr;
    if (m) copy_blk(Z + oG * ldZ, ldZ, T + oG * ldT, ldT, m, n, G);          // G_{i+1}
    if (withW) copy_blk(Z + oW * ldZ, ldZ, T + oW * ldT, ldT, n, n, G);      // W_{i+1}
    if ((i + 1 < g.len - 1) || g.hasF) load_blk<LU>(Z, ldZ, Dp(Ein, j + 1), none, n, n, false, G);
    gsync(G);
    if (withW) load_blk<LU>(T + oW * ldT, ldT, none, none, n, n, false, G);     // W_{i+2} <- 0
    if (i + 2 < g.len) {
      load_blk<LU>(T, ldT, Dp(Din, j + 2), Dp(D2, j + 2), n, n, false, G);
      if (m) load_blk<LU>(T + oG * ldT, ldT, Gp(Gin, j + 2), Gp(G2, j + 2), m, n, false, G);
    } else {
      load_blk<LU>(T, ldT, none, none, n, n, false, G);
      if (m) load_blk<LU>(T + oG * ldT, ldT, none, none, m, n, false, G);
    }
    gsync(G);
  }

  // the next level's slots of segment k (not on the top level)
  __device__ void store_slots(int k, bool eg, bool wr, Grp G) const {
    if (eg && g.hasF) {
      store_blk(d->DB + (size_t)k * nn, T, ldT, n, n, false, true, G);             // -F^ F^T
      if (m) store_blk(d->GB + (size_t)k * mn, T + oG * ldT, ldT, m, n, false, false, G);  // -G^ F^T
    }
    if (wr) {
      store_blk(d->DA + (size_t)(k - 1) * nn, T + oW * ldT + oW, ldT, n, n, false, true, G);  // A~_k
      if (m) store_blk(d->GA + (size_t)(k - 1) * mn, T + oW * ldT + oG, ldT, n, m, true, false, G);  // Q~_k
      if (g.hasF) store_blk(d->EN + (size_t)(k - 1) * nn, T + oW * ldT, ldT, n, n, true, false, G);  // H~_k
    }
    if (eg && m) store_blk(d->Rpart + (size_t)k * m * m, T + oG * ldT + oG, ldT, m, m, false, true, G);
  }
};

// Forward substitution task of the solve kernels (defined below); the factor
// kernel of a bordered pass runs it for the top level (corner solve and the
// backward sweep of the top level) right after the corner.
template <typename TS>
__device__ void forward_task(const Task tk, const LevelDesc* __restrict__ descs, double* b, int ldb, int nr,
                             const int* skip, unsigned char* smraw, Grp G, int fwd_done, int c0 = 0);

// MINB: CTAs per SM the register allocation must allow. Launches of CTA pairs
// (one CTA per SM, latency-bound) take the unconstrained allocation (1);
// the others four (at most 64 registers), so that several segment CTAs share
// an SM when shared memory allows it.
// TC: the instantiation with the tensor-core Schur products (mixed launches
// that use them); the others carry none of that code.
// One segment task of the factorization by the whole CTA (or, with `pair`,
// by this CTA's half of a two-CTA cluster): the body of k_factor, also run
// task after task by the persistent kernel. `bad`, `tslot`, `tbar`: shared
// variables of the caller (breakdown flag, TMEM address slot, mbarrier).
template <typename TZ, bool TC>
__device__ __forceinline__ void factor_task(const Task tk, const LevelDesc* __restrict__ descs,
                                            const double* __restrict__ uD, const double* __restrict__ uE,
                                            const double* __restrict__ uG, const double* __restrict__ uR,
                                            Info* info, int pair, double* yb, int ldyb, int top_solve, int dbl,
                                            int tcm, unsigned char* smraw, int& bad, uint32_t& tslot,
                                            uint64_t& tbar) {
  const unsigned rank = pair ? cluster_rank() : 0u;
  const LevelDesc& d = descs[tk.desc];
  constexpr bool mixed = sizeof(TZ) == 4;
  const FacLayout lay = fac_layout(d.n, d.m, (int)sizeof(TZ), d.P > 1, dbl != 0);
  if (!task_geometry_ok(d, tk.seg, smraw, lay.total)) return;  // debug build only (both CTAs of a pair alike)
  const FacCtx<TZ, 4> cx(d, tk.seg, smraw, lay, uD, uE, uG);
  const int n = cx.n, m = cx.m, R = cx.R, ldD = cx.ldD, ldZ = cx.ldZ, ldT = cx.ldT, oG = cx.oG, oW = cx.oW;
  double* const Dfac = cx.Dfac;
  double* const rinv = cx.rinv;
  double* const T = cx.T;
  TZ* const M = cx.M;
  TZ* const rinvZ = cx.rinvZ;
  TZ* const Z = cx.Z;
  int* const tab = cx.tab;
  const SegGeom g = cx.g;
  const int mode = pair ? kPair : (g.hasW && !mixed) ? kSplit : kWhole;
  // consumer buffers of the pair layout: buffer 0 is (M, rinvZ, Z rows [0, n+m)),
  // buffer 1 reuses the pivot block, rinv and the first rows of T, which a
  // consumer CTA has no other use for
  auto Mbuf = [&](int b) { return b ? (TZ*)Dfac : M; };
  auto rinvbuf = [&](int b) { return b ? (TZ*)rinv : rinvZ; };
  auto Zbuf = [&](int b) { return b ? (TZ*)T : Z; };
  const bool eg = mode != kPair || rank == 0;       // this CTA holds the E/G rows
  const bool wr = g.hasW && (mode != kPair || rank == 1);  // this CTA holds the W rows

  // tensor-core Schur products (mixed whole-CTA layout without the second
  // pivot buffer, whose region then stages the operands)
  const bool use_tc = TC && mixed && tcm && mode == kWhole && !dbl;
  const uint32_t tc_cols = ((lay.Rs + 15) & ~15) <= 64 ? 64u : 128u;
  uint32_t tmem = 0u, tphase = 0u;
  if constexpr (TC) {
    if (use_tc) {
      if (threadIdx.x < 32) tc::alloc(&tslot, tc_cols);
      if (threadIdx.x == 0) tc::mbar_init(&tbar);
      tc::fence_before();
    }
  }
  // An FP64 pair's consumer factors the first stage's pivot block as well,
  // in the second pivot buffer (no hand-off ever writes there), so that its
  // W-rows' panel solve of that stage runs while the producer's sweep and
  // hand-off are still under way; the result is bitwise the producer's
  // (potrf_sm + panel_operand is the fused sweep's arithmetic).
  const bool own0 = mode == kPair && rank == 1 && g.hasW && dbl && !mixed;
  double* const Dfac2c = (double*)(smraw + lay.oDfac2);
  double* const rinv2c = (double*)(smraw + lay.oRinv2);
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < lay.Rs * ldT; e += blockDim.x) T[e] = 0.0;
  if (eg || own0) potrf_table(tab, n);
  __syncthreads();
  if constexpr (TC) {
    if (use_tc) {
      tc::fence_after();
      tmem = tslot;
    }
  }
  cx.load_first(eg, wr, cta_grp());
  if (own0) cx.load_D(Dfac2c, g.f, cta_grp());
  __syncthreads();
  if (mode == kPair) {
    // both CTAs have started before any remote store
    cluster_arrive();
    cluster_wait();
  }

  const bool producer = mode == kWhole || (mode == kSplit && (int)threadIdx.x < kRoleThreads) ||
                        (mode == kPair && rank == 0);
  auto store_pivot = [&](int j, const double* Dp_, const double* rv, const TZ* Ms, Grp G) {
    cx.store_pivot(j, Dp_, rv, Ms, G);
  };
  auto store_panel = [&](int j, int r0, int r1, int rows, Grp G) { cx.store_panel(j, r0, r1, rows, G); };
  // hand the trsm operand (strict lower triangle of Msrc, ld ldD), its
  // 1/diag and panel rows [r0, r1) of stage i to the consumer CTA of a pair
  auto push_stage = [&](int i, const TZ* Msrc, const TZ* rsrc, int r0, int r1, Grp G) {
    const int b = i & 1;
    const unsigned aM = cluster_addr(Mbuf(b), 1), aR = cluster_addr(rinvbuf(b), 1),
                   aZ = cluster_addr(Zbuf(b), 1);
    const int ntri = (n - 1) * n / 2;
    for (int e = G.tid; e < ntri; e += G.nt) {
      int a, c;
      tri_rc(e, a, c);
      const int off = (a + 1) * ldD + c;
      st_cluster(aM + off * (unsigned)sizeof(TZ), Msrc[off]);
    }
    for (int e = G.tid; e < n; e += G.nt) st_cluster(aR + e * (unsigned)sizeof(TZ), rsrc[e]);
    for (int e = G.tid; e < (r1 - r0) * n; e += G.nt) {
      const int r = r0 + e / n, c = e - (r - r0) * n;
      const int off = r * ldZ + c;
      st_cluster(aZ + off * (unsigned)sizeof(TZ), Z[off]);
    }
  };
  auto rotate = [&](int i, int j, bool withW, Grp G) { cx.rotate(i, j, withW, G); };

  if (producer && mode == kSplit) {
    // FP64, E- and G-rows on warps 0-3 (the consumer warps run the W-rows)
    const Grp P{(int)threadIdx.x, kRoleThreads, kBarProd};
    const int pr1 = n + m;
    potrf_sm(Dfac, ldD, n, rinv, tab, &bad, false);
    for (int i = 0; i < g.len; ++i) {
      const int j = g.f + i;
      const bool eRows = (i < g.len - 1) || g.hasF;
      const int r0 = eRows ? 0 : n;
      if (threadIdx.x == 0 && bad) { record_breakdown(info, d.sys, d.nat[j], d.level); bad = 0; }
      if (i > 0) group_bar(kBarFreeM, kFactorThreads);
      panel_operand(M, Dfac, ldD, n, rinv, P);
      for (int e = P.tid; e < n; e += P.nt) rinvZ[e] = (TZ)rinv[e];
      gsync(P);
      group_arrive(kBarFullM, kFactorThreads);
      trsm_panel(Z, ldZ, r0, pr1, M, ldD, n, rinvZ, P);
      group_arrive(kBarFullZ, kFactorThreads);
      if (d.mr) cx.store_y(j, yb, ldyb, P);
      store_pivot(j, Dfac, rinv, M, P);
      store_panel(j, r0, pr1, pr1, P);
      syrk_trap(T, ldT, Z, Z, 0, ldZ, r0, pr1, r0, n, P);
      if (i + 1 < g.len) {
        // D_{i+1} is final: factor it now, then rotate the panel once the
        // consumer has read E-hat_i and G-hat_i
        copy_blk(Dfac, ldD, T, ldT, n, n, P);
        gsync(P);
        potrf_sm(Dfac, ldD, n, rinv, tab, &bad, false);
        group_bar(kBarFreeZ, kFactorThreads);
        rotate(i, j, false, P);
      }
    }
  } else if (producer) {
    // Whole CTA on the E- and G-rows (and the W-rows in the whole layout of a
    // mixed level; FP64 levels with fill-in rows split or pair). Per stage:
    // the fused pivot factorization and panel solve (warps 0-3 and 5-7)
    // while warp 4 writes the previous stage's pivot blocks from the other
    // pivot buffer; then the hand-off to the consumer, the Schur update and
    // the rotation.
    const Grp P = cta_grp();
    const Grp W4{(int)(threadIdx.x & 31), 32, -1};
    const bool w4 = (threadIdx.x >> 5) == 4;
    const int pr1 = n + m + (mode == kWhole && g.hasW ? n : 0);  // end of the CTA's panel rows
    const bool push = mode == kPair && g.hasW;
    double* const Dfac2 = (double*)(smraw + lay.oDfac2);
    double* const rinv2 = (double*)(smraw + lay.oRinv2);
    // without the second pivot buffer (dbl = 0) the pivot blocks of a stage
    // are written by the whole CTA right after its sweep
    auto Dbuf = [&](int b) { return b && dbl ? Dfac2 : Dfac; };
    auto rvbuf = [&](int b) { return b && dbl ? rinv2 : rinv; };
    for (int i = 0; i < g.len; ++i) {
      const int j = g.f + i;
      const int cur = i & 1;
      const bool eRows = (i < g.len - 1) || g.hasF;
      const int r0 = eRows ? 0 : n;
      if (!dbl) {
        potrf_trsm_sm(Dbuf(cur), ldD, n, rvbuf(cur), M, tab, &bad, Z, ldZ, r0, pr1, true);
      } else if (w4) {
        if (i > 0) store_pivot(j - 1, Dbuf(cur ^ 1), rvbuf(cur ^ 1), nullptr, W4);
      } else {
        potrf_trsm_sm(Dbuf(cur), ldD, n, rvbuf(cur), M, tab, &bad, Z, ldZ, r0, pr1);
      }
      __syncthreads();
      if (threadIdx.x == 0 && bad) { record_breakdown(info, d.sys, d.nat[j], d.level); bad = 0; }
      if (!dbl) store_pivot(j, Dfac, rinv, nullptr, P);  // read before the copy of D_{i+1} below
      if (d.mr) cx.store_y(j, yb, ldyb, P);
      if (push) {
        for (int e = P.tid; e < n; e += P.nt) rinvZ[e] = (TZ)rvbuf(cur)[e];
        __syncthreads();
        if (i > 0) cluster_wait();  // the consumer is done with stage i-2 (buffer i % 2)
        push_stage(i, M, rinvZ, r0, n + m, P);
        cluster_arrive();
      }
      store_panel(j, r0, pr1, mode == kWhole ? R : n + m, P);
      bool tc_done = false;
      if constexpr (mixed && TC) {
        if (use_tc) {
          if (!syrk_tc(T, ldT, (const float*)Z, ldZ, r0, pr1, n, smraw + lay.oDfac, tmem, &tbar, tphase & 1, tcm) &&
              threadIdx.x == 0)
            record_timeout(info, d.sys, d.nat[j], d.level);
          ++tphase;
          tc_done = true;
        }
      }
      if (!tc_done) syrk_trap(T, ldT, Z, Z, 0, ldZ, r0, pr1, r0, n, P);
      if (i + 1 < g.len) {
        copy_blk(Dbuf(cur ^ 1), ldD, T, ldT, n, n, P);                      // D_{i+1}
        rotate(i, j, mode == kWhole && g.hasW, P);
      } else if (dbl) {
        store_pivot(j, Dbuf(cur), rvbuf(cur), nullptr, P);
      }
    }
    if (push) cluster_wait();  // phase of the last stage
  } else if (wr) {
    // fill-in rows W
    const Grp C = mode == kSplit ? Grp{(int)threadIdx.x - kRoleThreads, kRoleThreads, kBarCons} : cta_grp();
    for (int i = 0; i < g.len; ++i) {
      const int j = g.f + i;
      const bool eRows = (i < g.len - 1) || g.hasF;
      const int r0 = eRows ? 0 : n;
      const int b = mode == kPair ? (i & 1) : 0;
      const bool own = i == 0 && own0;
      if (mode == kSplit) {
        group_bar(kBarFullM, kFactorThreads);
      } else if (own) {
        cluster_arrive();  // (stage -1)
        int bad0 = 0;      // a breakdown is the producer's to report
        potrf_sm(Dfac2c, ldD, n, rinv2c, tab, &bad0);
        panel_operand(Dfac2c, Dfac2c, ldD, n, rinv2c, cta_grp());  // in place: M_cj = L_cj / L_jj
        __syncthreads();
        trsm_panel(Z, ldZ, oW, R, (const TZ*)Dfac2c, ldD, n, (const TZ*)rinv2c, cta_grp());
        cluster_wait();    // stage 0's E- and G-rows are in buffer 0
      } else {
        cluster_arrive();  // done with stage i-1
        cluster_wait();    // stage i's blocks are in buffer b
      }
      if (!own) trsm_panel(Z, ldZ, oW, R, Mbuf(b), ldD, n, rinvbuf(b), C);
      if (mode == kSplit && i + 1 < g.len) group_arrive(kBarFreeM, kFactorThreads);
      {
        double* Pd = d.Lp + (size_t)j * R * n + (size_t)oW * n;
        float* Pf = mixed ? d.Lpf + (size_t)j * R * n + (size_t)oW * n : nullptr;
        for (int e = C.tid; e < n * n; e += C.nt) {
          const int r = e / n, c = e - r * n;
          const TZ v = Z[(oW + r) * ldZ + c];
          Pd[e] = (double)v;
          if (mixed) Pf[e] = (float)v;
        }
      }
      if (mode == kSplit) group_bar(kBarFullZ, kFactorThreads);
      syrk_trap(T, ldT, Zbuf(b), Z, oW, ldZ, oW, R, r0, n, C);
      if (i + 1 < g.len) {
        if (mode == kSplit) group_arrive(kBarFreeZ, kFactorThreads);
        copy_blk(Z + oW * ldZ, ldZ, T + oW * ldT, ldT, n, n, C);               // W_{i+1}
        gsync(C);
        load_blk(T + oW * ldT, ldT, (const double*)nullptr, (const double*)nullptr, n, n, false, C);  // W_{i+2} <- 0
        gsync(C);
      }
    }
  }
  __syncthreads();

  if (!d.is_top) {
    cx.store_slots(tk.seg, eg, wr, cta_grp());
  } else if (m) {
    // corner: R-hat = chol(R + sum_k R~_k over every level), in a fixed order:
    // the lower levels' partials are summed by the pair's idle CTA while this
    // one runs the stages (or here, without a pair), then R and this level's
    // own partial are added
    double* Psum = (double*)(smraw + lay.oCorner);
    auto part = [&](int p, int o) { return d.Rpart_all[(size_t)p * m * m + o]; };
    if (mode == kPair && rank == 1) {
      const unsigned aP = cluster_addr(Psum, 0);
      sum_partials(cta_grp(), m * m, d.nRpart_all, part,
                   [&](int o, double v) { st_cluster(aP + o * (unsigned)sizeof(double), v); });
    } else if (mode != kPair) {
      sum_partials(cta_grp(), m * m, d.nRpart_all, part, [&](int o, double v) { Psum[o] = v; });
    }
    if (mode == kPair) {
      cluster_arrive();
      cluster_wait();
    } else {
      __syncthreads();
    }
  }
  if (d.is_top && eg && m) {
    double* Psum = (double*)(smraw + lay.oCorner);
    double* Rs = Dfac;  // reuse
    const int ldR = odd(m);
    const double* Ru = uR + d.offR;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = e / m, c = e - r * m;
      Rs[r * ldR + c] = (Ru[e] + Psum[e]) + T[(oG + r) * ldT + oG + c];
    }
    __syncthreads();
    // by one warp: at m <= 16 a per-column block barrier costs more than the
    // column's work (the operations per element are potrf_sm's)
    if (threadIdx.x < 32)
      corner_factor<true>(Rs, ldR, m, d.mr, rinv, tab, d, info, nullptr, Grp{(int)threadIdx.x, 32, -1});
    __syncthreads();
  }
  if constexpr (!mixed) {
    // bordered pass, top level: the corner solve x_g = R-hat^{-T} y_g and the
    // backward sweep of the top level's stages (Algorithm 3, sequential
    // phase) here instead of in a launch of their own; the blocks it reads
    // were written by this CTA, and the shared memory is free by now
    if (top_solve && d.is_top && d.mr && yb && eg) {
      __syncthreads();
      forward_task<double>(tk, descs, yb, ldyb, 1, nullptr, smraw, cta_grp(), 1);
    }
  }
  if (mode == kPair) {
    // a segment without fill-in leaves its consumer idle; every CTA of the
    // pair then meets once more, after which no remote store is in flight
    cluster_arrive();
    cluster_wait();
  }
  if constexpr (TC) {
    if (use_tc) {
      tc::fence_before();
      __syncthreads();
      if (threadIdx.x < 32) tc::dealloc(tmem, tc_cols);
    }
  }
}

template <typename TZ, int MINB, bool TC = false>
__global__ void __launch_bounds__(kFactorThreads, MINB) k_factor(const LevelDesc* __restrict__ descs,
                                                           const Task* __restrict__ tasks,
                                                           const double* __restrict__ uD,
                                                           const double* __restrict__ uE,
                                                           const double* __restrict__ uG,
                                                           const double* __restrict__ uR,
                                                           Info* info, int pair, double* yb, int ldyb,
                                                           int top_solve, int dbl, int tcm) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  __shared__ uint32_t tslot;               // TMEM address of the tensor-core accumulator
  __shared__ __align__(8) uint64_t tbar;   // its completion mbarrier
  factor_task<TZ, TC>(tasks[pair ? blockIdx.x >> 1 : blockIdx.x], descs, uD, uE, uG, uR, info, pair, yb, ldyb,
                      top_solve, dbl, tcm, smraw, bad, tslot, tbar);
}

// ---------------------------------------------------------------------------
// One-stage segments on a cluster of C CTAs (2 <= C <= 8), FP64. On the deep
// levels of a recursive plan every segment is a single stage (its pivot
// block with the E-, G- and W-rows of its panel), and the levels have few
// tasks: one or two CTAs per task leave most SMs idle while the stage's
// panel solve and Schur update (Alg. 1) run at two FP64 FMAs per clock per
// SM. Here the stage is spread over the cluster:
//   - every CTA factors the pivot block itself and solves a contiguous band
//     of about 1/C of the panel rows with the fused sweep (potrf_trsm_sm),
//     then stores its solved rows into every other CTA's shared memory;
//   - every CTA applies the Schur update to a band of trapezoid rows holding
//     about 1/C of the elements and stores the results into the shared
//     memory of the CTA that writes that block's slots for the next level
//     (rank 0: E- and G-rows, rank 1: W-rows);
//   - the last rank writes the pivot blocks, each CTA its panel rows.
// Three split-phase cluster barriers order the exchanges. Every element is
// computed by the same operations in the same order as in the one- and
// two-CTA layouts, so the results are bitwise theirs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void clus_task(const Task tk, const LevelDesc* __restrict__ descs,
                                          const double* __restrict__ uD, const double* __restrict__ uE,
                                          const double* __restrict__ uG, Info* info, double* yb, int ldyb, int C,
                                          unsigned char* smraw, int& bad) {
  const int rank = (int)cluster_rank();
  const LevelDesc& d = descs[tk.desc];
  const FacLayout lay = fac_layout(d.n, d.m, 8, true, false);
  if (!task_geometry_ok(d, tk.seg, smraw, lay.total)) return;  // debug build only (every CTA alike)
  const FacCtx<double, 4> cx(d, tk.seg, smraw, lay, uD, uE, uG);
  const int n = cx.n, m = cx.m, ldD = cx.ldD, ldZ = cx.ldZ, ldT = cx.ldT, oG = cx.oG, oW = cx.oW;
  const SegGeom g = cx.g;
  const int j = g.f, s = cx.s, tid = threadIdx.x, nt = blockDim.x;
  double* const Dfac = cx.Dfac;
  double* const rinv = cx.rinv;
  double* const T = cx.T;
  double* const M = cx.M;
  double* const Z = cx.Z;
  // panel rows [r0, r1): the E-rows when a next separator exists, the G-rows,
  // the W-rows when a previous one does
  const int r0 = g.hasF ? 0 : n, r1 = g.hasW ? cx.R : n + m, h = r1 - r0;
  // this CTA's band of the panel solve: equal row counts
  const int t0 = r0 + h * rank / C, t1 = r0 + h * (rank + 1) / C;
  // its band of the Schur update: row r0 + a holds a + 1 elements; band q
  // starts at the first row whose preceding rows hold >= q/C of the total
  const int tot = h * (h + 1) / 2;
  auto band0 = [&](int q) {
    const int want = (tot * q + C - 1) / C;
    int a = 0;
    while (a < h && a * (a + 1) / 2 < want) ++a;
    return r0 + a;
  };
  const int s0 = band0(rank), s1 = band0(rank + 1);
  cluster_arrive();  // this CTA runs: the others may store into its shared memory after their wait
  if (tid == 0) bad = 0;
  potrf_table(cx.tab, n);
  // inputs: the pivot block D_j, the panel rows of the solve band, and the
  // initial values of the Schur band (A_k and Q_k^T in its W-rows, zero
  // elsewhere). Every load is an L2 round trip, so the three sets form one
  // list whose loads go out eight per thread before any store: element e
  // of the list is D_j's (e < nD), then the band's panel rows (< nD + nZ),
  // then the W-row part [oG, R) of the Schur band's rows (the rest of those
  // rows is zeroed separately). Sums of two slots add in the order of
  // load_blk, so the values are those of the other layouts.
  {
    const int nD = n * n, nZ = (t1 - t0) * n;
    const int wa0 = max(s0, oW), nTr = max(0, s1 - wa0), nTc = m + n;
    const int nIn = nD + nZ + nTr * nTc;
    const double* const D1 = cx.Din + (size_t)j * cx.nn;
    const double* const D2 = cx.D2 ? cx.D2 + (size_t)j * cx.nn : nullptr;
    constexpr int U = 8;
    for (int e0 = tid; e0 < nIn; e0 += U * nt) {
      double v[U];
      int dst[U];  // offset in doubles from smraw's Dfac (Dfac, Z and T are one allocation)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nt;
        dst[u] = -1;
        v[u] = 0.0;
        if (e < nD) {
          const int r = e / n, c = e - r * n;
          v[u] = D2 ? D1[e] + D2[e] : D1[e];
          dst[u] = (int)(&Dfac[r * ldD + c] - Dfac);
        } else if (e < nD + nZ) {
          const int f = e - nD, r = t0 + f / n, c = f - (r - t0) * n;
          if (r < n) v[u] = cx.Ein[(size_t)j * cx.nn + r * n + c];  // E_j
          else if (r < oW) {                                         // G_j (+ its second slot)
            const size_t o = (size_t)j * cx.mn + (r - oG) * n + c;
            v[u] = cx.G2 ? cx.Gin[o] + cx.G2[o] : cx.Gin[o];
          } else v[u] = cx.Ein[(size_t)s * cx.nn + c * n + (r - oW)];  // W_1 = E[s]^T
          dst[u] = (int)(&Z[r * ldZ + c] - Dfac);
        } else if (e < nIn) {
          const int f = e - nD - nZ, a = wa0 + f / nTc, b = oG + (f - (a - wa0) * nTc);
          if (b >= oW) {  // A_k = D_s (+ its second slot)
            const size_t o = (size_t)s * cx.nn + (a - oW) * n + (b - oW);
            v[u] = cx.D2 ? cx.Din[o] + cx.D2[o] : cx.Din[o];
          } else {        // Q_k^T = G_s^T
            const size_t o = (size_t)s * cx.mn + (b - oG) * n + (a - oW);
            v[u] = cx.G2 ? cx.Gin[o] + cx.G2[o] : cx.Gin[o];
          }
          dst[u] = (int)(&T[a * ldT + b] - Dfac);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dst[u] >= 0) Dfac[dst[u]] = v[u];
    }
    // the rest of the Schur band's rows: zero
    for (int e = tid; e < (s1 - s0) * ldT; e += nt) {
      const int a = s0 + e / ldT, b = e - (a - s0) * ldT;
      if (!(a >= oW && b >= oG && b < cx.R)) T[a * ldT + b] = 0.0;
    }
  }
  __syncthreads();
  potrf_trsm_sm(Dfac, ldD, n, rinv, M, cx.tab, &bad, Z, ldZ, t0, t1, true);
  __syncthreads();
  if (d.mr) {
    const int ry = oG + m - d.mr;  // the bordered row: y_j of the forward substitution
    if (ry >= t0 && ry < t1) cx.store_y(j, yb, ldyb, cta_grp());
  }
  cluster_wait();  // every CTA of the cluster runs
  {
    for (int q = 1; q < C; ++q) {
      const unsigned az = cluster_addr(Z, (unsigned)((rank + q) % C));
      for (int e = tid; e < (t1 - t0) * n; e += nt) {
        const int r = t0 + e / n, c = e - (r - t0) * n;
        const unsigned off = (unsigned)(r * ldZ + c) * 8u;
        st_cluster(az + off, Z[r * ldZ + c]);
      }
    }
  }
  cluster_arrive();
  // the pivot blocks: by the last rank, which stores no slots when C > 2
  if (rank == C - 1) {
    if (tid == 0 && bad) record_breakdown(info, d.sys, d.nat[j], d.level);
    cx.store_pivot(j, Dfac, rinv, M, cta_grp());
  }
  {
    double* Pd = d.Lp + (size_t)j * cx.R * n;
    const int p0 = rank == 0 ? 0 : t0;  // rank 0 also writes the zero rows [0, r0)
    for (int e = tid; e < (t1 - p0) * n; e += nt) {
      const int r = p0 + e / n, c = e - (r - p0) * n;
      Pd[(size_t)r * n + c] = r >= r0 ? Z[r * ldZ + c] : 0.0;
    }
  }
  cluster_wait();  // every solved panel row is here
  syrk_trap(T, ldT, Z, Z, 0, ldZ, s0, s1, r0, n, cta_grp());
  {
    const unsigned a0 = cluster_addr(T, 0u), a1 = cluster_addr(T, 1u);
    const int w0 = s0 - r0;  // row s0 + i holds w0 + i + 1 elements
    const int cnt = (s1 - s0) * w0 + (s1 - s0) * (s1 - s0 + 1) / 2;
    // (a, b) of element tid of the band, then advanced by nt along the rows
    int a = s0, b = r0 + tid;
    while (a < s1 && b > a) { b -= a - r0 + 1; ++a; }
    for (int e = tid; e < cnt; e += nt) {
      if (e != tid) {
        b += nt;
        while (b > a) { b -= a - r0 + 1; ++a; }
      }
      const int owner = a < oW ? 0 : 1;
      if (owner != rank)
        st_cluster((owner ? a1 : a0) + (unsigned)(a * ldT + b) * 8u, T[a * ldT + b]);
    }
  }
  cluster_arrive();
  cluster_wait();  // the slot owners hold their rows of the update
  if (rank == 0) cx.store_slots(tk.seg, true, false, cta_grp());
  else if (rank == 1) cx.store_slots(tk.seg, false, g.hasW, cta_grp());
}

__global__ void __launch_bounds__(kFactorThreads, 2) k_factor_clus(const LevelDesc* __restrict__ descs,
                                                                   const Task* __restrict__ tasks,
                                                                   const double* __restrict__ uD,
                                                                   const double* __restrict__ uE,
                                                                   const double* __restrict__ uG, Info* info,
                                                                   double* yb, int ldyb, int C) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  clus_task(tasks[blockIdx.x / C], descs, uD, uE, uG, info, yb, ldyb, C, smraw, bad);
}


// ---------------------------------------------------------------------------
// Small blocks (n <= kWarpMaxN): one warp per segment task, every step of a
// stage warp-synchronous, several tasks per CTA with a shared-memory slice
// each. The CTA kernel's role split needs blocks large enough to keep eight
// warps busy; at n = 6 a stage is a few hundred FMAs, and what counts is how
// many independent stage chains an SM interleaves. The operations per
// element are those of the CTA kernel, in the same order.
// ---------------------------------------------------------------------------

// Z[r0:r1) <- Z[r0:r1) L^{-T} by one warp, one panel row per lane: the
// division-free substitution of trsm_panel, in the same order per element.
template <typename TZ>
__device__ void trsm_w(TZ* Z, int ldz, int r0, int r1, const TZ* M, int ldm, int n, const TZ* rinv, int lane) {
  for (int r = r0 + lane; r < r1; r += 32) {
    TZ* z = Z + r * ldz;
    for (int j = 0; j < n - 1; ++j) {
      const TZ zj = z[j];
      for (int c = j + 1; c < n; ++c) z[c] = fma(-zj, M[c * ldm + j], z[c]);
    }
    for (int c = 0; c < n; ++c) z[c] *= rinv[c];
  }
  __syncwarp();
}

// One small-block segment task by one warp in its shared-memory slice `sm`:
// the body of k_factor_w, also run by the persistent kernel.
template <typename TZ>
__device__ __forceinline__ void factor_task_w(const Task tk, const LevelDesc* __restrict__ descs,
                                              const double* __restrict__ uD, const double* __restrict__ uE,
                                              const double* __restrict__ uG, const double* __restrict__ uR,
                                              Info* info, unsigned char* sm, int lane, double* yb, int ldyb) {
  const LevelDesc& d = descs[tk.desc];
  const FacLayout lay = fac_layout_w(d.n, d.m, (int)sizeof(TZ), d.P > 1);
  if (!task_geometry_ok(d, tk.seg, sm, lay.total)) return;  // debug build only
  const FacCtx<TZ, 1> cx(d, tk.seg, sm, lay, uD, uE, uG);
  const int n = cx.n, m = cx.m, R = cx.R, ldD = cx.ldD, ldZ = cx.ldZ, ldT = cx.ldT, oG = cx.oG;
  const SegGeom g = cx.g;
  const Grp W{lane, 32, -1};
  for (int e = lane; e < lay.Rs * ldT; e += 32) cx.T[e] = 0.0;
  pair_table_w(cx.tab, n, lane);
  cx.load_first(true, g.hasW, W);
  __syncwarp();
  const int pr1 = n + m + (g.hasW ? n : 0);
  for (int i = 0; i < g.len; ++i) {
    const int j = g.f + i;
    const bool eRows = (i < g.len - 1) || g.hasF;
    const int r0 = eRows ? 0 : n;
    const int bad = potrf_w(cx.Dfac, ldD, n, cx.rinv, cx.tab, lane);
    if (lane == 0 && bad) record_breakdown(info, d.sys, d.nat[j], d.level);
    panel_operand(cx.M, cx.Dfac, ldD, n, cx.rinv, W);
    for (int e = lane; e < n; e += 32) cx.rinvZ[e] = (TZ)cx.rinv[e];
    __syncwarp();
    trsm_w(cx.Z, ldZ, r0, pr1, cx.M, ldD, n, cx.rinvZ, lane);
    if (d.mr) cx.store_y(j, yb, ldyb, W);
    cx.store_pivot(j, cx.Dfac, cx.rinv, cx.M, W);
    cx.store_panel(j, r0, pr1, R, W);
    syrk_trap(cx.T, ldT, cx.Z, cx.Z, 0, ldZ, r0, pr1, r0, n, W);
    if (i + 1 < g.len) {
      copy_blk(cx.Dfac, ldD, cx.T, ldT, n, n, W);                                  // D_{i+1}
      __syncwarp();
      cx.rotate(i, j, g.hasW, W);
    }
  }
  __syncwarp();
  if (!d.is_top) {
    cx.store_slots(tk.seg, true, g.hasW, W);
  } else if (m) {
    // corner: R-hat = chol((R + sum of the lower levels' partials) + this level's)
    double* Rs = cx.Dfac;  // reuse (n >= m is not needed: the slice has room for q x q)
    double* Psum = (double*)(sm + lay.oCorner);
    const int ldR = odd(m);
    for (int o = lane; o < m * m; o += 32) {
      double a0 = 0.0, a1 = 0.0;
      int p = 0;
      for (; p + 1 < d.nRpart_all; p += 2) {
        a0 += d.Rpart_all[(size_t)p * m * m + o];
        a1 += d.Rpart_all[(size_t)(p + 1) * m * m + o];
      }
      if (p < d.nRpart_all) a0 += d.Rpart_all[(size_t)p * m * m + o];
      Psum[o] = a0 + a1;
    }
    __syncwarp();
    const double* Ru = uR + d.offR;
    for (int e = lane; e < m * m; e += 32) {
      const int r = e / m, c = e - r * m;
      Rs[r * ldR + c] = (Ru[e] + Psum[e]) + cx.T[(oG + r) * ldT + oG + c];
    }
    __syncwarp();
    corner_factor<true>(Rs, ldR, m, d.mr, cx.rinv, cx.tab, d, info, nullptr, W);
  }
}

template <typename TZ>
__global__ void __launch_bounds__(256, 4) k_factor_w(const LevelDesc* __restrict__ descs,
                                                  const Task* __restrict__ tasks, int ntasks,
                                                  const double* __restrict__ uD, const double* __restrict__ uE,
                                                  const double* __restrict__ uG, const double* __restrict__ uR,
                                                  Info* info, int slice, double* yb, int ldyb) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int t = blockIdx.x * (blockDim.x >> 5) + wid;
  if (t >= ntasks) return;  // whole warp
  factor_task_w<TZ>(tasks[t], descs, uD, uE, uG, uR, info, smraw + (size_t)wid * slice, lane, yb, ldyb);
}

// ---------------------------------------------------------------------------
// Persistent factorization: one launch runs every segment task of every level
// (Algorithm 1's parallel phase and, level by level, the reduced systems of
// Eq. (7)). CTAs take work items by ticket (atomicAdd) from a list in
// topological order: level by level, and within a level the most expensive
// first (longest-processing-time order), so long systems start first and the
// short ones fill the tail. An item of level >= 2 reads slots written by its
// feeder tasks one level down; its CTA waits (thread 0, acquire loads with a
// growing sleep, bounded by wait_cycles) until the feeders' release
// increments reach `need`. A CTA only ever waits on items with smaller
// tickets, which CTAs already running hold, so every wait has a producer in
// progress. A wait that runs out records KKT_ERR_TIMEOUT (with the waiting
// task's system, natural stage and level), skips its task and still releases
// its consumers, so nothing waits forever.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_release_gpu(int* p) {
  asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename TZ>
__global__ void __launch_bounds__(kFactorThreads, 3)
    k_factor_persist(const LevelDesc* __restrict__ descs, const Task* __restrict__ tasks,
                     const PItem* __restrict__ items, int nitems, const PCons* __restrict__ cons, int* ready,
                     const double* __restrict__ uD, const double* __restrict__ uE, const double* __restrict__ uG,
                     const double* __restrict__ uR, Info* info, int slice, int dbl, long long wait_cycles) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t tbar;
  __shared__ int cur, ok;
  int* const ticket = ready + nitems;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(ticket, 1);
    __syncthreads();
    const int it = cur;
    if (it >= nitems) break;
    const PItem w = items[it];
    if (threadIdx.x == 0) {
      int good = 1;
      if (w.need > 0) {
        const long long t0 = clock64();
        unsigned ns = 64;
        while (ld_acquire_gpu(ready + it) < w.need) {
          if (clock64() - t0 > wait_cycles) {
            good = 0;
            break;
          }
          __nanosleep(ns);
          if (ns < 2048) ns *= 2;
        }
        __threadfence();
      }
      ok = good;
      if (!good) {
        const Task tk = tasks[w.first];
        const LevelDesc& d = descs[tk.desc];
        record_timeout(info, d.sys, d.nat[d.seg[tk.seg]], d.level);
      }
    }
    __syncthreads();
    if (ok) {
      if (!w.warp) {
        factor_task<TZ, false>(tasks[w.first], descs, uD, uE, uG, uR, info, 0, nullptr, 1, 0, dbl, 0, smraw, bad,
                               tslot, tbar);
      } else {
        const int wid = threadIdx.x >> 5;
        if (wid < w.cnt)
          factor_task_w<TZ>(tasks[w.first + wid], descs, uD, uE, uG, uR, info, smraw + (size_t)wid * slice,
                            threadIdx.x & 31, nullptr, 1);
      }
    }
    __syncthreads();
    // release: every thread's writes of this item precede the barrier; the
    // fence makes them visible device-wide before the counters move
    if (threadIdx.x == 0) {
      __threadfence();
      for (int c = 0; c < w.ncons; ++c) atomicAdd(ready + cons[w.cons0 + c].item, cons[w.cons0 + c].weight);
    }
  }
}

// ---------------------------------------------------------------------------
// Solve. TS = double: FP64 factor and vectors. TS = float: the FP32 factor
// copy of a mixed level and FP32 vectors (the correction solves of iterative
// refinement). Global vectors are FP64 in both cases.
// ---------------------------------------------------------------------------

// rhs / solution rows of stage j at this level: the caller's b at level 1
// (rows offB + j n, stride ldb), this level's X array otherwise.
struct VecView {
  double* p;
  int ld;
};

__device__ __forceinline__ VecView level_vec(const LevelDesc& d, double* b, int ldb, int j, int c0) {
  VecView v;
  if (d.level == 1) { v.p = b + (size_t)(d.offB + (long long)j * d.n) * ldb; v.ld = ldb; }
  else { v.p = d.X + (size_t)j * d.n * kRhsChunk + c0; v.ld = kRhsChunk; }
  return v;
}

// dst (rows x nr, smem ld) <- src rows (global, stride lds) (+ src2, stride kRhsChunk)
template <typename TS>
__device__ void load_vec(TS* dst, int ldd, const double* src, int lds, const double* src2, int rows,
                         int nr, Grp G) {
  if (src2) {
    for (int e = G.tid; e < rows * nr; e += G.nt) {
      const int r = e / nr, c = e - r * nr;
      dst[r * ldd + c] = (TS)(src[(size_t)r * lds + c] + src2[(size_t)r * kRhsChunk + c]);
    }
  } else {
    for (int e = G.tid; e < rows * nr; e += G.nt) {
      const int r = e / nr, c = e - r * nr;
      dst[r * ldd + c] = (TS)src[(size_t)r * lds + c];
    }
  }
}

template <typename TS>
__device__ void store_vec(double* dst, int ldd, const TS* src, int lds, int rows, int nr, Grp G) {
  for (int e = G.tid; e < rows * nr; e += G.nt) {
    const int r = e / nr, c = e - r * nr;
    dst[(size_t)r * ldd + c] = (double)src[r * lds + c];
  }
}

__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Asynchronous global -> shared copy of one 4- or 8-byte element (no
// register staging; completes at cp_async_wait).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// every group but the two most recent ones complete
__device__ __forceinline__ void cp_async_wait_2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

// t <- L^{-1} t (forward) or t <- L^{-T} t (backward) for nr columns, one
// warp per column (warp-synchronous: shuffles, no block barriers). Rows i
// and i + 32 of a column live in lane i. Forward uses M (columns of L divided
// by their diagonal): u_i -= M_ij u_j, x = u * rinv. Backward uses MR (rows
// of L divided by their diagonal): u_i -= MR_ji u_j for i < j, x = u * rinv.
// The group's warps take the columns in turn; ends with the group's barrier.
template <typename TS>
__device__ void trsv_warp(TS* t, int ldt, const TS* M, int ldl, const TS* rinv, int n, int nr,
                          bool backward, Grp G) {
  const int lane = G.tid & 31, warp = G.tid >> 5, nw = G.nt >> 5;
  const int i0 = lane, i1 = lane + 32;
  for (int c = warp; c < nr; c += nw) {
    TS u0 = i0 < n ? t[i0 * ldt + c] : TS(0);
    if (n <= 32) {  // one row per lane (warp-uniform branch: no predicated FP64 slots)
      const int ir = i0 < n ? i0 : n - 1;  // clamp the multiplier row of idle lanes
      if (!backward) {
        int j = 0;
        for (; j + 4 < n; j += 4) {  // multipliers of four steps loaded ahead
          const TS m0 = M[ir * ldl + j], m1 = M[ir * ldl + j + 1], m2 = M[ir * ldl + j + 2],
                   m3 = M[ir * ldl + j + 3];
          TS uj = shfl_idx(u0, j);
          if (i0 > j) u0 = fma(-m0, uj, u0);
          uj = shfl_idx(u0, j + 1);
          if (i0 > j + 1) u0 = fma(-m1, uj, u0);
          uj = shfl_idx(u0, j + 2);
          if (i0 > j + 2) u0 = fma(-m2, uj, u0);
          uj = shfl_idx(u0, j + 3);
          if (i0 > j + 3) u0 = fma(-m3, uj, u0);
        }
        for (; j < n - 1; ++j) {
          const TS uj = shfl_idx(u0, j);
          if (i0 > j) u0 = fma(-M[ir * ldl + j], uj, u0);
        }
      } else {
        int j = n - 1;
        for (; j - 3 > 0; j -= 4) {
          const TS m0 = M[j * ldl + ir], m1 = M[(j - 1) * ldl + ir], m2 = M[(j - 2) * ldl + ir],
                   m3 = M[(j - 3) * ldl + ir];
          TS uj = shfl_idx(u0, j);
          if (i0 < j) u0 = fma(-m0, uj, u0);
          uj = shfl_idx(u0, j - 1);
          if (i0 < j - 1) u0 = fma(-m1, uj, u0);
          uj = shfl_idx(u0, j - 2);
          if (i0 < j - 2) u0 = fma(-m2, uj, u0);
          uj = shfl_idx(u0, j - 3);
          if (i0 < j - 3) u0 = fma(-m3, uj, u0);
        }
        for (; j > 0; --j) {
          const TS uj = shfl_idx(u0, j);
          if (i0 < j) u0 = fma(-M[j * ldl + ir], uj, u0);
        }
      }
    } else {
      TS u1 = i1 < n ? t[i1 * ldt + c] : TS(0);
      if (!backward) {
        for (int j = 0; j < n - 1; ++j) {
          const TS uj = shfl_idx(j < 32 ? u0 : u1, j & 31);
          if (i0 > j) u0 = fma(-M[i0 * ldl + j], uj, u0);
          if (i1 > j && i1 < n) u1 = fma(-M[i1 * ldl + j], uj, u1);
        }
      } else {
        for (int j = n - 1; j > 0; --j) {
          const TS uj = shfl_idx(j < 32 ? u0 : u1, j & 31);
          if (i0 < j) u0 = fma(-M[j * ldl + i0], uj, u0);
          if (i1 < j) u1 = fma(-M[j * ldl + i1], uj, u1);
        }
      }
      if (i1 < n) t[i1 * ldt + c] = u1 * rinv[i1];
    }
    if (i0 < n) t[i0 * ldt + c] = u0 * rinv[i0];
  }
  gsync(G);
}

// Shared-memory view of a substitution task: double-buffered factor blocks
// (selected by value, not by a run-time array index, which would put the
// pointers in local memory), the panel vector V and the stage vector t.
template <typename TS>
struct SolveSmem {
  TS *L0, *L1, *ri0, *ri1, *Z0, *Z1, *V, *t;
  int ldL, ldZ, ldV, Rs;  // Rs: panel rows held (2n + m, or n + m on a level with P = 1)
  __device__ TS* L(int q) const { return q ? L1 : L0; }
  __device__ TS* rinv(int q) const { return q ? ri1 : ri0; }
  __device__ TS* Z(int q) const { return q ? Z1 : Z0; }
};

template <typename TS>
__device__ __forceinline__ SolveSmem<TS> solve_smem(unsigned char* sm, int n, int m, bool fill) {
  SolveSmem<TS> S;
  const SolLayout L = sol_layout(n, m, (int)sizeof(TS), fill);
  S.Rs = L.R;
  S.ldL = odd(n);
  S.ldZ = L.ldZ;
  S.ldV = L.ldV;
  S.L0 = (TS*)(sm + L.oL[0]);
  S.L1 = (TS*)(sm + L.oL[1]);
  S.ri0 = (TS*)(sm + L.oRinv[0]);
  S.ri1 = (TS*)(sm + L.oRinv[1]);
  S.Z0 = (TS*)(sm + L.oZ[0]);
  S.Z1 = (TS*)(sm + L.oZ[1]);
  S.V = (TS*)(sm + L.oV);
  S.t = (TS*)(sm + L.oT);
  return S;
}

template <typename TS>
struct FactorView {
  const TS *M, *MR, *ri, *P;
};
__device__ __forceinline__ FactorView<double> factor_view(const LevelDesc& d, double) {
  return FactorView<double>{d.LdM, d.LdR, d.Lri, d.Lp};
}
__device__ __forceinline__ FactorView<float> factor_view(const LevelDesc& d, float) {
  return FactorView<float>{d.LdMf, d.LdRf, d.Lrif, d.Lpf};
}

// Start the asynchronous load of the factor blocks of stage j into buffer q
// (D-hat with its columns (forward) or rows (backward) divided by the
// diagonal, 1/diag, panel rows [r0, r1)).
template <typename TS>
__device__ void prefetch_stage_factor(const SolveSmem<TS>& S, int q, const LevelDesc& d, int j, int r0,
                                      int r1, bool backward, Grp G) {
  const int n = d.n, R = 2 * n + d.m;
  const FactorView<TS> F = factor_view(d, TS(0));
  // (the forward multipliers are stored transposed: element e is (e % n, e / n))
  const TS* Lg = (backward ? F.MR : F.M) + (size_t)j * n * n;
  for (int e = G.tid; e < n * n; e += G.nt) {
    const int a = e / n, c = e - a * n;
    cp_async_elem(S.L(q) + (backward ? a * S.ldL + c : c * S.ldL + a), Lg + e);
  }
  for (int e = G.tid; e < n; e += G.nt) cp_async_elem(S.rinv(q) + e, F.ri + (size_t)j * n + e);
  const TS* P = F.P + (size_t)j * R * n;
  for (int e = G.tid + r0 * n; e < r1 * n; e += G.nt) {
    const int r = e / n, c = e - r * n;
    cp_async_elem(S.Z(q) + r * S.ldZ + c, P + e);
  }
  cp_async_commit();
}

__device__ __forceinline__ void stage_rows(const SegGeom& g, int i, int n, int m, int& r0, int& r1) {
  const bool eRows = (i < g.len - 1) || g.hasF;
  r0 = eRows ? 0 : n;
  r1 = n + m + (g.hasW ? n : 0);
}

// Backward substitution over the stages of one segment (Algorithm 3,
// parallel phase; for the top level the whole sequential sweep). On entry
// S.V holds [x_next (E rows); x_g (G rows); x_sep (W rows)]. The factor
// blocks of the next stage stream in while the current one is solved.
// (prefetched: the last stage's factor blocks were already requested into
// buffer 0, see backward_prefetch)
template <typename TS>
__device__ void backward_segment(const SolveSmem<TS>& S, const LevelDesc& d, const SegGeom& g,
                                 double* b, int ldb, int nr, int c0, Grp G, bool prefetched = false) {
  const int n = d.n, m = d.m;
  int r0, r1;
  stage_rows(g, g.len - 1, n, m, r0, r1);
  if (!prefetched) prefetch_stage_factor(S, 0, d, g.f + g.len - 1, r0, r1, true, G);
  for (int i = g.len - 1; i >= 0; --i) {
    const int j = g.f + i, q = (g.len - 1 - i) & 1;
    stage_rows(g, i, n, m, r0, r1);
    const VecView y = level_vec(d, b, ldb, j, c0);
    cp_async_wait_all();
    gsync(G);
    if (i > 0) {
      int p0, p1;
      stage_rows(g, i - 1, n, m, p0, p1);
      prefetch_stage_factor(S, q ^ 1, d, j - 1, p0, p1, true, G);
    }
    const TS* Z = S.Z(q);
    // t = y_j - Z^T v over the active panel rows: four lanes per output (each
    // a quarter of the rows, two partial sums), shuffle-reduced
    {
      const int outs = n * nr, span = (outs * 4 + 31) & ~31, rows = r1 - r0;
      for (int e = G.tid; e < span; e += G.nt) {
        const int o = e >> 2, qq = e & 3;
        const bool act = o < outs;
        const int oo = act ? o : 0;
        const int c2 = oo / nr, c = oo - c2 * nr;
        const int ra = r0 + ((qq * rows) >> 2), rb = r0 + (((qq + 1) * rows) >> 2);
        TS a0 = 0, a1 = 0;
        int r = ra;
        if (act) {
          for (; r + 1 < rb; r += 2) {
            a0 = fma(Z[r * S.ldZ + c2], S.V[r * S.ldV + c], a0);
            a1 = fma(Z[(r + 1) * S.ldZ + c2], S.V[(r + 1) * S.ldV + c], a1);
          }
          if (r < rb) a0 = fma(Z[r * S.ldZ + c2], S.V[r * S.ldV + c], a0);
        }
        TS a = a0 + a1;
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (act && qq == 0) S.t[c2 * S.ldV + c] = (TS)y.p[(size_t)c2 * y.ld + c] - a;
      }
    }
    gsync(G);
    trsv_warp(S.t, S.ldV, S.L(q), S.ldL, S.rinv(q), n, nr, true, G);
    store_vec(y.p, y.ld, S.t, S.ldV, n, nr, G);
    for (int e = G.tid; e < n * nr; e += G.nt) {
      const int r = e / nr, c = e - r * nr;
      S.V[r * S.ldV + c] = S.t[r * S.ldV + c];
    }
  }
  gsync(G);
}

// Forward substitution (Algorithm 2) for one segment; the top level (P = 1)
// also solves the corner and runs its own backward sweep (Algorithm 3,
// sequential phase). `skip`: per-system flags; a set flag returns at once.
template <typename TS>
__device__ void forward_task(const Task tk, const LevelDesc* __restrict__ descs, double* b, int ldb, int nr,
                             const int* skip, unsigned char* smraw, Grp G, int fwd_done, int c0) {
  const LevelDesc& d = descs[tk.desc];
  if (skip && skip[d.sys]) return;
  if (fwd_done && !d.is_top) return;  // the factorization carried this forward sweep
  if (!task_geometry_ok(d, tk.seg, smraw, sol_layout(d.n, d.m, (int)sizeof(TS), d.P > 1).total)) return;
  const int n = d.n, m = d.m, mg = d.m - d.mr;  // mg: rows of the real arrow
  const SolveSmem<TS> S = solve_smem<TS>(smraw, n, m, d.P > 1);
  const int oG = n, oW = n + m;
  const SegGeom g = seg_geom(d, tk.seg);
  const int k = tk.seg;
  auto rhs = [&](int j, TS* dst) {  // this level's right-hand side of stage j
    if (d.level == 1) {
      const VecView v = level_vec(d, b, ldb, j, c0);
      load_vec(dst, S.ldV, v.p, v.ld, (const double*)nullptr, n, nr, G);
    } else {
      load_vec(dst, S.ldV, d.RA + (size_t)j * n * kRhsChunk + c0, kRhsChunk,
               d.RB + (size_t)j * n * kRhsChunk + c0, n, nr, G);
    }
  };
  int r0, r1;
  stage_rows(g, 0, n, m, r0, r1);
  if (!fwd_done) prefetch_stage_factor(S, 0, d, g.f, r0, r1, false, G);
  // V_G <- 0, V_W <- rhs of the separator, t <- rhs of the first stage
  for (int e = G.tid; e < S.Rs * S.ldV; e += G.nt) S.V[e] = TS(0);
  gsync(G);
  if (g.hasW) rhs(g.f - 1, S.V + oW * S.ldV);
  rhs(g.f, S.t);
  // a bordered factorization already carried this forward sweep (fwd_done)
  for (int i = 0; i < (fwd_done ? 0 : g.len); ++i) {
    const int j = g.f + i, q = i & 1;
    stage_rows(g, i, n, m, r0, r1);
    if (i + 1 < g.len) rhs(j + 1, S.V);  // V_E <- next stage's rhs (else 0: F-hat term)
    cp_async_wait_all();
    gsync(G);
    if (i + 1 < g.len) {
      int p0, p1;
      stage_rows(g, i + 1, n, m, p0, p1);
      prefetch_stage_factor(S, q ^ 1, d, j + 1, p0, p1, false, G);
    }
    trsv_warp(S.t, S.ldV, S.L(q), S.ldL, S.rinv(q), n, nr, false, G);
    const VecView y = level_vec(d, b, ldb, j, c0);
    store_vec(y.p, y.ld, S.t, S.ldV, n, nr, G);
    // [V_E; V_G; V_W] -= Z y over the active panel rows: four lanes per output
    // (each a quarter of the dot product, two partial sums), shuffle-reduced
    const TS* Z = S.Z(q);
    {
      const int outs = (r1 - r0) * nr, span = (outs * 4 + 31) & ~31;
      for (int e = G.tid; e < span; e += G.nt) {
        const int o = e >> 2, qq = e & 3;
        const bool act = o < outs;
        const int oo = act ? o : 0;
        const int r = r0 + oo / nr, c = oo - (oo / nr) * nr;
        const int k0 = (qq * n) >> 2, k1 = ((qq + 1) * n) >> 2;
        TS a0 = 0, a1 = 0;
        int t2 = k0;
        if (act) {
          for (; t2 + 1 < k1; t2 += 2) {
            a0 = fma(Z[r * S.ldZ + t2], S.t[t2 * S.ldV + c], a0);
            a1 = fma(Z[r * S.ldZ + t2 + 1], S.t[(t2 + 1) * S.ldV + c], a1);
          }
          if (t2 < k1) a0 = fma(Z[r * S.ldZ + t2], S.t[t2 * S.ldV + c], a0);
        }
        TS a = a0 + a1;
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (act && qq == 0) S.V[r * S.ldV + c] -= a;
      }
    }
    gsync(G);
    if (i + 1 < g.len) {
      for (int e = G.tid; e < n * nr; e += G.nt) {
        const int r = e / nr, c = e - r * nr;
        S.t[r * S.ldV + c] = S.V[r * S.ldV + c];
        S.V[r * S.ldV + c] = TS(0);
      }
      gsync(G);  // V_E is reloaded at the top of the next stage
    }
  }
  gsync(G);
  if (!d.is_top) {
    if (g.hasF) store_vec(d.YB + (size_t)k * n * kRhsChunk + c0, kRhsChunk, S.V, S.ldV, n, nr, G);
    if (g.hasW)
      store_vec(d.YA + (size_t)(k - 1) * n * kRhsChunk + c0, kRhsChunk, S.V + oW * S.ldV, S.ldV, n, nr, G);
    if (m) store_vec(d.ygpart + (size_t)k * m * kRhsChunk + c0, kRhsChunk, S.V + oG * S.ldV, S.ldV, m, nr, G);
    return;
  }
  // top level: corner y_g = R-hat^{-1} (r_g + sum of every yg partial + own),
  // x_g = R-hat^{-T} y_g, written to the caller's b; then the backward sweep.
  // After a bordered factorization y_g is the bordered row of R-hat itself.
  if (mg) {
    double* bg = b + (size_t)d.rowG * ldb;
    TS* gv = S.t;
    const int ldR = odd(mg);
    if (fwd_done) {
      for (int e = G.tid; e < mg * nr; e += G.nt) {
        const int r = e / nr, c = e - r * nr;
        gv[r * S.ldV + c] = (TS)d.Rhat[(size_t)(mg + c) * m + r];
      }
    } else {
      sum_partials(
          G, mg * nr, d.nyg_all,
          [&](int p, int o) { return d.yg_all[((size_t)p * m + o / nr) * kRhsChunk + c0 + o % nr]; },
          [&](int o, double v) {
            const int r = o / nr, c = o - r * nr;
            gv[r * S.ldV + c] = (TS)((bg[(size_t)r * ldb + c] + v) + (double)S.V[(oG + r) * S.ldV + c]);
          });
    }
    for (int e = G.tid; e < mg * mg; e += G.nt) {  // R-hat: columns scaled, rows scaled
      const int r = e / mg, c = e - r * mg;
      S.L(0)[r * ldR + c] = (TS)(d.Rhat[r * m + c] * d.Rri[c]);
      S.L(1)[r * ldR + c] = (TS)(d.Rhat[r * m + c] * d.Rri[r]);
    }
    for (int e = G.tid; e < mg; e += G.nt) S.rinv(0)[e] = (TS)d.Rri[e];
    gsync(G);
    if (!fwd_done) trsv_warp(gv, S.ldV, S.L(0), ldR, S.rinv(0), mg, nr, false, G);
    trsv_warp(gv, S.ldV, S.L(1), ldR, S.rinv(0), mg, nr, true, G);
    store_vec(bg, ldb, gv, S.ldV, mg, nr, G);
  }
  // V <- [0; x_g; 0; -] for the backward sweep of the top level (bordered rows 0)
  for (int e = G.tid; e < S.Rs * S.ldV; e += G.nt) {
    const int r = e / S.ldV;
    if (r < oG || r >= oG + mg) S.V[e] = TS(0);
    else S.V[e] = S.t[(r - oG) * S.ldV + (e - r * S.ldV)];
  }
  gsync(G);
  backward_segment(S, d, g, b, ldb, nr, c0, G);
}

// Backward substitution (Algorithm 3, parallel phase) for one segment below
// the top level: needs x_g (already in b), the separator solutions of the
// next level (x at s_k and s_{k+1}), and this level's y.
template <typename TS>
__device__ void backward_task(const Task tk, const LevelDesc* __restrict__ descs, double* b, int ldb, int nr,
                              const int* skip, unsigned char* smraw, Grp G, int c0 = 0, bool prefetched = false) {
  const LevelDesc& d = descs[tk.desc];
  if (skip && skip[d.sys]) return;
  if (!task_geometry_ok(d, tk.seg, smraw, sol_layout(d.n, d.m, (int)sizeof(TS), d.P > 1).total)) return;
  const int n = d.n, m = d.m;
  const SolveSmem<TS> S = solve_smem<TS>(smraw, n, m, d.P > 1);
  const int oG = n, oW = n + m;
  const SegGeom g = seg_geom(d, tk.seg);
  const int k = tk.seg;
  const double* none = nullptr;
  for (int e = G.tid; e < S.Rs * S.ldV; e += G.nt) S.V[e] = TS(0);
  gsync(G);
  if (g.hasF) load_vec(S.V, S.ldV, d.Xnext + (size_t)k * n * kRhsChunk + c0, kRhsChunk, none, n, nr, G);
  if (d.m - d.mr) load_vec(S.V + oG * S.ldV, S.ldV, b + (size_t)d.rowG * ldb, ldb, none, d.m - d.mr, nr, G);
  if (g.hasW) {
    load_vec(S.V + oW * S.ldV, S.ldV, d.Xnext + (size_t)(k - 1) * n * kRhsChunk + c0, kRhsChunk, none, n,
             nr, G);
    gsync(G);
    const VecView xs = level_vec(d, b, ldb, g.f - 1, c0);  // this level's copy of x at s_k
    store_vec(xs.p, xs.ld, S.V + oW * S.ldV, S.ldV, n, nr, G);
  }
  gsync(G);
  backward_segment(S, d, g, b, ldb, nr, c0, G, prefetched);
}

// The factor blocks of the backward sweep's first stage (the segment's last)
// into buffer 0: they do not depend on x, so a task can request them before
// the solutions it needs exist.
template <typename TS>
__device__ void backward_prefetch(const Task tk, const LevelDesc& d, unsigned char* smraw, Grp G) {
  const SolveSmem<TS> S = solve_smem<TS>(smraw, d.n, d.m, d.P > 1);
  const SegGeom g = seg_geom(d, tk.seg);
  int r0, r1;
  stage_rows(g, g.len - 1, d.n, d.m, r0, r1);
  prefetch_stage_factor(S, 0, d, g.f + g.len - 1, r0, r1, true, G);
}


// One CTA per task (blocks above kWarpMaxN), or one warp per task with a
// shared-memory slice each (small blocks; `slice` bytes per warp).
template <typename TS>
__global__ void __launch_bounds__(kSolveThreads) k_forward(const LevelDesc* __restrict__ descs,
                                                           const Task* __restrict__ tasks, double* b,
                                                           int ldb, int nr, const int* skip, int fwd_done,
                                                           int split) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // `split` CTAs per task, each on its own group of right-hand-side columns
  const int cg = blockIdx.x % split, nc = (nr + split - 1) / split, c0 = cg * nc, cn = min(nc, nr - c0);
  if (cn <= 0) return;
  forward_task<TS>(tasks[blockIdx.x / split], descs, b + c0, ldb, cn, skip, smraw, cta_grp(), fwd_done, c0);
}
template <typename TS>
__global__ void __launch_bounds__(kSolveThreads) k_backward(const LevelDesc* __restrict__ descs,
                                                            const Task* __restrict__ tasks, double* b,
                                                            int ldb, int nr, const int* skip, int split) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int cg = blockIdx.x % split, nc = (nr + split - 1) / split, c0 = cg * nc, cn = min(nc, nr - c0);
  if (cn <= 0) return;
  backward_task<TS>(tasks[blockIdx.x / split], descs, b + c0, ldb, cn, skip, smraw, cta_grp(), c0);
}
template <typename TS>
__global__ void __launch_bounds__(256) k_forward_w(const LevelDesc* __restrict__ descs,
                                                   const Task* __restrict__ tasks, int ntasks, double* b,
                                                   int ldb, int nr, const int* skip, int slice, int fwd_done) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int wid = threadIdx.x >> 5, t = blockIdx.x * (blockDim.x >> 5) + wid;
  if (t >= ntasks) return;  // whole warp
  forward_task<TS>(tasks[t], descs, b, ldb, nr, skip, smraw + (size_t)wid * slice,
                   Grp{(int)(threadIdx.x & 31), 32, -1}, fwd_done);
}
template <typename TS>
__global__ void __launch_bounds__(256) k_backward_w(const LevelDesc* __restrict__ descs,
                                                    const Task* __restrict__ tasks, int ntasks, double* b,
                                                    int ldb, int nr, const int* skip, int slice) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int wid = threadIdx.x >> 5, t = blockIdx.x * (blockDim.x >> 5) + wid;
  if (t >= ntasks) return;  // whole warp
  backward_task<TS>(tasks[t], descs, b, ldb, nr, skip, smraw + (size_t)wid * slice,
                    Grp{(int)(threadIdx.x & 31), 32, -1});
}

// Every backward level below the top (Algorithm 3, parallel phase of each
// level, top down) in one launch. Items are (segment task, column group)
// pairs in chain order: the levels from the one below the top down to level
// 1, each level's items together. CTAs take items by ticket, so a CTA only
// ever waits for items taken before its own, which running CTAs hold. An
// item first requests its stage's factor blocks (they do not depend on x),
// then waits until every item of the level above has released its counter
// (thread 0 polls with ld.acquire.gpu, bounded by `wait` clock cycles; a
// wait that runs out records KKT_ERR_TIMEOUT and skips the item), solves,
// and releases its own level's counter. ctr[0] is the ticket, ctr[1 + li]
// the finished items of chain level li; the host zeroes them before the
// launch. unmet: every wait expects one item more than its level has (a
// test of the timeout path).
template <typename TS>
__global__ void __launch_bounds__(kSolveThreads) k_backward_chain(const LevelDesc* __restrict__ descs,
                                                                  const Task* __restrict__ tasks, ChainPlan cp,
                                                                  int* ctr, double* b, int ldb, int nr,
                                                                  const int* skip, Info* info,
                                                                  long long wait_cycles, int unmet) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int cur, ok;
  const int total = cp.nlev > 0 ? cp.end[cp.nlev - 1] : 0;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(ctr, 1);
    __syncthreads();
    const int t = cur;
    if (t >= total) break;
    int li = 0;
    while (t >= cp.end[li]) ++li;
    const int u = t - (li ? cp.end[li - 1] : 0), sp = cp.split[li];
    const Task tk = tasks[cp.off[li] + u / sp];
    const LevelDesc& d = descs[tk.desc];
    const int nc = (nr + sp - 1) / sp, c0 = (u % sp) * nc, cn = min(nc, nr - c0);
    bool work = cn > 0 && !(skip && skip[d.sys]) &&
                task_geometry_ok(d, tk.seg, smraw, sol_layout(d.n, d.m, (int)sizeof(TS), d.P > 1).total);
    if (work) backward_prefetch<TS>(tk, d, smraw, cta_grp());
    if (threadIdx.x == 0) {
      int good = 1;
      if (li > 0) {
        const int need = cp.end[li - 1] - (li >= 2 ? cp.end[li - 2] : 0) + unmet;
        const long long t0 = clock64();
        while (ld_acquire_gpu(ctr + li) < need) {
          if (clock64() - t0 > wait_cycles) {
            good = 0;
            break;
          }
        }
      }
      ok = good;
      if (!good) record_timeout(info, d.sys, d.nat[d.seg[tk.seg]], d.level);
    }
    __syncthreads();
    work = work && ok;
    if (work) backward_task<TS>(tk, descs, b + c0, ldb, cn, nullptr, smraw, cta_grp(), c0, true);
    cp_async_wait_all();  // (a skipped item's requested blocks)
    __syncthreads();
    // release: the item's writes precede the barrier, and the release
    // reduction orders them (cumulatively) before the counter's increment
    if (threadIdx.x == 0) red_release_gpu(ctr + 1 + li);
  }
}

// ---------------------------------------------------------------------------
// Whole substitution of a system whose level plan is one level with P = 1
// (the sequential method), one right-hand side, one warp per system:
// Algorithm 2 over the N stages, the corner of Eq. (7), Algorithm 3 back.
// Stage j's n x n multipliers and its panel rows (the E-hat rows when a next
// stage exists, then the arrow rows) arrive by two bulk copies into one of
// `nbuf` (2 to 4) shared-memory buffers; the 2N stage visits (forward, then
// backward) form one sequence whose next nbuf - 1 visits are in flight while
// one is solved (the backward sweep's first stages arrive during the last
// forward stages and the corner). A
// lane owns rows `lane` (and `lane + 32` when RPL = 2) of a stage, so the
// warp needs no block barrier. Every shared-memory read is free of bank
// conflicts on the unpadded blocks: the forward multipliers are stored
// transposed (column c of L contiguous), the backward ones row-major, the
// backward panel product reads columns and the forward one walks a skewed
// diagonal (lane r reads column (r + kk) mod n of row r at step kk). The
// arrow rows' sums sum_j G-hat_j y_j stay in registers over the forward
// sweep (per lane, over its own rows) and are reduced across the warp once,
// before the corner. The right-hand side (forward) and y (backward) rows of
// the stages three ahead stream into a ring of shared-memory slots by
// cp.async, so no register waits on a load in flight.
// ---------------------------------------------------------------------------

// forward chain u_r -= (L_rc / L_cc) u_c for c < r; MT holds column c of L
// (divided by its diagonal) as row c
template <typename TS, int RPL>
__device__ __forceinline__ void seq_fwd_chain(TS& u0, TS& u1, const TS* MT, int n, int lane) {
  if (RPL == 1) {
    const int r0 = lane < n ? lane : n - 1;
    int c = 0;
#pragma unroll
    for (; c + 4 < n; c += 4) {  // multipliers of four steps loaded ahead
      const TS m0 = MT[c * n + r0], m1 = MT[(c + 1) * n + r0], m2 = MT[(c + 2) * n + r0],
               m3 = MT[(c + 3) * n + r0];
      TS uc = shfl_idx(u0, c);
      if (lane > c) u0 = fma(-m0, uc, u0);
      uc = shfl_idx(u0, c + 1);
      if (lane > c + 1) u0 = fma(-m1, uc, u0);
      uc = shfl_idx(u0, c + 2);
      if (lane > c + 2) u0 = fma(-m2, uc, u0);
      uc = shfl_idx(u0, c + 3);
      if (lane > c + 3) u0 = fma(-m3, uc, u0);
    }
#pragma unroll
    for (; c < n - 1; ++c) {
      const TS uc = shfl_idx(u0, c);
      if (lane > c) u0 = fma(-MT[c * n + r0], uc, u0);
    }
  } else {
    const int r1 = lane + 32 < n ? lane + 32 : n - 1;
#pragma unroll
    for (int c = 0; c < n - 1; ++c) {
      const TS m0 = MT[c * n + lane], m1 = MT[c * n + r1];
      const TS uc = shfl_idx(c < 32 ? u0 : u1, c & 31);
      if (lane > c) u0 = fma(-m0, uc, u0);
      if (lane + 32 > c && lane + 32 < n) u1 = fma(-m1, uc, u1);
    }
  }
}

// backward chain u_r -= (L_cr / L_cc) u_c for c > r; MR holds row c of L
// (divided by its diagonal)
template <typename TS, int RPL>
__device__ __forceinline__ void seq_bwd_chain(TS& u0, TS& u1, const TS* MR, int n, int lane) {
  if (RPL == 1) {
    const int r0 = lane < n ? lane : n - 1;
    int c = n - 1;
#pragma unroll
    for (; c - 3 > 0; c -= 4) {
      const TS m0 = MR[c * n + r0], m1 = MR[(c - 1) * n + r0], m2 = MR[(c - 2) * n + r0],
               m3 = MR[(c - 3) * n + r0];
      TS uc = shfl_idx(u0, c);
      if (lane < c) u0 = fma(-m0, uc, u0);
      uc = shfl_idx(u0, c - 1);
      if (lane < c - 1) u0 = fma(-m1, uc, u0);
      uc = shfl_idx(u0, c - 2);
      if (lane < c - 2) u0 = fma(-m2, uc, u0);
      uc = shfl_idx(u0, c - 3);
      if (lane < c - 3) u0 = fma(-m3, uc, u0);
    }
#pragma unroll
    for (; c > 0; --c) {
      const TS uc = shfl_idx(u0, c);
      if (lane < c) u0 = fma(-MR[c * n + r0], uc, u0);
    }
  } else {
    const int r1 = lane + 32 < n ? lane + 32 : n - 1;
#pragma unroll
    for (int c = n - 1; c > 0; --c) {
      const TS m0 = MR[c * n + lane], m1 = MR[c * n + r1];
      const TS uc = shfl_idx(c < 32 ? u0 : u1, c & 31);
      if (lane < c) u0 = fma(-m0, uc, u0);
      if (lane + 32 < c) u1 = fma(-m1, uc, u1);
    }
  }
}

// a_r = sum_k Z[r][k] y_k for the rows r = lane (a0) and lane + 32 (a1) of
// an n x n block, y_k held by lane k (k < 32, y0) or lane k - 32 (y1);
// lane r starts its walk over k at column r, so that the warp's reads of
// one step fall in distinct banks
template <typename TS, int RPL>
__device__ __forceinline__ void seq_fwd_panel(TS& a0, TS& a1, const TS* Z, TS y0, TS y1, int n, int lane) {
  if (RPL == 1) {
    const int r0 = lane < n ? lane : n - 1;
    const TS* zr = Z + r0 * n;
    int k = r0;
    TS s0 = TS(0), s1 = TS(0);
    int kk = 0;
#pragma unroll
    for (; kk + 1 < n; kk += 2) {
      const TS ya = shfl_idx(y0, k);
      const TS za = zr[k];
      k = k + 1 == n ? 0 : k + 1;
      const TS yb = shfl_idx(y0, k);
      const TS zb = zr[k];
      k = k + 1 == n ? 0 : k + 1;
      s0 = fma(za, ya, s0);
      s1 = fma(zb, yb, s1);
    }
    if (kk < n) s0 = fma(zr[k], shfl_idx(y0, k), s0);
    a0 = s0 + s1;
    a1 = TS(0);
  } else {
    const int r1 = lane + 32 < n ? lane + 32 : n - 1, h = n - 32;
    const TS *z0 = Z + lane * n, *z1 = Z + r1 * n;
    TS s0 = TS(0), s1 = TS(0);
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {  // columns 0..31: y from y0
      const int k = (lane + kk) & 31;
      const TS yk = shfl_idx(y0, k);
      s0 = fma(z0[k], yk, s0);
      s1 = fma(z1[k], yk, s1);
    }
    int k = lane % h;
#pragma unroll
    for (int kk = 0; kk < h; ++kk) {  // columns 32..n-1: y from y1
      const TS yk = shfl_idx(y1, k);
      s0 = fma(z0[32 + k], yk, s0);
      s1 = fma(z1[32 + k], yk, s1);
      k = k + 1 == h ? 0 : k + 1;
    }
    a0 = s0;
    a1 = s1;
  }
}

// NT > 0: every system of the launch has n = NT (the loops unroll with
// constant offsets); NT = 0: n from the descriptor, RPL rows per lane
template <typename TS, int RPL, int NT>
__global__ void __launch_bounds__(32) k_seq_solve(const LevelDesc* __restrict__ descs,
                                                  const Task* __restrict__ tasks, double* b, int ldb,
                                                  const int* skip, Info* info, long long wait_cycles,
                                                  int unmet, int nbuf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int sb = (int)sizeof(TS);
  const int lane = threadIdx.x;
  const Task tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  if (skip && skip[d.sys]) return;
  const int n = NT > 0 ? NT : d.n, m = d.m, N = d.N, R = 2 * n + m, mg = m - d.mr;
#ifdef KKT_DEBUG
  {
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (!dbg_ok(d.n == n && d.is_top && d.P == 1 && d.level == 1 && tk.seg == 0 && N >= 1 && seq_shape_ok(n, m, sb) &&
                    n <= 32 * RPL && mg >= 0 && d.nyg_all >= 0 && nbuf >= 2 && nbuf <= kSeqMaxBuf &&
                    seq_slice_bytes(n, m, sb, nbuf) <= (int)dyn,
                d))
      return;
  }
#endif
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);  // one mbarrier per buffer
  const int bufB = seq_buf_bytes(n, m, sb);
  auto bufp = [&](int q) { return reinterpret_cast<TS*>(smraw + kSeqHeader + q * bufB); };
  const int zo = seq_zoff_bytes(n, sb) / sb;  // panel rows follow the multipliers
  const size_t nn = (size_t)n * n;
  const FactorView<TS> F = factor_view(d, TS(0));
  double* const bs = b + (size_t)d.offB * ldb;  // the system's stage rows
  const bool own0 = lane < n, own1 = RPL == 2 && lane + 32 < n;
  const int c0 = own0 ? lane : n - 1, c1 = own1 ? lane + 32 : n - 1;  // rows for addresses
  if (lane == 0) {
    for (int q = 0; q < nbuf; ++q) bulk::init(bar + q);
    bulk::fence_async();
  }
  __syncwarp();
  uint32_t phase = 0, pend = 0;  // bit q: parity of buffer q's next phase; buffer q's copies in flight
  // visit t of the sequence (t < N: forward stage t; else backward stage
  // 2N - 1 - t) into buffer t % nbuf: lane 0 copies the stage's multipliers
  // and panel rows; every lane notes the copies in flight
  auto issue = [&](int t) {
    const bool backward = t >= N;
    const int j = backward ? 2 * N - 1 - t : t, q = t & (nbuf - 1);
    if (lane == 0) {
      const int e0 = j < N - 1 ? 0 : n;  // E-hat rows exist above the last stage only
      const uint32_t bM = (uint32_t)(nn * sb), bZ = (uint32_t)((n + m - e0) * n * sb);
      TS* B = bufp(q);
      bulk::fence_async();
      bulk::expect_tx(bar + q, bM + bZ + (unmet ? 16u : 0u));  // unmet: a phase that never completes
      bulk::g2s(B, (backward ? F.MR : F.M) + (size_t)j * nn, bM, bar + q);
      if (bZ) bulk::g2s(B + zo, F.P + ((size_t)j * R + e0) * n, bZ, bar + q);
    }
    pend |= 1u << q;
  };
  auto wait_buf = [&](int q) -> bool {
    const bool got = __all_sync(0xffffffffu, bulk::wait(bar + q, (phase >> q) & 1u, wait_cycles));
    if (got) {
      phase ^= 1u << q;
      pend &= ~(1u << q);
    }
    return got;
  };
  // a copy that did not arrive: record it; the copies still in flight land
  // in this warp's buffers, so wait for them (bounded) before returning
  auto fail = [&](int stage) {
    if (lane == 0) record_timeout(info, d.sys, stage, 1);
    for (int q = 0; q < nbuf; ++q)
      if ((pend >> q) & 1u) (void)bulk::wait(bar + q, (phase >> q) & 1u, wait_cycles);
    cp_async_wait_all();  // the ring's copies too
  };
  // ring of kSeqRing slots (rows lane and lane + 32 of one stage each);
  // stage j's rows of bs go to slot j % kSeqRing, one commit group per stage
  double* const ring = reinterpret_cast<double*>(smraw + kSeqHeader + nbuf * bufB);
  auto ring_load = [&](int j) {
    if (j >= 0 && j < N) {
      double* sl = ring + (j & (kSeqRing - 1)) * 64;
      if (own0) cp_async_elem(sl + lane, bs + ((size_t)j * n + lane) * ldb);
      if (own1) cp_async_elem(sl + 32 + lane, bs + ((size_t)j * n + lane + 32) * ldb);
    }
    cp_async_commit();
  };
  auto ring_get = [&](int j, TS& v0, TS& v1) {  // after the wait for stage j's group
    const double* sl = ring + (j & (kSeqRing - 1)) * 64;
    v0 = own0 ? (TS)sl[lane] : TS(0);
    v1 = own1 ? (TS)sl[32 + lane] : TS(0);
  };
  constexpr int kAhead = kSeqRing - 1;  // stages in flight besides the one read

  // ---- forward sweep (Algorithm 2): L y = b
  for (int jj = 0; jj < kAhead; ++jj) ring_load(jj);
  cp_async_wait_2();
  TS t0, t1;
  ring_get(0, t0, t1);
  TS pg[kMaxM];  // this lane's terms of sum_j G-hat_j y_j, per arrow row
#pragma unroll
  for (int g = 0; g < kMaxM; ++g) pg[g] = TS(0);
  for (int t = 0; t < nbuf - 1 && t < 2 * N; ++t) issue(t);
  for (int j = 0; j < N; ++j) {
    const int q = j & (nbuf - 1);
    if (!wait_buf(q)) {
      fail(j);
      return;
    }
    __syncwarp();  // every lane is done with the buffer of the previous visit
    if (j + nbuf - 1 < 2 * N) issue(j + nbuf - 1);
    ring_load(j + kAhead);
    const TS* MT = bufp(q);
    const TS* Z = MT + zo;
    TS u0 = t0, u1 = t1;
    seq_fwd_chain<TS, RPL>(u0, u1, MT, n, lane);
    const TS y0 = own0 ? u0 * MT[c0 * n + c0] : TS(0);
    const TS y1 = own1 ? u1 * MT[c1 * n + c1] : TS(0);
    if (own0) bs[((size_t)j * n + lane) * ldb] = (double)y0;
    if (own1) bs[((size_t)j * n + lane + 32) * ldb] = (double)y1;
    const int e0 = j < N - 1 ? 0 : n;
    const TS* ZG = Z + (size_t)(n - e0) * n;  // arrow rows
#pragma unroll
    for (int g = 0; g < kMaxM; ++g) {
      if (g >= m) break;  // warp-uniform; full unrolling keeps pg in registers
      pg[g] = fma(ZG[g * n + c0], y0, pg[g]);
      if (RPL == 2) pg[g] = fma(ZG[g * n + c1], y1, pg[g]);
    }
    if (j + 1 < N) {  // t_{j+1} = b_{j+1} - E-hat_j y_j
      TS a0, a1;
      seq_fwd_panel<TS, RPL>(a0, a1, Z, y0, y1, n, lane);
      cp_async_wait_2();  // stage j + 1's group (two newer ones may be in flight)
      TS bn0, bn1;
      ring_get(j + 1, bn0, bn1);
      t0 = bn0 - a0;
      t1 = bn1 - a1;
    }
  }

  // ---- corner (Eq. (7)): R-hat R-hat^T x_g = b_g - sum_j G-hat_j y_j
  TS vg = TS(0);  // lane g: sum_j G-hat_j y_j of arrow row g
#pragma unroll
  for (int g = 0; g < kMaxM; ++g) {
    if (g >= m) break;
    TS v = pg[g];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == g) vg = v;
  }
  TS xgl = TS(0);  // lane g: x_g of arrow row g (0 for a bordered row)
  if (mg > 0) {
    const int gl = lane < mg ? lane : 0;
    double bsum = 0.0;
    if (lane < mg) {
      double v = 0.0;
      for (int p = 0; p < d.nyg_all; ++p) v += d.yg_all[((size_t)p * m + lane) * kRhsChunk];
      bsum = b[(size_t)(d.rowG + lane) * ldb] + v;
    }
    TS u = lane < mg ? (TS)(bsum + (double)(-vg)) : TS(0);
    double rrow[kMaxM], rcol[kMaxM];  // row and column gl of R-hat
#pragma unroll
    for (int p = 0; p < kMaxM; ++p) {
      rrow[p] = p < mg ? d.Rhat[gl * m + p] : 0.0;
      rcol[p] = p < mg ? d.Rhat[p * m + gl] : 0.0;
    }
    // R-hat y = u: u_g -= (R_gp / R_pp) u_p for p < g, y_g = u_g / R_gg
#pragma unroll
    for (int p = 0; p < kMaxM - 1; ++p) {
      if (p >= mg - 1) break;
      const TS up = shfl_idx(u, p);
      if (lane > p && lane < mg) u = fma(-(TS)(rrow[p] * d.Rri[p]), up, u);
    }
    u = u * (TS)d.Rri[gl];
    // R-hat^T x = y: u_g -= (R_pg / R_pp) u_p for p > g, x_g = u_g / R_gg
#pragma unroll
    for (int p = kMaxM - 1; p >= 1; --p) {
      if (p >= mg) continue;
      const TS up = shfl_idx(u, p);
      if (lane < p) u = fma(-(TS)(rcol[p] * d.Rri[p]), up, u);
    }
    const TS x = u * (TS)d.Rri[gl];
    if (lane < mg) b[(size_t)(d.rowG + lane) * ldb] = (double)x;
    xgl = lane < mg ? x : TS(0);
  }
  TS xg[kMaxM];  // x_g, every lane
#pragma unroll
  for (int g = 0; g < kMaxM; ++g) xg[g] = g < m ? shfl_idx(xgl, g) : TS(0);

  // ---- backward sweep (Algorithm 3): L^T x = y
  TS xn0 = TS(0), xn1 = TS(0);  // x of stage j + 1
  __threadfence_block();  // this lane's y stores before its asynchronous reads of them
  for (int jj = 0; jj < kAhead; ++jj) ring_load(N - 1 - jj);
  cp_async_wait_2();
  TS yc0, yc1;
  ring_get(N - 1, yc0, yc1);
  for (int s = 0; s < N; ++s) {
    const int j = N - 1 - s, t = N + s, q = t & (nbuf - 1);
    if (!wait_buf(q)) {
      fail(j);
      return;
    }
    __syncwarp();
    if (t + nbuf - 1 < 2 * N) issue(t + nbuf - 1);
    ring_load(j - kAhead);
    const TS* MR = bufp(q);
    const TS* Z = MR + zo;
    const int e0 = j < N - 1 ? 0 : n;
    const TS* ZG = Z + (size_t)(n - e0) * n;
    // t_c = y_c - sum_g G-hat_j[g][c] x_g - sum_r E-hat_j[r][c] x_{j+1, r}
    TS s0 = TS(0), s1 = TS(0), s0b = TS(0), s1b = TS(0);
#pragma unroll
    for (int g = 0; g < kMaxM; ++g) {
      if (g >= m) break;
      s0 = fma(ZG[g * n + c0], xg[g], s0);
      if (RPL == 2) s1 = fma(ZG[g * n + c1], xg[g], s1);
    }
    if (e0 == 0) {
#pragma unroll
      for (int r = 0; r < n; ++r) {
        const TS xr = shfl_idx(RPL == 2 && r >= 32 ? xn1 : xn0, r & 31);
        s0b = fma(Z[r * n + c0], xr, s0b);
        if (RPL == 2) s1b = fma(Z[r * n + c1], xr, s1b);
      }
    }
    TS u0 = yc0 - (s0 + s0b), u1 = yc1 - (s1 + s1b);
    seq_bwd_chain<TS, RPL>(u0, u1, MR, n, lane);
    xn0 = u0 * MR[c0 * n + c0];
    xn1 = u1 * MR[c1 * n + c1];
    if (own0) bs[((size_t)j * n + lane) * ldb] = (double)xn0;
    if (own1) bs[((size_t)j * n + lane + 32) * ldb] = (double)xn1;
    if (j > 0) {
      cp_async_wait_2();  // stage j - 1's group
      ring_get(j - 1, yc0, yc1);
    }
  }
  cp_async_wait_all();  // (only empty groups remain)
}

// ---------------------------------------------------------------------------
// Iterative refinement support (FP64): x += c; c = b - Psi x with the blocks
// of Eq. (3) (lower triangles of D and R read); eta = ||c||_inf /
// (||Psi||_inf ||x||_inf + ||b||_inf), maxima taken over all right-hand
// sides of the system together.
// ---------------------------------------------------------------------------

// x += c over the stage rows of one chunk; each system's first chunk also
// does the g rows. c has leading dimension kRhsChunk.
__global__ void k_axpy(const LevelDesc* __restrict__ descs, const ResTask* __restrict__ tasks,
                       double* x, int ldx, const double* c, int nr, const int* skip) {
  const ResTask tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  if (skip && skip[d.sys]) return;
  const int j1 = min(tk.j0 + kResChunk, d.N);
  const long long row0 = d.offB + (long long)tk.j0 * d.n;
  const int rows = (j1 - tk.j0) * d.n;
  for (int e = threadIdx.x; e < rows * nr; e += blockDim.x) {
    const int r = e / nr, col = e - r * nr;
    x[(size_t)(row0 + r) * ldx + col] += c[(size_t)(row0 + r) * kRhsChunk + col];
  }
  if (tk.part == 0)
    for (int e = threadIdx.x; e < d.m * nr; e += blockDim.x) {
      const int r = e / nr, col = e - r * nr;
      x[(size_t)(d.rowG + r) * ldx + col] += c[(size_t)(d.rowG + r) * kRhsChunk + col];
    }
}

// FP64 residual c = b - Psi x (blocks of Eq. (3)) over the stage rows of one
// residual task (kResChunk consecutive stages of one system) per warp. A
// pass takes res_spw(n) consecutive stages, chosen so that their rows fill
// whole warps (up to three rows per lane: row r of the pass is lane r % 32,
// slot r / 32), since an FP64 instruction costs its issue slot whether a
// lane has a row or not. Each lane forms, for each of its rows,
//   (E_{j-1} x_{j-1} + D_j x_j + E_j^T x_{j+1} + G_j^T x_g)_i
// from the blocks in global memory (lower triangle of D_j by symmetry) as
// three independent FMA chains, with the pass's x rows (and its neighbour
// stages') staged in shared memory, so Psi is read once. A matrix-vector
// product does 2 flop per 8-byte element, more than the FP64 units sustain
// at full HBM bandwidth on this part, so the kernel keeps FP64 work to the
// products themselves: the row sums of |Psi| (for eta) are only formed when
// `norms` is set (the first sweep of a refinement; they depend on the matrix
// alone). Per task it writes the g-row partials sum_j G_j x_j (m x nr),
// max|c|, max|x|, max|b| and, with `norms`, the largest stage-row sum of
// |Psi| and the |G| sums of the g rows; k_residual_final combines them per
// system. MB: registers for up to MB arrow rows.
template <int MB>
__global__ void __launch_bounds__(256, 3) k_residual(const LevelDesc* __restrict__ descs,
                                                  const ResTask* __restrict__ tasks, int ntasks,
                                                  const double* __restrict__ uD, const double* __restrict__ uE,
                                                  const double* __restrict__ uG, const double* __restrict__ b,
                                                  int ldb, const double* __restrict__ x, int ldx, double* c,
                                                  int nr, double* parts, const int* skip, int norms,
                                                  int xs_doubles) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= ntasks) return;  // whole warp
  const ResTask tk = tasks[t];
  const LevelDesc& d = descs[tk.desc];
  if (skip && skip[d.sys]) return;
  const int n = d.n, m = d.m, N = d.N;
  const int spw = res_spw(n);  // stages per pass
  if (!dbg_ok(tk.j0 >= 0 && tk.j0 < d.N && d.n <= kMaxN && d.m <= MB && tk.part < tk.nparts &&
                  (spw + 2) * n <= xs_doubles,
              d))
    return;
  const int j0 = tk.j0, j1 = min(tk.j0 + kResChunk, N);
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  const double* D = uD + d.offD;
  const double* E = uE ? uE + d.offE : nullptr;
  const double* G = m ? uG + d.offG : nullptr;
  double* part = parts + (size_t)t * kResPartDoubles;
  // x rows of stages jb-1 .. jb+spw of the current pass: xs[(s + 1) n + k] is
  // row k of stage jb + s (zero outside 0..N-1)
  double* const xs = reinterpret_cast<double*>(smraw) + (size_t)(threadIdx.x >> 5) * xs_doubles;
  // this lane's rows of a pass: slot q is pass row lane + 32 q, i.e. row ri[q] of stage si[q]
  const int rows = spw * n, slots = (rows + 31) >> 5;
  int si[3], ri[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int r = lane + 32 * q;
    si[q] = r < rows ? r / n : 0;
    ri[q] = r < rows ? r - si[q] * n : 0;
  }
  double mr = 0.0, mx = 0.0, mb = 0.0;
  float mrow = 0.0f;
  for (int col = 0; col < nr; ++col) {
    const double xg_l = lane < m ? x[(size_t)(d.rowG + lane) * ldx + col] : 0.0;  // x_g, lane q holds row q
    double gacc[MB];  // this lane's terms of sum_j G_j x_j per g row
#pragma unroll
    for (int q = 0; q < MB; ++q) gacc[q] = 0.0;
    for (int jb = j0; jb < j1; jb += spw) {
      const int cnt = min(spw, j1 - jb);
      __syncwarp();  // the previous pass is done with xs
      for (int e = lane; e < (cnt + 2) * n; e += 32) {
        const int s = e / n - 1, k = e - (s + 1) * n, jj = jb + s;
        xs[e] = (jj >= 0 && jj < N) ? x[(size_t)(d.offB + (long long)jj * n + k) * ldx + col] : 0.0;
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= slots) break;  // warp-uniform
        const bool ok = lane + 32 * q < cnt * n;
        const int s = ok ? si[q] : 0, i = ok ? ri[q] : 0, j = jb + s;
        const long long rb = d.offB + (long long)j * n;
        const double* Dj = D + (size_t)j * nn;
        const bool hp = E && j > 0, hn = E && j < N - 1;
        const double* Ep = hp ? E + (size_t)(j - 1) * nn : D;
        const double* En = hn ? E + (size_t)j * nn : D;
        const double* xp = xs + (size_t)s * n;  // x_{j-1}, x_j, x_{j+1} follow at n apart
        // E_{j-1} x_{j-1}, D_j x_j (lower triangle by symmetry) and E_j^T
        // x_{j+1} as three independent chains over k, then summed
        double aP = 0.0, aD = 0.0, aN = 0.0;
        float rs = 0.0f;
        for (int k = 0; k < n; ++k) {
          const double dv = k <= i ? Dj[i * n + k] : Dj[k * n + i];
          const double pv = hp ? Ep[i * n + k] : 0.0, qv = hn ? En[k * n + i] : 0.0;
          aP = fma(pv, xp[k], aP);
          aD = fma(dv, xp[n + k], aD);
          aN = fma(qv, xp[2 * n + k], aN);
          if (norms) rs += (abs_lo(dv) + abs_lo(pv)) + abs_lo(qv);
        }
        double acc = (aP + aD) + aN;
        const double xo = ok ? xp[n + i] : 0.0;  // this row's x
        if (m) {
          const double* Gj = G + (size_t)j * mn;
#pragma unroll
          for (int g = 0; g < MB; ++g) {
            if (g >= m) break;  // warp-uniform; full unrolling keeps gacc in registers
            const double xq = __shfl_sync(0xffffffffu, xg_l, g);
            const double gv = Gj[g * n + i];
            acc = fma(gv, xq, acc);
            gacc[g] = fma(gv, xo, gacc[g]);  // xo = 0 on lanes without a row
            if (norms) rs += abs_lo(gv);
          }
        }
        if (ok) {
          const double bv = b ? b[(size_t)(rb + i) * ldb + col] : 0.0, r = bv - acc;
          c[(size_t)(rb + i) * kRhsChunk + col] = r;
          mr = fmax(mr, fabs(r)); mb = fmax(mb, fabs(bv)); mx = fmax(mx, fabs(xo));
          if (norms) mrow = fmaxf(mrow, rs);
        }
      }
    }
    // g-row partials of this column: lane sums, then a shuffle tree
#pragma unroll
    for (int g = 0; g < MB; ++g) {
      if (g >= m) break;
      double v = gacc[g];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) part[g * kRhsChunk + col] = v;
    }
  }
  float gab = 0.0f;  // |G| sum of g row `lane` (lane < m) over the task's stages
  if (norms && m && lane < m)
    for (int j = j0; j < j1; ++j) {
      const double* Gj = G + (size_t)j * mn;
      for (int i = 0; i < n; ++i) gab += abs_lo(Gj[lane * n + i]);
    }
  for (int o = 16; o > 0; o >>= 1) {
    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (norms) mrow = fmaxf(mrow, __shfl_xor_sync(0xffffffffu, mrow, o));
  }
  double* pm = part + kMaxM * kRhsChunk;
  if (lane == 0) {
    pm[0] = mr; pm[1] = mx; pm[2] = mb;
    if (norms) pm[3] = (double)mrow;
  }
  if (norms && lane < m) pm[4 + lane] = (double)gab;
}

// Finish the g rows of one system from the chunk partials, then eta and the
// stop flag (`stall`: the fallback is enabled, flag 3 below): 1 when eta <= tol, 2 when eta is at the rounding level of the
// FP64 residual (kEtaFloor) and the sweep cut the previous sweep's eta by
// less than 10 % (refinement has reached its floor; above that level a slow
// sweep is not taken as the end, since the normwise eta of an
// ill-conditioned system need not fall monotonically); 3 (only with `stall`)
// when eta is above that level and the sweep did not halve it (refinement
// stalls: the system is handed to the preconditioned conjugate-gradient
// fallback); a stopped system skips the remaining sweeps.
constexpr double kEtaFloor = 4.0 * 1.1102230246251565e-16;  // 4 u
__global__ void k_residual_final(const LevelDesc* __restrict__ descs, const int* __restrict__ sys_desc,
                                 const int* __restrict__ part0, const double* __restrict__ uG,
                                 const double* __restrict__ uR, const double* __restrict__ b, int ldb,
                                 const double* __restrict__ x, int ldx, double* c, int nr,
                                 const double* __restrict__ parts, double tol, double* eta_out,
                                 const double* __restrict__ eta_prev, int* converged, int stall) {
  __shared__ double red[4][256];
  __shared__ double gsum[kMaxM];
  const int s = blockIdx.x;
  const LevelDesc& d = descs[sys_desc[s]];
  if (converged && converged[s]) {  // keeps the eta of its converging sweep
    if (threadIdx.x == 0 && eta_prev) eta_out[s] = eta_prev[s];
    return;
  }
  const int m = d.m;
  const int p0 = part0[s], np = (d.N + kResChunk - 1) / kResChunk;
  const double* R = m ? uR + d.offR : nullptr;
  double mr = 0.0, mx = 0.0, mb = 0.0, mrow = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double* pm = parts + (size_t)(p0 + p) * kResPartDoubles + kMaxM * kRhsChunk;
    mr = fmax(mr, pm[0]); mx = fmax(mx, pm[1]); mb = fmax(mb, pm[2]); mrow = fmax(mrow, pm[3]);
  }
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    double ga = 0.0;
    for (int p = 0; p < np; ++p) ga += parts[(size_t)(p0 + p) * kResPartDoubles + kMaxM * kRhsChunk + 4 + q];
    for (int k = 0; k < m; ++k) ga += fabs(k <= q ? R[q * m + k] : R[k * m + q]);
    gsum[q] = ga;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * nr; e += blockDim.x) {
    const int q = e / nr, col = e - q * nr;
    double acc = 0.0;
    for (int p = 0; p < np; ++p) acc += parts[(size_t)(p0 + p) * kResPartDoubles + q * kRhsChunk + col];
    for (int k = 0; k < m; ++k)
      acc = fma(k <= q ? R[q * m + k] : R[k * m + q], x[(size_t)(d.rowG + k) * ldx + col], acc);
    const size_t row = (size_t)(d.rowG + q);
    const double bv = b ? b[row * ldb + col] : 0.0;
    const double r = bv - acc;
    c[row * kRhsChunk + col] = r;
    mr = fmax(mr, fabs(r));
    mb = fmax(mb, fabs(bv));
    mx = fmax(mx, fabs(x[row * ldx + col]));
  }
  for (int q = threadIdx.x; q < m; q += blockDim.x) mrow = fmax(mrow, gsum[q]);
  red[0][threadIdx.x] = mr; red[1][threadIdx.x] = mx; red[2][threadIdx.x] = mb; red[3][threadIdx.x] = mrow;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = fmax(red[q][threadIdx.x], red[q][threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double eta = red[0][0] / (red[3][0] * red[1][0] + red[2][0]);
    eta_out[s] = eta;
    // stop: 1 = eta <= tol; 2 = eta is at the rounding level of the FP64
    // residual (<= 4 u) and this sweep cut it by less than 10 %
    if (converged) {
      if (eta <= tol) converged[s] = 1;
      else if (tol >= 0.0 && eta_prev && eta <= kEtaFloor && eta > 0.9 * eta_prev[s]) converged[s] = 2;
      else if (stall && eta_prev && eta > kEtaFloor && eta > 0.5 * eta_prev[s]) converged[s] = 3;
    }
  }
}

// Gradients of a loss L(x), x = Psi^{-1} b, with respect to the stored
// blocks, given x and bbar = Psi^{-1} xbar (xbar = dL/dx): dPsi = -bbar x^T
// restricted to the blocks, each symmetric pair of entries perturbed
// together, summed over the right-hand sides:
//   dD_j[r][c] = -(bbar_r x_c + bbar_c x_r) (r > c), -bbar_r x_r (r = c), 0 above
//   dE_j       = -(bbar_{j+1} x_j^T + x_{j+1} bbar_j^T)
//   dG_j       = -(bbar_g x_j^T + x_g bbar_j^T),   dR like dD on the g rows.
__global__ void k_adjoint_grad(const LevelDesc* __restrict__ descs, const ResTask* __restrict__ tasks,
                               const double* __restrict__ x, int ldx, const double* __restrict__ xb,
                               int ldxb, int nr, double* dD, double* dE, double* dG, double* dR) {
  const ResTask tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  const int n = d.n, m = d.m, N = d.N;
  const int j1 = min(tk.j0 + kResChunk, N);
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  auto xr = [&](long long row, int c) { return x[(size_t)row * ldx + c]; };
  auto br = [&](long long row, int c) { return xb[(size_t)row * ldxb + c]; };
  // Every element costs two FP64 fmas per right-hand side, issued by every
  // lane alike (a predicated-off FP64 instruction still takes its issue
  // slot): v = fma(-a_r, b_c, fma(-a'_c, b'_r, v)). On a symmetric block's
  // diagonal the second term's factor is zeroed by an integer select (the
  // entry is one parameter: -bbar_r x_r); above it the stored value is 0.
  auto sym = [&](long long r0, long long c0, int r, int c) {  // dD / dR entry (r, c)
    double v = 0.0;
    for (int q = 0; q < nr; ++q) {
      const double bc = __longlong_as_double(c == r ? 0LL : __double_as_longlong(br(c0 + c, q)));
      v = fma(-br(r0 + r, q), xr(c0 + c, q), fma(-bc, xr(r0 + r, q), v));
    }
    return c > r ? 0.0 : v;
  };
  for (int j = tk.j0; j < j1; ++j) {
    const long long rj = d.offB + (long long)j * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      dD[d.offD + (size_t)j * nn + e] = sym(rj, rj, r, c);
    }
    if (j < N - 1)
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        double v = 0.0;
        for (int q = 0; q < nr; ++q) v = fma(-br(rj + n + r, q), xr(rj + c, q), fma(-xr(rj + n + r, q), br(rj + c, q), v));
        dE[d.offE + (size_t)j * nn + e] = v;
      }
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      double v = 0.0;
      for (int q = 0; q < nr; ++q) v = fma(-br(d.rowG + r, q), xr(rj + c, q), fma(-xr(d.rowG + r, q), br(rj + c, q), v));
      dG[d.offG + (size_t)j * mn + e] = v;
    }
  }
  if (tk.part == 0)
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = e / m, c = e - r * m;
      dR[d.offR + e] = sym(d.rowG, d.rowG, r, c);
    }
}

// ---------------------------------------------------------------------------
// Fallback of iterative refinement: preconditioned conjugate gradients on
// Psi x = b (Psi is SPD), preconditioned by the mixed factor, for the systems
// whose refinement stalled (flag 3) or ran out of sweeps (flag 0), as
// proposed for GMRES/CG-based refinement with a low-precision factor
// (Carson and Higham, SIAM J. Sci. Comput. 40, 2018). Vectors are FP64 with
// leading dimension kRhsChunk; per system and right-hand side the scalars rho
// and p^T q live in small device arrays, so the iteration needs no host
// synchronization.
// ---------------------------------------------------------------------------

// out[s][q] = sum over the system's rows of u[row][q] v[row][q] (rows offB ..
// offB + N n + m, contiguous), for the systems whose mask entry is set; a
// fixed-order tree over the CTA
__global__ void k_sys_dot(const LevelDesc* __restrict__ descs, const int* __restrict__ sys_desc,
                          const int* __restrict__ conv, const double* __restrict__ u, const double* __restrict__ v,
                          int nr, double* out) {
  __shared__ double red[256];
  const int s = blockIdx.x;
  if (conv[s] == 1 || conv[s] == 2) return;  // converged: not in the fallback
  const LevelDesc& d = descs[sys_desc[s]];
  const long long r0 = d.offB, rows = (long long)d.N * d.n + d.m;
  for (int q = 0; q < nr; ++q) {
    double a = 0.0;
    for (long long r = threadIdx.x; r < rows; r += blockDim.x)
      a = fma(u[(size_t)(r0 + r) * kRhsChunk + q], v[(size_t)(r0 + r) * kRhsChunk + q], a);
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)s * kRhsChunk + q] = red[0];
    __syncthreads();
  }
}

// mode 0: alpha = rho / (p^T Psi p) with Qn = -Psi p and pq = p^T Qn:
//         x += alpha p, r += alpha Qn (i.e. r -= alpha Psi p)
// mode 1: beta = rho_new / rho_old: p = z + beta p
// over the stage rows of each residual task (the g rows with the system's
// first task); systems outside the fallback are skipped
__global__ void k_pcg_update(const LevelDesc* __restrict__ descs, const ResTask* __restrict__ tasks,
                             const int* __restrict__ conv, int mode, int nr, double* x, int ldx, double* rr,
                             const double* __restrict__ qn, double* p, const double* __restrict__ z,
                             const double* __restrict__ num, const double* __restrict__ den) {
  const ResTask tk = tasks[blockIdx.x];
  const LevelDesc& d = descs[tk.desc];
  const int cs = conv[d.sys];
  if (cs == 1 || cs == 2) return;
  const int j1 = min(tk.j0 + kResChunk, d.N);
  const long long row0 = d.offB + (long long)tk.j0 * d.n;
  const int rows = (j1 - tk.j0) * d.n + (tk.part == 0 ? 0 : 0);
  auto one = [&](long long row, int col) {
    const size_t sc = (size_t)d.sys * kRhsChunk + col, i = (size_t)row * kRhsChunk + col;
    const double dn = den[sc];
    if (mode == 0) {
      const double alpha = dn != 0.0 ? -num[sc] / dn : 0.0;
      x[(size_t)row * ldx + col] = fma(alpha, p[i], x[(size_t)row * ldx + col]);
      rr[i] = fma(alpha, qn[i], rr[i]);
    } else {
      const double beta = dn != 0.0 ? num[sc] / dn : 0.0;
      p[i] = fma(beta, p[i], z[i]);
    }
  };
  for (int e = threadIdx.x; e < rows * nr; e += blockDim.x) one(row0 + e / nr, e % nr);
  if (tk.part == 0)
    for (int e = threadIdx.x; e < d.m * nr; e += blockDim.x) one(d.rowG + e / nr, e % nr);
}

// fallback mask for the solves and the matrix products: skip[s] = 1 unless
// the system's refinement stalled or did not converge
__global__ void k_pcg_mask(const int* __restrict__ conv, int* skip, int count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < count) skip[s] = (conv[s] == 1 || conv[s] == 2) ? 1 : 0;
}

// Identity pivot blocks and corner for every system of a batch (synthetic
// inputs of the autotuner: the kernels' run time does not depend on values).
__global__ void k_fill_identity(const LevelDesc* __restrict__ descs, const int* __restrict__ sys_desc,
                                double* D, double* R) {
  const LevelDesc& d = descs[sys_desc[blockIdx.x]];
  const long long nn = (long long)d.n * d.n, tot = (long long)d.N * nn;
  for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
    const long long r = e % nn;
    D[d.offD + e] = (r % (d.n + 1) == 0) ? 1.0 : 0.0;
  }
  for (int e = threadIdx.x; e < d.m * d.m; e += blockDim.x) R[d.offR + e] = (e % (d.m + 1) == 0) ? 1.0 : 0.0;
}

// Bordered inputs for a fused factor-and-solve pass: Gb_j = [G_j; b_j^T],
// Rb = [[R, b_g], [b_g^T, 0]]; db holds the bordered level-1 descriptors (m + 1
// arrow rows, offG and offR into Gb and Rb). Grid: x strides over a system's
// elements (one stage's row per 32-lane chunk), y = system.
__global__ void k_border(const LevelDesc* __restrict__ descs, const int* __restrict__ sys_desc,
                         const double* __restrict__ G, const double* __restrict__ R, const double* __restrict__ b,
                         int ldb, double* Gb, double* Rb, int j0, int j1, int corner) {
  const LevelDesc& d = descs[sys_desc[blockIdx.y]];
  const int n = d.n, mb = d.m, m = mb - 1, N = d.N;
  const long long offG = d.offGu, offR = d.offRu;  // the caller's arrays
  const int je = min(j1, N);
  const long long rows = je > j0 ? (long long)(je - j0) * mb : 0;  // rows of Gb of stages [j0, je)
  const long long base = (long long)j0 * mb * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < rows * n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / n, j = j0 + row / mb;
    const int r = (int)(row - (j - j0) * mb), c = (int)(e - row * n);
    Gb[d.offG + base + e] = r < m ? G[offG + (j * m + r) * n + c] : b[(size_t)(d.offB + j * n + c) * ldb];
  }
  if (corner && blockIdx.x == 0)
    for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
      const int r = e / mb, c = e - r * mb;
      double v = 0.0;
      if (r < m && c < m) v = R[offR + r * m + c];
      else if (r == m && c < m) v = b[(size_t)(d.rowG + c) * ldb];
      else if (c == m && r < m) v = b[(size_t)(d.rowG + r) * ldb];
      Rb[d.offR + e] = v;
    }
}

// Raises a kernel's dynamic shared memory limit to `bytes` on the current
// device (never lowers it: a captured graph replays earlier launches of the
// same kernel, which may need more than the latest one). The attribute is
// per device, so the record of what was granted is keyed by (device, kernel).
int set_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> granted[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return (int)cudaErrorInvalidDevice;
  if (dev < 0 || dev >= kMaxDevices)  // not recorded: set every time
    return (int)cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[dev][fn];
  if (bytes <= g) return 0;
  const int e = (int)cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (!e) g = bytes;
  return e;
}

}  // namespace

size_t factor_smem_bytes(int n, int m, int mixed, int fill, int dbl) {
  return (size_t)fac_layout(n, m, mixed ? 4 : 8, fill != 0, dbl != 0).total;
}

int debug_info(Info* out, int clear) {
#ifdef KKT_DEBUG
  if (cudaMemcpyFromSymbol(out, g_debug_info, sizeof(Info)) != cudaSuccess) return 1;
  if (clear) {
    const Info zero{};
    if (cudaMemcpyToSymbol(g_debug_info, &zero, sizeof(Info)) != cudaSuccess) return 1;
  }
#else
  *out = Info{};
  (void)clear;
#endif
  return 0;
}

size_t factor_w_slice_bytes(int n, int m, int mixed, int fill) {
  return (size_t)fac_layout_w(n, m, mixed ? 4 : 8, fill != 0).total;
}

int persist_occupancy(int mixed, size_t smem) {
  const void* fn = mixed ? (const void*)k_factor_persist<float> : (const void*)k_factor_persist<double>;
  if (set_smem(fn, smem)) return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kFactorThreads, smem) != cudaSuccess) return 0;
  return occ;
}

int launch_factor_persist(const LevelDesc* d, const Task* t, const PItem* items, int nitems, const PCons* cons,
                          int* ready, int mixed, const double* D, const double* E, const double* G,
                          const double* R, Info* info, int grid, size_t smem, int slice, int dbl,
                          long long wait_cycles, void* stream) {
  if (nitems <= 0) return 0;
  const void* fn = mixed ? (const void*)k_factor_persist<float> : (const void*)k_factor_persist<double>;
  int e = set_smem(fn, smem);
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  if (mixed)
    k_factor_persist<float><<<grid, kFactorThreads, smem, st>>>(d, t, items, nitems, cons, ready, D, E, G, R, info,
                                                                slice, dbl, wait_cycles);
  else
    k_factor_persist<double><<<grid, kFactorThreads, smem, st>>>(d, t, items, nitems, cons, ready, D, E, G, R,
                                                                 info, slice, dbl, wait_cycles);
  return (int)cudaGetLastError();
}

size_t solve_smem_bytes(int n, int m, int single, int fill) {
  return (size_t)sol_layout(n, m, single ? 4 : 8, fill != 0).total;
}

int launch_factor_w(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int mixed,
                    const double* D, const double* E, const double* G, const double* R, Info* info,
                    void* stream, double* b, int ldb, int fill) {
  if (ntasks <= 0) return 0;
  const int slice = fac_layout_w(maxn, maxm, mixed ? 4 : 8, fill != 0).total;
  const int wpc = std::max(1, std::min(8, (200 * 1024) / slice));  // tasks (warps) per CTA
  const size_t sm = (size_t)wpc * slice;
  const void* fn = mixed ? (const void*)k_factor_w<float> : (const void*)k_factor_w<double>;
  int e = set_smem(fn, sm);
  if (e) return e;
  const int grid = (ntasks + wpc - 1) / wpc;
  if (mixed)
    k_factor_w<float><<<grid, 32 * wpc, sm, (cudaStream_t)stream>>>(d, t, ntasks, D, E, G, R, info, slice, b, ldb);
  else
    k_factor_w<double><<<grid, 32 * wpc, sm, (cudaStream_t)stream>>>(d, t, ntasks, D, E, G, R, info, slice, b, ldb);
  return (int)cudaGetLastError();
}

// Tensor-core Schur products for a mixed launch of blocks n >= 32 when the
// pivot-buffer region of the layout without the second pivot buffer can stage
// the operand (Rs rows of K) and the packed product triangle, and the
// layout spans the 128 operand rows the MMA addresses; 0 otherwise.
int tc_mode_for(int tc, int mixed, int pair, int maxn, int maxm, int fill) {
  if (!tc || !mixed || pair || maxn < 32) return 0;
  const FacLayout L = fac_layout(maxn, maxm, 4, fill != 0, false);
  const int kin = tc == 2 ? 16 : 8, eb = tc == 2 ? 2 : 4;
  const long Kp = (maxn + kin - 1) / kin * kin;
  const long cap = L.oZ - L.oDfac;
  const bool fits = L.Rs <= 128 && (long)L.Rs * Kp * eb <= cap && (long)L.Rs * (L.Rs + 1) / 2 * 4 <= cap &&
                    128 * Kp * eb <= L.total;
  return fits ? tc : 0;
}

int launch_factor(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int mixed, int pair,
                  const double* D, const double* E, const double* G, const double* R, Info* info,
                  void* stream, double* b, int ldb, int fill, int top_solve, int tc) {
  if (ntasks <= 0) return 0;
  top_solve = top_solve && b && !mixed;
  const int tcm = tc_mode_for(tc, mixed, pair, maxn, maxm, fill);
  // Mixed launches go without the second pivot buffer: warp 4 then joins the
  // pivot sweep's workers, whose FP32 panel work keeps all four sub-partitions
  // busy, and the pivot blocks are written right after the sweep (the uneven
  // batch's mixed factorization 2-8 % faster). FP64 unpaired launches drop it
  // only when that lets more CTAs share an SM (below); CTA pairs keep it.
  int dbl = (mixed || tcm) ? 0 : 1;
  size_t sm = factor_smem_bytes(maxn, maxm, mixed, fill, dbl);
  if (top_solve) sm = std::max(sm, solve_smem_bytes(maxn, maxm, 0, fill));
  const void* fn = mixed ? (pair ? (const void*)k_factor<float, 1>
                                 : tcm ? (const void*)k_factor<float, 4, true> : (const void*)k_factor<float, 4>)
                          : (pair ? (const void*)k_factor<double, 1> : (const void*)k_factor<double, 4>);
  int e = set_smem(fn, sm);
  if (e) return e;
  if (dbl && !pair && !top_solve) {
    // the occupancy of this kernel with either request
    const size_t sm1 = factor_smem_bytes(maxn, maxm, mixed, fill, 0);
    int occ = 0, occ1 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kFactorThreads, sm) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, fn, kFactorThreads, sm1) == cudaSuccess &&
        occ1 > occ) {
      dbl = 0;
      sm = sm1;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3((unsigned)(pair ? 2 * ntasks : ntasks));
  cfg.blockDim = dim3(kFactorThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = (cudaStream_t)stream;
  if (pair) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  const int p = pair ? 1 : 0;
  if (mixed)
    return pair ? (int)cudaLaunchKernelEx(&cfg, k_factor<float, 1>, d, t, D, E, G, R, info, p, b, ldb, top_solve,
                                          dbl, 0)
                : tcm ? (int)cudaLaunchKernelEx(&cfg, k_factor<float, 4, true>, d, t, D, E, G, R, info, p, b, ldb,
                                                top_solve, dbl, tcm)
                      : (int)cudaLaunchKernelEx(&cfg, k_factor<float, 4>, d, t, D, E, G, R, info, p, b, ldb, top_solve,
                                                dbl, 0);
  return pair ? (int)cudaLaunchKernelEx(&cfg, k_factor<double, 1>, d, t, D, E, G, R, info, p, b, ldb, top_solve,
                                        dbl, 0)
              : (int)cudaLaunchKernelEx(&cfg, k_factor<double, 4>, d, t, D, E, G, R, info, p, b, ldb, top_solve,
                                        dbl, 0);
}

int factor_clus_size(int ntasks, int maxn, int maxm, int sms) {
  if (ntasks <= 0) return 0;
  const size_t sm = factor_smem_bytes(maxn, maxm, 0, 1, 0);
  if (set_smem((const void*)k_factor_clus, sm)) return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_factor_clus, kFactorThreads, sm) != cudaSuccess ||
      occ < 1)
    return 0;
  occ = std::min(occ, 2);
  for (int C = 8; C >= 2; C /= 2) {
    if ((long long)C * ntasks > (long long)occ * sms) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(C * ntasks));
    cfg.blockDim = dim3(kFactorThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_factor_clus, &cfg) == cudaSuccess && ncl >= ntasks) return C;
  }
  return 0;
}

int launch_factor_clus(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int C, const double* D,
                       const double* E, const double* G, Info* info, void* stream, double* b, int ldb) {
  if (ntasks <= 0) return 0;
  if (C < 2 || C > 8) return (int)cudaErrorInvalidValue;
  const size_t sm = factor_smem_bytes(maxn, maxm, 0, 1, 0);
  const int e = set_smem((const void*)k_factor_clus, sm);
  if (e) return e;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(C * ntasks));
  cfg.blockDim = dim3(kFactorThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = (cudaStream_t)stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, k_factor_clus, d, t, D, E, G, info, b, ldb, C);
}

int launch_forward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single,
                   double* b, int ldb, int nrhs, const int* skip, void* stream, int fwd_done, int split, int fill) {
  if (ntasks <= 0) return 0;
  const size_t sm = solve_smem_bytes(maxn, maxm, single, fill);
  const void* fn = single ? (const void*)k_forward<float> : (const void*)k_forward<double>;
  int e = set_smem(fn, sm);
  if (e) return e;
  split = std::max(1, std::min(split, nrhs));
  const unsigned grid = (unsigned)(ntasks * split);
  if (single)
    k_forward<float><<<grid, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, b, ldb, nrhs, skip, fwd_done, split);
  else
    k_forward<double><<<grid, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, b, ldb, nrhs, skip, fwd_done, split);
  return (int)cudaGetLastError();
}

int launch_backward(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single,
                    double* b, int ldb, int nrhs, const int* skip, void* stream, int split, int fill) {
  if (ntasks <= 0) return 0;
  const size_t sm = solve_smem_bytes(maxn, maxm, single, fill);
  const void* fn = single ? (const void*)k_backward<float> : (const void*)k_backward<double>;
  int e = set_smem(fn, sm);
  if (e) return e;
  split = std::max(1, std::min(split, nrhs));
  const unsigned grid = (unsigned)(ntasks * split);
  if (single)
    k_backward<float><<<grid, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, b, ldb, nrhs, skip, split);
  else
    k_backward<double><<<grid, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, b, ldb, nrhs, skip, split);
  return (int)cudaGetLastError();
}

int launch_backward_chain(const LevelDesc* d, const Task* t, const ChainPlan& cp, int* ctr, int maxn, int maxm,
                          int single, double* b, int ldb, int nrhs, const int* skip, Info* info, long long wait,
                          int unmet, int sms, void* stream) {
  if (cp.nlev <= 0) return 0;
  if (cp.nlev > kChainMax) return (int)cudaErrorInvalidValue;
  const size_t sm = solve_smem_bytes(maxn, maxm, single, 1);
  const void* fn = single ? (const void*)k_backward_chain<float> : (const void*)k_backward_chain<double>;
  int e = set_smem(fn, sm);
  if (e) return e;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSolveThreads, sm) != cudaSuccess || occ < 1)
    return (int)cudaErrorInvalidConfiguration;
  const int total = cp.end[cp.nlev - 1];
  const unsigned grid = (unsigned)std::max(1, std::min(total, occ * std::max(sms, 1)));
  const cudaError_t me = cudaMemsetAsync(ctr, 0, sizeof(int) * (cp.nlev + 1), (cudaStream_t)stream);
  if (me != cudaSuccess) return (int)me;
  if (single)
    k_backward_chain<float><<<grid, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, cp, ctr, b, ldb, nrhs, skip,
                                                                               info, wait, unmet ? 1 : 0);
  else
    k_backward_chain<double><<<grid, kSolveThreads, sm, (cudaStream_t)stream>>>(d, t, cp, ctr, b, ldb, nrhs, skip,
                                                                                info, wait, unmet ? 1 : 0);
  return (int)cudaGetLastError();
}

// warp-per-task substitutions (blocks n <= kWarpMaxN)
int launch_solve_w(bool backward, const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single,
                   double* b, int ldb, int nrhs, const int* skip, void* stream, int fwd_done, int fill) {
  if (ntasks <= 0) return 0;
  const int slice = (int)solve_smem_bytes(maxn, maxm, single, fill);
  const int wpc = std::max(1, std::min(8, (200 * 1024) / slice));
  const size_t sm = (size_t)wpc * slice;
  const void* fn = backward ? (single ? (const void*)k_backward_w<float> : (const void*)k_backward_w<double>)
                            : (single ? (const void*)k_forward_w<float> : (const void*)k_forward_w<double>);
  int e = set_smem(fn, sm);
  if (e) return e;
  const int grid = (ntasks + wpc - 1) / wpc;
  cudaStream_t st = (cudaStream_t)stream;
  if (backward) {
    if (single) k_backward_w<float><<<grid, 32 * wpc, sm, st>>>(d, t, ntasks, b, ldb, nrhs, skip, slice);
    else k_backward_w<double><<<grid, 32 * wpc, sm, st>>>(d, t, ntasks, b, ldb, nrhs, skip, slice);
  } else {
    if (single) k_forward_w<float><<<grid, 32 * wpc, sm, st>>>(d, t, ntasks, b, ldb, nrhs, skip, slice, fwd_done);
    else k_forward_w<double><<<grid, 32 * wpc, sm, st>>>(d, t, ntasks, b, ldb, nrhs, skip, slice, fwd_done);
  }
  return (int)cudaGetLastError();
}

int launch_seq_solve(const LevelDesc* d, const Task* t, int ntasks, int maxn, int maxm, int single, double* b,
                     int ldb, const int* skip, Info* info, long long wait, int unmet, int sms, int uniform,
                     void* stream) {
  if (ntasks <= 0) return 0;
  const int sb = single ? 4 : 8;
  if (maxn < 2 || maxn % 2 || maxn > kMaxN || maxm < 0 || maxm > kMaxM) return (int)cudaErrorInvalidValue;
  const int nbuf = seq_nbuf(maxn, maxm, sb, ntasks, sms);
  const size_t sm = (size_t)seq_slice_bytes(maxn, maxm, sb, nbuf);
  // block sizes with their own unrolled kernel (every system of the launch the same n)
  const int nt = uniform && (maxn == 12 || maxn == 24 || maxn == 32 || maxn == 48) ? maxn : 0;
  const bool two = maxn > 32;
  cudaStream_t st = (cudaStream_t)stream;
  auto go = [&](auto kern) -> int {
    const int e = set_smem((const void*)kern, sm);
    if (e) return e;
    kern<<<ntasks, 32, sm, st>>>(d, t, b, ldb, skip, info, wait, unmet, nbuf);
    return (int)cudaGetLastError();
  };
  if (single) {
    switch (nt) {
      case 12: return go(k_seq_solve<float, 1, 12>);
      case 24: return go(k_seq_solve<float, 1, 24>);
      case 32: return go(k_seq_solve<float, 1, 32>);
      case 48: return go(k_seq_solve<float, 2, 48>);
      default: return two ? go(k_seq_solve<float, 2, 0>) : go(k_seq_solve<float, 1, 0>);
    }
  }
  switch (nt) {
    case 12: return go(k_seq_solve<double, 1, 12>);
    case 24: return go(k_seq_solve<double, 1, 24>);
    case 32: return go(k_seq_solve<double, 1, 32>);
    case 48: return go(k_seq_solve<double, 2, 48>);
    default: return two ? go(k_seq_solve<double, 2, 0>) : go(k_seq_solve<double, 1, 0>);
  }
}

int launch_axpy(const LevelDesc* d, const ResTask* t, int ntasks, double* x, int ldx, const double* c,
                int nr, const int* skip, void* stream) {
  if (ntasks <= 0) return 0;
  k_axpy<<<ntasks, 256, 0, (cudaStream_t)stream>>>(d, t, x, ldx, c, nr, skip);
  return (int)cudaGetLastError();
}

int launch_fill_identity(const LevelDesc* d, const int* sys_desc, int count, double* D, double* R,
                         void* stream) {
  if (count <= 0) return 0;
  k_fill_identity<<<count, 256, 0, (cudaStream_t)stream>>>(d, sys_desc, D, R);
  return (int)cudaGetLastError();
}

int launch_border(const LevelDesc* db, const int* sys_desc, int count, long long max_elems, const double* G,
                  const double* R, const double* b, int ldb, double* Gb, double* Rb, void* stream, int j0, int j1,
                  int corner) {
  if (count <= 0) return 0;
  const long long bx = std::min<long long>(std::max<long long>((max_elems + 255) / 256, 1), 2048);
  k_border<<<dim3((unsigned)bx, (unsigned)count), 256, 0, (cudaStream_t)stream>>>(db, sys_desc, G, R, b, ldb, Gb,
                                                                                  Rb, j0, j1, corner);
  return (int)cudaGetLastError();
}

int launch_sys_dot(const LevelDesc* d, const int* sys_desc, const int* conv, int count, const double* u,
                   const double* v, int nr, double* out, void* stream) {
  if (count <= 0) return 0;
  k_sys_dot<<<count, 256, 0, (cudaStream_t)stream>>>(d, sys_desc, conv, u, v, nr, out);
  return (int)cudaGetLastError();
}

int launch_pcg_update(const LevelDesc* d, const ResTask* t, int ntasks, const int* conv, int mode, int nr,
                      double* x, int ldx, double* r, const double* qn, double* p, const double* z,
                      const double* num, const double* den, void* stream) {
  if (ntasks <= 0) return 0;
  k_pcg_update<<<ntasks, 256, 0, (cudaStream_t)stream>>>(d, t, conv, mode, nr, x, ldx, r, qn, p, z, num, den);
  return (int)cudaGetLastError();
}

int launch_pcg_mask(const int* conv, int* skip, int count, void* stream) {
  if (count <= 0) return 0;
  k_pcg_mask<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(conv, skip, count);
  return (int)cudaGetLastError();
}

int launch_adjoint_grad(const LevelDesc* d, const ResTask* t, int ntasks, const double* x, int ldx,
                        const double* xb, int ldxb, int nr, double* dD, double* dE, double* dG,
                        double* dR, void* stream) {
  if (ntasks <= 0) return 0;
  k_adjoint_grad<<<ntasks, 256, 0, (cudaStream_t)stream>>>(d, t, x, ldx, xb, ldxb, nr, dD, dE, dG, dR);
  return (int)cudaGetLastError();
}

int launch_residual(const LevelDesc* d, const ResTask* t, int ntasks, const double* D, const double* E,
                    const double* G, const double* b, int ldb, const double* x, int ldx, double* c, int nr,
                    double* parts, const int* skip, int norms, void* stream, int xs_doubles, int maxm) {
  if (ntasks <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((ntasks + 7) / 8);
  const size_t sm = (size_t)8 * xs_doubles * sizeof(double);
  auto go = [&](auto kern) -> int {
    const int e = set_smem((const void*)kern, sm);
    if (e) return e;
    kern<<<grid, 256, sm, st>>>(d, t, ntasks, D, E, G, b, ldb, x, ldx, c, nr, parts, skip, norms, xs_doubles);
    return (int)cudaGetLastError();
  };
  if (maxm <= 4) return go(k_residual<4>);
  if (maxm <= 8) return go(k_residual<8>);
  return go(k_residual<kMaxM>);
}

int launch_residual_final(const LevelDesc* d, const int* sys_desc, const int* part0, int count,
                          const double* G, const double* R, const double* b, int ldb, const double* x,
                          int ldx, double* c, int nr, const double* parts, double tol, double* eta_out,
                          const double* eta_prev, int* converged, void* stream, int stall) {
  if (count <= 0) return 0;
  k_residual_final<<<count, 256, 0, (cudaStream_t)stream>>>(d, sys_desc, part0, G, R, b, ldb, x, ldx, c,
                                                            nr, parts, tol, eta_out, eta_prev, converged, stall);
  return (int)cudaGetLastError();
}

}  // namespace kkt
