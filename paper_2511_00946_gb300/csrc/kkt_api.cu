// Host side of the C interface declared in include/kkt.h: the partition rule
// of Eq. (13), the level plan of every system, the device workspace (factor,
// fill-ins, reduced-system slots, solve vectors) and the kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/kkt.h"
#include "kkt_internal.h"

using kkt::LevelDesc;
using kkt::Task;

namespace {

struct LevelPlan {
  int N, P;
  int mixed = 0;           // FP32 panel arithmetic in this level's segments
  std::vector<int> start;  // segment k: stages start[k] .. start[k+1]-2; start[P] = N+1
  std::vector<int> nat;    // natural stage index of each stage
};

struct SysPlan {
  int N, n, m;
  std::vector<LevelPlan> lv;  // levels 1..L (last has P = 1)
  long long offD, offE, offG, offR, offB;
};

// Partition rule of Eq. (13): balance ratio sigma = 19/7 (first segment
// 7/3 N_1 vs the others 19/3 N_k flops per Table 1), constraint
// N_1 + (P-1) N_k + P - 1 = N, N_k the floor or ceil of
// (N - P + 1) / (P - 1 + sigma) with the smaller max(7/3 N_1, 19/3 N_k),
// the floor on a tie.
bool partition_rule(int N, int P, int* N1, int* Nk) {
  if (N < 1 || P < 1) return false;
  if (P == 1) { *N1 = N; *Nk = 0; return true; }
  if (P > (N + 1) / 2) return false;
  const double sigma = 19.0 / 7.0;
  const double ideal = double(N - P + 1) / (double(P - 1) + sigma);
  const int cand[2] = {int(std::floor(ideal)), int(std::ceil(ideal))};
  int best = -1;
  double best_cost = 0.0;
  for (int nk : cand) {
    if (nk < 1) continue;
    const int n1 = N - (P - 1) * (nk + 1);
    if (n1 < 1) continue;
    const double cost = std::max(7.0 / 3.0 * n1, 19.0 / 3.0 * nk);
    if (best < 0 || cost < best_cost) { best = nk; best_cost = cost; }
  }
  if (best < 0) return false;
  *Nk = best;
  *N1 = N - (P - 1) * (best + 1);
  return true;
}

int seg_first(const LevelPlan& L, int k) { return L.start[k]; }
int seg_len(const LevelPlan& L, int k) { return L.start[k + 1] - L.start[k] - 1; }

// FP64 flops of one stage of the segment kernel (standard convention):
// potrf of the n x n pivot, trsm and syrk of the stacked panel of R rows.
double stage_flops(int n, int R) {
  const double dn = n, dR = R;
  return dn * dn * dn / 3.0 + dn * dn / 2.0 + dn / 6.0 + dR * dn * dn + dR * (dR + 1.0) * dn;
}

// Segment lengths -> start array.
std::vector<int> starts_from(const std::vector<int>& len) {
  std::vector<int> st(len.size() + 1);
  st[0] = 0;
  for (size_t k = 0; k < len.size(); ++k) st[k + 1] = st[k] + len[k] + 1;
  return st;
}

// Balanced partition: the first segment's stages are cheaper (no fill-in
// rows), so stages go one at a time to the segment whose cost would grow the
// least (first-segment stage weight w1, others w2), lowest index on ties.
// Unlike Eq. (13) the other segments may differ in length by one stage, so
// the rounding slack of large P is spread instead of piled onto segment 1.
// Cost of a stage of a paired segment with fill-in relative to a first-
// segment stage (the producer CTA also hands its blocks to the consumer).
constexpr double kPairedStageCost = 1.05;

std::vector<int> balanced_lengths(int N, int P, double w1, double w2) {
  std::vector<int> len(P, 1);
  // bulk fill: every segment up to the common cost level, then one by one
  double lo = 0.0, hi = (double)N * std::max(w1, w2) + 1.0;
  for (int it = 0; it < 200; ++it) {  // largest cost level T with total length <= N-P+1
    const double T = 0.5 * (lo + hi);
    long long tot = std::max(1, (int)std::floor(T / w1));
    tot += (long long)(P - 1) * std::max(1, (int)std::floor(T / w2));
    if (tot <= N - P + 1) lo = T; else hi = T;
  }
  len[0] = std::max(1, (int)std::floor(lo / w1));
  for (int k = 1; k < P; ++k) len[k] = std::max(1, (int)std::floor(lo / w2));
  int rest = N - (P - 1);
  for (int k = 0; k < P; ++k) rest -= len[k];
  while (rest > 0) {
    int best = 0;
    double bc = 0.0;
    for (int k = 0; k < P; ++k) {
      const double c = (len[k] + 1) * (k == 0 ? w1 : w2);
      if (k == 0 || c < bc) { bc = c; best = k; }
    }
    ++len[best];
    --rest;
  }
  return len;
}

// `paired`: the level's factor tasks run as CTA pairs, whose fill-in rows
// are off the segment's critical path (every segment then costs about what
// the first one does per stage).
bool make_level(int N, int P, int mode, int n, int m, bool paired, LevelPlan* L) {
  L->N = N;
  L->P = P;
  if (N < 1 || P < 1) return false;
  if (P == 1) { L->start = {0, N + 1}; return true; }
  if (P > (N + 1) / 2) return false;
  std::vector<int> len(P);
  if (mode == KKT_PARTITION_BALANCED) {
    // a stage also pays a fixed latency (pivot chain, barriers) that does not
    // grow with the panel height; measured on GB300 it is about 5 n^3 flops
    const double fixed = 5.0 * double(n) * n * n;
    const double w1 = stage_flops(n, n + m) + fixed;
    len = balanced_lengths(N, P, w1, paired ? kPairedStageCost * w1 : stage_flops(n, 2 * n + m) + fixed);
  } else {
    int N1 = 0, Nk = 0;
    if (!partition_rule(N, P, &N1, &Nk)) return false;
    len[0] = N1;
    for (int k = 1; k < P; ++k) len[k] = Nk;
  }
  L->start = starts_from(len);
  return L->start[P] == N + 1;
}

}  // namespace

struct kkt_handle {
  int count = 0;
  int precision = 0;
  int tc = 0;                                // tensor-core Schur products: 1 = TF32, 2 = BF16
  int maxn = 0, maxm = 0, maxL = 0;
  std::vector<SysPlan> sys;
  std::vector<LevelDesc> hdesc;              // host copy of the descriptors
  std::vector<std::vector<int>> desc_of;     // desc_of[s][level-1]
  std::vector<int> fac_off, fac_cnt;         // task ranges per level (factor + forward)
  // launch groups of a level: tasks of one block-size class, contiguous in
  // the task array (small blocks, one warp per task, first; then one group
  // per larger block size, one CTA or CTA pair per task), each launched with
  // shared memory for its own largest n and m
  struct Group {
    int off, cnt, n, m;
    bool warp;
    bool fill;  // some task has fill-in rows (its system has P > 1 at this level)
    // every system's blocks suit the bulk copies of the one-warp substitution
    // (k_seq_solve): n even, and m n a multiple of 4 for the FP32 copies
    bool even = true, mn4 = true;
    int nmin = 1 << 30;  // smallest block size (the group's n is the largest)
    bool len1 = true;    // every task is a segment of one stage
    int clus = 0;        // cluster size of its FP64 factor launch (k_factor_clus), 0: one or two CTAs
  };
  std::vector<std::vector<Group>> fac_groups, bwd_groups;
  std::vector<int> bwd_off, bwd_cnt;         // task ranges per level (backward)
  // the backward levels in one launch (k_backward_chain): every backward
  // task has blocks n > 16 and every level below the top the same precision
  // kkt_set_code_warmup: a companion handle (one small system with the
  // same block sizes and a three-level plan) whose bordered pass runs on a
  // side stream at the start of every kkt_factor_solve, its inputs, and the
  // fork/join events
  kkt_handle* warm = nullptr;
  double* warm_mem = nullptr;
  cudaStream_t warm_stream = nullptr;
  cudaEvent_t warm_fork = nullptr, warm_join = nullptr;
  bool chain = false;
  bool chain_on = true;                      // kkt_set_backward_chain
  int* dchain = nullptr;                     // its counters (maxL ints)
  void* dmem = nullptr;                      // one allocation for everything
  size_t dbytes = 0;
  LevelDesc* ddesc = nullptr;
  Task* dtasks = nullptr;
  kkt::Info* dinfo = nullptr;
  bool factored = false;
  size_t tot_D = 0, tot_E = 0, tot_G = 0, tot_R = 0, tot_B = 0;
  std::vector<cudaEvent_t> events;           // optional per-launch events
  // iterative refinement
  std::vector<kkt::ResTask> hres;
  kkt::ResTask* dres = nullptr;
  int* dsys_desc = nullptr;                  // level-1 descriptor of each system
  int* dpart0 = nullptr;                     // first residual task of each system
  double* dcorr = nullptr;                   // correction / residual vectors [tot_B][chunk]
  double* dparts = nullptr;                  // residual partials
  int* dconv = nullptr;                      // per-system convergence flags
  double* deta = nullptr;                    // eta history [kMaxSweeps][count]
  std::vector<int> level_mixed;              // per level index (all systems alike)
  std::vector<int> level_pair;               // factor tasks of this level run as CTA pairs
  // fused factor-and-solve (kkt_factor_solve): one right-hand side bordered
  // onto the arrow; storage has room for m + border arrow rows
  int border = 0;                            // 1 when the fused pass is available
  LevelDesc* ddesc_b = nullptr;              // bordered descriptors (m + 1 arrow rows, mr = 1)
  double* Gb = nullptr;                      // bordered level-1 arrow blocks [sum N][m+1][n]
  double* Rb = nullptr;                      // bordered corners [sum (m+1)^2]
  bool cur_b = false;                        // the current factor is the bordered one
  long long max_gb = 0;                      // largest bordered arrow of one system (elements)
  std::vector<int> level_top;                // some system's top level is this level
  int pair_policy = KKT_PAIR_AUTO;
  int sms = 0;                               // SMs of the device the handle was built on
  // kkt_factor_solve_host: device copies of the inputs and the streams and
  // events of the overlapped transfer (created by the first call)
  static constexpr int kHostChunks = 8;
  void* hs_mem = nullptr;                    // device copies of D, E, G, R (only when a call copies them)
  void* hs_bmem = nullptr;                   // device copy of b
  double *hsD = nullptr, *hsE = nullptr, *hsG = nullptr, *hsR = nullptr, *hsB = nullptr;
  int hs_nrhs = 0;                           // columns the b copy has room for
  cudaStream_t hs_copy = nullptr, hs_lvl[kHostChunks] = {};
  cudaEvent_t hs_ev_start = nullptr, hs_ev_copy[kHostChunks] = {}, hs_ev_lvl[kHostChunks] = {};
  // refinement fallback (kkt_set_refine_fallback): preconditioned conjugate
  // gradients for stalled systems, its vectors and per-system scalars
  int cg_iters = 0;
  int res_xs = 1;  // x rows the residual kernel stages per warp (the largest res_xs_doubles)
  double adj_tol = 0.0;  // refinement tolerance of kkt_solve_adjoint on a mixed factor
  void* cg_mem = nullptr;
  double *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_rho0 = nullptr, *cg_rho1 = nullptr,
         *cg_pq = nullptr, *cg_eta = nullptr;
  int* cg_skip = nullptr;
  // persistent factorization (kkt_set_persistent): work items, their tasks,
  // consumer edges, ready counters + ticket, in one allocation
  int persistent = 0;
  void* pmem = nullptr;
  kkt::PItem* pitems = nullptr;
  kkt::PCons* pcons = nullptr;
  Task* ptasks = nullptr;
  int* pready = nullptr;        // [pn] counters, then the ticket
  int pn = 0, pgrid = 0, pslice = 0, pdbl = 1, pmixed = 0, punmet = 0;
  size_t psmem = 0;
  long long pwait = 1LL << 31;  // clock cycles a dependency wait may take (about a second)
  std::vector<kkt::PItem> hpitems;
};

constexpr int kMaxSweeps = 16;

namespace {
// Record the caller's event `i` (if attached) after a launch. Inside a
// stream capture the record becomes an external event-record node of the
// graph, so that every replay records the event.
inline bool mark(const kkt_handle* h, int i, void* stream) {
  if (i < (int)h->events.size() && h->events[i]) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) return false;
    const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    return cudaEventRecordWithFlags(h->events[i], (cudaStream_t)stream, flags) == cudaSuccess;
  }
  return true;
}
}  // namespace

namespace {

struct Carver {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

// Levels whose factor tasks run as CTA pairs by default: some segment has
// fill-in rows and the pairs fit on the device (two CTAs per task, at most
// one CTA per SM).
// The second CTA of a pair has work when a segment of the level has fill-in
// rows, or on a top level below which other levels left corner partials to
// sum (the sum then runs beside the top level's stages).
// Only systems with blocks above kWarpMaxN run on the CTA kernel (the others
// take one warp per task and never pair).
std::vector<int> paired_levels(const std::vector<std::vector<int>>& Plev, const int* n, int sms) {
  size_t L = 0;
  for (const auto& ps : Plev) L = std::max(L, ps.size());
  std::vector<int> pr(L, 0);
  for (size_t l = 0; l < L; ++l) {
    long long tasks = 0;
    bool work = false;
    for (size_t s = 0; s < Plev.size(); ++s) {
      const auto& ps = Plev[s];
      if (l < ps.size() && n[s] > kkt::kWarpMaxN) {
        tasks += ps[l];
        work = work || ps[l] > 1 || (l + 1 == ps.size() && l > 0);
      }
    }
    pr[l] = work && 2 * tasks <= sms;
  }
  return pr;
}

kkt_status build_handle(int count, const int* N, const int* n, const int* m,
                        const std::vector<std::vector<int>>& Plev, int mode, int precision,
                        kkt_handle** out) {
  if (!out) return KKT_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !N || !n || !m) return KKT_ERR_ARG;
  int dev = 0, optin = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return KKT_ERR_CUDA;
  const std::vector<int> pair_lv = paired_levels(Plev, n, sms);
  if (precision != KKT_FP64 && precision != KKT_MIXED_FP32 && precision != KKT_MIXED_FP32_ALL &&
      precision != KKT_MIXED_TF32 && precision != KKT_MIXED_BF16)
    return KKT_ERR_ARG;
  auto* h = new kkt_handle();
  h->count = count;
  h->precision = precision;
  h->tc = precision == KKT_MIXED_TF32 ? 1 : precision == KKT_MIXED_BF16 ? 2 : 0;
  h->sms = sms;
  h->sys.resize(count);
  for (int s = 0; s < count; ++s) {
    SysPlan& sp = h->sys[s];
    sp.N = N[s]; sp.n = n[s]; sp.m = m[s];
    if (sp.N < 1 || sp.n < 1 || sp.n > kkt::kMaxN || sp.m < 0 || sp.m > kkt::kMaxM) {
      delete h;
      return KKT_ERR_ARG;
    }
    const std::vector<int>& Ps = Plev[s];
    if (Ps.empty() || Ps.back() != 1) { delete h; return KKT_ERR_ARG; }
    int Nl = sp.N;
    std::vector<int> nat(sp.N);
    for (int j = 0; j < sp.N; ++j) nat[j] = j;
    for (size_t l = 0; l < Ps.size(); ++l) {
      LevelPlan L;
      if (!make_level(Nl, Ps[l], mode, sp.n, sp.m, pair_lv[l] != 0 && sp.n > kkt::kWarpMaxN, &L)) {
        delete h;
        return KKT_ERR_PARTITION;
      }
      L.nat = nat;
      L.mixed = (precision == KKT_MIXED_FP32_ALL) ||
                ((precision == KKT_MIXED_FP32 || precision == KKT_MIXED_TF32 || precision == KKT_MIXED_BF16) &&
                 l == 0);
      sp.lv.push_back(L);
      if (L.P == 1) {
        if (l + 1 != Ps.size()) { delete h; return KKT_ERR_ARG; }
        break;
      }
      std::vector<int> nn(L.P - 1);
      for (int k = 1; k < L.P; ++k) nn[k - 1] = nat[seg_first(L, k) - 1];
      nat = nn;
      Nl = L.P - 1;
    }
    sp.offD = h->tot_D; sp.offE = h->tot_E; sp.offG = h->tot_G; sp.offR = h->tot_R; sp.offB = h->tot_B;
    h->tot_D += size_t(sp.N) * sp.n * sp.n;
    h->tot_E += size_t(sp.N - 1) * sp.n * sp.n;
    h->tot_G += size_t(sp.N) * sp.m * sp.n;
    h->tot_R += size_t(sp.m) * sp.m;
    h->tot_B += size_t(sp.N) * sp.n + sp.m;
    h->maxn = std::max(h->maxn, sp.n);
    h->maxm = std::max(h->maxm, sp.m);
    h->maxL = std::max(h->maxL, (int)sp.lv.size());
  }
  // shared memory must fit: (n | 1)-padded blocks for the largest shapes
  h->level_pair.assign(h->maxL, 0);
  for (int l = 0; l < h->maxL && l < (int)pair_lv.size(); ++l) h->level_pair[l] = pair_lv[l];
  if (kkt::factor_smem_bytes(h->maxn, h->maxm, 0) > size_t(optin)) { delete h; return KKT_ERR_ARG; }
  // room for one bordered right-hand side (FP64 handles whose arrow has a spare row)
  h->border = (precision == KKT_FP64 && h->maxm + 1 <= kkt::kMaxM &&
               kkt::factor_smem_bytes(h->maxn, h->maxm + 1, 0) <= size_t(optin))
                  ? 1 : 0;
  const int bc = h->border;
  h->level_mixed.assign(h->maxL, 0);
  for (const SysPlan& sp : h->sys)
    for (size_t l = 0; l < sp.lv.size(); ++l) h->level_mixed[l] = sp.lv[l].mixed;

  // workspace carving (byte offsets), then one cudaMalloc
  const size_t D8 = sizeof(double), CH = kkt::kRhsChunk;
  Carver cv;
  struct Offs {
    size_t Ld, LdM, LdR, Lri, Lp, DA, DB, EN, GA, GB, X, YA, YB, nat, seg;
    size_t LdMf, LdRf, Lrif, Lpf;
  };
  std::vector<std::vector<Offs>> lo(count);
  std::vector<size_t> rhat(count), rri(count), rpart(count), ygall(count);
  std::vector<size_t> offGb(count), offRb(count);
  size_t tot_Gb = 0, tot_Rb = 0;
  for (int s = 0; s < count; ++s) {
    const SysPlan& sp = h->sys[s];
    const int ma = sp.m + bc;  // arrow rows with room for a bordered right-hand side
    const size_t nn = size_t(sp.n) * sp.n, mn = size_t(ma) * sp.n, R = 2 * sp.n + ma;
    offGb[s] = tot_Gb; offRb[s] = tot_Rb;
    tot_Gb += size_t(sp.N) * ma * sp.n;
    h->max_gb = std::max<long long>(h->max_gb, (long long)sp.N * ma * sp.n);
    tot_Rb += size_t(ma) * ma;
    size_t nparts = 0;
    for (const LevelPlan& L : sp.lv) {
      Offs o{};
      const bool top = (L.P == 1);
      o.Ld = cv.take(D8 * L.N * nn);
      o.LdM = cv.take(D8 * L.N * nn);
      o.LdR = cv.take(D8 * L.N * nn);
      o.Lri = cv.take(D8 * L.N * sp.n);
      o.Lp = cv.take(D8 * L.N * R * sp.n);
      if (L.mixed) {
        o.LdMf = cv.take(4 * L.N * nn);
        o.LdRf = cv.take(4 * L.N * nn);
        o.Lrif = cv.take(4 * L.N * sp.n);
        o.Lpf = cv.take(4 * L.N * R * sp.n);
      }
      if (!top) {
        o.DA = cv.take(D8 * (L.P - 1) * nn);
        o.DB = cv.take(D8 * (L.P - 1) * nn);
        o.EN = cv.take(D8 * std::max(L.P - 2, 1) * nn);
        o.GA = cv.take(D8 * (L.P - 1) * std::max<size_t>(mn, 1));
        o.GB = cv.take(D8 * (L.P - 1) * std::max<size_t>(mn, 1));
        o.YA = cv.take(D8 * (L.P - 1) * sp.n * CH);
        o.YB = cv.take(D8 * (L.P - 1) * sp.n * CH);
        nparts += L.P;
      }
      o.X = cv.take(D8 * L.N * sp.n * CH);
      o.nat = cv.take(sizeof(int) * L.N);
      o.seg = cv.take(sizeof(int) * (L.P + 1));
      lo[s].push_back(o);
    }
    rhat[s] = cv.take(D8 * std::max(ma * ma, 1));
    rri[s] = cv.take(D8 * std::max(ma, 1));
    rpart[s] = cv.take(D8 * std::max<size_t>(nparts * ma * ma, 1));
    ygall[s] = cv.take(D8 * std::max<size_t>(nparts * ma * CH, 1));
  }
  const size_t gb_off = bc ? cv.take(D8 * std::max<size_t>(tot_Gb, 1)) : 0;
  const size_t rb_off = bc ? cv.take(D8 * std::max<size_t>(tot_Rb, 1)) : 0;
  // descriptors and tasks
  std::vector<Task> tasks;
  h->desc_of.assign(count, {});
  for (int s = 0; s < count; ++s)
    for (size_t l = 0; l < h->sys[s].lv.size(); ++l) {
      h->desc_of[s].push_back((int)h->hdesc.size());
      h->hdesc.push_back(LevelDesc{});
    }
  const size_t desc_off = cv.take(sizeof(LevelDesc) * h->hdesc.size());
  const size_t descb_off2 = bc ? cv.take(sizeof(LevelDesc) * h->hdesc.size()) : 0;
  // task lists: factor/forward per level, then backward per level
  h->fac_off.assign(h->maxL, 0); h->fac_cnt.assign(h->maxL, 0);
  h->bwd_off.assign(h->maxL, 0); h->bwd_cnt.assign(h->maxL, 0);
  // tasks of a level ordered by block size (small blocks first), one launch group per size class
  auto build_groups = [&](int l, bool backward, std::vector<kkt_handle::Group>& groups) {
    std::vector<int> sys_at;
    for (int s = 0; s < count; ++s)
      if ((backward ? l + 1 : l) < (int)h->sys[s].lv.size()) sys_at.push_back(s);
    // one launch per block-size class and per layout: levels with P = 1 (no
    // fill-in rows) get the compact shared-memory layout and more CTAs per SM
    auto fill_of = [&](int s) { return h->sys[s].lv[l].P > 1; };
    // within a launch group the longest segments first (longest processing
    // time first: CTAs are dispatched in task order, so the long systems of an
    // uneven batch start in the first wave instead of forming the tail)
    auto seg_stages = [&](int s) { return (double)h->sys[s].lv[l].N / h->sys[s].lv[l].P; };
    std::stable_sort(sys_at.begin(), sys_at.end(), [&](int a, int b) {
      if (h->sys[a].n != h->sys[b].n) return h->sys[a].n < h->sys[b].n;
      if (fill_of(a) != fill_of(b)) return fill_of(a) < fill_of(b);
      return seg_stages(a) > seg_stages(b);
    });
    for (int s : sys_at) {
      const SysPlan& sp = h->sys[s];
      const bool warp = sp.n <= kkt::kWarpMaxN, fill = fill_of(s);
      if (groups.empty() || groups.back().warp != warp || (!warp && groups.back().n != sp.n) ||
          groups.back().fill != fill)
        groups.push_back(kkt_handle::Group{(int)tasks.size(), 0, sp.n, sp.m, warp, fill});
      kkt_handle::Group& gr = groups.back();
      for (int k = 0; k < sp.lv[l].P; ++k) {
        tasks.push_back(Task{h->desc_of[s][l], k});
        gr.len1 = gr.len1 && seg_len(sp.lv[l], k) == 1;
      }
      gr.cnt += sp.lv[l].P;
      gr.even = gr.even && sp.n % 2 == 0;
      gr.nmin = std::min(gr.nmin, sp.n);
      gr.mn4 = gr.mn4 && (sp.m * sp.n) % 4 == 0;
      gr.n = std::max(gr.n, sp.n);
      gr.m = std::max(gr.m, sp.m);
    }
  };
  h->fac_groups.assign(h->maxL, {});
  h->bwd_groups.assign(h->maxL, {});
  for (int l = 0; l < h->maxL; ++l) {
    h->fac_off[l] = (int)tasks.size();
    build_groups(l, false, h->fac_groups[l]);
    h->fac_cnt[l] = (int)tasks.size() - h->fac_off[l];
  }
  for (int l = 0; l < h->maxL; ++l) {
    h->bwd_off[l] = (int)tasks.size();
    build_groups(l, true, h->bwd_groups[l]);
    h->bwd_cnt[l] = (int)tasks.size() - h->bwd_off[l];
  }
  // FP64 levels whose segments are single stages with fill-in rows (the deep
  // levels of a recursive plan): clusters of up to eight CTAs per task where
  // they all fit at once (sized for the bordered arrow too)
  for (int l = 0; l < h->maxL; ++l)
    for (kkt_handle::Group& gr : h->fac_groups[l])
      if (!gr.warp && gr.fill && gr.len1 && !h->level_mixed[l])
        gr.clus = kkt::factor_clus_size(gr.cnt, gr.n, gr.m + bc, sms);
  const size_t task_off = cv.take(sizeof(Task) * std::max<size_t>(tasks.size(), 1));
  // the backward chain: at least two backward levels
  h->chain = h->maxL >= 3 && h->maxL - 1 <= kkt::kChainMax;
  for (int l = 0; l + 1 < h->maxL && h->chain; ++l) {
    h->chain = h->level_mixed[l] == h->level_mixed[0];
    for (const kkt_handle::Group& gr : h->bwd_groups[l]) h->chain = h->chain && !gr.warp;
  }
  const size_t chain_off = cv.take(sizeof(int) * (h->maxL + 1));
  // refinement: residual tasks (chunks of kResChunk stages per system)
  std::vector<int> sys_desc(count), part0(count);
  for (int s = 0; s < count; ++s) {
    sys_desc[s] = h->desc_of[s][0];
    part0[s] = (int)h->hres.size();
    const int np = (h->sys[s].N + kkt::kResChunk - 1) / kkt::kResChunk;
    for (int p = 0; p < np; ++p)
      h->hres.push_back(kkt::ResTask{h->desc_of[s][0], p * kkt::kResChunk, p, np});
  }
  const size_t res_off = cv.take(sizeof(kkt::ResTask) * h->hres.size());
  const size_t sysd_off = cv.take(sizeof(int) * count), part0_off = cv.take(sizeof(int) * count);
  const size_t corr_off = cv.take(sizeof(double) * h->tot_B * kkt::kRhsChunk);
  const size_t parts_off = cv.take(sizeof(double) * h->hres.size() * kkt::kResPartDoubles);
  const size_t conv_off = cv.take(sizeof(int) * count);
  const size_t eta_off = cv.take(sizeof(double) * count * kMaxSweeps);
  const size_t info_off = cv.take(sizeof(kkt::Info));
  h->dbytes = cv.off;
  if (cudaMalloc(&h->dmem, h->dbytes) != cudaSuccess) {
    h->dmem = nullptr;
    delete h;
    return KKT_ERR_CUDA;
  }
  char* base = (char*)h->dmem;
  auto dp = [&](size_t o) { return (double*)(base + o); };
  for (int s = 0; s < count; ++s) {
    const SysPlan& sp = h->sys[s];
    const int L = (int)sp.lv.size();
    size_t part_cursor = 0;
    for (int l = 0; l < L; ++l) {
      const LevelPlan& P = sp.lv[l];
      const Offs& o = lo[s][l];
      LevelDesc& d = h->hdesc[h->desc_of[s][l]];
      d.N = P.N; d.n = sp.n; d.m = sp.m; d.P = P.P;
      d.seg = (const int*)(base + o.seg);
      d.level = l + 1;
      d.is_top = (P.P == 1);
      d.sys = s;
      d.precision = precision;
      d.offD = sp.offD; d.offE = sp.offE; d.offG = sp.offG; d.offR = sp.offR; d.offB = sp.offB;
      d.rowG = sp.offB + (long long)sp.N * sp.n;
      d.Nnat = sp.N;
      d.nat = (const int*)(base + o.nat);
      d.Ld = dp(o.Ld); d.LdM = dp(o.LdM); d.LdR = dp(o.LdR);
      d.mixed = P.mixed;
      if (P.mixed) {
        d.LdMf = (float*)(base + o.LdMf); d.LdRf = (float*)(base + o.LdRf);
        d.Lrif = (float*)(base + o.Lrif); d.Lpf = (float*)(base + o.Lpf);
      } d.Lri = dp(o.Lri); d.Lp = dp(o.Lp);
      d.X = dp(o.X);
      if (!d.is_top) {
        d.DA = dp(o.DA); d.DB = dp(o.DB); d.EN = dp(o.EN); d.GA = dp(o.GA); d.GB = dp(o.GB);
        d.YA = dp(o.YA); d.YB = dp(o.YB);
        d.Rpart = dp(rpart[s]) + part_cursor * sp.m * sp.m;
        d.ygpart = dp(ygall[s]) + part_cursor * sp.m * kkt::kRhsChunk;
        d.Xnext = dp(lo[s][l + 1].X);
        part_cursor += P.P;
      }
      if (l > 0) {
        const Offs& up = lo[s][l - 1];
        d.Dw = dp(up.DA); d.D2w = dp(up.DB); d.Ew = dp(up.EN);
        d.Gw = sp.m ? dp(up.GA) : nullptr; d.G2w = sp.m ? dp(up.GB) : nullptr;
        d.RA = dp(up.YA); d.RB = dp(up.YB);
      }
      d.Rhat = dp(rhat[s]); d.Rri = dp(rri[s]);
      d.Rpart_all = dp(rpart[s]);
      d.yg_all = dp(ygall[s]);
    }
    for (int l = 0; l < L; ++l) {
      LevelDesc& d = h->hdesc[h->desc_of[s][l]];
      d.nRpart_all = (int)part_cursor;
      d.nyg_all = (int)part_cursor;
    }
  }
  // bordered descriptors: the same storage, the arrow one row longer (the
  // right-hand side), level 1 reading the bordered copies of G and R
  std::vector<LevelDesc> hdesc_b;
  if (bc) {
    hdesc_b = h->hdesc;
    for (int s = 0; s < count; ++s) {
      const SysPlan& sp = h->sys[s];
      const int ma = sp.m + 1;
      size_t cursor = 0;
      for (size_t l = 0; l < sp.lv.size(); ++l) {
        LevelDesc& d = hdesc_b[h->desc_of[s][l]];
        d.m = ma;
        d.mr = 1;
        d.offGu = sp.offG;
        d.offRu = sp.offR;
        d.offG = (long long)offGb[s];
        d.offR = (long long)offRb[s];
        if (!d.is_top) {
          d.Rpart = dp(rpart[s]) + cursor * ma * ma;
          d.ygpart = dp(ygall[s]) + cursor * ma * kkt::kRhsChunk;
          cursor += sp.lv[l].P;
        }
        if (l > 0) {
          d.Gw = dp(lo[s][l - 1].GA);
          d.G2w = dp(lo[s][l - 1].GB);
        }
      }
    }
  }
  h->dres = (kkt::ResTask*)(base + res_off);
  h->dsys_desc = (int*)(base + sysd_off);
  h->dpart0 = (int*)(base + part0_off);
  h->dcorr = (double*)(base + corr_off);
  h->dparts = (double*)(base + parts_off);
  h->dconv = (int*)(base + conv_off);
  h->deta = (double*)(base + eta_off);
  h->ddesc = (LevelDesc*)(base + desc_off);
  if (bc) {
    h->ddesc_b = (LevelDesc*)(base + descb_off2);
    h->Gb = dp(gb_off);
    h->Rb = dp(rb_off);
  }
  h->dtasks = (Task*)(base + task_off);
  h->dchain = (int*)(base + chain_off);
  h->dinfo = (kkt::Info*)(base + info_off);
  bool ok = cudaMemset(h->dmem, 0, h->dbytes) == cudaSuccess;
  ok = ok && cudaMemcpy(h->ddesc, h->hdesc.data(), sizeof(LevelDesc) * h->hdesc.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
  if (bc)
    ok = ok && cudaMemcpy(h->ddesc_b, hdesc_b.data(), sizeof(LevelDesc) * hdesc_b.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
  h->level_top.assign(h->maxL, 0);
  for (const SysPlan& sp : h->sys) {
    h->level_top[sp.lv.size() - 1] = 1;
    h->res_xs = std::max(h->res_xs, kkt::res_xs_doubles(sp.n));
  }
  if (!tasks.empty())
    ok = ok && cudaMemcpy(h->dtasks, tasks.data(), sizeof(Task) * tasks.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(h->dres, h->hres.data(), sizeof(kkt::ResTask) * h->hres.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(h->dsys_desc, sys_desc.data(), sizeof(int) * count, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  ok = ok && cudaMemcpy(h->dpart0, part0.data(), sizeof(int) * count, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  for (int s = 0; s < count && ok; ++s)
    for (size_t l = 0; l < h->sys[s].lv.size() && ok; ++l) {
      const std::vector<int>& nat = h->sys[s].lv[l].nat;
      const std::vector<int>& st = h->sys[s].lv[l].start;
      ok = cudaMemcpy(base + lo[s][l].nat, nat.data(), sizeof(int) * nat.size(),
                      cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(base + lo[s][l].seg, st.data(), sizeof(int) * st.size(),
                      cudaMemcpyHostToDevice) == cudaSuccess;
    }
  if (!ok) {
    cudaFree(h->dmem);
    delete h;
    return KKT_ERR_CUDA;
  }
  *out = h;
  return KKT_OK;
}

// FP64 flops of one segment of `len` stages (standard convention).
void seg_flops(int len, int n, int m, bool hasW, bool hasF, double* fac, double* sol) {
  const double dn = n;
  for (int i = 0; i < len; ++i) {
    const bool eRows = (i < len - 1) || hasF;
    const double rows = (eRows ? n : 0) + m + (hasW ? n : 0);
    *fac += dn * dn * dn / 3.0 + dn * dn / 2.0 + dn / 6.0;   // potrf
    *fac += rows * dn * dn;                                  // trsm
    *fac += rows * (rows + 1) * dn;                          // syrk
    *sol += 2.0 * (dn * dn + 2.0 * rows * dn);               // trsv + gemv, both sweeps
  }
}

}  // namespace

extern "C" {

kkt_status kkt_create(int N, int n, int m, int P, int precision, kkt_handle** out) {
  std::vector<int> Ps;
  if (P == 1) Ps = {1};
  else Ps = {P, 1};
  if (P < 1) return KKT_ERR_PARTITION;
  return build_handle(1, &N, &n, &m, {Ps}, KKT_PARTITION_PAPER, precision, out);
}

kkt_status kkt_create_levels(int N, int n, int m, int nlevels, const int* P_levels, int precision,
                             kkt_handle** out) {
  if (nlevels < 1 || !P_levels) return KKT_ERR_ARG;
  std::vector<int> Ps(P_levels, P_levels + nlevels);
  for (int p : Ps)
    if (p < 1) return KKT_ERR_PARTITION;
  return build_handle(1, &N, &n, &m, {Ps}, KKT_PARTITION_PAPER, precision, out);
}

kkt_status kkt_create_plan(int N, int n, int m, int nlevels, const int* P_levels, int partition,
                           int precision, kkt_handle** out) {
  if (nlevels < 1 || !P_levels) return KKT_ERR_ARG;
  if (partition != KKT_PARTITION_PAPER && partition != KKT_PARTITION_BALANCED) return KKT_ERR_ARG;
  std::vector<int> Ps(P_levels, P_levels + nlevels);
  for (int p : Ps)
    if (p < 1) return KKT_ERR_PARTITION;
  return build_handle(1, &N, &n, &m, {Ps}, partition, precision, out);
}

kkt_status kkt_batch_create(int count, const int* N, const int* n, const int* m, const int* P,
                            int precision, kkt_handle** out) {
  if (!P) return kkt_batch_create_tuned(count, N, n, m, precision, nullptr, out);
  if (count < 1 || !N || !n || !m) return KKT_ERR_ARG;
  std::vector<std::vector<int>> Ps(count);
  for (int s = 0; s < count; ++s) {
    const int p = P[s];
    if (p < 1) return KKT_ERR_PARTITION;
    Ps[s] = (p == 1) ? std::vector<int>{1} : std::vector<int>{p, 1};
  }
  return build_handle(count, N, n, m, Ps, KKT_PARTITION_PAPER, precision, out);
}

namespace {
// Segments per level for one system: P1 on level 1, then every level has
// 1/ratio as many segments as the one below, down to a sequential top level.
std::vector<int> level_plan(int N, int P1, int ratio) {
  std::vector<int> v;
  int Nl = N, P = P1;
  for (;;) {
    P = std::min(P, (Nl + 1) / 2);
    if (P <= 1) {
      v.push_back(1);
      return v;
    }
    v.push_back(P);
    Nl = P - 1;
    P /= ratio;
  }
}

// Device time (ms) of one factor + one single-RHS solve of the handle, median
// of `reps` runs on the legacy stream; < 0 on a CUDA error.
float time_handle(kkt_handle* h, const double* D, const double* E, const double* G, const double* R,
                  double* b, int reps) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1.f; }
  std::vector<float> t;
  bool ok = true;
  for (int r = 0; r <= reps && ok; ++r) {  // the first run warms up
    ok = cudaEventRecord(e0, 0) == cudaSuccess && kkt_factor(h, D, E, G, R, nullptr) == KKT_OK &&
         kkt_solve(h, b, 1, 1, nullptr) == KKT_OK && cudaEventRecord(e1, 0) == cudaSuccess &&
         cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (ok && r > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || t.empty()) return -1.f;
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}
}  // namespace

kkt_status kkt_batch_create_tuned(int count, const int* N, const int* n, const int* m, int precision,
                                  int* levels_out, kkt_handle** out) {
  if (!out) return KKT_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !N || !n || !m) return KKT_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return KKT_ERR_CUDA;
  double sumN = 0.0;
  for (int s = 0; s < count; ++s) {
    if (N[s] < 1) return KKT_ERR_ARG;
    sumN += N[s];
  }
  // candidates: every system sequential, then level-1 segment totals of
  // 1/2 .. 64 per SM (small blocks run one warp per segment, many per SM)
  // spread over the systems by stage count, with 4x or 8x fewer segments per
  // level above
  std::vector<std::vector<std::vector<int>>> cands;
  cands.push_back(std::vector<std::vector<int>>(count, std::vector<int>{1}));
  for (int T1 : {sms / 2, sms, 2 * sms, 4 * sms, 8 * sms, 16 * sms, 32 * sms, 64 * sms})
    for (int ratio : {4, 8}) {
      std::vector<std::vector<int>> pl(count);
      for (int s = 0; s < count; ++s)
        pl[s] = level_plan(N[s], std::max(1, (int)std::llround((double)T1 * N[s] / sumN)), ratio);
      bool dup = false;
      for (const auto& c : cands) dup = dup || c == pl;
      if (!dup) cands.push_back(pl);
    }
  // synthetic inputs of the batch's shapes: identity pivot blocks and corners
  kkt_handle* h = nullptr;
  kkt_status st = build_handle(count, N, n, m, cands[0], KKT_PARTITION_BALANCED, precision, &h);
  if (st != KKT_OK) return st;
  const size_t nD = h->tot_D, nE = std::max<size_t>(h->tot_E, 1), nG = std::max<size_t>(h->tot_G, 1),
               nR = std::max<size_t>(h->tot_R, 1), nB = h->tot_B;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (nD + nE + nG + nR + nB)) != cudaSuccess) {
    kkt_destroy(h);
    return KKT_ERR_CUDA;
  }
  double *D = buf, *E = D + nD, *G = E + nE, *R = G + nG, *b = R + nR;
  bool ok = cudaMemset(buf, 0, sizeof(double) * (nD + nE + nG + nR + nB)) == cudaSuccess &&
            kkt::launch_fill_identity(h->ddesc, h->dsys_desc, count, D, R, nullptr) == 0 &&
            cudaDeviceSynchronize() == cudaSuccess;
  size_t best = 0;
  float best_ms = -1.f;
  for (size_t c = 0; c < cands.size() && ok; ++c) {
    if (c > 0) {
      kkt_destroy(h);
      h = nullptr;
      st = build_handle(count, N, n, m, cands[c], KKT_PARTITION_BALANCED, precision, &h);
      if (st != KKT_OK) { h = nullptr; continue; }  // a candidate that does not fit is skipped
    }
    const float ms = time_handle(h, D, E, G, R, b, 3);
    if (ms < 0.f) { ok = false; break; }
    if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = c; }
  }
  if (h) kkt_destroy(h);
  cudaFree(buf);
  if (!ok || best_ms < 0.f) return KKT_ERR_CUDA;
  st = build_handle(count, N, n, m, cands[best], KKT_PARTITION_BALANCED, precision, out);
  if (st == KKT_OK && levels_out)
    for (int s = 0; s < count; ++s) levels_out[s] = (int)cands[best][s].size();
  return st;
}

namespace {
void warm_release(kkt_handle* h) {
  if (h->warm) kkt_destroy(h->warm);
  if (h->warm_mem) cudaFree(h->warm_mem);
  if (h->warm_stream) cudaStreamDestroy(h->warm_stream);
  if (h->warm_fork) cudaEventDestroy(h->warm_fork);
  if (h->warm_join) cudaEventDestroy(h->warm_join);
  h->warm = nullptr;
  h->warm_mem = nullptr;
  h->warm_stream = nullptr;
  h->warm_fork = h->warm_join = nullptr;
}
}  // namespace

kkt_status kkt_destroy(kkt_handle* h) {
  if (!h) return KKT_OK;
  warm_release(h);
  if (h->dmem) cudaFree(h->dmem);
  if (h->pmem) cudaFree(h->pmem);
  if (h->cg_mem) cudaFree(h->cg_mem);
  if (h->hs_mem) cudaFree(h->hs_mem);
  if (h->hs_bmem) cudaFree(h->hs_bmem);
  if (h->hs_copy) cudaStreamDestroy(h->hs_copy);
  if (h->hs_ev_start) cudaEventDestroy(h->hs_ev_start);
  for (int c = 0; c < kkt_handle::kHostChunks; ++c) {
    if (h->hs_lvl[c]) cudaStreamDestroy(h->hs_lvl[c]);
    if (h->hs_ev_copy[c]) cudaEventDestroy(h->hs_ev_copy[c]);
    if (h->hs_ev_lvl[c]) cudaEventDestroy(h->hs_ev_lvl[c]);
  }
  delete h;
  return KKT_OK;
}

kkt_status kkt_partition(const kkt_handle* h, int system, int level, int* P_out, int* seg) {
  if (!h || system < 0 || system >= h->count) return KKT_ERR_ARG;
  const SysPlan& sp = h->sys[system];
  if (level < 1 || level > (int)sp.lv.size()) return KKT_ERR_ARG;
  const LevelPlan& L = sp.lv[level - 1];
  if (P_out) *P_out = L.P;
  if (seg)
    for (int k = 0; k < L.P; ++k) seg[k] = seg_len(L, k);
  return KKT_OK;
}

kkt_status kkt_partition_rule(int N, int P, int* seg) {
  int N1 = 0, Nk = 0;
  if (!seg) return KKT_ERR_ARG;
  if (!partition_rule(N, P, &N1, &Nk)) return KKT_ERR_PARTITION;
  seg[0] = N1;
  for (int k = 1; k < P; ++k) seg[k] = Nk;
  return KKT_OK;
}

kkt_status kkt_partition_balanced(int N, int n, int m, int P, int paired, int* seg) {
  if (!seg || n < 1 || m < 0) return KKT_ERR_ARG;
  LevelPlan L;
  if (!make_level(N, P, KKT_PARTITION_BALANCED, n, m, paired != 0, &L)) return KKT_ERR_PARTITION;
  for (int k = 0; k < P; ++k) seg[k] = seg_len(L, k);
  return KKT_OK;
}

kkt_status kkt_batch_offsets(const kkt_handle* h, size_t* oD, size_t* oE, size_t* oG, size_t* oR,
                             size_t* oB) {
  if (!h) return KKT_ERR_ARG;
  for (int s = 0; s <= h->count; ++s) {
    const bool end = (s == h->count);
    if (oD) oD[s] = end ? h->tot_D : h->sys[s].offD;
    if (oE) oE[s] = end ? h->tot_E : h->sys[s].offE;
    if (oG) oG[s] = end ? h->tot_G : h->sys[s].offG;
    if (oR) oR[s] = end ? h->tot_R : h->sys[s].offR;
    if (oB) oB[s] = end ? h->tot_B : h->sys[s].offB;
  }
  return KKT_OK;
}

namespace {
// Layout of a level's factor launch: the plan's choice (paired_levels)
// unless the caller forced one.
int level_paired(const kkt_handle* h, int l) {
  if (h->pair_policy == KKT_PAIR_OFF) return 0;
  if (h->pair_policy == KKT_PAIR_ON) return 1;  // (KKT_PAIR_AUTO_PAIRS: the automatic choice)
  return h->level_pair[l];
}

// Cluster size of a group's FP64 factor launch (0: the one- and two-CTA
// layouts); the automatic policy only.
int clus_of(const kkt_handle* h, int l, const kkt_handle::Group& gr) {
  return h->pair_policy == KKT_PAIR_AUTO && !h->level_mixed[l] ? gr.clus : 0;
}

// A bordered pass runs the top level's corner solve and backward sweep at the
// end of the top level's factor kernel (CTA-size blocks, and few enough top
// tasks that the larger shared-memory request costs no occupancy); the
// separate launch of that step is then left out.
bool top_in_factor(const kkt_handle* h, int l, const kkt_handle::Group& gr) {
  return h->level_top[l] && !gr.warp && gr.cnt <= h->sms;
}
}  // namespace

kkt_status kkt_set_pairing(kkt_handle* h, int policy) {
  if (!h || policy < KKT_PAIR_AUTO || policy > KKT_PAIR_AUTO_PAIRS) return KKT_ERR_ARG;
  h->pair_policy = policy;
  return KKT_OK;
}

namespace {
// FP64 flops of one factor task (segment of `len` stages), the LPT cost
double task_cost(int len, int n, int m, bool hasW, bool hasF) {
  double f = 0.0, sv = 0.0;
  seg_flops(len, n, m, hasW, hasF, &f, &sv);
  return f;
}

// The work items of the persistent factorization: level by level; within a
// level the CTA-size tasks one item each and the small-block tasks (n <=
// kWarpMaxN) in bundles of `wpc`, each group in decreasing cost, the items
// of the level then merged in decreasing cost (longest processing time
// first). Segment k' of level l + 1 (stages f'..e', separator f' - 1 when
// k' >= 1) reads the slots of level-l segments max(f' - 1, 0) .. e' + 1
// (level-(l+1) stage t is the separator between level-l segments t and
// t + 1): those are its feeders.
kkt_status build_persistent(kkt_handle* h) {
  int mixed = -1;
  for (int v : h->level_mixed) {
    if (mixed >= 0 && v != mixed) return KKT_ERR_ARG;  // one precision for every level
    mixed = v;
  }
  mixed = mixed > 0 ? 1 : 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return KKT_ERR_CUDA;
  // shared memory: the largest CTA task layout and a bundle of warp slices
  int cn = 0, cm = 0, wn = 0, wm = 0;
  bool cfill = false, wfill = false, any_cta = false, any_w = false;
  for (const SysPlan& sp : h->sys) {
    bool fill = false;
    for (const LevelPlan& L : sp.lv) fill = fill || L.P > 1;
    if (sp.n > kkt::kWarpMaxN) {
      any_cta = true; cn = std::max(cn, sp.n); cm = std::max(cm, sp.m); cfill = cfill || fill;
    } else {
      any_w = true; wn = std::max(wn, sp.n); wm = std::max(wm, sp.m); wfill = wfill || fill;
    }
  }
  const int slice = any_w ? (int)kkt::factor_w_slice_bytes(wn, wm, mixed, wfill) : 0;
  const int wpc = any_w ? std::max(1, std::min(8, (200 * 1024) / slice)) : 8;
  int dbl = 1, best_occ = -1;
  size_t smem = 0;
  // mixed levels without the second pivot buffer (warp 4 joins the sweep's
  // workers), FP64 with it unless dropping it lets more CTAs share an SM
  for (int db = mixed ? 0 : 1; db >= 0; --db) {
    const size_t sc = any_cta ? kkt::factor_smem_bytes(cn, cm, mixed, cfill, db) : 0;
    const size_t sm = std::max(sc, (size_t)wpc * slice);
    const int occ = kkt::persist_occupancy(mixed, sm);
    if (occ > best_occ) { best_occ = occ; dbl = db; smem = sm; }
    if (!any_cta) break;
  }
  if (best_occ < 1) return KKT_ERR_ARG;
  // items
  struct Cand { double cost; std::vector<std::pair<int, int>> tasks; bool warp; };
  std::vector<kkt::PItem> items;
  std::vector<Task> ptasks;
  std::vector<std::vector<std::vector<int>>> item_of(h->count);
  for (int s = 0; s < h->count; ++s) {
    item_of[s].resize(h->sys[s].lv.size());
    for (size_t l = 0; l < h->sys[s].lv.size(); ++l) item_of[s][l].assign(h->sys[s].lv[l].P, -1);
  }
  for (int l = 0; l < h->maxL; ++l) {
    std::vector<std::pair<double, std::pair<int, int>>> ct, wt;  // (cost, (system, segment))
    for (int s = 0; s < h->count; ++s) {
      const SysPlan& sp = h->sys[s];
      if (l >= (int)sp.lv.size()) continue;
      const LevelPlan& L = sp.lv[l];
      for (int k = 0; k < L.P; ++k) {
        const double c = task_cost(seg_len(L, k), sp.n, sp.m, k >= 1, k < L.P - 1);
        (sp.n > kkt::kWarpMaxN ? ct : wt).push_back({c, {s, k}});
      }
    }
    auto desc = [](const std::pair<double, std::pair<int, int>>& a, const std::pair<double, std::pair<int, int>>& b) {
      return a.first != b.first ? a.first > b.first : a.second < b.second;
    };
    std::sort(ct.begin(), ct.end(), desc);
    std::sort(wt.begin(), wt.end(), desc);
    std::vector<Cand> cands;
    for (const auto& t : ct) cands.push_back(Cand{t.first, {t.second}, false});
    for (size_t i = 0; i < wt.size(); i += wpc) {
      Cand c{wt[i].first, {}, true};
      for (size_t j = i; j < std::min(wt.size(), i + (size_t)wpc); ++j) c.tasks.push_back(wt[j].second);
      cands.push_back(c);
    }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.cost > b.cost; });
    for (const Cand& c : cands) {
      kkt::PItem it{};
      it.first = (int)ptasks.size();
      it.cnt = (int)c.tasks.size();
      it.warp = c.warp ? 1 : 0;
      for (const auto& t : c.tasks) {
        ptasks.push_back(Task{h->desc_of[t.first][l], t.second});
        item_of[t.first][l][t.second] = (int)items.size();
      }
      items.push_back(it);
    }
  }
  // dependency edges (producer item, consumer item) -> feeder tasks
  std::map<std::pair<int, int>, int> w;
  for (int s = 0; s < h->count; ++s) {
    const SysPlan& sp = h->sys[s];
    for (size_t l = 1; l < sp.lv.size(); ++l) {
      const LevelPlan& L = sp.lv[l];
      for (int k = 0; k < L.P; ++k) {
        const int f = seg_first(L, k), e = f + seg_len(L, k) - 1;
        const int lo = k >= 1 ? f - 1 : f, hi = e + 1;
        const int ci = item_of[s][l][k];
        for (int q = lo; q <= hi; ++q) {
          ++w[{item_of[s][l - 1][q], ci}];
          ++items[ci].need;
        }
      }
    }
  }
  std::vector<kkt::PCons> cons;
  for (size_t i = 0; i < items.size(); ++i) {
    items[i].cons0 = (int)cons.size();
    auto itr = w.lower_bound({(int)i, -1});
    for (; itr != w.end() && itr->first.first == (int)i; ++itr) cons.push_back(kkt::PCons{itr->first.second, itr->second});
    items[i].ncons = (int)cons.size() - items[i].cons0;
  }
  const size_t n_it = items.size(), n_c = std::max<size_t>(cons.size(), 1), n_t = ptasks.size();
  Carver cv;
  const size_t o_it = cv.take(sizeof(kkt::PItem) * n_it), o_c = cv.take(sizeof(kkt::PCons) * n_c),
               o_t = cv.take(sizeof(Task) * n_t), o_r = cv.take(sizeof(int) * (n_it + 1));
  if (h->pmem) cudaFree(h->pmem);
  h->pmem = nullptr;
  if (cudaMalloc(&h->pmem, cv.off) != cudaSuccess) {
    h->pmem = nullptr;
    return KKT_ERR_CUDA;
  }
  char* base = (char*)h->pmem;
  h->pitems = (kkt::PItem*)(base + o_it);
  h->pcons = (kkt::PCons*)(base + o_c);
  h->ptasks = (Task*)(base + o_t);
  h->pready = (int*)(base + o_r);
  bool ok = cudaMemcpy(h->pitems, items.data(), sizeof(kkt::PItem) * n_it, cudaMemcpyHostToDevice) == cudaSuccess &&
            (cons.empty() || cudaMemcpy(h->pcons, cons.data(), sizeof(kkt::PCons) * cons.size(),
                                        cudaMemcpyHostToDevice) == cudaSuccess) &&
            cudaMemcpy(h->ptasks, ptasks.data(), sizeof(Task) * n_t, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaFree(h->pmem);
    h->pmem = nullptr;
    return KKT_ERR_CUDA;
  }
  h->hpitems = items;
  h->pn = (int)n_it;
  h->pgrid = (int)std::min<long long>((long long)n_it, (long long)best_occ * sms);
  h->psmem = smem;
  h->pslice = slice;
  h->pdbl = dbl;
  h->pmixed = mixed;
  h->punmet = 0;
  return KKT_OK;
}
}  // namespace

kkt_status kkt_set_persistent(kkt_handle* h, int on) {
  if (!h) return KKT_ERR_ARG;
  if (on && !h->pmem) {
    const kkt_status st = build_persistent(h);
    if (st != KKT_OK) return st;
  }
  h->persistent = on ? 1 : 0;
  return KKT_OK;
}

// Companion system of the code warm-up: N = 7 stages with the handle's
// largest block sizes, plan [4, 2, 1] (one-stage segments on both lower
// levels, a top level of one stage), D_j = I, E_j = 0, G_j = 0, R = I, b = 0.
kkt_status kkt_set_code_warmup(kkt_handle* h, int on) {
  if (!h) return KKT_ERR_ARG;
  if (!on) {
    warm_release(h);
    return KKT_OK;
  }
  if (h->warm) return KKT_OK;
  if (!h->border || h->precision != KKT_FP64) return KKT_OK;  // nothing of the bordered pass to warm
  const int N = 7, n = h->maxn, m = h->maxm, P[3] = {4, 2, 1};
  kkt_handle* w = nullptr;
  kkt_status st = kkt_create_plan(N, n, m, 3, P, KKT_PARTITION_BALANCED, KKT_FP64, &w);
  if (st != KKT_OK) return st;
  const size_t nD = (size_t)N * n * n, nE = (size_t)(N - 1) * n * n, nG = (size_t)N * m * n,
               nR = (size_t)m * m, nB = (size_t)N * n + m;
  std::vector<double> host(nD + nE + nG + nR + nB, 0.0);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < n; ++i) host[(size_t)j * n * n + (size_t)i * n + i] = 1.0;
  for (int i = 0; i < m; ++i) host[nD + nE + nG + (size_t)i * m + i] = 1.0;
  double* mem = nullptr;
  if (cudaMalloc(&mem, sizeof(double) * host.size()) != cudaSuccess) {
    kkt_destroy(w);
    return KKT_ERR_CUDA;
  }
  h->warm = w;
  h->warm_mem = mem;
  if (cudaMemcpy(mem, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->warm_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->warm_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->warm_join, cudaEventDisableTiming) != cudaSuccess) {
    warm_release(h);
    return KKT_ERR_CUDA;
  }
  return KKT_OK;
}

kkt_status kkt_set_backward_chain(kkt_handle* h, int on) {
  if (!h) return KKT_ERR_ARG;
  h->chain_on = on != 0;
  return KKT_OK;
}

kkt_status kkt_set_wait_limit(kkt_handle* h, long long cycles, int unmet) {
  if (!h || cycles < 1) return KKT_ERR_ARG;
  h->pwait = cycles;
  unmet = unmet ? 1 : 0;
  if (h->pmem && unmet != h->punmet) {
    std::vector<kkt::PItem> it = h->hpitems;
    if (unmet)
      for (kkt::PItem& x : it)
        if (x.need > 0) ++x.need;
    if (cudaMemcpy(h->pitems, it.data(), sizeof(kkt::PItem) * it.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return KKT_ERR_CUDA;
  }
  h->punmet = unmet;
  return KKT_OK;
}

kkt_status kkt_factor(kkt_handle* h, const double* D, const double* E, const double* G,
                      const double* R, void* stream) {
  if (!h || !D) return KKT_ERR_ARG;
  if (h->tot_E > 0 && !E) return KKT_ERR_ARG;
  if (h->maxm > 0 && (!G || !R)) return KKT_ERR_ARG;
  if (h->persistent) {
    if (cudaMemsetAsync(h->pready, 0, sizeof(int) * (h->pn + 1), (cudaStream_t)stream) != cudaSuccess ||
        kkt::launch_factor_persist(h->ddesc, h->ptasks, h->pitems, h->pn, h->pcons, h->pready, h->pmixed, D, E, G, R,
                                   h->dinfo, h->pgrid, h->psmem, h->pslice, h->pdbl, h->pwait, stream) ||
        !mark(h, 0, stream))
      return KKT_ERR_CUDA;
    h->factored = true;
    h->cur_b = false;
    return KKT_OK;
  }
  int li = 0;
  for (int l = 0; l < h->maxL; ++l)
    for (const kkt_handle::Group& gr : h->fac_groups[l]) {
      const int C = clus_of(h, l, gr);
      const int e = C ? kkt::launch_factor_clus(h->ddesc, h->dtasks + gr.off, gr.cnt, gr.n, gr.m, C, D, E, G,
                                                h->dinfo, stream)
                    : gr.warp ? kkt::launch_factor_w(h->ddesc, h->dtasks + gr.off, gr.cnt, gr.n, gr.m,
                                                   h->level_mixed[l], D, E, G, R, h->dinfo, stream, nullptr, 1,
                                                   gr.fill)
                            : kkt::launch_factor(h->ddesc, h->dtasks + gr.off, gr.cnt, gr.n, gr.m,
                                                 h->level_mixed[l], level_paired(h, l), D, E, G, R,
                                                 h->dinfo, stream, nullptr, 1, gr.fill, 0,
                                                 h->level_mixed[l] ? h->tc : 0);
      if (e || !mark(h, li++, stream)) return KKT_ERR_CUDA;
    }
  h->factored = true;
  h->cur_b = false;
  return KKT_OK;
}

namespace {
// One forward/backward sweep over every level for up to kRhsChunk columns,
// with the descriptors of the current factor. fwd_done: the factorization
// carried the forward sweep (bordered pass), so only the top levels' corner
// and backward sweep run among the forward launches.
constexpr int kSeqSmemMax = 227 * 1024;  // shared memory a CTA can opt in to
kkt_status solve_chunk(kkt_handle* h, double* b, int ldb, int nr, const int* skip, void* stream, int* li,
                       int fwd_done = 0) {
  const LevelDesc* dd = h->cur_b ? h->ddesc_b : h->ddesc;
  const int dm = h->cur_b ? 1 : 0;  // arrow rows beyond each group's m
  // one launch per group: small blocks one warp per task, the others one CTA per task
  auto run = [&](bool backward, int l, const std::vector<kkt_handle::Group>& groups) -> bool {
    for (const kkt_handle::Group& gr : groups) {
      if (fwd_done && !backward && top_in_factor(h, l, gr)) continue;  // done by the factor kernel
      const Task* t = h->dtasks + gr.off;
      const int mx = h->level_mixed[l], gm = gr.m + dm;
      // several right-hand sides on a level with few tasks: the columns are
      // split over up to four CTAs per task (at least four columns each) while
      // the CTAs fit one wave (three substitution CTAs per SM)
      const int slots = 3 * std::max(h->sms, 1);
      const int split = std::max(1, std::min(nr / 4, slots / std::max(gr.cnt, 1)));
      // whole systems (level 1 with P = 1) and one right-hand side: one warp
      // per system solves forward, corner and backward with the stage blocks
      // streamed by bulk copies
      const bool seq = l == 0 && !backward && !gr.fill && nr == 1 && !fwd_done && gr.even &&
                       (!mx || (gr.mn4 && !dm)) && gr.n <= kkt::kMaxN && gm <= kkt::kMaxM &&
                       kkt::seq_slice_bytes(gr.n, gm, mx ? 4 : 8, 2) <= kSeqSmemMax;
      const int e = seq ? kkt::launch_seq_solve(dd, t, gr.cnt, gr.n, gm, mx, b, ldb, skip, h->dinfo, h->pwait,
                                                h->punmet, h->sms, gr.nmin == gr.n, stream)
                    : gr.warp ? kkt::launch_solve_w(backward, dd, t, gr.cnt, gr.n, gm, mx, b, ldb, nr, skip,
                                                  stream, fwd_done, gr.fill)
                    : backward ? kkt::launch_backward(dd, t, gr.cnt, gr.n, gm, mx, b, ldb, nr, skip, stream, split,
                                                      gr.fill)
                               : kkt::launch_forward(dd, t, gr.cnt, gr.n, gm, mx, b, ldb, nr, skip, stream,
                                                     fwd_done, split, gr.fill);
      if (e || (li && !mark(h, (*li)++, stream))) return false;
    }
    return true;
  };
  for (int l = 0; l < h->maxL; ++l)
    if ((!fwd_done || h->level_top[l]) && !run(false, l, h->fac_groups[l])) return KKT_ERR_CUDA;
  if (h->chain && h->chain_on && nr == 1) {
    // every backward level in one launch, top down (one right-hand side: with
    // several, an item's stages take longer and the items that wait for the
    // level above hold CTAs that lower levels' items need, so the per-level
    // launches below are faster: 532 against 586 us for 16 columns)
    kkt::ChainPlan cp{};
    int acc = 0, maxn = 1, maxm = 0;
    for (int l = h->maxL - 2; l >= 0; --l) {
      const int cnt = h->bwd_cnt[l];
      const int split = 1;
      acc += cnt * split;
      cp.off[cp.nlev] = h->bwd_off[l];
      cp.end[cp.nlev] = acc;
      cp.split[cp.nlev] = split;
      ++cp.nlev;
      for (const kkt_handle::Group& gr : h->bwd_groups[l]) {
        maxn = std::max(maxn, gr.n);
        maxm = std::max(maxm, gr.m + dm);
      }
    }
    const int e = kkt::launch_backward_chain(dd, h->dtasks, cp, h->dchain, maxn, maxm, h->level_mixed[0], b, ldb, nr,
                                             skip, h->dinfo, h->pwait, h->punmet, h->sms, stream);
    if (e || (li && !mark(h, (*li)++, stream))) return KKT_ERR_CUDA;
    return KKT_OK;
  }
  for (int l = h->maxL - 2; l >= 0; --l)
    if (!run(true, l, h->bwd_groups[l])) return KKT_ERR_CUDA;
  return KKT_OK;
}
}  // namespace

kkt_status kkt_solve(kkt_handle* h, double* b, int nrhs, int ldb, void* stream) {
  if (!h || !b || nrhs < 1 || ldb < nrhs) return KKT_ERR_ARG;
  if (!h->factored) return KKT_ERR_STATE;
  // attached events: the factor's launches take the first slots, then the
  // solve's launches in order
  int li = 0;
  kkt_launch_counts(h, &li, nullptr);
  for (int c0 = 0; c0 < nrhs; c0 += kkt::kRhsChunk) {
    const int nr = std::min(kkt::kRhsChunk, nrhs - c0);
    const kkt_status st = solve_chunk(h, b + c0, ldb, nr, nullptr, stream, &li);
    if (st != KKT_OK) return st;
  }
  return KKT_OK;
}

namespace {
kkt_status factor_solve_bordered(kkt_handle* h, const double* D, const double* E, const double* G,
                                 const double* R, double* b, int ldb, void* stream);
}  // namespace

kkt_status kkt_factor_solve(kkt_handle* h, const double* D, const double* E, const double* G,
                            const double* R, double* b, int nrhs, int ldb, void* stream) {
  if (!h || !D || !b || nrhs < 1 || ldb < nrhs) return KKT_ERR_ARG;
  if (h->tot_E > 0 && !E) return KKT_ERR_ARG;
  if (h->maxm > 0 && (!G || !R)) return KKT_ERR_ARG;
  if (!h->border || nrhs != 1) {  // no room for the bordered row: the two passes
    const kkt_status st = kkt_factor(h, D, E, G, R, stream);
    return st != KKT_OK ? st : kkt_solve(h, b, nrhs, ldb, stream);
  }
  // code warm-up: the companion system's bordered pass on the side stream,
  // forked here and joined at the end of the call
  if (h->warm) {
    kkt_handle* w = h->warm;
    const size_t nD = (size_t)w->tot_D, nE = (size_t)w->tot_E, nG = (size_t)w->tot_G, nR = (size_t)w->tot_R;
    double* wm = h->warm_mem;
    if (cudaEventRecord(h->warm_fork, (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamWaitEvent(h->warm_stream, h->warm_fork, 0) != cudaSuccess)
      return KKT_ERR_CUDA;
    const kkt_status ws = kkt_factor_solve(w, wm, wm + nD, wm + nD + nE, wm + nD + nE + nG,
                                           wm + nD + nE + nG + nR, 1, 1, h->warm_stream);
    if (ws != KKT_OK || cudaEventRecord(h->warm_join, h->warm_stream) != cudaSuccess) return KKT_ERR_CUDA;
  }
  const kkt_status st = factor_solve_bordered(h, D, E, G, R, b, ldb, stream);
  if (h->warm && cudaStreamWaitEvent((cudaStream_t)stream, h->warm_join, 0) != cudaSuccess) return KKT_ERR_CUDA;
  return st;
}

namespace {
kkt_status factor_solve_bordered(kkt_handle* h, const double* D, const double* E, const double* G,
                                 const double* R, double* b, int ldb, void* stream) {
  // the right-hand side bordered onto the arrow: the factorization carries the
  // forward substitution and writes y where the backward sweep reads it
  int li = 0;
  if (kkt::launch_border(h->ddesc_b, h->dsys_desc, h->count, h->max_gb, G, R, b, ldb, h->Gb, h->Rb, stream) ||
      !mark(h, li++, stream))
    return KKT_ERR_CUDA;
  for (int l = 0; l < h->maxL; ++l)
    for (const kkt_handle::Group& gr : h->fac_groups[l]) {
      const int C = clus_of(h, l, gr);
      const int e = C ? kkt::launch_factor_clus(h->ddesc_b, h->dtasks + gr.off, gr.cnt, gr.n, gr.m + 1, C, D, E,
                                                h->Gb, h->dinfo, stream, b, ldb)
                    : gr.warp ? kkt::launch_factor_w(h->ddesc_b, h->dtasks + gr.off, gr.cnt, gr.n, gr.m + 1, 0, D, E,
                                                   h->Gb, h->Rb, h->dinfo, stream, b, ldb, gr.fill)
                            : kkt::launch_factor(h->ddesc_b, h->dtasks + gr.off, gr.cnt, gr.n, gr.m + 1, 0,
                                                 level_paired(h, l), D, E, h->Gb, h->Rb, h->dinfo, stream, b, ldb,
                                                 gr.fill, top_in_factor(h, l, gr));
      if (e || !mark(h, li++, stream)) return KKT_ERR_CUDA;
    }
  h->factored = true;
  h->cur_b = true;
  return solve_chunk(h, b, ldb, 1, nullptr, stream, &li, 1);
}
}  // namespace

namespace {
// Device buffers and the overlap streams of kkt_factor_solve_host: the copy
// of b always, copies of D, E, G, R only for inputs that are not read in
// place (`inputs`).
kkt_status host_prepare(kkt_handle* h, int nrhs, bool inputs) {
  const size_t d8 = sizeof(double);
  if (!h->hs_bmem || h->hs_nrhs < nrhs) {
    if (h->hs_bmem) cudaFree(h->hs_bmem);
    h->hs_bmem = nullptr;
    if (cudaMalloc(&h->hs_bmem, std::max<size_t>(h->tot_B * (size_t)nrhs, 1) * d8) != cudaSuccess) {
      h->hs_bmem = nullptr;
      h->hs_nrhs = 0;
      return KKT_ERR_CUDA;
    }
    h->hsB = (double*)h->hs_bmem;
    h->hs_nrhs = nrhs;
  }
  if (inputs && !h->hs_mem) {
    const size_t tot = h->tot_D + h->tot_E + h->tot_G + h->tot_R;
    if (cudaMalloc(&h->hs_mem, std::max<size_t>(tot, 1) * d8) != cudaSuccess) {
      h->hs_mem = nullptr;
      return KKT_ERR_CUDA;
    }
    double* p = (double*)h->hs_mem;
    h->hsD = p; p += h->tot_D;
    h->hsE = p; p += h->tot_E;
    h->hsG = p; p += h->tot_G;
    h->hsR = p;
  }
  if (!h->hs_copy) {
    if (cudaStreamCreateWithFlags(&h->hs_copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->hs_ev_start, cudaEventDisableTiming) != cudaSuccess)
      return KKT_ERR_CUDA;
    for (int c = 0; c < kkt_handle::kHostChunks; ++c)
      if (cudaStreamCreateWithFlags(&h->hs_lvl[c], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->hs_ev_copy[c], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->hs_ev_lvl[c], cudaEventDisableTiming) != cudaSuccess)
        return KKT_ERR_CUDA;
  }
  return KKT_OK;
}

// The device address of host array p when it is page-locked memory that the
// current device can read (cudaHostAlloc / cudaHostRegister with unified
// addressing); nullptr for pageable memory and anything else. The query
// enqueues nothing; the thread's capture mode is relaxed around it so that it
// is also allowed while the caller captures a graph.
const double* device_view(const double* p) {
  if (!p) return nullptr;
  cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  if (cudaThreadExchangeStreamCaptureMode(&mode) != cudaSuccess) return nullptr;
  cudaPointerAttributes a;
  const bool ok = cudaPointerGetAttributes(&a, p) == cudaSuccess;
  cudaThreadExchangeStreamCaptureMode(&mode);  // back to the caller's mode
  if (!ok) {
    cudaGetLastError();  // clear the error an unknown pointer may leave
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer ? (const double*)a.devicePointer : nullptr;
}
}  // namespace

kkt_status kkt_factor_solve_host(kkt_handle* h, const double* D, const double* E, const double* G,
                                 const double* R, double* b, int nrhs, int ldb, void* stream) {
  if (!h || !D || !b || nrhs < 1 || ldb < nrhs) return KKT_ERR_ARG;
  if (h->tot_E > 0 && !E) return KKT_ERR_ARG;
  if (h->maxm > 0 && (!G || !R)) return KKT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t d8 = sizeof(double);
  auto h2d = [&](double* dst, const double* src, size_t cnt, cudaStream_t st) {
    return cnt == 0 || cudaMemcpyAsync(dst, src, cnt * d8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  // b: (N n + m) rows of ldb on the host, nrhs packed columns on the device;
  // one linear copy when the host rows are packed too (a pitched copy of
  // 8-byte rows moves one row at a time)
  auto rows_copy = [&](double* dst, size_t dld, const double* src, size_t sld, size_t rows, cudaMemcpyKind kind,
                       cudaStream_t st) {
    if (dld == (size_t)nrhs && sld == (size_t)nrhs)
      return cudaMemcpyAsync(dst, src, rows * nrhs * d8, kind, st) == cudaSuccess;
    return cudaMemcpy2DAsync(dst, dld * d8, src, sld * d8, nrhs * d8, rows, kind, st) == cudaSuccess;
  };
  auto b_in = [&]() { return rows_copy(h->hsB, nrhs, b, ldb, h->tot_B, cudaMemcpyHostToDevice, s); };
  auto b_out = [&]() {
    return rows_copy(b, ldb, h->hsB, nrhs, h->tot_B, cudaMemcpyDeviceToHost, s) ? KKT_OK : KKT_ERR_CUDA;
  };
  // page-locked inputs: the factorization reads D, E, G and R in place over
  // the host link (each element once, by the launch that factors its stage),
  // so only b is copied in and x out
  const double *vD = device_view(D), *vE = h->tot_E ? device_view(E) : nullptr,
               *vG = h->tot_G ? device_view(G) : nullptr, *vR = h->tot_R ? device_view(R) : nullptr;
  const bool in_place = vD && (vE || !h->tot_E) && (vG || !h->tot_G) && (vR || !h->tot_R);
  const kkt_status ps = host_prepare(h, nrhs, !in_place);
  if (ps != KKT_OK) return ps;
  if (in_place) {
    if (!b_in()) return KKT_ERR_CUDA;
    std::vector<cudaEvent_t> ev;
    ev.swap(h->events);  // no launch events on this path
    const kkt_status st = kkt_factor_solve(h, vD, vE, h->maxm ? vG : nullptr, h->maxm ? vR : nullptr, h->hsB,
                                           nrhs, nrhs, stream);
    h->events.swap(ev);
    return st != KKT_OK ? st : b_out();
  }
  const bool chunked = h->count == 1 && h->border && nrhs == 1 && h->sys[0].lv[0].P >= 2 &&
                       h->fac_groups[0].size() == 1;
  if (!chunked) {
    if (!b_in() || !h2d(h->hsD, D, h->tot_D, s) || !h2d(h->hsE, E, h->tot_E, s) || !h2d(h->hsG, G, h->tot_G, s) ||
        !h2d(h->hsR, R, h->tot_R, s))
      return KKT_ERR_CUDA;
    std::vector<cudaEvent_t> ev;
    ev.swap(h->events);  // no launch events on this path
    const kkt_status st = kkt_factor_solve(h, h->hsD, h->tot_E ? h->hsE : nullptr, h->maxm ? h->hsG : nullptr,
                                           h->maxm ? h->hsR : nullptr, h->hsB, nrhs, nrhs, stream);
    h->events.swap(ev);
    return st != KKT_OK ? st : b_out();
  }
  // one system, bordered pass: the stage rows of D, E, G and b in chunks that
  // end at separator stages, on the copy stream; each chunk's bordered arrow
  // copy and level-1 segments on a stream of their own as soon as its rows
  // have arrived (the first chunk also brings the corner and the g-rows of b)
  const SysPlan& sp = h->sys[0];
  const LevelPlan& L1 = sp.lv[0];
  const int P = L1.P, K = std::min(kkt_handle::kHostChunks, P);
  const size_t nn = (size_t)sp.n * sp.n, mn = (size_t)sp.m * sp.n;
  // the copy stream starts after the work already queued on `stream`
  if (cudaEventRecord(h->hs_ev_start, s) != cudaSuccess ||
      cudaStreamWaitEvent(h->hs_copy, h->hs_ev_start, 0) != cudaSuccess)
    return KKT_ERR_CUDA;
  const kkt_handle::Group& g1 = h->fac_groups[0][0];
  for (int c = 0; c < K; ++c) {
    const int k0 = (int)((long long)P * c / K), k1 = (int)((long long)P * (c + 1) / K);
    // stages [lo, hi): segments k0..k1-1 with the separator in front of k0
    const int lo = k0 ? L1.start[k0] - 1 : 0, hi = k1 < P ? L1.start[k1] - 1 : sp.N;
    const int ehi = std::min(hi, sp.N - 1);
    cudaStream_t cs = h->hs_copy;
    if (!h2d(h->hsD + lo * nn, D + lo * nn, (size_t)(hi - lo) * nn, cs) ||
        (ehi > lo && !h2d(h->hsE + lo * nn, E + lo * nn, (size_t)(ehi - lo) * nn, cs)) ||
        !h2d(h->hsG + lo * mn, G + lo * mn, (size_t)(hi - lo) * mn, cs) ||
        !rows_copy(h->hsB + (size_t)lo * sp.n, 1, b + (size_t)lo * sp.n * ldb, ldb, (size_t)(hi - lo) * sp.n,
                   cudaMemcpyHostToDevice, cs))
      return KKT_ERR_CUDA;
    if (c == 0 && sp.m > 0 &&
        (!h2d(h->hsR, R, h->tot_R, cs) ||
         !rows_copy(h->hsB + (size_t)sp.N * sp.n, 1, b + (size_t)sp.N * sp.n * ldb, ldb, (size_t)sp.m,
                    cudaMemcpyHostToDevice, cs)))
      return KKT_ERR_CUDA;
    if (cudaEventRecord(h->hs_ev_copy[c], cs) != cudaSuccess) return KKT_ERR_CUDA;
    cudaStream_t ls = h->hs_lvl[c];
    if (cudaStreamWaitEvent(ls, h->hs_ev_copy[c], 0) != cudaSuccess ||
        kkt::launch_border(h->ddesc_b, h->dsys_desc, 1, (long long)(hi - lo) * (sp.m + 1) * sp.n, h->hsG, h->hsR,
                           h->hsB, 1, h->Gb, h->Rb, ls, lo, hi, c == 0))
      return KKT_ERR_CUDA;
    const Task* t = h->dtasks + g1.off + k0;
    const int e = g1.warp ? kkt::launch_factor_w(h->ddesc_b, t, k1 - k0, g1.n, g1.m + 1, 0, h->hsD, h->hsE, h->Gb,
                                                 h->Rb, h->dinfo, ls, h->hsB, 1, g1.fill)
                          : kkt::launch_factor(h->ddesc_b, t, k1 - k0, g1.n, g1.m + 1, 0, level_paired(h, 0),
                                               h->hsD, h->hsE, h->Gb, h->Rb, h->dinfo, ls, h->hsB, 1, g1.fill);
    if (e || cudaEventRecord(h->hs_ev_lvl[c], ls) != cudaSuccess ||
        cudaStreamWaitEvent(s, h->hs_ev_lvl[c], 0) != cudaSuccess)
      return KKT_ERR_CUDA;
  }
  for (int l = 1; l < h->maxL; ++l)
    for (const kkt_handle::Group& gr : h->fac_groups[l]) {
      const int C = clus_of(h, l, gr);
      const int e = C ? kkt::launch_factor_clus(h->ddesc_b, h->dtasks + gr.off, gr.cnt, gr.n, gr.m + 1, C, h->hsD,
                                                h->hsE, h->Gb, h->dinfo, stream, h->hsB, 1)
                    : gr.warp ? kkt::launch_factor_w(h->ddesc_b, h->dtasks + gr.off, gr.cnt, gr.n, gr.m + 1, 0,
                                                   h->hsD, h->hsE, h->Gb, h->Rb, h->dinfo, stream, h->hsB, 1,
                                                   gr.fill)
                            : kkt::launch_factor(h->ddesc_b, h->dtasks + gr.off, gr.cnt, gr.n, gr.m + 1, 0,
                                                 level_paired(h, l), h->hsD, h->hsE, h->Gb, h->Rb, h->dinfo,
                                                 stream, h->hsB, 1, gr.fill, top_in_factor(h, l, gr));
      if (e) return KKT_ERR_CUDA;
    }
  h->factored = true;
  h->cur_b = true;
  const kkt_status st = solve_chunk(h, h->hsB, 1, 1, nullptr, stream, nullptr, 1);
  return st != KKT_OK ? st : b_out();
}

namespace {
// Preconditioned conjugate gradients for the systems whose refinement stalled
// or did not converge (flags 0 and 3), started from the refined x and its
// residual (in dcorr), preconditioned by the factor's solve: r = b - Psi x,
// z = M^{-1} r, p = z, rho = r.z; then cg_iters times q = Psi p, alpha =
// rho / p.q, x += alpha p, r -= alpha q, z = M^{-1} r, rho' = r.z, p = z +
// (rho'/rho) p. The eta of those systems after the last iteration replaces
// that of the last sweep.
kkt_status refine_fallback(kkt_handle* h, const double* D, const double* E, const double* G, const double* R,
                           const double* b, int ldb, double* x, int ldx, int nr, int sweeps, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int CH = kkt::kRhsChunk, nres = (int)h->hres.size(), cnt = h->count;
  const size_t vec = sizeof(double) * h->tot_B * CH;
  auto matvec = [&](const double* v, double* out) {  // out = -Psi v (b = 0)
    return kkt::launch_residual(h->ddesc, h->dres, nres, D, E, G, nullptr, 1, v, CH, out, nr, h->dparts,
                                h->cg_skip, 0, stream, h->res_xs, h->maxm) == 0 &&
           kkt::launch_residual_final(h->ddesc, h->dsys_desc, h->dpart0, cnt, G, R, nullptr, 1, v, CH, out, nr,
                                      h->dparts, -1.0, h->cg_eta, nullptr, h->cg_skip, stream) == 0;
  };
  auto precond = [&]() {  // z = M^{-1} r
    return cudaMemcpyAsync(h->cg_z, h->dcorr, vec, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
           solve_chunk(h, h->cg_z, CH, nr, h->cg_skip, stream, nullptr) == KKT_OK;
  };
  bool ok = kkt::launch_pcg_mask(h->dconv, h->cg_skip, cnt, stream) == 0 && precond() &&
            cudaMemcpyAsync(h->cg_p, h->cg_z, vec, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
            kkt::launch_sys_dot(h->ddesc, h->dsys_desc, h->dconv, cnt, h->dcorr, h->cg_z, nr, h->cg_rho0,
                                stream) == 0;
  for (int it = 0; it < h->cg_iters && ok; ++it) {
    double* rho = (it & 1) ? h->cg_rho1 : h->cg_rho0;
    double* rho_next = (it & 1) ? h->cg_rho0 : h->cg_rho1;
    ok = matvec(h->cg_p, h->cg_q) &&
         kkt::launch_sys_dot(h->ddesc, h->dsys_desc, h->dconv, cnt, h->cg_p, h->cg_q, nr, h->cg_pq, stream) == 0 &&
         kkt::launch_pcg_update(h->ddesc, h->dres, nres, h->dconv, 0, nr, x, ldx, h->dcorr, h->cg_q, h->cg_p,
                                nullptr, rho, h->cg_pq, stream) == 0 &&
         precond() &&
         kkt::launch_sys_dot(h->ddesc, h->dsys_desc, h->dconv, cnt, h->dcorr, h->cg_z, nr, rho_next, stream) == 0 &&
         kkt::launch_pcg_update(h->ddesc, h->dres, nres, h->dconv, 1, nr, x, ldx, h->dcorr, h->cg_q, h->cg_p,
                                h->cg_z, rho_next, rho, stream) == 0;
  }
  // the true residual and eta of the fallback's systems
  ok = ok &&
       kkt::launch_residual(h->ddesc, h->dres, nres, D, E, G, b, ldb, x, ldx, h->dcorr, nr, h->dparts, h->cg_skip, 0,
                            stream, h->res_xs, h->maxm) == 0 &&
       kkt::launch_residual_final(h->ddesc, h->dsys_desc, h->dpart0, cnt, G, R, b, ldb, x, ldx, h->dcorr, nr,
                                  h->dparts, -1.0, h->deta + (size_t)(sweeps - 1) * cnt, nullptr, h->cg_skip,
                                  stream) == 0;
  return ok ? KKT_OK : KKT_ERR_CUDA;
}
}  // namespace

kkt_status kkt_set_refine_tol(kkt_handle* h, double tol) {
  if (!h || !(tol == tol)) return KKT_ERR_ARG;
  h->adj_tol = tol;
  return KKT_OK;
}

kkt_status kkt_set_refine_fallback(kkt_handle* h, int cg_iters) {
  if (!h || cg_iters < 0 || cg_iters > 256) return KKT_ERR_ARG;
  if (cg_iters > 0 && !h->cg_mem) {
    const size_t vec = sizeof(double) * h->tot_B * kkt::kRhsChunk, sc = sizeof(double) * h->count * kkt::kRhsChunk;
    Carver cv;
    const size_t oz = cv.take(vec), op = cv.take(vec), oq = cv.take(vec), o0 = cv.take(sc), o1 = cv.take(sc),
                 opq = cv.take(sc), oe = cv.take(sizeof(double) * h->count), os = cv.take(sizeof(int) * h->count);
    if (cudaMalloc(&h->cg_mem, cv.off) != cudaSuccess) {
      h->cg_mem = nullptr;
      return KKT_ERR_CUDA;
    }
    char* base = (char*)h->cg_mem;
    if (cudaMemset(h->cg_mem, 0, cv.off) != cudaSuccess) return KKT_ERR_CUDA;
    h->cg_z = (double*)(base + oz); h->cg_p = (double*)(base + op); h->cg_q = (double*)(base + oq);
    h->cg_rho0 = (double*)(base + o0); h->cg_rho1 = (double*)(base + o1); h->cg_pq = (double*)(base + opq);
    h->cg_eta = (double*)(base + oe); h->cg_skip = (int*)(base + os);
  }
  h->cg_iters = cg_iters;
  return KKT_OK;
}

kkt_status kkt_solve_refined(kkt_handle* h, const double* D, const double* E, const double* G,
                             const double* R, const double* b, int ldb, double* x, int ldx, int nrhs,
                             int sweeps, double tol, void* stream) {
  if (!h || !D || !b || !x || nrhs < 1 || ldb < nrhs || ldx < nrhs || sweeps < 1 ||
      sweeps > kMaxSweeps)
    return KKT_ERR_ARG;
  if (h->tot_E > 0 && !E) return KKT_ERR_ARG;
  if (h->maxm > 0 && (!G || !R)) return KKT_ERR_ARG;
  if (!h->factored) return KKT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  const int CH = kkt::kRhsChunk, nres = (int)h->hres.size();
  for (int c0 = 0; c0 < nrhs; c0 += CH) {
    const int nr = std::min(CH, nrhs - c0);
    // x = 0, c = b (this chunk's columns), flags cleared
    if (cudaMemset2DAsync(x + c0, sizeof(double) * ldx, 0, sizeof(double) * nr, h->tot_B, st) != cudaSuccess ||
        cudaMemcpy2DAsync(h->dcorr, sizeof(double) * CH, b + c0, sizeof(double) * ldb, sizeof(double) * nr,
                          h->tot_B, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(h->dconv, 0, sizeof(int) * h->count, st) != cudaSuccess)
      return KKT_ERR_CUDA;
    for (int sw = 0; sw < sweeps; ++sw) {
      // correction c <- Psi~^{-1} c with the (mixed) factor, then x += c,
      // c <- b - Psi x in FP64, eta and the per-system flags
      kkt_status s2 = solve_chunk(h, h->dcorr, CH, nr, h->dconv, stream, nullptr);
      if (s2 != KKT_OK) return s2;
      if (kkt::launch_axpy(h->ddesc, h->dres, nres, x + c0, ldx, h->dcorr, nr, h->dconv, stream) ||
          kkt::launch_residual(h->ddesc, h->dres, nres, D, E, G, b + c0, ldb, x + c0, ldx, h->dcorr, nr,
                               h->dparts, h->dconv, c0 == 0 && sw == 0, stream, h->res_xs, h->maxm) ||
          kkt::launch_residual_final(h->ddesc, h->dsys_desc, h->dpart0, h->count, G, R, b + c0, ldb,
                                     x + c0, ldx, h->dcorr, nr, h->dparts, tol,
                                     h->deta + (size_t)sw * h->count,
                                     sw > 0 ? h->deta + (size_t)(sw - 1) * h->count : nullptr, h->dconv,
                                     stream, h->cg_iters > 0))
        return KKT_ERR_CUDA;
    }
    if (h->cg_iters > 0) {
      const kkt_status s3 = refine_fallback(h, D, E, G, R, b + c0, ldb, x + c0, ldx, nr, sweeps, stream);
      if (s3 != KKT_OK) return s3;
    }
  }
  return KKT_OK;
}

kkt_status kkt_solve_adjoint(kkt_handle* h, const double* D, const double* E, const double* G,
                             const double* R, const double* x, int ldx, const double* xbar, int ldxb,
                             double* bbar, int ldbb, int nrhs, double* dD, double* dE, double* dG,
                             double* dR, int sweeps, void* stream) {
  if (!h || !x || !xbar || !bbar || nrhs < 1 || ldx < nrhs || ldxb < nrhs || ldbb < nrhs || !dD)
    return KKT_ERR_ARG;
  if (h->tot_E > 0 && !dE) return KKT_ERR_ARG;
  if (h->maxm > 0 && (!dG || !dR)) return KKT_ERR_ARG;
  if (!h->factored) return KKT_ERR_STATE;
  bool mixed = false;
  for (int v : h->level_mixed) mixed = mixed || v;
  // bbar = Psi^{-1} xbar (Psi is symmetric): the same factor; refined when it is mixed
  if (mixed) {
    if (!D || (h->tot_E > 0 && !E) || (h->maxm > 0 && (!G || !R))) return KKT_ERR_ARG;
    const kkt_status st = kkt_solve_refined(h, D, E, G, R, xbar, ldxb, bbar, ldbb, nrhs,
                                            sweeps < 1 ? 4 : sweeps, h->adj_tol, stream);
    if (st != KKT_OK) return st;
  } else {
    if (cudaMemcpy2DAsync(bbar, sizeof(double) * ldbb, xbar, sizeof(double) * ldxb, sizeof(double) * nrhs,
                          h->tot_B, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
      return KKT_ERR_CUDA;
    const kkt_status st = kkt_solve(h, bbar, nrhs, ldbb, stream);
    if (st != KKT_OK) return st;
  }
  if (kkt::launch_adjoint_grad(h->ddesc, h->dres, (int)h->hres.size(), x, ldx, bbar, ldbb, nrhs, dD, dE,
                               dG, dR, stream))
    return KKT_ERR_CUDA;
  return KKT_OK;
}

kkt_status kkt_refine_eta(kkt_handle* h, int sweep, double* eta) {
  if (!h || !eta || sweep < 0 || sweep >= kMaxSweeps) return KKT_ERR_ARG;
  if (cudaMemcpy(eta, h->deta + (size_t)sweep * h->count, sizeof(double) * h->count,
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return KKT_ERR_CUDA;
  return KKT_OK;
}

kkt_status kkt_get_info(kkt_handle* h, kkt_info* info, int clear) {
  if (!h || !info) return KKT_ERR_ARG;
  kkt::Info hi{};
  if (cudaMemcpy(&hi, h->dinfo, sizeof(hi), cudaMemcpyDeviceToHost) != cudaSuccess) return KKT_ERR_CUDA;
  kkt::Info dbg{};
  if (kkt::debug_info(&dbg, clear)) return KKT_ERR_CUDA;
  if (hi.status == 0 && dbg.status == 8) hi = dbg;  // an index check of the debug build failed
  info->status = hi.status == 3 ? KKT_ERR_NOT_SPD : hi.status == 5 ? KKT_ERR_TIMEOUT
                 : hi.status == 8 ? KKT_ERR_BOUNDS : KKT_OK;
  info->system = hi.system;
  info->stage = hi.stage;
  info->level = hi.level;
  if (clear && cudaMemset(h->dinfo, 0, sizeof(kkt::Info)) != cudaSuccess) return KKT_ERR_CUDA;
  return KKT_OK;
}

kkt_status kkt_get_factor(kkt_handle* h, int system, double* Ld, double* Le, double* Lw, double* Lh,
                          double* Lg, double* Lr) {
  if (!h || system < 0 || system >= h->count) return KKT_ERR_ARG;
  const SysPlan& sp = h->sys[system];
  if (sp.lv.size() > 2) return KKT_ERR_ARG;
  if (!h->factored || h->cur_b) return KKT_ERR_STATE;
  if (cudaDeviceSynchronize() != cudaSuccess) return KKT_ERR_CUDA;
  const int N = sp.N, n = sp.n, m = sp.m, R = 2 * n + m;
  const size_t nn = size_t(n) * n, mn = size_t(m) * n;
  auto fetch = [&](const LevelDesc& d, std::vector<double>& hd, std::vector<double>& hp) {
    hd.resize(size_t(d.N) * nn);
    hp.resize(size_t(d.N) * R * n);
    return cudaMemcpy(hd.data(), d.Ld, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost) == cudaSuccess &&
           cudaMemcpy(hp.data(), d.Lp, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
  };
  std::vector<double> d1, p1, d2, p2;
  const LevelDesc& L1 = h->hdesc[h->desc_of[system][0]];
  if (!fetch(L1, d1, p1)) return KKT_ERR_CUDA;
  if (Ld) std::memset(Ld, 0, sizeof(double) * N * nn);
  if (Le && N > 1) std::memset(Le, 0, sizeof(double) * (N - 1) * nn);
  if (Lw) std::memset(Lw, 0, sizeof(double) * N * nn);
  if (Lh) std::memset(Lh, 0, sizeof(double) * N * nn);
  if (Lg && m) std::memset(Lg, 0, sizeof(double) * N * mn);
  const LevelPlan& P1 = sp.lv[0];
  auto panel = [&](const std::vector<double>& p, int j, int row0, int rows, double* dst) {
    std::memcpy(dst, p.data() + (size_t(j) * R + row0) * n, sizeof(double) * rows * n);
  };
  for (int k = 0; k < P1.P; ++k) {
    const int f = seg_first(P1, k), len = seg_len(P1, k);
    for (int j = f; j < f + len; ++j) {
      if (Ld) std::memcpy(Ld + j * nn, d1.data() + j * nn, sizeof(double) * nn);
      if (Le && j < N - 1 && (j < f + len - 1 || k < P1.P - 1)) panel(p1, j, 0, n, Le + j * nn);
      if (Lg && m) panel(p1, j, n, m, Lg + j * mn);
      if (Lw && k >= 1) panel(p1, j, n + m, n, Lw + j * nn);
    }
  }
  if (sp.lv.size() == 2) {
    const LevelDesc& L2 = h->hdesc[h->desc_of[system][1]];
    if (!fetch(L2, d2, p2)) return KKT_ERR_CUDA;
    for (int k = 1; k < P1.P; ++k) {
      const int s = seg_first(P1, k) - 1, j2 = k - 1;
      if (Ld) std::memcpy(Ld + s * nn, d2.data() + j2 * nn, sizeof(double) * nn);
      if (Lg && m) panel(p2, j2, n, m, Lg + s * mn);
      if (Lh && k < P1.P - 1) panel(p2, j2, 0, n, Lh + s * nn);
    }
  }
  if (Lr && m) {
    const LevelDesc& top = h->hdesc[h->desc_of[system].back()];
    if (cudaMemcpy(Lr, top.Rhat, sizeof(double) * m * m, cudaMemcpyDeviceToHost) != cudaSuccess)
      return KKT_ERR_CUDA;
  }
  return KKT_OK;
}

kkt_status kkt_set_launch_events(kkt_handle* h, void* const* events, int count) {
  if (!h || count < 0) return KKT_ERR_ARG;
  h->events.clear();
  if (events)
    for (int i = 0; i < count; ++i) h->events.push_back((cudaEvent_t)events[i]);
  return KKT_OK;
}

kkt_status kkt_factor_ctas_per_task(const kkt_handle* h, int level, int* ctas) {
  if (!h || !ctas || level < 0 || level >= h->maxL) return KKT_ERR_ARG;
  int c = 1;
  for (const kkt_handle::Group& gr : h->fac_groups[level])
    if (!gr.warp) {
      const int C = clus_of(h, level, gr);
      c = std::max(c, C ? C : level_paired(h, level) ? 2 : 1);
    }
  *ctas = c;
  return KKT_OK;
}

kkt_status kkt_launch_counts(const kkt_handle* h, int* fl, int* sl) {
  if (!h) return KKT_ERR_ARG;
  int f = 0, sv = 0;
  for (int l = 0; l < h->maxL; ++l) {
    f += (int)h->fac_groups[l].size();
    sv += (int)h->fac_groups[l].size() + (h->chain && h->chain_on ? 0 : (int)h->bwd_groups[l].size());
  }
  if (h->chain && h->chain_on) sv += 1;
  if (h->persistent) f = 1;
  if (fl) *fl = f;
  if (sl) *sl = sv;
  return KKT_OK;
}

static void plan_flops(const std::vector<SysPlan>& sys, double* ff, double* sf, double* seqf) {
  double fac = 0.0, sol = 0.0, seq = 0.0, seqsol = 0.0;
  for (const SysPlan& sp : sys) {
    for (const LevelPlan& L : sp.lv)
      for (int k = 0; k < L.P; ++k)
        seg_flops(seg_len(L, k), sp.n, sp.m, k >= 1, k < L.P - 1, &fac, &sol);
    seg_flops(sp.N, sp.n, sp.m, false, false, &seq, &seqsol);
    const double dm = sp.m;
    const double corner = sp.m ? dm * dm * dm / 3.0 + dm * dm / 2.0 + dm / 6.0 : 0.0;
    fac += corner;
    seq += corner;
    sol += 2.0 * dm * dm;
  }
  if (ff) *ff = fac;
  if (sf) *sf = sol;
  if (seqf) *seqf = seq;
}

kkt_status kkt_flops(const kkt_handle* h, double* ff, double* sf, double* seqf) {
  if (!h) return KKT_ERR_ARG;
  plan_flops(h->sys, ff, sf, seqf);
  return KKT_OK;
}

kkt_status kkt_plan_flops(int N, int n, int m, int nlevels, const int* P_levels, int partition, int sms,
                          double* ff, double* sf, double* seqf) {
  if (N < 1 || n < 1 || m < 0 || nlevels < 1 || !P_levels || P_levels[nlevels - 1] != 1 || sms < 0)
    return KKT_ERR_ARG;
  SysPlan sp;
  sp.N = N; sp.n = n; sp.m = m;
  const std::vector<int> pair_lv = paired_levels({std::vector<int>(P_levels, P_levels + nlevels)}, &n, sms);
  int Nl = N;
  for (int l = 0; l < nlevels; ++l) {
    LevelPlan L;
    if (!make_level(Nl, P_levels[l], partition, n, m, pair_lv[l] != 0, &L)) return KKT_ERR_PARTITION;
    sp.lv.push_back(L);
    if (L.P == 1) {
      if (l + 1 != nlevels) return KKT_ERR_ARG;
      break;
    }
    Nl = L.P - 1;
  }
  plan_flops({sp}, ff, sf, seqf);
  return KKT_OK;
}

const char* kkt_status_string(int s) {
  switch (s) {
    case KKT_OK: return "ok";
    case KKT_ERR_ARG: return "invalid argument";
    case KKT_ERR_PARTITION: return "no partition (P > floor((N+1)/2))";
    case KKT_ERR_NOT_SPD: return "pivot block not positive definite";
    case KKT_ERR_CUDA: return "CUDA runtime error";
    case KKT_ERR_TIMEOUT: return "device wait timed out";
    case KKT_ERR_STATE: return "call out of order";
    case KKT_ERR_CAPACITY: return "problem exceeds the fixed buffer capacity";
    case KKT_ERR_BOUNDS: return "index check failed (debug build)";
    default: return "unknown status";
  }
}

}  // extern "C"
