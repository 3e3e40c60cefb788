// kkt_solve_noalloc: factor and solve one system without allocating memory.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: a real-time control loop that must not touch the allocator, a
// plugin whose host framework owns every allocation, or a process whose
// memory pool is already exhausted. For them this entry point keeps its
// factor and scratch space in a fixed, library-owned device array instead of
// a handle's cudaMalloc.
//
// The array is a file-scope __device__ variable of kNoallocBytes (16 MiB).
// Every GPU on which the library is loaded holds it until the process exits.
// Its host-side name is only a stand-in, not a device address: the device
// address is looked up with cudaGetSymbolAddress once per device (on the
// first call made with that device current) and cached. Each call stages a
// few small tables (level descriptors, task list, index maps) from a static
// host buffer into the array with cudaMemcpyAsync from pageable memory, which
// may block the host until the data is staged.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/kkt.h"
#include "kkt_internal.h"

namespace {

constexpr size_t kNoallocBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;
constexpr int kMaxP = 1024;        // largest segment count
constexpr int kMaxStages = 16384;  // largest N

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Host staging for the small tables (descriptors, tasks, index maps) copied
// into the scratch array on every call; guarded by g_mu.
struct Staging {
  kkt::LevelDesc desc[2];
  kkt::Task tasks[2 * kMaxP + 1];
  int nat1[kMaxStages];
  int nat2[kMaxP];
  int seg1[kMaxP + 1];
  int seg2[2];
};
Staging g_stage;

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace

extern "C" kkt_status kkt_solve_noalloc(int N, int n, int m, int P, const double* D, const double* E,
                                        const double* G, const double* R, double* b, int nrhs, int ldb,
                                        int* info, void* stream) {
  if (N < 1 || n < 1 || n > kkt::kMaxN || m < 0 || m > kkt::kMaxM || P < 1 || !D || !b ||
      nrhs < 1 || ldb < nrhs || (N > 1 && !E) || (m > 0 && (!G || !R)))
    return KKT_ERR_ARG;
  if (N > kMaxStages || P > kMaxP) return KKT_ERR_CAPACITY;
  int seg[kMaxP];
  if (kkt_partition_rule(N, P, seg) != KKT_OK) return KKT_ERR_PARTITION;

  // layout of the scratch array for this shape
  const size_t D8 = sizeof(double), CH = kkt::kRhsChunk;
  const size_t nn = size_t(n) * n, mn = size_t(m) * n, Rr = 2 * n + m;
  const bool two = P > 1;
  const int N2 = P - 1;
  Carve cv;
  const size_t oLd1 = cv.take(D8 * N * nn), oLdM1 = cv.take(D8 * N * nn), oLdR1 = cv.take(D8 * N * nn);
  const size_t oLri1 = cv.take(D8 * N * n), oLp1 = cv.take(D8 * N * Rr * n);
  size_t oDA = 0, oDB = 0, oEN = 0, oGA = 0, oGB = 0, oYA = 0, oYB = 0;
  size_t oLd2 = 0, oLdM2 = 0, oLdR2 = 0, oLri2 = 0, oLp2 = 0, oX2 = 0;
  if (two) {
    oDA = cv.take(D8 * N2 * nn); oDB = cv.take(D8 * N2 * nn);
    oEN = cv.take(D8 * (N2 > 1 ? N2 - 1 : 1) * nn);
    oGA = cv.take(D8 * N2 * (mn ? mn : 1)); oGB = cv.take(D8 * N2 * (mn ? mn : 1));
    oYA = cv.take(D8 * N2 * n * CH); oYB = cv.take(D8 * N2 * n * CH);
    oLd2 = cv.take(D8 * N2 * nn); oLdM2 = cv.take(D8 * N2 * nn); oLdR2 = cv.take(D8 * N2 * nn);
    oLri2 = cv.take(D8 * N2 * n); oLp2 = cv.take(D8 * N2 * Rr * n); oX2 = cv.take(D8 * N2 * n * CH);
  }
  const int nparts = two ? P : 0;
  const size_t oRhat = cv.take(D8 * (m ? m * m : 1)), oRri = cv.take(D8 * (m ? m : 1));
  const size_t oRpart = cv.take(D8 * (nparts * m * m ? nparts * m * m : 1));
  const size_t oYg = cv.take(D8 * (nparts * m ? nparts * m * CH : 1));
  const size_t oDesc = cv.take(sizeof(kkt::LevelDesc) * 2);
  const size_t oTask = cv.take(sizeof(kkt::Task) * (2 * P + 1));
  const size_t oNat1 = cv.take(sizeof(int) * N), oNat2 = cv.take(sizeof(int) * (two ? N2 : 1));
  const size_t oSeg1 = cv.take(sizeof(int) * (P + 1)), oSeg2 = cv.take(sizeof(int) * 2);
  const size_t oInfo = cv.take(sizeof(kkt::Info));
  if (cv.off > kNoallocBytes) return KKT_ERR_CAPACITY;
  if (kkt::factor_smem_bytes(n, m, 0) > 227 * 1024) return KKT_ERR_ARG;

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KKT_ERR_CUDA;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KKT_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  char* base = (char*)g_scratch_addr[dev];
  auto dp = [&](size_t o) { return (double*)(base + o); };

  // index maps and segment starts (Eq. (13))
  Staging& S = g_stage;
  std::memset(S.desc, 0, sizeof(S.desc));
  S.seg1[0] = 0;
  for (int k = 0; k < P; ++k) S.seg1[k + 1] = S.seg1[k] + seg[k] + 1;
  for (int j = 0; j < N; ++j) S.nat1[j] = j;
  for (int k = 1; k < P; ++k) S.nat2[k - 1] = S.seg1[k] - 1;
  S.seg2[0] = 0;
  S.seg2[1] = N2 + 1;

  kkt::LevelDesc& d1 = S.desc[0];
  d1.N = N; d1.n = n; d1.m = m; d1.P = P;
  d1.seg = (const int*)(base + oSeg1);
  d1.level = 1;
  d1.is_top = !two;
  d1.rowG = (long long)N * n;
  d1.Nnat = N;
  d1.nat = (const int*)(base + oNat1);
  d1.Ld = dp(oLd1); d1.LdM = dp(oLdM1); d1.LdR = dp(oLdR1); d1.Lri = dp(oLri1); d1.Lp = dp(oLp1);
  d1.Rhat = dp(oRhat); d1.Rri = dp(oRri);
  d1.Rpart_all = dp(oRpart); d1.nRpart_all = nparts;
  d1.yg_all = dp(oYg); d1.nyg_all = nparts;
  if (two) {
    d1.DA = dp(oDA); d1.DB = dp(oDB); d1.EN = dp(oEN); d1.GA = dp(oGA); d1.GB = dp(oGB);
    d1.YA = dp(oYA); d1.YB = dp(oYB);
    d1.Rpart = dp(oRpart); d1.ygpart = dp(oYg);
    d1.Xnext = dp(oX2);
    kkt::LevelDesc& d2 = S.desc[1];
    d2 = d1;
    d2.N = N2; d2.P = 1;
    d2.seg = (const int*)(base + oSeg2);
    d2.level = 2;
    d2.is_top = 1;
    d2.nat = (const int*)(base + oNat2);
    d2.Ld = dp(oLd2); d2.LdM = dp(oLdM2); d2.LdR = dp(oLdR2); d2.Lri = dp(oLri2); d2.Lp = dp(oLp2);
    d2.DA = d2.DB = d2.EN = d2.GA = d2.GB = d2.YA = d2.YB = nullptr;
    d2.Rpart = d2.ygpart = d2.Xnext = nullptr;
    d2.X = dp(oX2);
    d2.Dw = dp(oDA); d2.D2w = dp(oDB); d2.Ew = dp(oEN);
    d2.Gw = m ? dp(oGA) : nullptr; d2.G2w = m ? dp(oGB) : nullptr;
    d2.RA = dp(oYA); d2.RB = dp(oYB);
  }
  // tasks: level-1 factor/forward [0, P), level-2 [P, P+1), level-1 backward [P+1, 2P+1)
  for (int k = 0; k < P; ++k) S.tasks[k] = kkt::Task{0, k};
  S.tasks[P] = kkt::Task{1, 0};
  for (int k = 0; k < P; ++k) S.tasks[P + 1 + k] = kkt::Task{0, k};

  cudaStream_t st = (cudaStream_t)stream;
  kkt::Info* dinfo = info ? (kkt::Info*)info : (kkt::Info*)(base + oInfo);
  bool ok = cudaMemcpyAsync(base + oDesc, S.desc, sizeof(kkt::LevelDesc) * (two ? 2 : 1),
                            cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(base + oTask, S.tasks, sizeof(kkt::Task) * (2 * P + 1),
                             cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(base + oNat1, S.nat1, sizeof(int) * N, cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(base + oSeg1, S.seg1, sizeof(int) * (P + 1), cudaMemcpyHostToDevice, st) ==
                 cudaSuccess;
  if (two) {
    ok = ok && cudaMemcpyAsync(base + oNat2, S.nat2, sizeof(int) * N2, cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(base + oSeg2, S.seg2, sizeof(int) * 2, cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
  }
  // the breakdown record is the only state that must start at zero
  ok = ok && cudaMemsetAsync(dinfo, 0, sizeof(kkt::Info), st) == cudaSuccess;
  if (!ok) return KKT_ERR_CUDA;

  const kkt::LevelDesc* ddesc = (const kkt::LevelDesc*)(base + oDesc);
  const kkt::Task* dtask = (const kkt::Task*)(base + oTask);
  if (kkt::launch_factor(ddesc, dtask, P, n, m, 0, 0, D, E, G, R, dinfo, stream)) return KKT_ERR_CUDA;
  if (two && kkt::launch_factor(ddesc, dtask + P, 1, n, m, 0, 0, D, E, G, R, dinfo, stream)) return KKT_ERR_CUDA;
  for (int c0 = 0; c0 < nrhs; c0 += kkt::kRhsChunk) {
    const int nr = nrhs - c0 < kkt::kRhsChunk ? nrhs - c0 : kkt::kRhsChunk;
    if (kkt::launch_forward(ddesc, dtask, P, n, m, 0, b + c0, ldb, nr, nullptr, stream)) return KKT_ERR_CUDA;
    if (two) {
      if (kkt::launch_forward(ddesc, dtask + P, 1, n, m, 0, b + c0, ldb, nr, nullptr, stream))
        return KKT_ERR_CUDA;
      if (kkt::launch_backward(ddesc, dtask + P + 1, P, n, m, 0, b + c0, ldb, nr, nullptr, stream))
        return KKT_ERR_CUDA;
    }
  }
  return KKT_OK;
}
