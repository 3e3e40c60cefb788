// Test helper: runs the library's device arithmetic helpers (kkt_numerics.cuh)
// elementwise over an array so that tests can compare them with exact
// references. Built by the tests with nvcc; not part of the library.
#include <cuda_runtime.h>

#include "../../paper_2511_00946_gb300/csrc/kkt_numerics.cuh"

namespace {
__global__ void k_probe(int what, const double* in, double* out, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double v = in[i];
  if (what == 0) out[i] = kkt::pivot_rsqrt(v);
  else if (what == 1) out[i] = (double)kkt::abs_lo(v);
  else out[i] = kkt::not_positive(v) ? 1.0 : 0.0;
}
}  // namespace

// what: 0 = pivot_rsqrt, 1 = abs_lo (as double), 2 = not_positive (0/1).
// in, out: device arrays of `count` doubles. Returns the cudaError_t of the
// launch and of the synchronization.
extern "C" int numerics_probe(int what, const double* in, double* out, long long count) {
  if (count <= 0) return 0;
  const long long blocks = (count + 255) / 256;
  k_probe<<<(unsigned)blocks, 256>>>(what, in, out, count);
  int e = (int)cudaGetLastError();
  if (e) return e;
  return (int)cudaDeviceSynchronize();
}
