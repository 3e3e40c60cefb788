// Test helper: measures the FP64 arithmetic rates that the kernels' design
// rests on, on the device it runs on: FP64 FMA throughput over every SM,
// the cycles a warp waits for one dependent FP64 FMA, the throughput of the
// warp-level FP64 matrix multiply-accumulate (mma.sync m8n8k4 with FP64
// operands and accumulators), and the FP32 FMA throughput for comparison.
// Built by the tests with nvcc; not part of the library.
#include <cuda_runtime.h>

namespace {
constexpr int kChains = 8;

// every thread: kChains independent FMA chains of `iters` steps
template <typename T>
__global__ void k_fma(T* out, int iters, T a, T b) {
  T acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one warp, one dependent chain: clock cycles per step
__global__ void k_dfma_latency(double* out, long long* cycles, int iters, double a, double b) {
  double acc = threadIdx.x * 1e-3;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) acc = fma(acc, a, b);
  const long long t1 = clock64();
  out[threadIdx.x] = acc;
  if (threadIdx.x == 0) *cycles = t1 - t0;
}

// every warp: kChains / 2 independent accumulators of mma.sync m8n8k4 FP64
// (each MMA is 8 x 8 x 4 = 256 multiply-adds)
__global__ void k_dmma(double* out, int iters, double a, double b) {
  double d[kChains / 2][2];
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) d[k][0] = d[k][1] = threadIdx.x * 1e-3 + k;
  const double av = a + threadIdx.x * 1e-6, bv = b - threadIdx.x * 1e-6;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[k][0]), "+d"(d[k][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) s += d[k][0] + d[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
float time_ms(F launch) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();  // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}
}  // namespace

// out[0] FP64 FMA TFLOP/s, out[1] cycles per dependent FP64 FMA (one warp),
// out[2] FP64 mma.sync TFLOP/s, out[3] FP32 FMA TFLOP/s, out[4] SM count,
// out[5] the SM clock the driver reports (MHz). Returns the first CUDA error.
extern "C" int fp64_rates(double* out) {
  int dev = 0, sms = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  const int blocks = sms * 8, threads = 256, n = blocks * threads;
  double* dbuf = nullptr;
  float* fbuf = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&dbuf, sizeof(double) * n) != cudaSuccess) return 2;
  if (cudaMalloc(&fbuf, sizeof(float) * n) != cudaSuccess) return 2;
  if (cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) return 2;
  const int it64 = 4096, itmma = 2048, it32 = 65536;
  const float t64 = time_ms([&] { k_fma<double><<<blocks, threads>>>(dbuf, it64, 0.999999, 1e-7); });
  out[0] = 2.0 * kChains * (double)it64 * n / (t64 * 1e-3) / 1e12;
  k_dfma_latency<<<1, 32>>>(dbuf, cyc, it64, 0.999999, 1e-7);
  long long c = 0;
  cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
  out[1] = (double)c / it64;
  const float tm = time_ms([&] { k_dmma<<<blocks, threads>>>(dbuf, itmma, 0.999999, 1e-7); });
  out[2] = 2.0 * 256.0 * (kChains / 2) * (double)itmma * (n / 32) / (tm * 1e-3) / 1e12;
  const float t32 = time_ms([&] { k_fma<float><<<blocks, threads>>>(fbuf, it32, 0.9999f, 1e-4f); });
  out[3] = 2.0 * kChains * (double)it32 * n / (t32 * 1e-3) / 1e12;
  out[4] = sms;
  out[5] = khz / 1000.0;
  const int e = (int)cudaDeviceSynchronize();
  cudaFree(dbuf);
  cudaFree(fbuf);
  cudaFree(cyc);
  return e;
}
