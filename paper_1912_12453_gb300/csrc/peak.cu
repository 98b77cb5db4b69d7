// Non-tensor FMA pipe peaks of the GPU, measured in the run that reports a
// roofline fraction against them: every thread runs independent chains of
// fused multiply-adds on registers (flop = 2 per FMA), all SMs busy, best of
// five CUDA-event timings.  Built into libchns_peak.so, a library of its own
// that only the benchmark loads; the solver does not use it.
#include <cuda_runtime.h>

namespace {

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma(T *out, int iters, T a, T b) {
  T x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  if (s == T(12345.678)) out[0] = s;  // keeps the chains live; never true
}

template <typename T, int CH>
int run(int blocks, int iters, double *tflops) {
  T *out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma<T, CH><<<blocks, 256>>>(out, iters, T(0.999999), T(1e-7));  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma<T, CH><<<blocks, 256>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *tflops = 2.0 * CH * double(iters) * blocks * 256 / (best * 1e-3) / 1e12;
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace

// FP32 and FP64 FMA peaks (TFLOP/s) of the current device; returns 0 on success.
extern "C" int chns_peak_fma(double *fp32_tflops, double *fp64_tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  if (run<float, 16>(blocks, 20000, fp32_tflops)) return 1;
  return run<double, 16>(blocks, 500, fp64_tflops);
}
