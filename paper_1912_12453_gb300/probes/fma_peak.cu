// Non-tensor FMA pipe peaks of the GPU (FP32 and FP64): every thread runs
// independent chains of fused multiply-adds on registers; flop = 2 per FMA.
// The FP32 number is the roofline denominator of the FP32 element kernels,
// the FP64 number that of the FP64 ones.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fma_peak fma_peak.cu && ./fma_peak
#include <cstdio>
#include <cuda_runtime.h>

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
double run(int blocks, int iters) {
  T *out = nullptr;
  cudaMalloc(&out, sizeof(T));
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
  cudaFree(out);
  return 2.0 * CH * double(iters) * blocks * 256 / (best * 1e-3) / 1e12;
}

int main() {
  int dev = 0, sms = 0, clk = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  const int blocks = sms * 8;
  const double f32 = run<float, 16>(blocks, 20000);
  const double f64 = run<double, 16>(blocks, 500);
  printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"fp32_fma_tflops\": %.2f, \"fp64_fma_tflops\": %.3f}\n", sms,
         clk / 1e3, f32, f64);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    printf("CUDA error: %s\n", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}
