// Host stand-ins for the CUDA runtime calls of the library's mesh builder, so
// that its host code (mesh.cpp) can be built and checked without a GPU: the
// "device" arrays are host allocations.  Test infrastructure only.
#include <cstdlib>
#include <cstring>

#include <cuda_runtime.h>

extern "C" {
cudaError_t cudaMalloc(void **p, size_t n) {
  *p = std::malloc(n ? n : 1);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void *p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaMemcpy(void *d, const void *s, size_t n, cudaMemcpyKind) {
  std::memcpy(d, s, n);
  return cudaSuccess;
}
cudaError_t cudaGetDevice(int *d) {
  *d = 0;
  return cudaSuccess;
}
const char *cudaGetErrorString(cudaError_t) { return "host stand-in"; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaFreeHost(void *p) {
  std::free(p);
  return cudaSuccess;
}
}
