// chns_energy_mass_noalloc: the energy / mass / bubble-volume diagnostics
// without any device allocation.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- code issued while a stream is being captured into a CUDA graph
// (cudaMalloc is not allowed during a global-mode capture), and host
// frameworks that hand all device memory to their own pool at start-up and
// forbid allocation afterwards.  chns_energy_mass allocates its reduction
// scratch lazily on first use; this variant never does.
//
// The per-block partial sums live in a file-scope device array of fixed size
// (kMaxBlocks x 3 doubles = 1.5 MiB), which every GPU that loads the library
// keeps until the process exits.  Host code cannot pass the array's name to
// a kernel (on the host it is only a stand-in symbol), so the first call on
// each device looks up its device address with cudaGetSymbolAddress and
// caches it for the life of the process; make that first call before any
// stream capture begins.  The cached address belongs to the device's primary
// context: after cudaDeviceReset (or anything else that destroys that
// context) it is stale, so this library must not be used across a device
// reset.  All calls share the array: calls that overlap on the GPU
// (different streams, no ordering between them) race on it.  Every call
// overwrites the partials it uses before reading them, so nothing needs to
// start at zero.
#include <cstdint>
#include <mutex>

#include "chns_internal.h"
#include "kernels.h"

namespace chns {

namespace {

constexpr int64_t kMaxBlocks = 65536;      // energy kernel blocks (256 threads, 2^dim per element)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxBlocks * 3];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

// out[k] = sum over blocks b of g_partials[b * 3 + k] in a fixed order: one
// block of 256 threads, thread t sums the blocks t, t + 256, ... in
// increasing order, then a fixed shuffle tree per warp and a fixed sum over
// the warps.  Deterministic; the order differs from chns_energy_mass's host
// loop only by rounding.
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) k_sum3(int64_t nb, double *__restrict__ out) {
  double s[3] = {0.0, 0.0, 0.0};
  for (int64_t b = threadIdx.x; b < nb; b += kSumThreads)
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] += g_partials[b * 3 + k];
  __shared__ double part[3][kSumThreads / 32];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
    if ((threadIdx.x & 31) == 0) part[k][threadIdx.x >> 5] = s[k];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) t += part[threadIdx.x][w];
    out[threadIdx.x] = t;
  }
}

chns_status scratch_address(double **p) {
  int dev = 0;
  CHNS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) { set_error("device index %d out of range", dev); return CHNS_ERR_ARG; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *a = nullptr;
    CHNS_CUDA_TRY(cudaGetSymbolAddress(&a, g_partials));
    g_addr[dev] = static_cast<double *>(a);
  }
  *p = g_addr[dev];
  return CHNS_OK;
}

}  // namespace

}  // namespace chns

using namespace chns;

extern "C" chns_status chns_energy_mass_noalloc(const chns_mesh *m, const chns_params *p, const double *U,
                                                double *out3, void *stream) {
  chns_status ps = check_params(m, p);  // the same checks as chns_energy_mass
  if (ps != CHNS_OK) return ps;
  if (!U || !out3) { set_error("null argument"); return CHNS_ERR_ARG; }
  const int64_t nb = energy_blocks(m);
  if (nb > kMaxBlocks) {
    set_error("mesh too large for chns_energy_mass_noalloc: %lld elements need %lld reduction blocks, "
              "the fixed scratch holds %lld (at most %lld leaves in 3D, %lld in 2D)",
              (long long)m->n_elem, (long long)nb, (long long)kMaxBlocks, (long long)(kMaxBlocks * 256 / 8),
              (long long)(kMaxBlocks * 256 / 4));
    return CHNS_ERR_ARG;
  }
  int dev = 0;
  CHNS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != m->device) { set_error("the mesh lives on device %d, current device is %d", m->device, dev); return CHNS_ERR_ARG; }
  double *scratch = nullptr;
  chns_status s = scratch_address(&scratch);
  if (s != CHNS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PhysCoef pc = make_coef(*p, m->lo, m->hi);
  launch_energy(m, pc, U, scratch, st);
  k_sum3<<<1, kSumThreads, 0, st>>>(nb, out3);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error("kernel launch failed: %s", cudaGetErrorString(e)); return CHNS_ERR_CUDA; }
  return CHNS_OK;
}
