// Krylov vector kernels (FGMRES with classical Gram-Schmidt applied twice),
// nodal block-Jacobi preconditioner, deterministic double reductions.
#include <algorithm>
#include <cstdint>

#include "chns_internal.h"
#include "vector.h"

namespace chns {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kB = 256;
constexpr int kRedBlocks = 152 * 4;  // fixed: reductions are deterministic

inline unsigned grid_n(int64_t n) {
  int64_t b = (n + kB - 1) / kB;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 8);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

// block sum of NV values per thread -> out[NV * blockIdx.x + k]
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double *out) {
  __shared__ double sh[NV][kB / 32];
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(v[k]);
    if (ln == 0) sh[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < kB / 32; ++w) s += sh[threadIdx.x][w];
    out[(int64_t)gridDim.x * threadIdx.x + blockIdx.x] = s;
  }
}

// partial[k * nblocks + b] for k < nv -> res[k]; fixed order
__global__ void k_sum_partials(const double *__restrict__ partial, int nblocks, int nv,
                               double *__restrict__ res) {
  const int k = blockIdx.x;
  if (k >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)k * nblocks + b];
  __shared__ double sh[kB / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    res[k] = t;
  }
}

// h[i] = V_i . w for i in [i0, i0 + NV)   (V_i at V + i * ld)
template <int NV>
__global__ void __launch_bounds__(kB) k_multidot(const double *__restrict__ V, int64_t ld, int i0, int nv,
                                                 const double *__restrict__ w, int64_t n,
                                                 double *__restrict__ partial) {
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) {
    double x = w[t];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nv) acc[k] += V[(int64_t)(i0 + k) * ld + t] * x;
  }
  block_sum_store<NV>(acc, partial + (int64_t)i0 * gridDim.x);
}

// w -= sum_i h[i] V_i, i < nv
__global__ void __launch_bounds__(kB) k_update(const double *__restrict__ V, int64_t ld, int nv,
                                               const double *__restrict__ h, double *__restrict__ w,
                                               int64_t n) {
  __shared__ double hs[kMaxRestart + 1];
  for (int i = threadIdx.x; i < nv; i += kB) hs[i] = h[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) {
    double s = w[t];
    for (int i = 0; i < nv; ++i) s -= hs[i] * V[(int64_t)i * ld + t];
    w[t] = s;
  }
}

// w -= sum_i h[i] V_i (i < nv) and per-block partial sums of the new |w|^2;
// skipped entirely when flag is given and *flag == 0
__global__ void __launch_bounds__(kB) k_update_norm(const double *__restrict__ V, int64_t ld, int nv,
                                                    const double *__restrict__ h, double *__restrict__ w,
                                                    int64_t n, const int *__restrict__ flag,
                                                    double *__restrict__ partial) {
  if (flag && *flag == 0) return;
  __shared__ double hs[kMaxRestart + 1];
  for (int i = threadIdx.x; i < nv; i += kB) hs[i] = h[i];
  __syncthreads();
  double acc[1] = {0.0};
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) {
    double s = w[t];
    for (int i = 0; i < nv; ++i) s -= hs[i] * V[(int64_t)i * ld + t];
    w[t] = s;
    acc[0] += s * s;
  }
  block_sum_store<1>(acc, partial);
}

// multi-dot that is skipped when *flag == 0
template <int NV>
__global__ void __launch_bounds__(kB) k_multidot_if(const double *__restrict__ V, int64_t ld, int i0, int nv,
                                                    const double *__restrict__ w, int64_t n,
                                                    double *__restrict__ partial, const int *__restrict__ flag) {
  if (*flag == 0) return;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) {
    double x = w[t];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nv) acc[k] += V[(int64_t)(i0 + k) * ld + t] * x;
  }
  block_sum_store<NV>(acc, partial + (int64_t)i0 * gridDim.x);
}

__global__ void k_sum_partials_if(const double *__restrict__ partial, int nblocks, int nv, double *__restrict__ res,
                                  const int *__restrict__ flag) {
  const int k = blockIdx.x;
  if (k >= nv) return;
  if (*flag == 0) {
    if (threadIdx.x == 0) res[k] = 0.0;
    return;
  }
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)k * nblocks + b];
  __shared__ double sh[kB / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    res[k] = t;
  }
}

// Reorthogonalise only on severe cancellation: the first projection removed
// more than 99.99% of |w|^2 (|w| dropped below 1% of its length); the
// Newton corrections need a linear reduction of ~1e-3 only
__global__ void k_reorth_flag(const double *__restrict__ before, const double *__restrict__ after,
                              int *__restrict__ flag) {
  *flag = (after[0] < 1e-4 * before[0]) ? 1 : 0;
}

// out = x / sqrt(chosen |w|^2): n2[0] if *flag else n1[0]
__global__ void k_normalize(double *__restrict__ w, int64_t n, const double *__restrict__ n1,
                            const double *__restrict__ n2, const int *__restrict__ flag) {
  const double q = *flag ? n2[0] : n1[0];
  if (!(q > 0.0)) return;
  const double s = 1.0 / sqrt(q);
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) w[t] *= s;
}

// out = x / nrm[0]
__global__ void k_scale_by(const double *__restrict__ x, const double *__restrict__ nrm, double *__restrict__ out,
                           int64_t n) {
  double s = 1.0 / nrm[0];
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) out[t] = x[t] * s;
}

template <typename A, typename B>
__global__ void k_convert(const A *__restrict__ x, B *__restrict__ y, int64_t n, double a) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    y[t] = B(a * double(x[t]));
}

// x += sum_j c[j] Z_j
template <typename T>
__global__ void k_combine(const T *__restrict__ Z, int64_t ld, int nz, const double *__restrict__ c,
                          double *__restrict__ x, int64_t n) {
  __shared__ double cs[kMaxRestart];
  for (int i = threadIdx.x; i < nz; i += kB) cs[i] = c[i];
  __syncthreads();
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) {
    double s = x[t];
    for (int j = 0; j < nz; ++j) s += cs[j] * double(Z[(int64_t)j * ld + t]);
    x[t] = s;
  }
}

// y = a x + b y
__global__ void k_axpby(double a, const double *__restrict__ x, double b, double *__restrict__ y, int64_t n) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    y[t] = a * x[t] + b * y[t];
}

// z = a x + b y (out of place)
__global__ void k_lincomb(double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                          double *__restrict__ z, int64_t n) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    z[t] = a * x[t] + b * y[t];
}

// keep field k of each node block, scaled; zero the others
__global__ void k_mask_field(double *__restrict__ y, int64_t n_nodes, int nf, int k, double s) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n_nodes * nf; t += int64_t(gridDim.x) * kB)
    y[t] = (t % nf == k) ? s * y[t] : 0.0;
}

// probing vector: 1 in field f of the nodes of one node colour
template <typename T>
__global__ void k_probe_set(const int32_t *__restrict__ nodes, int64_t cnt, int nf, int f, T *__restrict__ w) {
  int64_t i = blockIdx.x * int64_t(kB) + threadIdx.x;
  if (i < cnt) w[int64_t(nodes[i]) * nf + f] = T(1);
}

// B[a][r][f] = y[a*nf + r] for the probed nodes
template <typename T>
__global__ void k_probe_get(const int32_t *__restrict__ nodes, int64_t cnt, int nf, int f,
                            const T *__restrict__ y, T *__restrict__ B) {
  int64_t i = blockIdx.x * int64_t(kB) + threadIdx.x;
  if (i < cnt) {
    int64_t a = nodes[i];
    for (int r = 0; r < nf; ++r) B[(a * nf + r) * nf + f] = y[a * nf + r];
  }
}

// in-place inverse of each nf x nf nodal block (Gauss-Jordan, partial pivoting, double)
template <typename T, int NF>
__global__ void k_invert_blocks(T *__restrict__ B, int64_t n_nodes, int *__restrict__ bad) {
  int64_t a = blockIdx.x * int64_t(kB) + threadIdx.x;
  if (a >= n_nodes) return;
  double M[NF][2 * NF];
  for (int r = 0; r < NF; ++r)
    for (int c = 0; c < NF; ++c) {
      M[r][c] = double(B[(a * NF + r) * NF + c]);
      M[r][NF + c] = r == c ? 1.0 : 0.0;
    }
  for (int c = 0; c < NF; ++c) {
    int p = c;
    double best = fabs(M[c][c]);
    for (int r = c + 1; r < NF; ++r)
      if (fabs(M[r][c]) > best) { best = fabs(M[r][c]); p = r; }
    if (!(best > 0.0)) { *bad = 1; return; }
    if (p != c)
      for (int k = 0; k < 2 * NF; ++k) { double t = M[c][k]; M[c][k] = M[p][k]; M[p][k] = t; }
    double inv = 1.0 / M[c][c];
    for (int k = 0; k < 2 * NF; ++k) M[c][k] *= inv;
    for (int r = 0; r < NF; ++r) {
      if (r == c) continue;
      double f = M[r][c];
      if (f != 0.0)
        for (int k = 0; k < 2 * NF; ++k) M[r][k] -= f * M[c][k];
    }
  }
  for (int r = 0; r < NF; ++r)
    for (int c = 0; c < NF; ++c) B[(a * NF + r) * NF + c] = T(M[r][NF + c]);
}

// z = Binv v  (v double, z and Binv in T)
template <typename T, int NF>
__global__ void __launch_bounds__(kB) k_block_apply(const T *__restrict__ Binv, const double *__restrict__ v,
                                                    T *__restrict__ z, int64_t n_nodes) {
  for (int64_t a = blockIdx.x * int64_t(kB) + threadIdx.x; a < n_nodes; a += int64_t(gridDim.x) * kB) {
    T x[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) x[c] = T(v[a * NF + c]);
    const T *b = Binv + a * NF * NF;
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < NF; ++c) s += b[r * NF + c] * x[c];
      z[a * NF + r] = s;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers
int red_blocks() { return kRedBlocks; }

void vec_multidot(const double *V, int64_t ld, int nv, const double *w, int64_t n, double *partial,
                  double *h, cudaStream_t st) {
  for (int i0 = 0; i0 < nv; i0 += 8) {
    int c = std::min(8, nv - i0);
    k_multidot<8><<<kRedBlocks, kB, 0, st>>>(V, ld, i0, c, w, n, partial);
    note_launches(1);
  }
  k_sum_partials<<<nv, kB, 0, st>>>(partial, kRedBlocks, nv, h);
  note_launches(1);
}

void vec_dot(const double *x, const double *y, int64_t n, double *partial, double *res, cudaStream_t st) {
  k_multidot<1><<<kRedBlocks, kB, 0, st>>>(x, 0, 0, 1, y, n, partial);
  note_launches(1);
  k_sum_partials<<<1, kB, 0, st>>>(partial, kRedBlocks, 1, res);
  note_launches(1);
}

// One Arnoldi orthogonalisation of w = V_{nv} against V_0..V_{nv-1} (classical
// Gram-Schmidt, a second pass only on severe cancellation), then
// normalisation of w when its norm is nonzero.  Device outputs (no host sync):
// h1[0..nv-1] first-pass coefficients, h1[nv] = |w|^2 before; h2[0..nv-1]
// second-pass coefficients (0 if skipped); nrm[0] = |w|^2 after pass 1,
// nrm[1] = after pass 2, flag[0] = whether pass 2 ran.
void vec_orthogonalize(double *V, int64_t ld, int nv, int64_t n, double *partial, double *h1, double *h2,
                       double *nrm, int *flag, cudaStream_t st) {
  // pass 1 dots include w itself (stored right after V_{nv-1}): |w|^2
  vec_multidot(V, ld, nv + 1, V + (int64_t)nv * ld, n, partial, h1, st);
  double *w = V + (int64_t)nv * ld;
  k_update_norm<<<kRedBlocks, kB, 0, st>>>(V, ld, nv, h1, w, n, nullptr, partial);
  k_sum_partials<<<1, kB, 0, st>>>(partial, kRedBlocks, 1, nrm);
  k_reorth_flag<<<1, 1, 0, st>>>(h1 + nv, nrm, flag);
  for (int i0 = 0; i0 < nv; i0 += 8) {
    int c = std::min(8, nv - i0);
    k_multidot_if<8><<<kRedBlocks, kB, 0, st>>>(V, ld, i0, c, w, n, partial, flag);
  }
  k_sum_partials_if<<<nv, kB, 0, st>>>(partial, kRedBlocks, nv, h2, flag);
  k_update_norm<<<kRedBlocks, kB, 0, st>>>(V, ld, nv, h2, w, n, flag, partial);
  k_sum_partials_if<<<1, kB, 0, st>>>(partial, kRedBlocks, 1, nrm + 1, flag);
  note_launches(6 + (nv + 7) / 8 + (nv + 1 + 7) / 8 + 1);
}

void vec_normalize(double *w, int64_t n, const double *nrm, const int *flag, cudaStream_t st) {
  k_normalize<<<grid_n(n), kB, 0, st>>>(w, n, nrm, nrm + 1, flag);
  note_launches(1);
}

void vec_update(const double *V, int64_t ld, int nv, const double *h, double *w, int64_t n, cudaStream_t st) {
  k_update<<<grid_n(n), kB, 0, st>>>(V, ld, nv, h, w, n);
  note_launches(1);
}

void vec_scale_by(const double *x, const double *nrm2_sqrt, double *out, int64_t n, cudaStream_t st) {
  k_scale_by<<<grid_n(n), kB, 0, st>>>(x, nrm2_sqrt, out, n);
  note_launches(1);
}

template <typename A, typename B>
void vec_convert(const A *x, B *y, int64_t n, double a, cudaStream_t st) {
  k_convert<A, B><<<grid_n(n), kB, 0, st>>>(x, y, n, a);
  note_launches(1);
}
template void vec_convert<float, double>(const float *, double *, int64_t, double, cudaStream_t);
template void vec_convert<double, float>(const double *, float *, int64_t, double, cudaStream_t);
template void vec_convert<double, double>(const double *, double *, int64_t, double, cudaStream_t);

template <typename T>
void vec_combine(const T *Z, int64_t ld, int nz, const double *c, double *x, int64_t n, cudaStream_t st) {
  k_combine<T><<<grid_n(n), kB, 0, st>>>(Z, ld, nz, c, x, n);
  note_launches(1);
}
template void vec_combine<float>(const float *, int64_t, int, const double *, double *, int64_t, cudaStream_t);
template void vec_combine<double>(const double *, int64_t, int, const double *, double *, int64_t, cudaStream_t);

void vec_axpby(double a, const double *x, double b, double *y, int64_t n, cudaStream_t st) {
  k_axpby<<<grid_n(n), kB, 0, st>>>(a, x, b, y, n);
  note_launches(1);
}

void vec_lincomb(double a, const double *x, double b, const double *y, double *z, int64_t n, cudaStream_t st) {
  k_lincomb<<<grid_n(n), kB, 0, st>>>(a, x, b, y, z, n);
  note_launches(1);
}

void vec_mask_field(double *y, int64_t n_nodes, int nf, int k, double s, cudaStream_t st) {
  k_mask_field<<<grid_n(n_nodes * nf), kB, 0, st>>>(y, n_nodes, nf, k, s);
  note_launches(1);
}

template <typename T>
void probe_set(const int32_t *nodes, int64_t cnt, int nf, int f, T *w, cudaStream_t st) {
  if (cnt > 0) { k_probe_set<T><<<(unsigned)((cnt + kB - 1) / kB), kB, 0, st>>>(nodes, cnt, nf, f, w); note_launches(1); }
}
template <typename T>
void probe_get(const int32_t *nodes, int64_t cnt, int nf, int f, const T *y, T *B, cudaStream_t st) {
  if (cnt > 0) { k_probe_get<T><<<(unsigned)((cnt + kB - 1) / kB), kB, 0, st>>>(nodes, cnt, nf, f, y, B); note_launches(1); }
}
template void probe_set<float>(const int32_t *, int64_t, int, int, float *, cudaStream_t);
template void probe_set<double>(const int32_t *, int64_t, int, int, double *, cudaStream_t);
template void probe_get<float>(const int32_t *, int64_t, int, int, const float *, float *, cudaStream_t);
template void probe_get<double>(const int32_t *, int64_t, int, int, const double *, double *, cudaStream_t);

template <typename T>
void invert_blocks(T *B, int64_t n_nodes, int nf, int *bad, cudaStream_t st) {
  unsigned g = (unsigned)((n_nodes + kB - 1) / kB);
  if (nf == 5) { k_invert_blocks<T, 5><<<g, kB, 0, st>>>(B, n_nodes, bad); note_launches(1); }
  else { k_invert_blocks<T, 6><<<g, kB, 0, st>>>(B, n_nodes, bad); note_launches(1); }
}
template void invert_blocks<float>(float *, int64_t, int, int *, cudaStream_t);
template void invert_blocks<double>(double *, int64_t, int, int *, cudaStream_t);

template <typename T>
void block_apply(const T *Binv, const double *v, T *z, int64_t n_nodes, int nf, cudaStream_t st) {
  if (nf == 5) { k_block_apply<T, 5><<<grid_n(n_nodes), kB, 0, st>>>(Binv, v, z, n_nodes); note_launches(1); }
  else { k_block_apply<T, 6><<<grid_n(n_nodes), kB, 0, st>>>(Binv, v, z, n_nodes); note_launches(1); }
}
template void block_apply<float>(const float *, const double *, float *, int64_t, int, cudaStream_t);
template void block_apply<double>(const double *, const double *, double *, int64_t, int, cudaStream_t);

}  // namespace chns
