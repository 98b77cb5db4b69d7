// Krylov vector kernels (FGMRES with classical Gram-Schmidt, a second pass on
// a device flag), nodal block-Jacobi probing and inversion, deterministic
// reductions (element-precision partials, one double sum per result).
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

// FP64 instructions run on a narrow pipe on this part (tens of times slower
// than FP32, per warp instruction, whatever the active lanes), so the FP32
// Krylov kernels keep every per-element and per-block step in float: 16-byte
// loads, float products and sums within a thread, a warp and a block (fixed
// order), one float partial per block.  Only the final sum of the block
// partials is in double.  With the FP64 path (T = double) the same kernels
// run in double.

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

// 16 bytes of T: 4 floats or 2 doubles
template <typename T>
struct alignas(16) V16 {
  static constexpr int L = 16 / sizeof(T);
  T a[L];
};

// block sums of NV per-thread values (fixed order) -> out[k * gridDim.x + blockIdx.x]
template <typename T, int NV>
__device__ __forceinline__ void block_sum_store(T (&v)[NV], T *out) {
  __shared__ T sh[NV][kB / 32];
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const T s = warp_sum(v[k]);
    if (ln == 0) sh[k][wid] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    T s = T(0);
#pragma unroll
    for (int w = 0; w < kB / 32; ++w) s += sh[threadIdx.x][w];
    out[(int64_t)gridDim.x * threadIdx.x + blockIdx.x] = s;
  }
}

// Grid reductions without a second launch: every block stores its partials,
// then the last block to finish (ticket counter, reset for the next launch)
// sums each row over the blocks in block order -- in T within a lane and a
// warp, one conversion to double per row.
__device__ __forceinline__ bool last_block(unsigned *counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

template <typename T>
__device__ __forceinline__ void sum_rows(const T *partial, int nrows, double *res) {
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
  for (int k = wid; k < nrows; k += kB / 32) {
    T s = T(0);
    for (int b = ln; b < (int)gridDim.x; b += 32) s += __ldcg(partial + (int64_t)k * gridDim.x + b);
    s = warp_sum(s);
    if (ln == 0) res[k] = double(s);
  }
}

// res[k] = sum_b partial[k * nblocks + b] (double, fixed order), k < nv
template <typename P>
__global__ void k_sum_partials(const P *__restrict__ partial, int nblocks, int nv, double *__restrict__ res) {
  const int k = blockIdx.x;
  if (k >= nv) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += double(partial[(int64_t)k * nblocks + b]);
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

// partial sums of V_k . w for all k < nv, eight vectors at a time (w is
// re-read per group, from L2); V_i at V + i * ld with ld a multiple of 16
// bytes / sizeof(T) and V 16-byte aligned; skipped when flag is given and
// *flag == 0
template <typename T>
__global__ void __launch_bounds__(kB) k_multidot(const T *__restrict__ V, int64_t ld, int nv,
                                                 const T *__restrict__ w, int64_t n, T *__restrict__ partial,
                                                 const int *__restrict__ flag, unsigned *__restrict__ counter,
                                                 double *__restrict__ h) {
  if (flag && *flag == 0) return;
  constexpr int L = V16<T>::L, NV = 8;
  const int64_t nl = n / L;
  const V16<T> *wv = reinterpret_cast<const V16<T> *>(w);
  for (int i0 = 0; i0 < nv; i0 += NV) {
    const int c = nv - i0;
    T acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = T(0);
    for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < nl; t += int64_t(gridDim.x) * kB) {
      const V16<T> x = wv[t];
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < c) {
          const V16<T> a = reinterpret_cast<const V16<T> *>(V + (int64_t)(i0 + k) * ld)[t];
#pragma unroll
          for (int l = 0; l < L; ++l) acc[k] = fma(a.a[l], x.a[l], acc[k]);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < n - nl * L) {
      const int64_t t = nl * L + threadIdx.x;
      const T x = w[t];
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < c) acc[k] = fma(V[(int64_t)(i0 + k) * ld + t], x, acc[k]);
    }
    block_sum_store<T, NV>(acc, partial + (int64_t)i0 * gridDim.x);
    __syncthreads();  // the block-sum scratch is reused by the next group
  }
  if (last_block(counter)) {
    sum_rows<T>(partial, nv, h);
    if (threadIdx.x == 0) *counter = 0;
  }
}

// w -= sum_i h[i] V_i (i < nv) and block partial sums of the new |w|^2;
// skipped when flag is given and *flag == 0.  Layout as k_multidot.
// The last block writes |w|^2 to *nrm, the normalisation factor 1/|w| (0 if
// |w| = 0) to *scale and, given `before` (|w|^2 before the projection), the
// DGKS flag = (|w|^2 < 1e-4 before): the projection removed more than 99.99%
// of |w|^2, so a second Gram-Schmidt pass is needed.
template <typename T>
__global__ void __launch_bounds__(kB) k_update_norm(const T *__restrict__ V, int64_t ld, int nv,
                                                    const double *__restrict__ h, T *__restrict__ w, int64_t n,
                                                    const int *__restrict__ flag, T *__restrict__ partial,
                                                    unsigned *__restrict__ counter, double *__restrict__ nrm,
                                                    T *__restrict__ scale, const double *__restrict__ before,
                                                    int *__restrict__ flag_out) {
  if (flag && *flag == 0) return;
  constexpr int L = V16<T>::L;
  __shared__ T hs[kMaxRestart + 1];
  for (int i = threadIdx.x; i < nv; i += kB) hs[i] = T(-h[i]);
  __syncthreads();
  T acc[1] = {T(0)};
  const int64_t nl = n / L;
  V16<T> *wv = reinterpret_cast<V16<T> *>(w);
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < nl; t += int64_t(gridDim.x) * kB) {
    V16<T> s = wv[t];
#pragma unroll 4
    for (int i = 0; i < nv; ++i) {
      const V16<T> a = reinterpret_cast<const V16<T> *>(V + (int64_t)i * ld)[t];
#pragma unroll
      for (int l = 0; l < L; ++l) s.a[l] = fma(hs[i], a.a[l], s.a[l]);
    }
    wv[t] = s;
#pragma unroll
    for (int l = 0; l < L; ++l) acc[0] = fma(s.a[l], s.a[l], acc[0]);
  }
  if (blockIdx.x == 0 && threadIdx.x < n - nl * L) {
    const int64_t t = nl * L + threadIdx.x;
    T s = w[t];
    for (int i = 0; i < nv; ++i) s = fma(hs[i], V[(int64_t)i * ld + t], s);
    w[t] = s;
    acc[0] = fma(s, s, acc[0]);
  }
  block_sum_store<T, 1>(acc, partial);
  if (last_block(counter)) {
    __shared__ double tot;
    sum_rows<T>(partial, 1, &tot);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double t = tot;
      *nrm = t;
      *scale = t > 0.0 ? T(1.0 / sqrt(t)) : T(0);
      if (flag_out) *flag_out = (t < 1e-4 * before[0]) ? 1 : 0;
      *counter = 0;
    }
  }
}

// partial sums of x . y (double, any alignment)
__global__ void __launch_bounds__(kB) k_dot(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                            double *__restrict__ partial) {
  double acc[1] = {0.0};
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    acc[0] = fma(x[t], y[t], acc[0]);
  block_sum_store<double, 1>(acc, partial);
}

// w *= *scale (a zero scale: |w| = 0, w is left as is)
template <typename T>
__global__ void k_normalize(T *__restrict__ w, int64_t n, const T *__restrict__ scale) {
  const T s = *scale;
  if (s == T(0)) return;
  constexpr int L = V16<T>::L;
  const int64_t nl = n / L;
  V16<T> *wv = reinterpret_cast<V16<T> *>(w);
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < nl; t += int64_t(gridDim.x) * kB) {
    V16<T> x = wv[t];
#pragma unroll
    for (int l = 0; l < L; ++l) x.a[l] *= s;
    wv[t] = x;
  }
  if (blockIdx.x == 0 && threadIdx.x < n - nl * L) w[nl * L + threadIdx.x] *= s;
}

template <typename A, typename B>
__global__ void k_convert(const A *__restrict__ x, B *__restrict__ y, int64_t n, double a) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    y[t] = B(a * double(x[t]));
}

// x += sum_j c[j] Z_j: the combination in the precision T of Z (it is a
// Krylov correction, accurate to the Krylov tolerance), added to x in double
template <typename T>
__global__ void k_combine(const T *__restrict__ Z, int64_t ld, int nz, const double *__restrict__ c,
                          double *__restrict__ x, int64_t n) {
  __shared__ T cs[kMaxRestart];
  for (int i = threadIdx.x; i < nz; i += kB) cs[i] = T(c[i]);
  __syncthreads();
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) {
    T s = T(0);
    for (int j = 0; j < nz; ++j) s = fma(cs[j], Z[(int64_t)j * ld + t], s);
    x[t] += double(s);
  }
}

// r = b - y  (y in the element precision)
template <typename T>
__global__ void k_sub(const double *__restrict__ b, const T *__restrict__ y, double *__restrict__ r, int64_t n) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    r[t] = b[t] - double(y[t]);
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

// zero the fields of each node block whose bit in fmask is clear
__global__ void k_mask_fields(double *__restrict__ y, int64_t n_nodes, int nf, uint32_t fmask) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n_nodes * nf; t += int64_t(gridDim.x) * kB)
    if (!((fmask >> (t % nf)) & 1u)) y[t] = 0.0;
}

// max over i of |x_i - y_i| as a per-block maximum, then the maximum of the
// block maxima (order-independent: exact)
__global__ void k_maxabs_diff(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                              double *__restrict__ partial) {
  double m = 0.0;
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB)
    m = fmax(m, fabs(x[t] - y[t]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(FULL, m, o));
  __shared__ double sh[kB / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kB / 32; ++w) r = fmax(r, sh[w]);
    partial[blockIdx.x] = r;
  }
}

__global__ void k_max_partials(const double *__restrict__ partial, int nb, double *__restrict__ res) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmax(m, partial[b]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(FULL, m, o));
  __shared__ double sh[kB / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    *res = r;
  }
}

// field k of each node block = v, the others 0
__global__ void k_fill_field(double *__restrict__ y, int64_t n_nodes, int nf, int k, double v) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n_nodes * nf; t += int64_t(gridDim.x) * kB)
    y[t] = (t % nf == k) ? v : 0.0;
}

// z = r / d in field k of each node block (d > 0 there), 0 in the others
__global__ void k_div_field(const double *__restrict__ r, const double *__restrict__ d, double *__restrict__ z,
                            int64_t n_nodes, int nf, int k) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n_nodes * nf; t += int64_t(gridDim.x) * kB)
    z[t] = (t % nf == k && d[t] > 0.0) ? r[t] / d[t] : 0.0;
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

// in-place scale * inverse of each nf x nf nodal block (Gauss-Jordan, partial
// pivoting, double)
template <typename T, int NF>
__global__ void k_invert_blocks(T *__restrict__ B, int64_t n_nodes, int *__restrict__ bad, double scale) {
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
    for (int c = 0; c < NF; ++c) B[(a * NF + r) * NF + c] = T(scale * M[r][NF + c]);
}

}  // namespace

// ---------------------------------------------------------------- launchers
int red_blocks() { return kRedBlocks; }

template <typename T>
void vec_multidot(const T *V, int64_t ld, int nv, const T *w, int64_t n, double *partial, double *h,
                  cudaStream_t st, const int *flag, unsigned *counter) {
  T *pt = reinterpret_cast<T *>(partial);
  k_multidot<T><<<kRedBlocks, kB, 0, st>>>(V, ld, nv, w, n, pt, flag, counter, h);
  note_launches(1);
}
template void vec_multidot<float>(const float *, int64_t, int, const float *, int64_t, double *, double *,
                                  cudaStream_t, const int *, unsigned *);
template void vec_multidot<double>(const double *, int64_t, int, const double *, int64_t, double *, double *,
                                   cudaStream_t, const int *, unsigned *);

void vec_dot(const double *x, const double *y, int64_t n, double *partial, double *res, cudaStream_t st) {
  k_dot<<<kRedBlocks, kB, 0, st>>>(x, y, n, partial);
  k_sum_partials<double><<<1, kB, 0, st>>>(partial, kRedBlocks, 1, res);
  note_launches(2);
}

// One Arnoldi orthogonalisation of w = V_{nv} against V_0..V_{nv-1} (classical
// Gram-Schmidt, a second pass only on severe cancellation).  Device outputs
// (no host sync): h1[0..nv-1] first-pass coefficients, h1[nv] = |w|^2
// before; h2[0..nv-1] second-pass coefficients (0 if skipped); nrm[0] =
// |w|^2 after pass 1, nrm[1] = after pass 2, flag[0] = whether pass 2 ran,
// *scale = 1/|w| for vec_normalize.
template <typename T>
void vec_orthogonalize(T *V, int64_t ld, int nv, int64_t n, double *partial, double *h1, double *h2,
                       double *nrm, int *flag, T *scale, unsigned *counter, cudaStream_t st) {
  T *pt = reinterpret_cast<T *>(partial);
  T *w = V + (int64_t)nv * ld;
  // pass 1 dots include w itself (stored right after V_{nv-1}): |w|^2 = h1[nv]
  vec_multidot<T>(V, ld, nv + 1, w, n, partial, h1, st, nullptr, counter);
  k_update_norm<T><<<kRedBlocks, kB, 0, st>>>(V, ld, nv, h1, w, n, nullptr, pt, counter, nrm, scale, h1 + nv,
                                              flag);
  // pass 2, on the device flag
  vec_multidot<T>(V, ld, nv, w, n, partial, h2, st, flag, counter);
  k_update_norm<T><<<kRedBlocks, kB, 0, st>>>(V, ld, nv, h2, w, n, flag, pt, counter, nrm + 1, scale, nullptr,
                                              nullptr);
  note_launches(2);
}
template void vec_orthogonalize<float>(float *, int64_t, int, int64_t, double *, double *, double *, double *,
                                       int *, float *, unsigned *, cudaStream_t);
template void vec_orthogonalize<double>(double *, int64_t, int, int64_t, double *, double *, double *, double *,
                                        int *, double *, unsigned *, cudaStream_t);

template <typename T>
void vec_normalize(T *w, int64_t n, const T *scale, cudaStream_t st) {
  k_normalize<T><<<grid_n(n / V16<T>::L + 1), kB, 0, st>>>(w, n, scale);
  note_launches(1);
}
template void vec_normalize<float>(float *, int64_t, const float *, cudaStream_t);
template void vec_normalize<double>(double *, int64_t, const double *, cudaStream_t);

template <typename T>
void vec_sub(const double *b, const T *y, double *r, int64_t n, cudaStream_t st) {
  k_sub<T><<<grid_n(n), kB, 0, st>>>(b, y, r, n);
  note_launches(1);
}
template void vec_sub<float>(const double *, const float *, double *, int64_t, cudaStream_t);
template void vec_sub<double>(const double *, const double *, double *, int64_t, cudaStream_t);

template <typename A, typename B>
void vec_convert(const A *x, B *y, int64_t n, double a, cudaStream_t st) {
  k_convert<A, B><<<grid_n(n), kB, 0, st>>>(x, y, n, a);
  note_launches(1);
}
template void vec_convert<float, double>(const float *, double *, int64_t, double, cudaStream_t);
template void vec_convert<double, float>(const double *, float *, int64_t, double, cudaStream_t);
template void vec_convert<double, double>(const double *, double *, int64_t, double, cudaStream_t);
template void vec_convert<float, float>(const float *, float *, int64_t, double, cudaStream_t);

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

void vec_mask_fields(double *y, int64_t n_nodes, int nf, uint32_t fmask, cudaStream_t st) {
  k_mask_fields<<<grid_n(n_nodes * nf), kB, 0, st>>>(y, n_nodes, nf, fmask);
  note_launches(1);
}

void vec_maxabs_diff(const double *x, const double *y, int64_t n, double *partial, double *res, cudaStream_t st) {
  k_maxabs_diff<<<kRedBlocks, kB, 0, st>>>(x, y, n, partial);
  k_max_partials<<<1, kB, 0, st>>>(partial, kRedBlocks, res);
  note_launches(2);
}

void vec_fill_field(double *y, int64_t n_nodes, int nf, int k, double v, cudaStream_t st) {
  k_fill_field<<<grid_n(n_nodes * nf), kB, 0, st>>>(y, n_nodes, nf, k, v);
  note_launches(1);
}

void vec_div_field(const double *r, const double *d, double *z, int64_t n_nodes, int nf, int k, cudaStream_t st) {
  k_div_field<<<grid_n(n_nodes * nf), kB, 0, st>>>(r, d, z, n_nodes, nf, k);
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
void invert_blocks(T *B, int64_t n_nodes, int nf, int *bad, double scale, cudaStream_t st) {
  unsigned g = (unsigned)((n_nodes + kB - 1) / kB);
  if (nf == 5) { k_invert_blocks<T, 5><<<g, kB, 0, st>>>(B, n_nodes, bad, scale); note_launches(1); }
  else { k_invert_blocks<T, 6><<<g, kB, 0, st>>>(B, n_nodes, bad, scale); note_launches(1); }
}
template void invert_blocks<float>(float *, int64_t, int, int *, double, cudaStream_t);
template void invert_blocks<double>(double *, int64_t, int, int *, double, cudaStream_t);

}  // namespace chns
