// Host-side launchers of the Krylov vector and preconditioner kernels (vector.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace chns {

constexpr int kMaxRestart = 64;

int red_blocks();
// Krylov vectors: V_i at V + i * ld, ld a multiple of kVecAlign elements and
// V 16-byte aligned (16-byte loads); products and sums in T, the final sum
// of block partials in double (vector.cu)
constexpr int64_t kVecAlign = 64;
inline int64_t vec_ld(int64_t n) { return (n + kVecAlign - 1) / kVecAlign * kVecAlign; }

// h[i] = V_i . w for i < nv; partial: (nv + 8) * red_blocks() doubles;
// counter: a device word that is zero between launches (grid reduction
// ticket); skipped (h unchanged) when flag is given and *flag == 0
template <typename T>
void vec_multidot(const T *V, int64_t ld, int nv, const T *w, int64_t n, double *partial, double *h,
                  cudaStream_t st, const int *flag, unsigned *counter);
// x . y (double)
void vec_dot(const double *x, const double *y, int64_t n, double *partial, double *res, cudaStream_t st);
template <typename T>
void vec_orthogonalize(T *V, int64_t ld, int nv, int64_t n, double *partial, double *h1, double *h2,
                       double *nrm, int *flag, T *scale, unsigned *counter, cudaStream_t st);
template <typename T>
void vec_normalize(T *w, int64_t n, const T *scale, cudaStream_t st);
// r = b - y
template <typename T>
void vec_sub(const double *b, const T *y, double *r, int64_t n, cudaStream_t st);
template <typename A, typename B>
void vec_convert(const A *x, B *y, int64_t n, double a, cudaStream_t st);
template <typename T>
void vec_combine(const T *Z, int64_t ld, int nz, const double *c, double *x, int64_t n, cudaStream_t st);
void vec_axpby(double a, const double *x, double b, double *y, int64_t n, cudaStream_t st);
void vec_lincomb(double a, const double *x, double b, const double *y, double *z, int64_t n, cudaStream_t st);
void vec_mask_field(double *y, int64_t n_nodes, int nf, int k, double s, cudaStream_t st);
// field k = v, the other fields 0
void vec_fill_field(double *y, int64_t n_nodes, int nf, int k, double v, cudaStream_t st);
// z = r / d in field k (where d > 0), 0 elsewhere
void vec_div_field(const double *r, const double *d, double *z, int64_t n_nodes, int nf, int k, cudaStream_t st);
// zero the fields whose bit in fmask is clear
void vec_mask_fields(double *y, int64_t n_nodes, int nf, uint32_t fmask, cudaStream_t st);
// *res = max_i |x_i - y_i| (partial: red_blocks() doubles)
void vec_maxabs_diff(const double *x, const double *y, int64_t n, double *partial, double *res, cudaStream_t st);
template <typename T>
void probe_set(const int32_t *nodes, int64_t cnt, int nf, int f, T *w, cudaStream_t st);
template <typename T>
void probe_get(const int32_t *nodes, int64_t cnt, int nf, int f, const T *y, T *B, cudaStream_t st);
// B <- scale * B^{-1} for each nf x nf nodal block
template <typename T>
void invert_blocks(T *B, int64_t n_nodes, int nf, int *bad, double scale, cudaStream_t st);

}  // namespace chns
