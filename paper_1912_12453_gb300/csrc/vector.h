// Host-side launchers of the Krylov vector and preconditioner kernels (vector.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace chns {

constexpr int kMaxRestart = 64;

int red_blocks();
// h[i] = V_i . w for i < nv; partial: (nv + 8) * red_blocks() doubles
void vec_multidot(const double *V, int64_t ld, int nv, const double *w, int64_t n, double *partial,
                  double *h, cudaStream_t st);
void vec_dot(const double *x, const double *y, int64_t n, double *partial, double *res, cudaStream_t st);
void vec_update(const double *V, int64_t ld, int nv, const double *h, double *w, int64_t n, cudaStream_t st);
void vec_orthogonalize(double *V, int64_t ld, int nv, int64_t n, double *partial, double *h1, double *h2,
                       double *nrm, int *flag, cudaStream_t st);
void vec_normalize(double *w, int64_t n, const double *nrm, const int *flag, cudaStream_t st);
void vec_scale_by(const double *x, const double *nrm, double *out, int64_t n, cudaStream_t st);
template <typename A, typename B>
void vec_convert(const A *x, B *y, int64_t n, double a, cudaStream_t st);
template <typename T>
void vec_combine(const T *Z, int64_t ld, int nz, const double *c, double *x, int64_t n, cudaStream_t st);
void vec_axpby(double a, const double *x, double b, double *y, int64_t n, cudaStream_t st);
void vec_lincomb(double a, const double *x, double b, const double *y, double *z, int64_t n, cudaStream_t st);
void vec_mask_field(double *y, int64_t n_nodes, int nf, int k, double s, cudaStream_t st);
template <typename T>
void probe_set(const int32_t *nodes, int64_t cnt, int nf, int f, T *w, cudaStream_t st);
template <typename T>
void probe_get(const int32_t *nodes, int64_t cnt, int nf, int f, const T *y, T *B, cudaStream_t st);
template <typename T>
void invert_blocks(T *B, int64_t n_nodes, int nf, int *bad, cudaStream_t st);
template <typename T>
void block_apply(const T *Binv, const double *v, T *z, int64_t n_nodes, int nf, cudaStream_t st);

}  // namespace chns
