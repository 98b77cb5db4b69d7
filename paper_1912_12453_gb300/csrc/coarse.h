// Two-level (coarse-space) part of the Krylov preconditioner (coarse.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "chns_internal.h"

namespace chns {

#define TRY_CHNS(expr)              \
  do {                              \
    chns_status s_ = (expr);        \
    if (s_ != CHNS_OK) return s_;   \
  } while (0)

// y = J w for the current linearisation (supplied by the Newton driver)
template <typename T>
using JvFn = chns_status (*)(void *ctx, const T *w, T *y);

chns_status coarse_setup(chns_mesh *m, int level);
template <typename T>
chns_status coarse_build(chns_mesh *m, JvFn<T> jv, void *ctx, T *w, T *y, cudaStream_t st);
// z = B^{-1} v + P A_c^{-1} R v: B^{-1} the nodal inverse diagonal blocks
// (n_nodes x nf x nf; nullptr: no block term), the coarse term only when
// `coarse` and the coarse operator is built
template <typename T>
void precond_apply(chns_mesh *m, const T *Binv, bool coarse, const T *v, T *z, cudaStream_t st);

}  // namespace chns
