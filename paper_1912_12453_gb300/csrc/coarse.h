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
// z += P A_c^{-1} R v
template <typename T>
void coarse_apply_add(chns_mesh *m, const double *v, T *z, cudaStream_t st);

}  // namespace chns
