// Pieces of the Newton-Krylov solver shared by the C ABI (api.cu) and the
// multigrid preconditioner (multigrid.cu).
#pragma once

#include <cuda_runtime.h>

#include "chns_internal.h"

namespace chns {

chns_status check_launch();
// CN averages and increments of (U_new, U_old) in precision T, in the mesh's workspace
template <typename T>
chns_status prepare(chns_mesh *m, const double *Un, const double *Uo, cudaStream_t st, T **ut, T **dl);
// element-local J.w buffer of the mesh (allocated on first use)
template <typename T>
chns_status ensure_ebuf(chns_mesh *m, T **E);
// y = J w for the linearisation given by the prepared fields (ut, dl)
template <typename T>
chns_status jacvec_prepared(chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, const T *w, T *y,
                            cudaStream_t st);
// scale * (nodal diagonal blocks of J)^{-1}, by probing, into out
template <typename T>
chns_status build_block_jacobi(chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, DevBuf &out,
                               cudaStream_t st, double scale);

// pick the mesh's FP32 J.w schedule by timing all of them (once per mesh)
chns_status autotune_jacvec(chns_mesh *m, const PhysCoef &pc, const float *ut, const float *dl, cudaStream_t st);

}  // namespace chns
