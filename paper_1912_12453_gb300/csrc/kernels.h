// Host-side launchers of the device kernels (element.cu, vector.cu).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "chns_internal.h"

namespace chns {

template <typename T>
void launch_prep(const chns_mesh *m, const double *Un, const double *Uo, T *ut, T *dl, cudaStream_t st);
void launch_residual(const chns_mesh *m, const PhysCoef &pc, const double *ut, const double *dl,
                     const double *f, double *F, cudaStream_t st);
// J.w with schedule `variant` (-1: the mesh's tuned schedule for float,
// schedule 0 for double); see element.cu for the schedules
constexpr int kJacvecVariants = 7;
template <typename T>
void launch_jacvec(const chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, const T *w, T *E, T *y,
                   cudaStream_t st, int variant = -1);
void launch_tau_floor_count(const chns_mesh *m, const PhysCoef &pc, const double *ut, const double *dl,
                            unsigned long long *count, cudaStream_t st);
void launch_dirichlet_res(const chns_mesh *m, const double *Un, const double *bc, double *F, cudaStream_t st);
int64_t energy_blocks(const chns_mesh *m);
// per-instance element coefficients of a batched (union) mesh
chns_status upload_coef_tables(chns_mesh *m, const std::vector<PhysCoef> &pcs, cudaStream_t st);
chns_status copy_coef_tables(const chns_mesh *src, chns_mesh *dst);
void launch_energy(const chns_mesh *m, const PhysCoef &pc, const double *U, double *partial, cudaStream_t st);

}  // namespace chns
