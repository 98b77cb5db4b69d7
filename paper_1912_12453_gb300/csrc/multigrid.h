// Geometric multigrid preconditioner over the octree levels (multigrid.cu).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "chns_internal.h"

namespace chns {

struct MgLevel {
  chns_mesh *mesh = nullptr;             // level 0: the mesh itself (not owned); l >= 1: owned
  // transfers between this level (l >= 1) and level l-1
  int32_t *pptr = nullptr, *pcol = nullptr;  // per node of level l-1: its level-l nodes ...
  float *pw = nullptr;                       // ... and weights (prolongation P_l)
  int32_t *rptr = nullptr, *rcol = nullptr;  // per node of level l: the level-(l-1) nodes ...
  float *rw = nullptr;                       // ... and weights (restriction P_l^T)
  int32_t *inj = nullptr;                    // per node of level l: the level-(l-1) node at its position
  int64_t nnz = 0;
  DevBuf ut[2], dl[2];                       // injected linearisation state (l >= 1), [float, double]
  DevBuf binv[2];                            // omega * inverse nodal diagonal blocks, [float, double]
  DevBuf x, b, y;                            // V-cycle vectors (sized for double)
};

struct Multigrid {
  std::vector<MgLevel> lv;
  int bottom_level = -1;                     // uniform octree level of the coarsest mesh
  bool ready[2] = {false, false};            // smoothers and bottom inverse built: [float, double]
  double omega = 0.7;
  int smooth = 1;
  uint64_t generation = 0;                   // bumped at every build (graph keys)
  bool autotune = false;                     // tune the J.w schedule of every level
  bool finish64 = false;                     // the FP64 finish needs double V-cycles on this mesh
};

// hierarchy of coarsened meshes and transfers down to a uniform level `bottom`
// (at most the coarsest leaf level); kept until the mesh is destroyed
chns_status mg_setup(chns_mesh *m, int bottom);
// inject the fine linearisation (ut0, dl0) down the levels
template <typename T>
chns_status mg_update_state(chns_mesh *m, const T *ut0, const T *dl0, cudaStream_t st);
// injected states, damped block-Jacobi smoothers, bottom dense inverse in
// precision T; keep_other: the other precision's operators stay valid
template <typename T>
chns_status mg_build(chns_mesh *m, const PhysCoef &pc, const T *ut0, const T *dl0, double omega, int smooth,
                     cudaStream_t st, bool keep_other = false);
// z = V-cycle(v): allocates nothing, so it can be captured into a graph
template <typename T>
chns_status mg_apply(chns_mesh *m, const PhysCoef &pc, const T *ut0, const T *dl0, const T *v, T *z,
                     cudaStream_t st);

}  // namespace chns
