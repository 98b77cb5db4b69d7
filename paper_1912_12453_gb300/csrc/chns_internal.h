// Internal declarations shared by the translation units of libchns.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/chns.h"

namespace chns {

void set_error(const char *fmt, ...);
void note_launches(int n);  // tracing counter of kernel launches
void set_capture_sink(int *sink);  // while set, this thread's launches count into *sink

#define CHNS_CUDA_TRY(expr)                                                      \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ::chns::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                     \
      return e_ == cudaErrorMemoryAllocation ? CHNS_ERR_OOM : CHNS_ERR_CUDA;     \
    }                                                                            \
  } while (0)

// Device buffer owned by the library.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  chns_status ensure(size_t n);
  void release();
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// Element-kernel coefficients that do not depend on the element.
struct PhysCoef {
  double dt, inv_dt, four_dt2;
  double alpha, beta, gamma, xi;   // rho = alpha phi* + beta, eta = gamma phi* + xi
  double jc;                       // flux J = jc grad mu, jc = (rho_r - 1)/2
  double inv_Pe, inv_We, inv_Re, inv_Fr, CnWe, inv_PeCn, Cn2, C_I;
  double g[3];
  double ext[3];                   // box extent per axis
  double lo[3];
  // fields solved for (bit k: field k of [v_1..v_d, p, phi, mu]); the rows of
  // the other fields are identity rows of J.w (block iteration, Sec. 3.1)
  uint32_t fmask;
};

PhysCoef make_coef(const chns_params &p, const double *lo, const double *hi);

struct Multigrid;
void mg_release(Multigrid *g);
// parameter checks shared by the entry points (dimension match, positivity)
chns_status check_params(const chns_mesh *m, const chns_params *p);

// Solver scratch, sized on first use.
struct Workspace {
  DevBuf ut, dl, ut32, dl32, f;        // prepared nodal fields (time averages / increments)
  DevBuf F, dU, r;                     // double n_dof
  DevBuf Ublk;                         // double n_dof: the previous block-iteration state
  DevBuf p32a, p32b;                   // float n_dof: float V-cycle input / output in the FP64 finish
  DevBuf V;                            // double (m+1) n_dof Krylov basis
  DevBuf Z;                            // (m) n_dof preconditioned directions (float or double)
  DevBuf wv, yv;                       // float/double n_dof work vectors
  DevBuf e32, e64;                     // element-local J.w contributions (n_elem * 2^dim * nf)
  DevBuf ctr;                          // grid-reduction tickets
  DevBuf count;                        // diagnostic counter (tau_m floors)
  DevBuf binv;                         // n_nodes * nf * nf inverse diagonal blocks (element precision)
  DevBuf binv64;                       // the same blocks in double (FP64 J.w iterations)
  DevBuf red;                          // reduction partials
  DevBuf hdev;                         // device copy of Gram-Schmidt coefficients
  double *hpinned = nullptr;           // pinned host mirror of reduction results
  // preconditioner kept across steps: valid for `pc_steps_left` more steps
  // with the same precision, parameters and coarse level
  int pc_steps_left = 0;
  int pc_precision = -1, pc_coarse = -1, pc_kind = -1, pc_smooth = -1;
  double pc_omega = -1.0;
  chns_params pc_params{};
  // CUDA graphs of the Arnoldi steps, one per step index and element
  // precision (0 float, 1 double), valid while `key` (the pointers and
  // parameters they were captured with) is unchanged
  struct StepGraphs {
    std::vector<cudaGraphExec_t> exec;
    std::vector<int> launches;         // kernel launches per replay
    std::vector<cudaEvent_t> jv;       // J.w start/end event of each step
    std::vector<unsigned char> key;
    void clear();
  } kg[2];
  cudaStream_t cap = nullptr;          // capture stream
  std::vector<cudaEvent_t> ev;         // general events (Krylov column slots 0, 1; residual timing)
  std::vector<cudaEvent_t> tev;        // J.w timing ring
  ~Workspace();
};

// Coarse space of the two-level preconditioner (coarse.cu): uniform octree
// level `level`, all fields, trilinear prolongation.
struct Coarse {
  int level = -1, nc1 = 0;
  int n_inst = 1;                   // one coarse grid per problem instance
  int64_t ncn_inst = 0, nc0 = 0;    // coarse nodes / unknowns of one instance
  int64_t ncn = 0, nc = 0;          // coarse nodes, coarse unknowns (all instances)
  float *pos = nullptr;             // n_nodes * dim: node positions in coarse units
  int64_t *rstart = nullptr;        // ncn + 1: restriction lists per coarse node (operator build)
  int32_t *rnode = nullptr;
  float *rw = nullptr;
  // restriction in the Krylov loop: mesh nodes grouped by coarse cell and cut
  // into pieces of at most kPiece nodes
  int64_t ncell_inst = 0, ncell = 0, n_pieces = 0;
  int32_t *cnodes = nullptr;        // n_nodes: node ids, cell by cell
  int32_t *piece_cell = nullptr;    // n_pieces
  int32_t *piece_begin = nullptr;   // n_pieces + 1: ranges in cnodes
  int32_t *cell_piece = nullptr;    // ncell + 1: pieces of each cell
  int32_t *sptr = nullptr;          // ncn + 1: restriction-sum entries of each coarse node
  int32_t *sent = nullptr;          // entries piece * 2^dim + corner
  DevBuf M;                         // per instance A_c -> A_c^{-1} (double), nc0 x nc0
  DevBuf Minv32;                    // per instance A_c^{-1} in float, nc0 x nc0
  DevBuf piv;                       // Gauss-Jordan row interchanges, nc0 per instance
  DevBuf vec;                       // coarse work vectors and operator-build partials
  DevBuf rpart;                     // restriction partials, n_pieces x 2^dim x nf doubles
  bool ready = false;
  ~Coarse();
  void release();
};

}  // namespace chns

struct chns_mesh {
  int dim = 0, max_level = 0, min_level = 0, nc = 0, nf = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int64_t n_elem = 0, n_nodes = 0, n_hang = 0;
  bool uniform = false;
  int n_colours = 0;
  std::vector<int64_t> colour_start;   // n_colours + 1, elements are stored colour by colour
  int n_node_colours = 0;
  std::vector<int64_t> node_colour_start;  // nodes of each node colour (for probing)
  int64_t origin = -1;                 // node at the box origin (pressure pin)
  // pinned pressure nodes (one per problem instance)
  int32_t *pins = nullptr;
  int64_t n_pins = 0;
  // batched (union) meshes: several independent problems in one mesh
  int n_inst = 1;
  uint16_t *elem_inst = nullptr;       // n_elem instance of each element (device)
  int32_t *node_inst = nullptr;        // n_nodes instance of each node (device)
  void *coef32 = nullptr, *coef64 = nullptr;  // per-instance element coefficients (device)
  std::vector<int64_t> inst_node_start;      // n_inst + 1 (host)
  std::vector<int> inst_max_level;           // n_inst (host)
  std::vector<const chns_mesh *> inst_meshes;  // union: the instance meshes (not owned)
  int64_t n_wall = 0;
  std::vector<int64_t> node_xyz;       // host: n_nodes * dim integer coordinates
  std::vector<uint8_t> leaf_level;     // host: the leaves as given (Morton order), plain meshes
  std::vector<uint32_t> leaf_anchor;   // host: n_elem * dim
  // device arrays
  int32_t *conn = nullptr;             // n_elem * nc: node index, or -(h+1) for hanging corner h
  uint8_t *level = nullptr;            // n_elem
  uint32_t *anchor = nullptr;          // n_elem * dim
  int32_t *hang = nullptr;             // n_hang * 4 parent nodes (-1 padded for edge midpoints)
  int32_t *wall = nullptr;             // n_wall node indices on the box boundary
  int32_t *node_perm = nullptr;        // n_nodes node indices grouped by node colour
  // node gather of element-local J.w contributions: the (element, corner)
  // slots feeding node i are gent[gptr[i] .. gptr[i+1]), each slot e*nc+c
  // with its hanging-node weight in the top two bits (0: 1, 1: 1/2, 2: 1/4),
  // in increasing slot order; nflag: bit 0 wall node, bit 1 pinned pressure
  int32_t *gptr = nullptr;             // n_nodes + 1
  int32_t *gent = nullptr;
  uint8_t *nflag = nullptr;            // n_nodes
  int device = 0;
  // FP32 J.w schedule picked by the autotuner (0 until tuned), its measured
  // times per schedule (ms; negative: not measured)
  int jv_variant = 0;
  bool jv_tuned = false;
  double jv_times[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  chns::Workspace ws;
  chns::Coarse coarse;
  chns::Multigrid *mg = nullptr;       // multigrid hierarchy (built on first use)
};

// Instances of one dimension fused into a union mesh.
struct BatchGroup {
  std::vector<int> members;            // batch indices, in union order
  chns_mesh *u = nullptr;              // union mesh (owned)
  chns::DevBuf Un, Unm1, Unp1;         // union state vectors
};

struct chns_batch {
  std::vector<chns_mesh *> meshes;
  std::vector<chns_params> params;
  std::vector<BatchGroup> groups;
};
