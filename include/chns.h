/*
 * chns.h -- C ABI of the GB300 (sm_103a) matrix-free CHNS operator library.
 *
 * The library applies the fully discrete Crank-Nicolson, residual-based VMS
 * weak form of the Cahn-Hilliard-Navier-Stokes system (Sec. 3.1 time scheme,
 * Definition of the fully discrete VMS problem in Sec. 3.4) on trilinear
 * (bilinear in 2D) continuous Galerkin elements over the leaves of a 2:1
 * balanced octree (quadtree), with hanging nodes interpolated before and
 * eliminated after each element operation (Sec. 4, "Handling hanging nodes"),
 * and advances one time step by Newton's method (Sec. 3.5).
 *
 * Unknowns.  Every independent (non-hanging) mesh node carries dim+3 values,
 * interleaved per node in the order [v_1 .. v_dim, p, phi, mu]; a state
 * vector has n_dof = n_nodes * (dim+3) entries.  The library numbers nodes
 * itself; chns_mesh_node_coords returns their integer coordinates so callers
 * can map their data.
 *
 * Memory.  Meshes and batches are opaque, library-owned objects holding device
 * arrays and the solver's scratch.  Every state vector passed to the calls
 * below is a DEVICE pointer owned by the caller (n_dof entries, 16-byte
 * aligned), unless the comment says "host".  Calls are asynchronous on the
 * given CUDA stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream) except where they return host values; those synchronise the stream.
 *
 * Errors.  Every call returns a chns_status; on failure chns_last_error()
 * gives a message (thread-local, valid until the next call on that thread).
 * No call traps or aborts the process; kernels never spin without a bound.
 *
 * Boundary conditions (Sec. 3.1): no-slip walls on every face of the box
 * (velocity rows of wall nodes are replaced by v - g), zero normal flux of
 * phi and mu (natural), and the pressure pinned at the node at the box
 * origin (its continuity row is replaced by p - g).
 */
#ifndef CHNS_H
#define CHNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chns_mesh chns_mesh;
typedef struct chns_batch chns_batch;

typedef enum {
  CHNS_OK = 0,
  CHNS_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad option) */
  CHNS_ERR_MESH = 2,       /* leaves unsorted, overlapping, or not 2:1 balanced */
  CHNS_ERR_CUDA = 3,       /* a CUDA runtime call failed */
  CHNS_ERR_NONFINITE = 4,  /* NaN or Inf in a residual or Krylov norm */
  CHNS_ERR_NEWTON = 5,     /* Newton did not reach its tolerance in newton_max_it */
  CHNS_ERR_KRYLOV = 6,     /* FGMRES breakdown, or a singular nodal / coarse block in the
                              preconditioner */
  /* 7 is not used: no kernel of this library waits on a device-side flag */
  CHNS_ERR_OOM = 8         /* device allocation failed */
} chns_status;

typedef enum {
  CHNS_FP64 = 0,           /* everything in double precision */
  CHNS_FP32_BULK = 1       /* element and Krylov-vector kernels in float, Newton in double */
} chns_precision;

/* Nondimensional parameters (Sec. 2).  rho_ratio = rho_-/rho_+ and
 * eta_ratio = eta_-/eta_+ (fluid "+" at phi = +1 is the reference, rho = eta = 1).
 * gravity is the unit vector g^ (the paper's default is (0,-1,0)); C_I is the
 * constant of tau_m (6 in the paper). */
typedef struct {
  int dim;
  double dt, Cn, Re, We, Pe, Fr, rho_ratio, eta_ratio, C_I;
  double gravity[3];
} chns_params;

typedef enum {
  CHNS_PC_TWO_LEVEL = 0,   /* nodal block-Jacobi + additive Galerkin coarse space (coarse_level) */
  CHNS_PC_MULTIGRID = 1    /* geometric multigrid V-cycle over the octree levels (mg_* fields) */
} chns_preconditioner;

typedef struct {
  double newton_rtol;      /* stop when ||F||_2 <= newton_rtol ||F(initial guess)||_2 ... */
  double newton_atol;      /* ... or ||F||_2 <= newton_atol */
  int newton_max_it;
  double krylov_rtol;      /* FGMRES relative tolerance of each Newton correction */
  int krylov_restart;      /* FGMRES restart length m (1..64) */
  int krylov_max_it;       /* total FGMRES iterations per Newton correction */
  chns_precision precision;
  int reuse_preconditioner;/* k >= 1: the preconditioner built at the first Newton iteration of a
                              step serves that step and the next k-1 steps of the same mesh
                              (same precision, parameters, coarse level); 0: rebuilt at every
                              Newton iteration */
  int coarse_level;        /* two-level preconditioner: coarse octree level L_c >= 1 (at most one
                              below the coarsest leaf); 0 = block-Jacobi only; -1 = automatic
                              (L_c = min(3, coarsest leaf level - 1), off if that is < 1) */
  int use_graph;           /* 1: each Arnoldi step is captured once as a CUDA graph and replayed;
                              0: launched kernel by kernel (same arithmetic, same results) */
  chns_preconditioner preconditioner;
  int mg_coarsest;         /* multigrid: uniform octree level of the coarsest mesh, solved exactly
                              by a dense inverse (clamped to the coarsest leaf level); -1 = 2 in 3D,
                              3 in 2D */
  int mg_smooth;           /* multigrid: damped block-Jacobi sweeps before and after each coarse
                              correction (1..8) */
  double mg_omega;         /* multigrid: damping of the block-Jacobi sweeps (0 < omega <= 1; 0.4
                              measured best on the droplet and bubble workloads, 0.6 and above
                              let the smoother amplify some modes) */
  int block_iteration;     /* 0: coupled Newton on all fields; 1: the block iteration of Sec. 3.1
                              (Fig. flowchart_block): Newton on the Navier-Stokes fields (v, p) with
                              phi, mu frozen, then on the Cahn-Hilliard fields (phi, mu) with v, p
                              frozen, repeated until a block iteration after the first changes no
                              entry of (v, p, phi, mu) by more than block_tol */
  double block_tol;        /* block iteration: tolerance on the max-norm change (the paper: 1e-4) */
  int block_max_it;        /* block iteration: at most this many block iterations (else
                              CHNS_ERR_NEWTON) */
  int autotune;            /* 1: at its first FP32-bulk step a mesh (and each multigrid level)
                              times every FP32 J.w schedule of the library (element-local buffer +
                              node gather at several block shapes and register budgets, or element
                              colours with in-place adds) and keeps the fastest; 0: the default
                              schedule.  Results are identical up to the summation order of a
                              node's contributions. */
} chns_solver_opts;

typedef struct {
  int newton_its;
  int krylov_its_total;
  double res0, res_final;          /* ||F|| at the initial guess and at exit */
  double energy_old, energy_new;   /* energy functional of U_n and U_{n+1} */
  double mass_old, mass_new;       /* integral of phi */
  double seconds;                  /* host wall time of the call */
  double jacvec_ms;                /* device time of the Krylov J.w applies (CUDA events) */
  int jacvec_calls;
  double residual_ms;              /* device time of the FP64 residual applies */
  int residual_calls;
  double precond_ms;               /* host time of building the preconditioner (block-Jacobi and
                                      coarse space); 0 when a previous build was reused */
  int fp64_newton_its;             /* CHNS_FP32_BULK: Newton iterations finished with FP64 J.w */
  int block_its;                   /* block iterations (0 with the coupled Newton); newton_its then
                                      counts the Newton iterations of all sub-solves, and res_final is
                                      the coupled residual of the result */
  int jacvec_variant;              /* the mesh's FP32 J.w schedule (0 until autotuned) */
} chns_step_stats;

/* ---------------------------------------------------------------- meshes */

/* Build a mesh from the leaves of a linear octree (dim = 3) or quadtree
 * (dim = 2) given in Morton order (Sec. 4 "Meshing").  Host arrays:
 * level[n_leaves] (0..max_level) and anchor[n_leaves*dim] (integer lower
 * corner of each leaf at max_level resolution, x fastest).  The domain is the
 * box [lo, hi].  The leaves must tile the box, be sorted by Morton key, and
 * be 2:1 balanced across faces, edges and corners (Sec. 4 "2:1 Balancing");
 * otherwise CHNS_ERR_MESH.  Colours the elements so that elements of one
 * colour touch disjoint node sets (hanging constraints included), which
 * makes the residual's scatter-add free of atomics and deterministic, and
 * builds the node gather lists that sum the element-local J.w contributions
 * of each node in a fixed order. */
chns_status chns_mesh_create(int dim, int64_t n_leaves, const uint8_t *level,
                             const uint32_t *anchor, int max_level, const double lo[3],
                             const double hi[3], chns_mesh **out);

/* Host outputs; any pointer may be NULL. */
chns_status chns_mesh_info(const chns_mesh *mesh, int64_t *n_nodes, int64_t *n_dof,
                           int *n_colours, int64_t *n_hanging);

/* Integer coordinates (max_level resolution) of the independent nodes in the
 * library's numbering.  Host output xyz[n_nodes*dim]. */
chns_status chns_mesh_node_coords(const chns_mesh *mesh, int64_t *xyz);

/* Host-side validation of a built mesh (reads its device arrays back):
 * elements of one colour touch disjoint sets of independent nodes, hanging
 * parents expanded (so the residual's colour-by-colour scatter-add needs no
 * atomics); every independent node's gather list holds exactly the (element,
 * corner) slots that reach it, with weight 1 directly or 1/2 (edge) / 1/4
 * (face) through a hanging corner, in increasing slot order; every hanging
 * node has 2 or 4 independent parents.  CHNS_OK or CHNS_ERR_MESH with the
 * first violation in chns_last_error(). */
chns_status chns_mesh_check(const chns_mesh *mesh);

/* The FP32 J.w schedule of a mesh (the autotuner's choice, see
 * chns_solver_opts.autotune): variant in [0, 7) fixes it (and marks the mesh
 * tuned); times_ms (host, nullable, 7 entries) receives the autotuner's
 * median time per schedule, negative where none was measured.  Schedules:
 * 0-3, 5, 6 element-local buffer + node gather with (block size, blocks per
 * SM) = (128, 6), (256, 3), (64, 12), (128, 8), -, (128, 5), (128, 4); 4
 * element colours with in-place adds.  variant = -1 only reads. */
chns_status chns_mesh_jacvec_schedule(chns_mesh *mesh, int variant, int *current, double *times_ms);

void chns_mesh_destroy(chns_mesh *mesh);

/* ---------------------------------------------------------------- operators */

/* Nonlinear residual F(U_new; U_old) of the fully discrete CN-VMS problem
 * (Sec. 3.4 Definition with the time derivative replaced by the CN scheme of
 * Sec. 3.1), in double precision.  forcing (nullable): nodal source at
 * t_{k+1/2}, subtracted from every row and inside the strong residuals.
 * bc (nullable, 0 if NULL): prescribed values of the constrained rows (wall
 * velocities at t_{k+1}, pinned pressure); other entries are ignored.
 * F is overwritten. */
chns_status chns_residual(const chns_mesh *mesh, const chns_params *params,
                          const double *U_new, const double *U_old, const double *forcing,
                          const double *bc, double *F, void *stream);

/* Jacobian-vector product y = (dF/dU_new)(U_new; U_old) w (Sec. 3.5: the
 * analytic Jacobian), exact directional derivative including tau_m, tau_c,
 * the phi* clip and rho(phi^{k+1}).  prec = CHNS_FP64: w, y are double*.
 * prec = CHNS_FP32_BULK: w, y are float* and the element arithmetic is
 * float (the states are rounded to float after forming their CN averages
 * and increments in double).  Constrained rows give y = w. */
chns_status chns_jacvec(const chns_mesh *mesh, const chns_params *params,
                        const double *U_new, const double *U_old, const void *w, void *y,
                        chns_precision prec, void *stream);

/* Replace the chemical potential of U (in place) by the L2 projection of
 * psi'(phi) - Cn^2 lap(phi), i.e. solve M mu = (N, psi'(phi)) + Cn^2 (grad N,
 * grad phi) (the chemical-potential row with U_new = U_old). */
chns_status chns_init_mu(const chns_mesh *mesh, const chns_params *params, double *U,
                         void *stream);

/* One Crank-Nicolson step (Sec. 3.1, 3.5): Newton on F(U; U_n) = 0 from the
 * guess U_n (or 2 U_n - U_nm1 when U_nm1 is not NULL), each correction by
 * right-preconditioned FGMRES(m).  Preconditioners: CHNS_PC_TWO_LEVEL, nodal
 * block-Jacobi plus, optionally, an additive coarse-space correction
 * P (R J P)^{-1} R on a uniform coarse octree level (R = P^T, P trilinear);
 * CHNS_PC_MULTIGRID, a V-cycle over the meshes obtained by repeatedly merging
 * the finest leaves (each level applies the same J.w on its own leaves,
 * linearised at the injected state; damped nodal block-Jacobi smoothing;
 * transfers by Q1 interpolation with hanging constraints and its transpose;
 * the coarsest uniform level solved by a dense inverse; the hierarchy is
 * built at the first multigrid step of a mesh and kept).  The residual and
 * the Newton update are double; with CHNS_FP32_BULK the Krylov basis, J.w,
 * Gram-Schmidt and preconditioner run in float (dot products summed per
 * block in float, across blocks in double), refined by the outer double
 * residual; once a float-Krylov Newton iteration cuts ||F|| by less than
 * 10x, the remaining iterations apply J in double with the float
 * preconditioner promoted.  With opts->use_graph each Arnoldi step is
 * replayed as a CUDA graph captured at its first use.  U_np1 receives the
 * result (may not alias U_n).  stats (host, nullable).  Errors:
 * CHNS_ERR_NONFINITE when a residual or Krylov norm is NaN/Inf (e.g. NaN in
 * U_n), CHNS_ERR_NEWTON after newton_max_it iterations without reaching the
 * tolerance, CHNS_ERR_KRYLOV on an FGMRES breakdown or a singular
 * preconditioner block.  Setting the environment variable CHNS_TRACE=1
 * prints each Newton iteration to stderr; CHNS_INJECT=krylov makes the next
 * FGMRES report a breakdown (a host-side fault injection for tests of the
 * caller's error handling).  A mesh is used by one host thread at a time. */
chns_status chns_step(const chns_mesh *mesh, const chns_params *params,
                      const chns_solver_opts *opts, const double *U_n, const double *U_nm1,
                      const double *forcing, const double *bc, double *U_np1,
                      chns_step_stats *stats, void *stream);

/* Number of Gauss points, over all leaves, at which the tau_m radicand of
 * Sec. 3.4 (4/dt^2 + v~.G v~ + v~.G J~/(rho Pe) + C_I (eta/(rho Re))^2 G:G)
 * falls below 4/dt^2 and is raised to it (v~.J~ < 0 can make it small or
 * negative; the paper does not discuss the case).  Evaluated in double
 * precision at U_new, U_old exactly as chns_residual evaluates tau_m.  count:
 * host output; synchronises the stream. */
chns_status chns_tau_floor_count(const chns_mesh *mesh, const chns_params *params,
                                 const double *U_new, const double *U_old, int64_t *count,
                                 void *stream);

/* Diagnostics with the same 2^dim Gauss rule (host outputs, synchronises):
 * energy functional (Eq. energy_functional, gravity potential (1/Fr) rho(phi*)
 * (-g.x)), integral of phi (Prop. mass_conservation) and the volume where
 * phi < 0 (the bubble mass of Sec. 5.2).  Any output pointer may be NULL. */
chns_status chns_energy_mass(const chns_mesh *mesh, const chns_params *params,
                             const double *U, double *energy, double *mass,
                             double *bubble_mass, void *stream);

/* Allocation-free variant of chns_energy_mass, for callers that may not
 * allocate device memory while they run: work issued during a CUDA graph
 * stream capture (cudaMalloc is refused there) and host frameworks that give
 * all device memory to their own pool up front.  The paper has no
 * counterpart; it computes the same three integrals as chns_energy_mass, in
 * the same order.  out3: caller-owned DEVICE array of 3 doubles receiving
 * (energy, integral of phi, volume with phi < 0); asynchronous on stream.
 * The reduction scratch is a fixed 1.5 MiB array inside the library, held
 * by every GPU that loads it until the process exits; meshes of more than
 * 2,097,152 leaves in 3D (4,194,304 in 2D) are rejected with CHNS_ERR_ARG.
 * The first call on each device looks up that array's device address; make
 * it before any stream capture.  Calls that overlap on the GPU share the
 * scratch and race; order them on one stream.  Never calls cudaMalloc or
 * cudaFree. */
chns_status chns_energy_mass_noalloc(const chns_mesh *mesh, const chns_params *params,
                                     const double *U, double *out3, void *stream);

/* ---------------------------------------------------------------- batches */

/* Many independent problems (meshes of any size, own parameters) advanced
 * together.  The instances of each dimension are fused into one union mesh:
 * the element kernels run over the concatenated leaves of all of them in one
 * launch per colour, each element reading its own instance's coefficients;
 * the Newton-Krylov solve runs on the union with one coarse grid per instance
 * (block-diagonal coarse operator) and a per-instance Newton tolerance.
 * meshes and params: host arrays of n entries; the meshes must outlive the
 * batch. */
chns_status chns_batch_create(int n, chns_mesh *const *meshes, const chns_params *params,
                              chns_batch **out);

/* One CN step of every instance; U_n[i], U_nm1[i] (U_nm1 nullable),
 * U_np1[i] are device vectors of instance i.  Every instance stops when its
 * own ||F_i|| <= newton_rtol ||F_i(guess)|| (or atol).  stats: host array of
 * n entries or NULL; Newton/Krylov counts and times are those of the
 * instance's dimension group, energies and masses the instance's own. */
chns_status chns_batch_step(chns_batch *batch, const chns_solver_opts *opts,
                            double *const *U_n, double *const *U_nm1, double *const *U_np1,
                            chns_step_stats *stats, void *stream);

void chns_batch_destroy(chns_batch *batch);

/* ---------------------------------------------------------- remeshing (host)
 *
 * Sec. 4: every few time steps the octree is re-refined around the current
 * interface, 2:1 balanced, meshed again, and the fields are carried from the
 * old mesh to the new one by interpolation ("Refinement", "2:1 Balancing",
 * "Intergrid transfers").  These calls work on HOST arrays only and need no
 * GPU.  Leaf lists follow chns_mesh_create: level[n] and anchor[n*dim] (x
 * fastest, max_level resolution), in Morton order, tiling the box; a leaf
 * list passed in must satisfy that (otherwise CHNS_ERR_MESH), but need not be
 * balanced.  Nodal fields are host arrays U[n_nodes*nf] over the independent
 * nodes of the leaf list's mesh, whose integer coordinates are
 * xyz[n_nodes*dim] (chns_mesh_node_coords); hanging nodes take the mean of
 * the corners of the coarser edge or face they lie on.  Leaf lists that a
 * call returns are allocated by the library: release each array with
 * chns_leaves_free. */

/* The leaves a mesh was built from (host outputs level[n_leaves],
 * anchor[n_leaves*dim], Morton order).  CHNS_ERR_ARG for a batch's union
 * mesh. */
chns_status chns_mesh_leaves(const chns_mesh *mesh, uint8_t *level, uint32_t *anchor);

/* One adaptation pass: mark[e] = +1 splits leaf e into its 2^dim children
 * (ignored at max_level), -1 merges a family into its parent when all 2^dim
 * children are leaves marked -1 (ignored at level 0), 0 keeps it (mark NULL:
 * all 0).  Then the tree is 2:1 balanced across faces, edges and corners by
 * splitting leaves only (a merge that would break the balance is undone): the
 * result is the coarsest balanced refinement of the marked tree.  Outputs
 * *n_out, *level_out, *anchor_out (library-allocated, Morton order). */
chns_status chns_leaves_adapt(int dim, int max_level, int64_t n, const uint8_t *level,
                              const uint32_t *anchor, const int8_t *mark, int64_t *n_out,
                              uint8_t **level_out, uint32_t **anchor_out);

/* Intergrid transfer: the values at n_points integer points
 * (points[n_points*dim], each in [0, 2^max_level]^dim) of the nodal Q1 field
 * U on the leaf list (level, anchor): multilinear interpolation in the leaf
 * whose cell holds the point, hanging corners interpolated.  Evaluated at
 * the nodes of a refined or coarsened mesh this is the parent-to-child
 * interpolation (refinement) and injection (coarsening) of the paper's
 * transfer.  Host output out[n_points*nf].  A point outside the box is
 * CHNS_ERR_ARG; a leaf corner that is neither a node in xyz nor a hanging
 * node is CHNS_ERR_MESH. */
chns_status chns_leaves_transfer(int dim, int max_level, int64_t n_leaves, const uint8_t *level,
                                 const uint32_t *anchor, int64_t n_nodes, const int64_t *xyz,
                                 int nf, const double *U, int64_t n_points, const int64_t *points,
                                 double *out);

/* Interface marks of the leaf list (level, anchor) against component
 * phi_index of the field U on the source leaf list (src_level, src_anchor):
 * a leaf meets the interface when the field's phi, interpolated at one of its
 * corners, has |phi| <= band, or its corners carry both signs of phi (the
 * corner test of Sec. 4 "Refinement" applied to the diffuse interface).  Its
 * target level is level_max if it meets the interface, level_min otherwise;
 * mark[e] = +1 below the target, -1 above it, 0 at it (host output mark[n]).
 * A non-finite phi is CHNS_ERR_NONFINITE. */
chns_status chns_leaves_mark_interface(int dim, int max_level, int64_t n_src,
                                       const uint8_t *src_level, const uint32_t *src_anchor,
                                       int64_t n_nodes, const int64_t *xyz, int nf, const double *U,
                                       int phi_index, double band, int level_min, int level_max,
                                       int64_t n, const uint8_t *level, const uint32_t *anchor,
                                       int8_t *mark);

/* Remesh around the interface of U's phi component: starting from the
 * source leaf list, alternate chns_leaves_mark_interface (always against the
 * source field) and chns_leaves_adapt until no leaf is marked or a pass
 * changes nothing (at most 2 max_level + 2 passes; *passes, nullable, gets
 * the count).  Outputs as chns_leaves_adapt. */
chns_status chns_leaves_remesh(int dim, int max_level, int64_t n_src, const uint8_t *src_level,
                               const uint32_t *src_anchor, int64_t n_nodes, const int64_t *xyz,
                               int nf, const double *U, int phi_index, double band, int level_min,
                               int level_max, int64_t *n_out, uint8_t **level_out,
                               uint32_t **anchor_out, int *passes);

/* Releases an array returned by chns_leaves_adapt or chns_leaves_remesh. */
void chns_leaves_free(void *p);

const char *chns_last_error(void);

/* Tracing: number of kernels this library has launched in this process so
 * far (all devices, all streams).  Read it before and after a region to count
 * the region's launches. */
uint64_t chns_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* CHNS_H */
