// C ABI of libchns: meshes, operator applies, the Newton-Krylov CN step
// (Sec. 3.5), diagnostics and batches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "chns_internal.h"
#include "coarse.h"
#include "kernels.h"
#include "vector.h"
#include "solver.h"
#include "multigrid.h"

namespace chns {
chns_status build_mesh(int dim, int64_t n, const uint8_t *level, const uint32_t *anchor, int max_level,
                       const double lo[3], const double hi[3], chns_mesh *m);
chns_status build_union(const std::vector<const chns_mesh *> &ms, chns_mesh *u);
chns_status build_gather(chns_mesh *m);
chns_status validate_mesh(const chns_mesh *m);
const char *last_error();
uint64_t launches();
}  // namespace chns

using namespace chns;

#define TRY(expr)                               \
  do {                                          \
    chns_status s_ = (expr);                    \
    if (s_ != CHNS_OK) return s_;               \
  } while (0)

namespace chns {
chns_status check_params(const chns_mesh *m, const chns_params *p) {
  if (!m || !p) { set_error("null mesh or params"); return CHNS_ERR_ARG; }
  if (p->dim != m->dim) { set_error("params.dim %d != mesh dim %d", p->dim, m->dim); return CHNS_ERR_ARG; }
  if (!(p->dt > 0) || !(p->Cn > 0) || !(p->Re > 0) || !(p->We > 0) || !(p->Pe > 0) || !(p->Fr > 0) ||
      !(p->rho_ratio > 0) || !(p->eta_ratio > 0) || !(p->C_I >= 0)) {
    set_error("parameters must be positive");
    return CHNS_ERR_ARG;
  }
  return CHNS_OK;
}

chns_status check_launch() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("kernel launch failed: %s", cudaGetErrorString(e));
    return CHNS_ERR_CUDA;
  }
  return CHNS_OK;
}

// prepared nodal fields (CN averages and increments) in precision T
template <typename T>
chns_status prepare(chns_mesh *m, const double *Un, const double *Uo, cudaStream_t st, T **ut, T **dl) {
  Workspace &ws = m->ws;
  DevBuf &bu = sizeof(T) == 8 ? ws.ut : ws.ut32;
  DevBuf &bd = sizeof(T) == 8 ? ws.dl : ws.dl32;
  TRY(bu.ensure(sizeof(T) * m->n_nodes * m->nf));
  TRY(bd.ensure(sizeof(T) * m->n_nodes * (m->dim + 1)));
  launch_prep<T>(m, Un, Uo, bu.as<T>(), bd.as<T>(), st);
  *ut = bu.as<T>();
  *dl = bd.as<T>();
  return check_launch();
}

chns_status residual_prepared(chns_mesh *m, const PhysCoef &pc, const double *Un, const double *ut,
                              const double *dl, const double *forcing, const double *bc, double *F,
                              cudaStream_t st) {
  CHNS_CUDA_TRY(cudaMemsetAsync(F, 0, sizeof(double) * m->n_nodes * m->nf, st));
  launch_residual(m, pc, ut, dl, forcing, F, st);
  launch_dirichlet_res(m, Un, bc, F, st);
  return check_launch();
}

// element-local J.w buffer of precision T (n_elem * 2^dim * nf values)
template <typename T>
chns_status ensure_ebuf(chns_mesh *m, T **E) {
  DevBuf &b = sizeof(T) == 8 ? m->ws.e64 : m->ws.e32;
  TRY(b.ensure(sizeof(T) * (m->n_elem << m->dim) * m->nf));
  *E = b.as<T>();
  return CHNS_OK;
}

template <typename T>
chns_status jacvec_prepared(chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, const T *w, T *y,
                            cudaStream_t st) {
  T *E = nullptr;
  TRY(ensure_ebuf<T>(m, &E));
  launch_jacvec<T>(m, pc, ut, dl, w, E, y, st);
  return check_launch();
}
template chns_status prepare<float>(chns_mesh *, const double *, const double *, cudaStream_t, float **, float **);
template chns_status prepare<double>(chns_mesh *, const double *, const double *, cudaStream_t, double **, double **);
template chns_status ensure_ebuf<float>(chns_mesh *, float **);
template chns_status ensure_ebuf<double>(chns_mesh *, double **);
template chns_status jacvec_prepared<float>(chns_mesh *, const PhysCoef &, const float *, const float *, const float *,
                                            float *, cudaStream_t);
template chns_status jacvec_prepared<double>(chns_mesh *, const PhysCoef &, const double *, const double *,
                                             const double *, double *, cudaStream_t);

// ---------------------------------------------------------------- block-Jacobi by probing
// The nodal (nf x nf) diagonal blocks of J are read off J applied to the
// indicator of one field on the nodes of one node colour: nodes of a colour
// never share an element, so each probed node sees only its own block.
template <typename T>
chns_status build_block_jacobi(chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, DevBuf &out,
                               cudaStream_t st, double scale) {
  Workspace &ws = m->ws;
  const int nf = m->nf;
  const int64_t n = m->n_nodes * nf;
  TRY(out.ensure(sizeof(T) * m->n_nodes * nf * nf + 16));
  TRY(ws.wv.ensure(sizeof(T) * n));
  TRY(ws.yv.ensure(sizeof(T) * n));
  T *w = ws.wv.as<T>(), *y = ws.yv.as<T>(), *B = out.as<T>();
  for (int c = 0; c < m->n_node_colours; ++c) {
    int64_t b = m->node_colour_start[c], e = m->node_colour_start[c + 1];
    for (int f = 0; f < nf; ++f) {
      CHNS_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(T) * n, st));
      probe_set<T>(m->node_perm + b, e - b, nf, f, w, st);
      TRY(jacvec_prepared<T>(m, pc, ut, dl, w, y, st));
      probe_get<T>(m->node_perm + b, e - b, nf, f, y, B, st);
    }
  }
  int *bad = reinterpret_cast<int *>(reinterpret_cast<char *>(B) + sizeof(T) * m->n_nodes * nf * nf);
  CHNS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
  invert_blocks<T>(B, m->n_nodes, nf, bad, scale, st);
  int hbad = 0;
  CHNS_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHNS_CUDA_TRY(cudaStreamSynchronize(st));
  if (hbad) { set_error("singular nodal diagonal block in the preconditioner"); return CHNS_ERR_KRYLOV; }
  return check_launch();
}
template chns_status build_block_jacobi<float>(chns_mesh *, const PhysCoef &, const float *, const float *, DevBuf &,
                                              cudaStream_t, double);
template chns_status build_block_jacobi<double>(chns_mesh *, const PhysCoef &, const double *, const double *, DevBuf &,
                                               cudaStream_t, double);



// Autotuner of the FP32 J.w schedule of a mesh: every schedule of
// launch_jacvec is timed with CUDA events on the launching stream (one
// warm-up, then the median of five applies to the prepared state) and the
// fastest is kept for the mesh's later FP32 applies.  Runs once per mesh.
chns_status autotune_jacvec(chns_mesh *m, const PhysCoef &pc, const float *ut, const float *dl, cudaStream_t st) {
  if (m->jv_tuned) return CHNS_OK;
  const int64_t n = m->n_nodes * m->nf;
  DevBuf w, y;
  TRY(w.ensure(sizeof(float) * n + 16));
  TRY(y.ensure(sizeof(float) * n + 16));
  float *E = nullptr;
  TRY(ensure_ebuf<float>(m, &E));
  CHNS_CUDA_TRY(cudaMemcpyAsync(w.as<float>(), ut, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
  cudaEvent_t e[2];
  CHNS_CUDA_TRY(cudaEventCreate(&e[0]));
  CHNS_CUDA_TRY(cudaEventCreate(&e[1]));
  int best = 0;
  double tbest = 1e300;
  for (int v = 0; v < kJacvecVariants; ++v) {
    launch_jacvec<float>(m, pc, ut, dl, w.as<float>(), E, y.as<float>(), st, v);
    std::vector<float> ts;
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e[0], st);
      launch_jacvec<float>(m, pc, ut, dl, w.as<float>(), E, y.as<float>(), st, v);
      cudaEventRecord(e[1], st);
      cudaEventSynchronize(e[1]);
      float t = 0.f;
      cudaEventElapsedTime(&t, e[0], e[1]);
      ts.push_back(t);
    }
    std::sort(ts.begin(), ts.end());
    m->jv_times[v] = ts[2];
    if (ts[2] < tbest) { tbest = ts[2]; best = v; }
  }
  cudaEventDestroy(e[0]);
  cudaEventDestroy(e[1]);
  w.release();
  y.release();
  TRY(check_launch());
  m->jv_variant = best;
  m->jv_tuned = true;
  return CHNS_OK;
}
}  // namespace chns

namespace {

inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }


chns_status ensure_events(Workspace &ws, size_t n) {
  while (ws.ev.size() < n) {
    cudaEvent_t e;
    CHNS_CUDA_TRY(cudaEventCreate(&e));
    ws.ev.push_back(e);
  }
  return CHNS_OK;
}

// Hessenberg column slot: h (pass 1), h (pass 2), norms/flag/scale
constexpr int kHessSlot = kMaxRestart + 8;

chns_status ensure_pinned(Workspace &ws) {
  if (!ws.hpinned) CHNS_CUDA_TRY(cudaMallocHost(&ws.hpinned, sizeof(double) * 8 * kHessSlot));
  return CHNS_OK;
}

chns_status norm2(chns_mesh *m, const double *x, double *out_host, cudaStream_t st) {
  Workspace &ws = m->ws;
  int64_t n = m->n_nodes * m->nf;
  TRY(ws.red.ensure(sizeof(double) * (kMaxRestart + 16) * red_blocks()));
  TRY(ws.hdev.ensure(sizeof(double) * 8 * kHessSlot));
  TRY(ensure_pinned(ws));
  double *hd = ws.hdev.as<double>();
  vec_dot(x, x, n, ws.red.as<double>(), hd, st);
  CHNS_CUDA_TRY(cudaMemcpyAsync(ws.hpinned, hd, sizeof(double), cudaMemcpyDeviceToHost, st));
  CHNS_CUDA_TRY(cudaStreamSynchronize(st));
  *out_host = std::sqrt(ws.hpinned[0]);
  return CHNS_OK;
}

// Per-call timing of a group of launches with CUDA events on the stream: a
// ring of event pairs in the workspace; pairs are read once they completed
// (the Krylov loop runs ahead of the host by one iteration).
struct Timer {
  static constexpr int kPairs = 32;
  double ms = 0.0;
  int calls = 0;
  int64_t head = 0, tail = 0;  // pending pairs: [tail, head)
  Workspace *ws = nullptr;
  bool on = false;
  chns_status begin(cudaStream_t st, int *slot) {
    if (!on) return CHNS_OK;
    if (ws->tev.empty()) {
      for (int i = 0; i < 2 * kPairs; ++i) {
        cudaEvent_t e;
        CHNS_CUDA_TRY(cudaEventCreate(&e));
        ws->tev.push_back(e);
      }
    }
    if (head - tail == kPairs) {  // ring full: wait for the oldest pair
      CHNS_CUDA_TRY(cudaEventSynchronize(ws->tev[2 * (tail % kPairs) + 1]));
      TRY(collect());
    }
    *slot = int(head % kPairs);
    CHNS_CUDA_TRY(cudaEventRecord(ws->tev[2 * *slot], st));
    return CHNS_OK;
  }
  chns_status end(cudaStream_t st, int slot) {
    if (!on) return CHNS_OK;
    CHNS_CUDA_TRY(cudaEventRecord(ws->tev[2 * slot + 1], st));
    ++head;
    return CHNS_OK;
  }
  // add the pairs that have completed, oldest first
  chns_status collect() {
    while (tail < head) {
      const int sl = int(tail % kPairs);
      cudaError_t q = cudaEventQuery(ws->tev[2 * sl + 1]);
      if (q == cudaErrorNotReady) break;
      CHNS_CUDA_TRY(q);
      float t = 0.f;
      CHNS_CUDA_TRY(cudaEventElapsedTime(&t, ws->tev[2 * sl], ws->tev[2 * sl + 1]));
      ms += t;
      ++calls;
      ++tail;
    }
    return CHNS_OK;
  }
  // after the stream has drained
  chns_status finish() {
    if (tail < head) CHNS_CUDA_TRY(cudaEventSynchronize(ws->tev[2 * ((head - 1) % kPairs) + 1]));
    return collect();
  }
};

// What an Arnoldi-step graph bakes in: buffers, sizes, coarse-space state and
// the element coefficients (kernel arguments by value)
struct StepKey {
  const void *p[16];
  int64_t i[8];
  PhysCoef pc;
};

// CHNS_INJECT=krylov: the next FGMRES reports a breakdown (host-side fault
// injection; read at every solve so a test can set and clear it)
bool inject_krylov_fault() {
  const char *e = std::getenv("CHNS_INJECT");
  return e && std::strcmp(e, "krylov") == 0;
}

// ---------------------------------------------------------------- FGMRES
// Solve J x = b (b = -F) with right-preconditioned flexible GMRES(m).  The
// basis V, the preconditioned directions Z, J.z and the Gram-Schmidt
// (classical, a second pass on severe cancellation) are in the element
// precision T, with double accumulation of the dot products; the Hessenberg
// least squares, x, r = b - J x and its norm are in double.
//
// The host needs column j of the Hessenberg matrix only for the Givens
// rotations and the convergence test, so Arnoldi step j + 1 is queued on the
// stream before the host waits for column j (two result slots, a pinned
// mirror each): the GPU never idles on the host.  When step j converges,
// the queued step j + 1 is discarded.
// The float multigrid hierarchy as the preconditioner of a double FGMRES
// (the FP64 finish of the mixed path): the V-cycle runs in float on the float
// linearisation (ut, dl), between conversions of v and z.
struct Mg32 {
  const float *ut = nullptr, *dl = nullptr;
  float *vin = nullptr, *zout = nullptr;
};

template <typename T>
chns_status fgmres(chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, const T *Binv, bool coarse,
                   bool mg, const double *b, double *x, const chns_solver_opts &o, int *its_out, Timer &tj,
                   cudaStream_t st, const Mg32 *mg32 = nullptr, bool *converged = nullptr) {
  Workspace &ws = m->ws;
  const int nf = m->nf;
  const int64_t n = m->n_nodes * nf;
  const int mr = o.krylov_restart;
  const int64_t ld = vec_ld(n);  // basis stride: 16-byte aligned vectors
  constexpr int K = kHessSlot;
  TRY(ws.V.ensure(sizeof(T) * (mr + 1) * ld));
  TRY(ws.Z.ensure(sizeof(T) * mr * ld));
  TRY(ws.r.ensure(sizeof(double) * n));
  TRY(ws.wv.ensure(sizeof(T) * n));
  TRY(ws.yv.ensure(sizeof(T) * n));
  TRY(ws.red.ensure(sizeof(double) * (kMaxRestart + 16) * red_blocks()));
  TRY(ws.hdev.ensure(sizeof(double) * 8 * K));
  TRY(ensure_pinned(ws));
  TRY(ensure_events(ws, 2));
  double *r = ws.r.as<double>();
  T *V = ws.V.as<T>(), *Z = ws.Z.as<T>(), *yv = ws.yv.as<T>(), *tv = ws.wv.as<T>();
  double *part = ws.red.as<double>(), *hd = ws.hdev.as<double>();
  double *cz = hd + 6 * K;
  // grid-reduction ticket of the Gram-Schmidt kernels (zero between launches)
  TRY(ws.ctr.ensure(64));
  unsigned *ctr = ws.ctr.as<unsigned>();
  CHNS_CUDA_TRY(cudaMemsetAsync(ctr, 0, 64, st));

  CHNS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
  CHNS_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  double beta0 = 0.0;
  TRY(norm2(m, r, &beta0, st));
  if (!std::isfinite(beta0)) { set_error("non-finite right-hand side"); return CHNS_ERR_NONFINITE; }
  *its_out = 0;
  if (beta0 == 0.0) return CHNS_OK;
  const double target = o.krylov_rtol * beta0;
  double beta = beta0;

  // Arnoldi step j: z_j = M^{-1} v_j, w = J z_j orthogonalised against
  // v_0..v_j and normalised into v_{j+1}; column j to pinned slot j % 2.
  // Launched on stream s; with `cap` (stream capture) the J.w bracket is
  // recorded as external events of the graph.
  Workspace::StepGraphs &G = ws.kg[sizeof(T) == 8 ? 1 : 0];
  auto arnoldi_body = [&](int j, cudaStream_t s, bool cap) -> chns_status {
    const int sl = j & 1;
    double *h1 = hd + 3 * K * sl, *h2 = h1 + K, *nr = h1 + 2 * K;
    T *vj = V + (int64_t)j * ld, *w = V + (int64_t)(j + 1) * ld;
    T *zj = Z + (int64_t)j * ld;
    if (mg32) {
      vec_convert<T, float>(vj, mg32->vin, n, 1.0, s);
      TRY(mg_apply<float>(m, pc, mg32->ut, mg32->dl, mg32->vin, mg32->zout, s));
      vec_convert<float, T>(mg32->zout, zj, n, 1.0, s);
    } else if (mg) {
      TRY(mg_apply<T>(m, pc, ut, dl, vj, zj, s));
    }
    else precond_apply<T>(m, Binv, coarse, vj, zj, s);
    int ev = 0;
    if (cap) CHNS_CUDA_TRY(cudaEventRecordWithFlags(G.jv[2 * j], s, cudaEventRecordExternal));
    else TRY(tj.begin(s, &ev));
    TRY(jacvec_prepared<T>(m, pc, ut, dl, zj, w, s));
    if (cap) CHNS_CUDA_TRY(cudaEventRecordWithFlags(G.jv[2 * j + 1], s, cudaEventRecordExternal));
    else TRY(tj.end(s, ev));
    int *flag = reinterpret_cast<int *>(nr + 2);
    T *scale = reinterpret_cast<T *>(nr + 3);
    vec_orthogonalize<T>(V, ld, j + 1, n, part, h1, h2, nr, flag, scale, ctr, s);
    vec_normalize<T>(w, n, scale, s);
    CHNS_CUDA_TRY(cudaMemcpyAsync(ws.hpinned + 3 * K * sl, h1, sizeof(double) * 3 * K, cudaMemcpyDeviceToHost, s));
    return CHNS_OK;
  };
  // Arnoldi steps as CUDA graphs (one per j, captured at first use): a step
  // is ~25 launches of mostly short kernels, and host launch cost, not the
  // GPU, bounds a step launched one kernel at a time
  const bool graphs = o.use_graph != 0;
  T *Ebuf = nullptr;
  TRY(ensure_ebuf<T>(m, &Ebuf));
  if (graphs) {
    StepKey key;
    std::memset(&key, 0, sizeof(key));
    key.p[0] = V; key.p[1] = Z; key.p[2] = ut; key.p[3] = dl; key.p[4] = Binv; key.p[5] = part;
    key.p[6] = hd; key.p[7] = ws.hpinned; key.p[8] = m->coarse.vec.as<void>();
    key.p[9] = m->coarse.rpart.as<void>(); key.p[10] = m->coarse.M.as<void>();
    key.p[11] = m->coarse.Minv32.as<void>(); key.p[12] = m->coarse.cnodes; key.p[13] = Ebuf;
    key.p[14] = ctr; key.p[15] = mg ? m->mg : nullptr;
    key.i[0] = ld; key.i[1] = n; key.i[2] = coarse; key.i[3] = m->coarse.ready; key.i[4] = m->coarse.level;
    key.i[5] = mg ? (int64_t)m->mg->generation : -1; key.i[6] = o.use_graph + 2 * (mg32 != nullptr);
    key.i[7] = m->jv_variant;
    key.pc = pc;
    const unsigned char *kb = reinterpret_cast<const unsigned char *>(&key);
    if (G.key.size() != sizeof(key) || std::memcmp(G.key.data(), kb, sizeof(key)) != 0) {
      G.clear();
      G.key.assign(kb, kb + sizeof(key));
    }
    if ((int)G.exec.size() < mr) {
      G.exec.resize(mr, nullptr);
      G.launches.resize(mr, 0);
    }
    while ((int)G.jv.size() < 2 * mr) {
      cudaEvent_t e;
      CHNS_CUDA_TRY(cudaEventCreate(&e));
      G.jv.push_back(e);
    }
    if (!ws.cap) CHNS_CUDA_TRY(cudaStreamCreateWithFlags(&ws.cap, cudaStreamNonBlocking));
  }
  auto capture = [&](int j) -> chns_status {
    int cnt = 0;
    set_capture_sink(&cnt);
    cudaError_t e = cudaStreamBeginCapture(ws.cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      set_capture_sink(nullptr);
      CHNS_CUDA_TRY(e);
    }
    chns_status sb = arnoldi_body(j, ws.cap, true);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(ws.cap, &gr);
    set_capture_sink(nullptr);
    if (sb != CHNS_OK || e != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      if (sb != CHNS_OK) return sb;
      CHNS_CUDA_TRY(e);
    }
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, gr, 0);
    cudaGraphDestroy(gr);
    CHNS_CUDA_TRY(e);
    G.exec[j] = ge;
    G.launches[j] = cnt;
    return CHNS_OK;
  };
  auto arnoldi = [&](int j) -> chns_status {
    if (graphs) {
      if (!G.exec[j]) TRY(capture(j));
      CHNS_CUDA_TRY(cudaGraphLaunch(G.exec[j], st));
      note_launches(G.launches[j]);
    } else {
      TRY(arnoldi_body(j, st, false));
    }
    CHNS_CUDA_TRY(cudaEventRecord(ws.ev[j & 1], st));
    return CHNS_OK;
  };
  std::vector<double> H((mr + 1) * mr), cs(mr), sn(mr), g(mr + 1), yk(mr);
  int total = 0;
  bool conv = false;
  while (true) {
    // V_0 = r / beta
    vec_convert<double, T>(r, V, n, 1.0 / beta, st);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j_end = 0;
    bool done = false;
    for (int j = 0; j < mr; ++j) {
      if (j == 0) TRY(arnoldi(0));
      if (j + 1 < mr && total + 1 < o.krylov_max_it) TRY(arnoldi(j + 1));  // queued ahead
      CHNS_CUDA_TRY(cudaEventSynchronize(ws.ev[j & 1]));
      if (graphs && tj.on) {
        float t = 0.f;
        CHNS_CUDA_TRY(cudaEventElapsedTime(&t, G.jv[2 * j], G.jv[2 * j + 1]));
        tj.ms += t;
        ++tj.calls;
      }
      TRY(tj.collect());
      const double *hp = ws.hpinned + 3 * K * (j & 1);
      const double *hnr = hp + 2 * K;
      const int hflag = *reinterpret_cast<const int *>(hnr + 2);
      double hn = std::sqrt(hflag ? hnr[1] : hnr[0]);
      if (!std::isfinite(hn)) { set_error("non-finite Krylov vector"); return CHNS_ERR_NONFINITE; }
      for (int i = 0; i <= j; ++i) H[i * mr + j] = hp[i] + (hflag ? hp[K + i] : 0.0);
      H[(j + 1) * mr + j] = hn;
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        double a = H[i * mr + j], c = H[(i + 1) * mr + j];
        H[i * mr + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * mr + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * mr + j], c = H[(j + 1) * mr + j];
      double rr = std::hypot(a, c);
      if (rr == 0.0 || inject_krylov_fault()) {
        CHNS_CUDA_TRY(cudaStreamSynchronize(st));  // the queued step j + 1 has finished
        set_error("FGMRES breakdown at iteration %d", total + 1);
        return CHNS_ERR_KRYLOV;
      }
      cs[j] = a / rr;
      sn[j] = c / rr;
      H[j * mr + j] = rr;
      H[(j + 1) * mr + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      j_end = j + 1;
      if (std::fabs(g[j + 1]) <= target || hn == 0.0) { done = true; break; }
      if (total >= o.krylov_max_it) break;
    }
    // y = H^{-1} g, x += Z y
    for (int i = j_end - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j_end; ++k) s -= H[i * mr + k] * yk[k];
      yk[i] = s / H[i * mr + i];
    }
    CHNS_CUDA_TRY(cudaMemcpyAsync(cz, yk.data(), sizeof(double) * j_end, cudaMemcpyHostToDevice, st));
    vec_combine<T>(Z, ld, j_end, cz, x, n, st);
    if (done) conv = true;
    if (done || total >= o.krylov_max_it) break;
    // restart: r = b - J x
    vec_convert<double, T>(x, tv, n, 1.0, st);
    int ev = 0;
    TRY(tj.begin(st, &ev));
    TRY(jacvec_prepared<T>(m, pc, ut, dl, tv, yv, st));
    TRY(tj.end(st, ev));
    vec_sub<T>(b, yv, r, n, st);
    TRY(norm2(m, r, &beta, st));
    TRY(tj.collect());
    if (!std::isfinite(beta)) { set_error("non-finite Krylov residual"); return CHNS_ERR_NONFINITE; }
    if (beta <= target) { conv = true; break; }
  }
  *its_out = total;
  if (converged) *converged = conv;
  TRY(tj.finish());
  return check_launch();
}

template <typename T>
struct JvCtx {
  chns_mesh *m;
  const PhysCoef *pc;
  const T *ut, *dl;
  cudaStream_t st;
};

template <typename T>
chns_status jv_callback(void *ctx, const T *w, T *y) {
  JvCtx<T> *c = static_cast<JvCtx<T> *>(ctx);
  return jacvec_prepared<T>(c->m, *c->pc, c->ut, c->dl, w, y, c->st);
}

template <typename T>
chns_status build_coarse_operator(chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, cudaStream_t st) {
  Workspace &ws = m->ws;
  const int64_t n = m->n_nodes * m->nf;
  TRY(ws.wv.ensure(sizeof(T) * n));
  TRY(ws.yv.ensure(sizeof(T) * n));
  JvCtx<T> ctx{m, &pc, ut, dl, st};
  return coarse_build<T>(m, &jv_callback<T>, &ctx, ws.wv.as<T>(), ws.yv.as<T>(), st);
}

// An FP32-Krylov Newton iteration must cut ||F|| by at least this factor;
// otherwise the rest of the step uses FP64 J.w (FP64 finish).
constexpr double kFp32MinReduction = 10.0;

bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char *e = std::getenv("CHNS_TRACE");
    on = (e && *e && *e != '0') ? 1 : 0;
  }
  return on == 1;
}

// Newton on F(U; U_n) = 0 (Sec. 3.5).  FP64 residual and update; each
// correction by FGMRES in the element precision.  With CHNS_FP32_BULK the
// correction uses FP32 J.w and an FP32 block-Jacobi until an iteration fails
// to cut ||F|| by kFp32MinReduction (the FP32 operator cannot resolve the
// weakly stabilised pressure modes below that level); the remaining
// iterations use FP64 J.w with the FP32 block-Jacobi promoted to FP64.
chns_status newton_step(chns_mesh *m, const chns_params *p, const chns_solver_opts &o, const double *Un,
                        const double *Unm1, const double *forcing, const double *bc, double *U,
                        chns_step_stats *stats, cudaStream_t st) {
  Workspace &ws = m->ws;
  const int nf = m->nf;
  const int64_t n = m->n_nodes * nf;
  const int64_t nb = m->n_nodes * nf * nf;
  PhysCoef pc = make_coef(*p, m->lo, m->hi);
  TRY(ws.F.ensure(sizeof(double) * n));
  TRY(ws.dU.ensure(sizeof(double) * n));
  double *F = ws.F.as<double>(), *dU = ws.dU.as<double>();
  Timer tj, tr, tp;  // accumulated J.w, residual and preconditioner times
  const bool mixed = o.precision == CHNS_FP32_BULK;
  const bool use_mg = o.preconditioner == CHNS_PC_MULTIGRID;
  int Lc = o.coarse_level;
  if (Lc < 0) Lc = std::min(3, m->min_level - 1);
  const bool coarse = !use_mg && Lc >= 1;
  if (coarse) TRY(coarse_setup(m, Lc));
  if (use_mg) {
    TRY(mg_setup(m, o.mg_coarsest > 0 ? o.mg_coarsest : (m->dim == 3 ? 2 : 3)));
    Lc = m->mg->bottom_level;
    m->mg->autotune = o.autotune != 0;
  }
  // a preconditioner from an earlier step is reused while it is young enough
  // and was built for the same precision, parameters and preconditioner
  bool have_pc = ws.pc_steps_left > 0 && ws.pc_precision == (int)o.precision && ws.pc_coarse == Lc &&
                 ws.pc_kind == (int)o.preconditioner && ws.pc_smooth == o.mg_smooth && ws.pc_omega == o.mg_omega &&
                 std::memcmp(&ws.pc_params, p, sizeof(chns_params)) == 0 && o.reuse_preconditioner > 0 &&
                 (!use_mg || m->mg->ready[mixed ? 0 : 1]);
  if (have_pc) --ws.pc_steps_left;
  auto mark_built = [&]() {
    ws.pc_precision = (int)o.precision;
    ws.pc_coarse = Lc;
    ws.pc_kind = (int)o.preconditioner;
    ws.pc_smooth = o.mg_smooth;
    ws.pc_omega = o.mg_omega;
    ws.pc_params = *p;
    ws.pc_steps_left = o.reuse_preconditioner > 0 ? o.reuse_preconditioner - 1 : 0;
  };

  if (Unm1) vec_lincomb(2.0, Un, -1.0, Unm1, U, n, st);
  else CHNS_CUDA_TRY(cudaMemcpyAsync(U, Un, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));

  // fields solved for: all (coupled Newton), or one block of the NS <-> CH
  // block iteration (Sec. 3.1, Fig. flowchart_block); the other block's rows
  // are identity rows of J.w and zero rows of the residual
  uint32_t fmask = 0xffu;
  double *ut = nullptr, *dl = nullptr;
  auto residual = [&](double *fn) -> chns_status {
    TRY(prepare<double>(m, U, Un, st, &ut, &dl));
    if (stats) { TRY(ensure_events(ws, 64)); CHNS_CUDA_TRY(cudaEventRecord(ws.ev[60], st)); }
    TRY(residual_prepared(m, pc, U, ut, dl, forcing, bc, F, st));
    if (fmask != 0xffu) vec_mask_fields(F, m->n_nodes, nf, fmask, st);
    if (stats) CHNS_CUDA_TRY(cudaEventRecord(ws.ev[61], st));
    TRY(norm2(m, F, fn, st));
    if (stats) {
      float t = 0.f;
      CHNS_CUDA_TRY(cudaEventElapsedTime(&t, ws.ev[60], ws.ev[61]));
      tr.ms += t;
      tr.calls++;
    }
    if (!std::isfinite(*fn)) { set_error("non-finite residual norm"); return CHNS_ERR_NONFINITE; }
    return CHNS_OK;
  };
  // batched meshes: every instance must meet its own tolerance; converged
  // instances get a zero right-hand side (their correction is then exactly
  // zero: the operator and the preconditioner are block diagonal)
  const int ni = m->n_inst;
  std::vector<double> fi0, fi(ni, 0.0);
  auto instance_norms = [&]() -> chns_status {
    if (ni == 1) return CHNS_OK;
    TRY(ws.red.ensure(sizeof(double) * (kMaxRestart + 16) * red_blocks()));
    TRY(ws.hdev.ensure(sizeof(double) * std::max<int64_t>(8 * kHessSlot, ni + 8)));
    double *hd = ws.hdev.as<double>();
    for (int q = 0; q < ni; ++q) {
      const int64_t a = m->inst_node_start[q] * nf, b = m->inst_node_start[q + 1] * nf;
      vec_dot(F + a, F + a, b - a, ws.red.as<double>(), hd + q, st);
    }
    std::vector<double> h(ni);
    CHNS_CUDA_TRY(cudaMemcpyAsync(h.data(), hd, sizeof(double) * ni, cudaMemcpyDeviceToHost, st));
    CHNS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < ni; ++q) fi[q] = std::sqrt(h[q]);
    return CHNS_OK;
  };
  int its = 0, kits = 0, its64 = 0;
  double f0_all = -1.0, fn_last = 0.0;

  // Newton on the fields of fmask from the current U, to newton_rtol of its
  // initial residual (Sec. 3.5).  In the block iteration the reference is
  // the initial residual of the first sub-solve of the same block: later
  // sub-solves start close to their root, and a tolerance relative to their
  // own tiny initial residual would ask for more than double precision holds.
  double f0_block[2] = {-1.0, -1.0};
  std::vector<double> fi0_block[2];
  auto solve = [&](uint32_t mask) -> chns_status {
    fmask = mask;
    PhysCoef pcs = pc;
    pcs.fmask = mask;
    bool use64 = !mixed;
    bool have_pc64 = false;
    if (mask != 0xffu) have_pc = false;  // the operator differs per block: build for each sub-solve
    double fn = 0.0;
    TRY(residual(&fn));
    double f0 = fn;
    if (f0_all < 0.0) f0_all = f0;
    TRY(instance_norms());
    fi0 = fi;
    if (mask != 0xffu) {
      const int kind = (mask & 1u) ? 0 : 1;  // NS block holds v_1
      if (f0_block[kind] < 0.0) {
        f0_block[kind] = f0;
        fi0_block[kind] = fi0;
      }
      f0 = std::max(f0, f0_block[kind]);
      for (int q = 0; q < ni; ++q) fi0[q] = std::max(fi0[q], fi0_block[kind][q]);
    }
    auto converged = [&]() {
      if (ni == 1) return fn <= std::max(o.newton_rtol * f0, o.newton_atol);
      for (int q = 0; q < ni; ++q)
        if (!(fi[q] <= std::max(o.newton_rtol * fi0[q], o.newton_atol))) return false;
      return true;
    };
    int sub_its = 0;
    while (!converged()) {
      if (ni > 1)
        for (int q = 0; q < ni; ++q)
          if (fi[q] <= std::max(o.newton_rtol * fi0[q], o.newton_atol)) {
            const int64_t a = m->inst_node_start[q] * nf, b = m->inst_node_start[q + 1] * nf;
            CHNS_CUDA_TRY(cudaMemsetAsync(F + a, 0, sizeof(double) * (b - a), st));
          }
      if (sub_its >= o.newton_max_it) {
        ws.pc_steps_left = 0;
        set_error("Newton reached %d iterations with ||F|| = %.3e (start %.3e)", sub_its, fn, f0);
        if (stats) { stats->newton_its = its; stats->res_final = fn; stats->res0 = f0; }
        return CHNS_ERR_NEWTON;
      }
      int k = 0;
      Timer tk;  // event slots 0.. (the residual uses slots 60, 61)
      tk.ws = &ws;
      tk.on = stats != nullptr;
      // forcing term: never ask the linear solve for more than the Newton
      // target needs (with a factor-2 margin), never less than krylov_rtol
      chns_solver_opts oi = o;
      const double target = std::max(o.newton_rtol * f0, o.newton_atol);
      oi.krylov_rtol = std::max(o.krylov_rtol, std::min(0.5, 0.5 * target / fn));
      vec_axpby(-1.0, F, 0.0, F, n, st);  // b = -F
      auto a = std::chrono::steady_clock::now();
      if (!use64) {
        float *ut_t = nullptr, *dl_t = nullptr;
        TRY(prepare<float>(m, U, Un, st, &ut_t, &dl_t));
        if (o.autotune && !m->jv_tuned) TRY(autotune_jacvec(m, pcs, ut_t, dl_t, st));
        if (!have_pc || !o.reuse_preconditioner || (use_mg && !m->mg->ready[0])) {
          if (use_mg) {
            TRY(mg_build<float>(m, pcs, ut_t, dl_t, o.mg_omega, o.mg_smooth, st));
          } else {
            TRY(build_block_jacobi<float>(m, pcs, ut_t, dl_t, ws.binv, st, 1.0));
            if (coarse) TRY(build_coarse_operator<float>(m, pcs, ut_t, dl_t, st));
          }
          have_pc = true;
          mark_built();
          tp.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
        } else if (use_mg) {
          TRY(mg_update_state<float>(m, ut_t, dl_t, st));  // coarse levels follow the Newton iterate
        }
        TRY(fgmres<float>(m, pcs, ut_t, dl_t, ws.binv.as<float>(), coarse, use_mg, F, dU, oi, &k, tk, st));
      } else {
        double *ut_t = nullptr, *dl_t = nullptr;
        TRY(prepare<double>(m, U, Un, st, &ut_t, &dl_t));
        Mg32 mg32;
        bool use_mg32 = false;
        if (mixed) {
          if (use_mg && !m->mg->finish64) {
            // the FP64 finish first keeps the float hierarchy as its
            // preconditioner (FGMRES is flexible): float V-cycles, cheap
            float *u32 = nullptr, *d32 = nullptr;
            TRY(prepare<float>(m, U, Un, st, &u32, &d32));
            if (!m->mg->ready[0]) {
              TRY(mg_build<float>(m, pcs, u32, d32, o.mg_omega, o.mg_smooth, st));
              tp.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
            } else {
              TRY(mg_update_state<float>(m, u32, d32, st));
            }
            TRY(ws.p32a.ensure(sizeof(float) * n + 16));
            TRY(ws.p32b.ensure(sizeof(float) * n + 16));
            mg32.ut = u32;
            mg32.dl = d32;
            mg32.vin = ws.p32a.as<float>();
            mg32.zout = ws.p32b.as<float>();
            use_mg32 = true;
          } else if (use_mg) {
            // float V-cycles could not precondition the FP64 operator on this
            // mesh (FGMRES missed its tolerance): V-cycles with operators and
            // smoother blocks probed in double (the weakly determined modes
            // the finish must resolve are where float probes fall short);
            // built once and kept next to the float ones until the next float
            // build
            if (!m->mg->ready[1]) {
              TRY(mg_build<double>(m, pcs, ut_t, dl_t, o.mg_omega, o.mg_smooth, st, true));
              tp.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
            } else {
              TRY(mg_update_state<double>(m, ut_t, dl_t, st));
            }
          } else if (!have_pc64) {  // promote the FP32 blocks (built by an earlier FP32 iteration or step)
            TRY(ws.binv64.ensure(sizeof(double) * nb));
            vec_convert<float, double>(ws.binv.as<float>(), ws.binv64.as<double>(), nb, 1.0, st);
            have_pc64 = true;
          }
        } else if (!have_pc || !o.reuse_preconditioner || (use_mg && !m->mg->ready[1])) {
          if (use_mg) {
            TRY(mg_build<double>(m, pcs, ut_t, dl_t, o.mg_omega, o.mg_smooth, st));
          } else {
            TRY(build_block_jacobi<double>(m, pcs, ut_t, dl_t, ws.binv64, st, 1.0));
            if (coarse) TRY(build_coarse_operator<double>(m, pcs, ut_t, dl_t, st));
          }
          have_pc = true;
          mark_built();
          tp.ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
        } else if (use_mg) {
          TRY(mg_update_state<double>(m, ut_t, dl_t, st));
        }
        if (use_mg32) {
          // a bounded trial: if the float V-cycles cannot bring the FP64
          // correction to its tolerance within two restart cycles, this mesh
          // switches to double V-cycles for every later finish
          chns_solver_opts ot = oi;
          ot.krylov_max_it = std::min(o.krylov_max_it, 2 * o.krylov_restart);
          bool conv = false;
          TRY(fgmres<double>(m, pcs, ut_t, dl_t, ws.binv64.as<double>(), coarse, use_mg, F, dU, ot, &k, tk, st,
                             &mg32, &conv));
          if (!conv) m->mg->finish64 = true;
        } else {
          TRY(fgmres<double>(m, pcs, ut_t, dl_t, ws.binv64.as<double>(), coarse, use_mg, F, dU, oi, &k, tk, st));
        }
        if (mixed) ++its64;
      }
      tj.ms += tk.ms;
      tj.calls += tk.calls;
      kits += k;
      vec_axpby(1.0, dU, 1.0, U, n, st);
      ++its;
      ++sub_its;
      const double prev = fn;
      TRY(residual(&fn));
      TRY(instance_norms());
      if (trace_on())
        fprintf(stderr, "[chns] newton %d (fields %#x) |F|/|F0| = %.3e krylov %d (%s J.w)\n", its, mask, fn / f0, k,
                use64 ? "fp64" : "fp32");
      if (mixed && !use64 && fn * kFp32MinReduction > prev) use64 = true;
    }
    fn_last = fn;
    return CHNS_OK;
  };

  int blocks = 0;
  if (!o.block_iteration) {
    TRY(solve(0xffu));
  } else {
    const int d = m->dim;
    const uint32_t ns = (1u << (d + 1)) - 1u;            // v_1..v_d, p
    const uint32_t ch = (1u << (d + 1)) | (1u << (d + 2));  // phi, mu
    TRY(ws.Ublk.ensure(sizeof(double) * n));
    double *Uprev = ws.Ublk.as<double>();
    TRY(ws.red.ensure(sizeof(double) * (kMaxRestart + 16) * red_blocks()));
    TRY(ws.hdev.ensure(sizeof(double) * 8 * kHessSlot));
    TRY(ensure_pinned(ws));
    bool done = false;
    for (int l = 0; l < o.block_max_it && !done; ++l) {
      CHNS_CUDA_TRY(cudaMemcpyAsync(Uprev, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      TRY(solve(ns));
      TRY(solve(ch));
      ++blocks;
      // stop once a block iteration after the first changes no entry of
      // (v, p, phi, mu) by more than block_tol
      vec_maxabs_diff(U, Uprev, n, ws.red.as<double>(), ws.hdev.as<double>(), st);
      CHNS_CUDA_TRY(cudaMemcpyAsync(ws.hpinned, ws.hdev.as<double>(), sizeof(double), cudaMemcpyDeviceToHost, st));
      CHNS_CUDA_TRY(cudaStreamSynchronize(st));
      const double change = ws.hpinned[0];
      if (trace_on()) fprintf(stderr, "[chns] block iteration %d max|dU| = %.3e\n", l, change);
      if (!std::isfinite(change)) { set_error("non-finite block iteration change"); return CHNS_ERR_NONFINITE; }
      if (l >= 1 && change <= o.block_tol) done = true;
    }
    ws.pc_steps_left = 0;  // the last build was for one block only
    if (!done) {
      set_error("block iteration did not reach block_tol %.3e in %d iterations", o.block_tol, o.block_max_it);
      if (stats) { stats->newton_its = its; stats->block_its = blocks; }
      return CHNS_ERR_NEWTON;
    }
    // coupled residual of the block-iteration result (reported, not used)
    fmask = 0xffu;
    TRY(residual(&fn_last));
  }
  if (stats) {
    stats->newton_its = its;
    stats->krylov_its_total = kits;
    stats->res0 = f0_all;
    stats->res_final = fn_last;
    stats->jacvec_ms = tj.ms;
    stats->jacvec_calls = tj.calls;
    stats->residual_ms = tr.ms;
    stats->residual_calls = tr.calls;
    stats->precond_ms = tp.ms;
    stats->fp64_newton_its = its64;
    stats->block_its = blocks;
    stats->jacvec_variant = m->jv_variant;
  }
  return CHNS_OK;
}

chns_status step_impl(chns_mesh *m, const chns_params *p, const chns_solver_opts *o, const double *U_n,
                      const double *U_nm1, const double *forcing, const double *bc, double *U_np1,
                      chns_step_stats *stats, cudaStream_t st);

chns_status energy_mass_impl(chns_mesh *m, const chns_params *p, const double *U, double out[3],
                             cudaStream_t st) {
  PhysCoef pc = make_coef(*p, m->lo, m->hi);
  int64_t nb = energy_blocks(m);
  TRY(m->ws.red.ensure(sizeof(double) * std::max<int64_t>(3 * nb, (kMaxRestart + 16) * red_blocks())));
  launch_energy(m, pc, U, m->ws.red.as<double>(), st);
  TRY(check_launch());
  std::vector<double> h(3 * nb);
  CHNS_CUDA_TRY(cudaMemcpyAsync(h.data(), m->ws.red.as<double>(), sizeof(double) * 3 * nb,
                                cudaMemcpyDeviceToHost, st));
  CHNS_CUDA_TRY(cudaStreamSynchronize(st));
  out[0] = out[1] = out[2] = 0.0;
  for (int64_t b = 0; b < nb; ++b)
    for (int k = 0; k < 3; ++k) out[k] += h[b * 3 + k];
  return CHNS_OK;
}

chns_status step_impl(chns_mesh *m, const chns_params *p, const chns_solver_opts *o, const double *U_n,
                      const double *U_nm1, const double *forcing, const double *bc, double *U_np1,
                      chns_step_stats *stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  if (!o || !U_n || !U_np1) { set_error("null argument"); return CHNS_ERR_ARG; }
  if (U_np1 == U_n) { set_error("U_np1 may not alias U_n"); return CHNS_ERR_ARG; }
  if (o->krylov_restart < 1 || o->krylov_restart > kMaxRestart || o->krylov_max_it < 1 || o->newton_max_it < 0 ||
      o->coarse_level > 16 || o->use_graph < 0 || o->use_graph > 1 ||
      (o->preconditioner != CHNS_PC_TWO_LEVEL && o->preconditioner != CHNS_PC_MULTIGRID) ||
      (o->preconditioner == CHNS_PC_MULTIGRID && (o->mg_smooth < 1 || o->mg_smooth > 8 || !(o->mg_omega > 0.0) ||
                                                  !(o->mg_omega <= 1.0) || o->mg_coarsest > 16)) ||
      o->block_iteration < 0 || o->block_iteration > 1 || o->autotune < 0 || o->autotune > 1 ||
      (o->block_iteration && (!(o->block_tol > 0.0) || o->block_max_it < 1))) {
    set_error("invalid solver options");
    return CHNS_ERR_ARG;
  }
  chns_status s;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    double em[3];
    TRY(energy_mass_impl(m, p, U_n, em, st));
    stats->energy_old = em[0];
    stats->mass_old = em[1];
  }
  if (o->precision == CHNS_FP64 || o->precision == CHNS_FP32_BULK)
    s = newton_step(m, p, *o, U_n, U_nm1, forcing, bc, U_np1, stats, st);
  else {
    set_error("unknown precision");
    return CHNS_ERR_ARG;
  }
  if (s != CHNS_OK) return s;
  if (stats) {
    double em[3];
    TRY(energy_mass_impl(m, p, U_np1, em, st));
    stats->energy_new = em[0];
    stats->mass_new = em[1];
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return CHNS_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

const char *chns_last_error(void) { return chns::last_error(); }

uint64_t chns_kernel_launches(void) { return chns::launches(); }

chns_status chns_mesh_create(int dim, int64_t n_leaves, const uint8_t *level, const uint32_t *anchor,
                             int max_level, const double lo[3], const double hi[3], chns_mesh **out) {
  if (!out) { set_error("null output"); return CHNS_ERR_ARG; }
  *out = nullptr;
  chns_mesh *m = new chns_mesh;
  chns_status s = build_mesh(dim, n_leaves, level, anchor, max_level, lo, hi, m);
  if (s == CHNS_OK) s = build_gather(m);
  if (s != CHNS_OK) {
    chns_mesh_destroy(m);
    return s;
  }
  *out = m;
  return CHNS_OK;
}

chns_status chns_mesh_info(const chns_mesh *m, int64_t *n_nodes, int64_t *n_dof, int *n_colours,
                           int64_t *n_hanging) {
  if (!m) { set_error("null mesh"); return CHNS_ERR_ARG; }
  if (n_nodes) *n_nodes = m->n_nodes;
  if (n_dof) *n_dof = m->n_nodes * m->nf;
  if (n_colours) *n_colours = m->n_colours;
  if (n_hanging) *n_hanging = m->n_hang;
  return CHNS_OK;
}

chns_status chns_mesh_node_coords(const chns_mesh *m, int64_t *xyz) {
  if (!m || !xyz) { set_error("null argument"); return CHNS_ERR_ARG; }
  std::memcpy(xyz, m->node_xyz.data(), sizeof(int64_t) * m->node_xyz.size());
  return CHNS_OK;
}

void chns_mesh_destroy(chns_mesh *m) {
  if (!m) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(m->device);
  cudaFree(m->conn);
  cudaFree(m->level);
  cudaFree(m->anchor);
  cudaFree(m->hang);
  cudaFree(m->wall);
  cudaFree(m->node_perm);
  cudaFree(m->gptr);
  cudaFree(m->gent);
  cudaFree(m->nflag);
  cudaFree(m->pins);
  cudaFree(m->elem_inst);
  cudaFree(m->node_inst);
  cudaFree(m->coef32);
  cudaFree(m->coef64);
  chns::mg_release(m->mg);
  m->mg = nullptr;
  m->coarse.release();
  m->ws.ut.release(); m->ws.dl.release(); m->ws.ut32.release(); m->ws.dl32.release(); m->ws.f.release();
  m->ws.F.release(); m->ws.dU.release(); m->ws.r.release(); m->ws.V.release(); m->ws.Z.release();
  m->ws.wv.release(); m->ws.yv.release(); m->ws.binv.release(); m->ws.binv64.release(); m->ws.red.release(); m->ws.hdev.release();
  m->ws.e32.release(); m->ws.e64.release(); m->ws.ctr.release(); m->ws.count.release();
  m->ws.Ublk.release(); m->ws.p32a.release(); m->ws.p32b.release();
  delete m;
  cudaSetDevice(prev);
}

chns_status chns_residual(const chns_mesh *mc, const chns_params *p, const double *U_new, const double *U_old,
                          const double *forcing, const double *bc, double *F, void *stream) {
  TRY(check_params(mc, p));
  if (!U_new || !U_old || !F) { set_error("null vector"); return CHNS_ERR_ARG; }
  chns_mesh *m = const_cast<chns_mesh *>(mc);
  cudaStream_t st = S(stream);
  double *ut = nullptr, *dl = nullptr;
  TRY(prepare<double>(m, U_new, U_old, st, &ut, &dl));
  PhysCoef pc = make_coef(*p, m->lo, m->hi);
  return residual_prepared(m, pc, U_new, ut, dl, forcing, bc, F, st);
}

chns_status chns_jacvec(const chns_mesh *mc, const chns_params *p, const double *U_new, const double *U_old,
                        const void *w, void *y, chns_precision prec, void *stream) {
  TRY(check_params(mc, p));
  if (!U_new || !U_old || !w || !y) { set_error("null vector"); return CHNS_ERR_ARG; }
  chns_mesh *m = const_cast<chns_mesh *>(mc);
  cudaStream_t st = S(stream);
  PhysCoef pc = make_coef(*p, m->lo, m->hi);
  if (prec == CHNS_FP64) {
    double *ut = nullptr, *dl = nullptr;
    TRY(prepare<double>(m, U_new, U_old, st, &ut, &dl));
    return jacvec_prepared<double>(m, pc, ut, dl, static_cast<const double *>(w), static_cast<double *>(y), st);
  } else if (prec == CHNS_FP32_BULK) {
    float *ut = nullptr, *dl = nullptr;
    TRY(prepare<float>(m, U_new, U_old, st, &ut, &dl));
    return jacvec_prepared<float>(m, pc, ut, dl, static_cast<const float *>(w), static_cast<float *>(y), st);
  }
  set_error("unknown precision %d", (int)prec);
  return CHNS_ERR_ARG;
}

chns_status chns_init_mu(const chns_mesh *mc, const chns_params *p, double *U, void *stream) {
  TRY(check_params(mc, p));
  if (!U) { set_error("null vector"); return CHNS_ERR_ARG; }
  chns_mesh *m = const_cast<chns_mesh *>(mc);
  cudaStream_t st = S(stream);
  Workspace &ws = m->ws;
  const int nf = m->nf, imu = m->dim + 2;
  const int64_t n = m->n_nodes * nf;
  PhysCoef pc = make_coef(*p, m->lo, m->hi);
  // M mu_new = M mu + F_mu(U; U), M = -2 (dF_mu / d mu_new): conjugate
  // gradients preconditioned by the lumped mass (the row sums of M, from one
  // J.w on the indicator of the mu field), which keeps the iteration count
  // bounded however much the leaf sizes differ
  TRY(ws.F.ensure(sizeof(double) * n));
  TRY(ws.dU.ensure(sizeof(double) * n));
  TRY(ws.r.ensure(sizeof(double) * n));
  TRY(ws.V.ensure(sizeof(double) * 4 * n));
  double *r = ws.r.as<double>(), *x = ws.dU.as<double>(), *pv = ws.V.as<double>(), *q = pv + n, *d = pv + 2 * n,
         *z = pv + 3 * n;
  double *ut = nullptr, *dl = nullptr;
  TRY(prepare<double>(m, U, U, st, &ut, &dl));
  TRY(residual_prepared(m, pc, U, ut, dl, nullptr, nullptr, r, st));
  vec_mask_field(r, m->n_nodes, nf, imu, 1.0, st);
  // lumped mass: d = M 1 on the mu field (z holds the indicator of the mu field)
  TRY(ws.red.ensure(sizeof(double) * (kMaxRestart + 16) * red_blocks()));
  TRY(ws.hdev.ensure(sizeof(double) * 8 * kHessSlot));
  TRY(ensure_pinned(ws));
  vec_fill_field(z, m->n_nodes, nf, imu, 1.0, st);
  TRY(jacvec_prepared<double>(m, pc, ut, dl, z, d, st));
  vec_mask_field(d, m->n_nodes, nf, imu, -2.0, st);
  CHNS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
  auto dot = [&](const double *a, const double *b, double *out) -> chns_status {
    vec_dot(a, b, n, ws.red.as<double>(), ws.hdev.as<double>(), st);
    CHNS_CUDA_TRY(cudaMemcpyAsync(ws.hpinned, ws.hdev.as<double>(), sizeof(double), cudaMemcpyDeviceToHost, st));
    CHNS_CUDA_TRY(cudaStreamSynchronize(st));
    *out = ws.hpinned[0];
    return CHNS_OK;
  };
  vec_div_field(r, d, z, m->n_nodes, nf, imu, st);
  CHNS_CUDA_TRY(cudaMemcpyAsync(pv, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  double rz = 0.0, rr = 0.0;
  TRY(dot(r, z, &rz));
  TRY(dot(r, r, &rr));
  const double stop = 1e-26 * std::max(rr, 1e-300);
  for (int it = 0; it < 10000 && rr > stop && rz > 0.0; ++it) {
    TRY(jacvec_prepared<double>(m, pc, ut, dl, pv, q, st));
    vec_mask_field(q, m->n_nodes, nf, imu, -2.0, st);
    double pq = 0.0;
    TRY(dot(pv, q, &pq));
    if (!(pq > 0.0)) { set_error("mass matrix not positive in CG"); return CHNS_ERR_KRYLOV; }
    const double a = rz / pq;
    vec_axpby(a, pv, 1.0, x, n, st);
    vec_axpby(-a, q, 1.0, r, n, st);
    vec_div_field(r, d, z, m->n_nodes, nf, imu, st);
    double rz2 = 0.0;
    TRY(dot(r, z, &rz2));
    TRY(dot(r, r, &rr));
    vec_axpby(1.0, z, rz2 / rz, pv, n, st);
    rz = rz2;
  }
  vec_axpby(1.0, x, 1.0, U, n, st);
  return check_launch();
}

chns_status chns_step(const chns_mesh *mc, const chns_params *p, const chns_solver_opts *o, const double *U_n,
                      const double *U_nm1, const double *forcing, const double *bc, double *U_np1,
                      chns_step_stats *stats, void *stream) {
  TRY(check_params(mc, p));
  return step_impl(const_cast<chns_mesh *>(mc), p, o, U_n, U_nm1, forcing, bc, U_np1, stats, S(stream));
}

chns_status chns_tau_floor_count(const chns_mesh *mc, const chns_params *p, const double *U_new,
                                 const double *U_old, int64_t *count, void *stream) {
  TRY(check_params(mc, p));
  if (!U_new || !U_old || !count) { set_error("null argument"); return CHNS_ERR_ARG; }
  chns_mesh *m = const_cast<chns_mesh *>(mc);
  cudaStream_t st = S(stream);
  double *ut = nullptr, *dl = nullptr;
  TRY(prepare<double>(m, U_new, U_old, st, &ut, &dl));
  Workspace &ws = m->ws;
  TRY(ws.count.ensure(sizeof(unsigned long long)));
  TRY(ensure_pinned(ws));
  unsigned long long *cnt = ws.count.as<unsigned long long>();
  CHNS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  launch_tau_floor_count(m, make_coef(*p, m->lo, m->hi), ut, dl, cnt, st);
  TRY(check_launch());
  CHNS_CUDA_TRY(cudaMemcpyAsync(ws.hpinned, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CHNS_CUDA_TRY(cudaStreamSynchronize(st));
  unsigned long long v = 0;
  std::memcpy(&v, ws.hpinned, sizeof(v));
  *count = (int64_t)v;
  return CHNS_OK;
}

chns_status chns_mesh_jacvec_schedule(chns_mesh *m, int variant, int *current, double *times_ms) {
  if (!m) { set_error("null mesh"); return CHNS_ERR_ARG; }
  if (variant < -1 || variant >= kJacvecVariants) { set_error("schedule %d out of range", variant); return CHNS_ERR_ARG; }
  if (variant >= 0) {
    m->jv_variant = variant;
    m->jv_tuned = true;
  }
  if (current) *current = m->jv_variant;
  if (times_ms)
    for (int v = 0; v < kJacvecVariants; ++v) times_ms[v] = m->jv_times[v];
  return CHNS_OK;
}

chns_status chns_mesh_check(const chns_mesh *m) {
  if (!m) { set_error("null mesh"); return CHNS_ERR_ARG; }
  return validate_mesh(m);
}

chns_status chns_energy_mass(const chns_mesh *mc, const chns_params *p, const double *U, double *energy,
                             double *mass, double *bubble_mass, void *stream) {
  TRY(check_params(mc, p));
  if (!U) { set_error("null vector"); return CHNS_ERR_ARG; }
  double em[3];
  TRY(energy_mass_impl(const_cast<chns_mesh *>(mc), p, U, em, S(stream)));
  if (energy) *energy = em[0];
  if (mass) *mass = em[1];
  if (bubble_mass) *bubble_mass = em[2];
  return CHNS_OK;
}

chns_status chns_batch_create(int n, chns_mesh *const *meshes, const chns_params *params, chns_batch **out) {
  if (!out || n <= 0 || !meshes || !params) { set_error("invalid batch arguments"); return CHNS_ERR_ARG; }
  *out = nullptr;
  for (int i = 0; i < n; ++i) TRY(check_params(meshes[i], &params[i]));
  chns_batch *b = new chns_batch;
  b->meshes.assign(meshes, meshes + n);
  b->params.assign(params, params + n);
  for (int dim = 2; dim <= 3; ++dim) {
    BatchGroup g;
    std::vector<const chns_mesh *> ms;
    std::vector<PhysCoef> pcs;
    for (int i = 0; i < n; ++i)
      if (meshes[i]->dim == dim) {
        g.members.push_back(i);
        ms.push_back(meshes[i]);
        pcs.push_back(make_coef(params[i], meshes[i]->lo, meshes[i]->hi));
      }
    if (ms.empty()) continue;
    g.u = new chns_mesh;
    chns_status s = build_union(ms, g.u);
    if (s == CHNS_OK) s = build_gather(g.u);
    if (s == CHNS_OK) s = upload_coef_tables(g.u, pcs, nullptr);
    if (s != CHNS_OK) {
      chns_mesh_destroy(g.u);
      for (auto &h : b->groups) chns_mesh_destroy(h.u);
      delete b;
      return s;
    }
    b->groups.push_back(std::move(g));
  }
  *out = b;
  return CHNS_OK;
}

chns_status chns_batch_step(chns_batch *b, const chns_solver_opts *o, double *const *U_n, double *const *U_nm1,
                            double *const *U_np1, chns_step_stats *stats, void *stream) {
  if (!b || !o || !U_n || !U_np1) { set_error("null argument"); return CHNS_ERR_ARG; }
  cudaStream_t st = S(stream);
  for (auto &g : b->groups) {
    chns_mesh *u = g.u;
    const int64_t n = u->n_nodes * u->nf;
    TRY(g.Un.ensure(sizeof(double) * n));
    TRY(g.Unp1.ensure(sizeof(double) * n));
    if (U_nm1) TRY(g.Unm1.ensure(sizeof(double) * n));
    double *un = g.Un.as<double>(), *up = g.Unp1.as<double>(), *um = U_nm1 ? g.Unm1.as<double>() : nullptr;
    for (size_t q = 0; q < g.members.size(); ++q) {
      const int i = g.members[q];
      const int64_t a = u->inst_node_start[q] * u->nf, len = (u->inst_node_start[q + 1] - u->inst_node_start[q]) * u->nf;
      if (!U_n[i] || !U_np1[i]) { set_error("null vector of instance %d", i); return CHNS_ERR_ARG; }
      CHNS_CUDA_TRY(cudaMemcpyAsync(un + a, U_n[i], sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
      if (um) {
        if (!U_nm1[i]) { set_error("U_nm1 given but null for instance %d", i); return CHNS_ERR_ARG; }
        CHNS_CUDA_TRY(cudaMemcpyAsync(um + a, U_nm1[i], sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
      }
    }
    chns_step_stats gs;
    std::memset(&gs, 0, sizeof(gs));
    auto t0 = std::chrono::steady_clock::now();
    chns_status s = newton_step(u, &b->params[g.members[0]], *o, un, um, nullptr, nullptr, up, &gs, st);
    if (s != CHNS_OK) return s;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (size_t q = 0; q < g.members.size(); ++q) {
      const int i = g.members[q];
      const int64_t a = u->inst_node_start[q] * u->nf, len = (u->inst_node_start[q + 1] - u->inst_node_start[q]) * u->nf;
      CHNS_CUDA_TRY(cudaMemcpyAsync(U_np1[i], up + a, sizeof(double) * len, cudaMemcpyDeviceToDevice, st));
      if (stats) {
        chns_step_stats &x = stats[i];
        x = gs;  // shared Newton / Krylov counts and timings of the group
        x.seconds = secs;
        double em[3];
        TRY(energy_mass_impl(b->meshes[i], &b->params[i], U_n[i], em, st));
        x.energy_old = em[0];
        x.mass_old = em[1];
        TRY(energy_mass_impl(b->meshes[i], &b->params[i], U_np1[i], em, st));
        x.energy_new = em[0];
        x.mass_new = em[1];
      }
    }
  }
  return CHNS_OK;
}

void chns_batch_destroy(chns_batch *b) {
  if (!b) return;
  for (auto &g : b->groups) {
    chns_mesh_destroy(g.u);
    g.Un.release();
    g.Unm1.release();
    g.Unp1.release();
  }
  delete b;
}

}  // extern "C"
