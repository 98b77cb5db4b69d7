// Geometric multigrid preconditioner over the octree hierarchy for the Krylov
// solve of Sec. 3.5 (the paper preconditioned with algebraic multigrid and
// additive Schwarz on assembled matrices; this is a matrix-free geometric
// counterpart on the octree levels of Sec. 4).
//
// Hierarchy.  Level 0 is the mesh itself.  Level l+1 merges every family of
// leaves at the finest leaf level of level l into their parent; merging the
// finest leaves of a 2:1 balanced octree keeps it 2:1 balanced, and the
// meshes are nested (each coarse leaf is a fine leaf or the parent of 2^d
// fine leaves).  Coarsening stops at a uniform octree level L_b (the
// "bottom").
//
// Operators.  Level l applies the same CN-VMS Jacobian-vector product as the
// fine mesh (the element kernel on the level's own leaves, so the
// stabilisation parameters see the level's element size), linearised at the
// fine state injected to the level's nodes (every coarse node is a node of
// the finer mesh).  The bottom level is solved exactly: its operator is
// probed into a dense matrix and inverted (coarse.cu, with the coarse grid
// equal to the bottom mesh).
//
// Transfers.  P_l (level l -> l-1) evaluates the level-l Q1 field, hanging
// constraints included, at the nodes of level l-1; restriction is P_l^T.
// Both are stored as node lists with dyadic weights (exact in float) and
// applied by gathers in a fixed order: no atomics, deterministic.  The
// constrained rows (wall velocities, the pinned pressure) are homogeneous on
// the coarse levels: restricted residuals and prolonged corrections are zero
// there.
//
// Cycle.  V-cycle with nu pre- and nu post-smoothing sweeps of damped nodal
// block-Jacobi, x <- x + omega D^{-1} (b - A x), D the probed nodal diagonal
// blocks of the level's operator.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "chns_internal.h"
#include "coarse.h"
#include "host_util.h"
#include "kernels.h"
#include "multigrid.h"
#include "solver.h"

namespace chns {

chns_status build_mesh(int dim, int64_t n, const uint8_t *level, const uint32_t *anchor, int max_level,
                       const double lo[3], const double hi[3], chns_mesh *m);
chns_status build_gather(chns_mesh *m);
chns_status build_union(const std::vector<const chns_mesh *> &ms, chns_mesh *u);

namespace {

constexpr int kB = 256;

inline unsigned grid_n(int64_t n) {
  int64_t b = (n + kB - 1) / kB;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}

#define TRY_MG(expr)               \
  do {                             \
    chns_status s_ = (expr);       \
    if (s_ != CHNS_OK) return s_;  \
  } while (0)

// ---------------------------------------------------------------- kernels
// prepared state of level l from level l-1 at the same node positions
template <typename T, int NF>
__global__ void k_inject(int64_t n, const int32_t *__restrict__ inj, const T *__restrict__ utf,
                         const T *__restrict__ dlf, T *__restrict__ utc, T *__restrict__ dlc) {
  constexpr int ND = NF - 2;
  for (int64_t j = blockIdx.x * int64_t(kB) + threadIdx.x; j < n; j += int64_t(gridDim.x) * kB) {
    const int64_t i = inj[j];
#pragma unroll
    for (int k = 0; k < NF; ++k) utc[j * NF + k] = utf[i * NF + k];
#pragma unroll
    for (int k = 0; k < ND; ++k) dlc[j * ND + k] = dlf[i * ND + k];
  }
}

template <typename T, int NF>
__device__ __forceinline__ void block_mv(const T *__restrict__ B, int64_t i, const T *r, T *out) {
  const T *b = B + i * NF * NF;
#pragma unroll
  for (int q = 0; q < NF; ++q) {
    T s = T(0);
#pragma unroll
    for (int c = 0; c < NF; ++c) s = fma(b[q * NF + c], r[c], s);
    out[q] = s;
  }
}

// x = B b (y == nullptr), or x += B (b - y): one damped block-Jacobi sweep
template <typename T, int NF>
__global__ void __launch_bounds__(kB) k_smooth(int64_t n, const T *__restrict__ B, const T *__restrict__ b,
                                               const T *__restrict__ y, T *__restrict__ x) {
  for (int64_t i = blockIdx.x * int64_t(kB) + threadIdx.x; i < n; i += int64_t(gridDim.x) * kB) {
    T r[NF], d[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) r[k] = y ? b[i * NF + k] - y[i * NF + k] : b[i * NF + k];
    block_mv<T, NF>(B, i, r, d);
#pragma unroll
    for (int k = 0; k < NF; ++k) x[i * NF + k] = y ? x[i * NF + k] + d[k] : d[k];
  }
}

// bc[j] = sum over the restriction list of coarse node j of w (b - y)[i];
// zero in the constrained rows of the coarse level.  Eight lanes per coarse
// node (lane s takes the list entries s, s + 8, ...), then a fixed xor
// butterfly over the eight lanes: deterministic, and eight times the
// parallelism of a thread per coarse node on these short scattered lists.
constexpr int kRLanes = 8;
template <typename T, int NF>
__global__ void __launch_bounds__(kB) k_restrict_res(int64_t nc, int dim, const int32_t *__restrict__ rptr,
                                                     const int32_t *__restrict__ rcol, const float *__restrict__ rw,
                                                     const T *__restrict__ b, const T *__restrict__ y,
                                                     const uint8_t *__restrict__ cflag, T *__restrict__ bc) {
  const int64_t j = (blockIdx.x * int64_t(kB) + threadIdx.x) / kRLanes;
  const int sub = threadIdx.x % kRLanes;
  T acc[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) acc[k] = T(0);
  if (j < nc) {
    for (int e = rptr[j] + sub; e < rptr[j + 1]; e += kRLanes) {
      const int64_t i = rcol[e];
      const T w = T(rw[e]);
#pragma unroll
      for (int k = 0; k < NF; ++k) acc[k] = fma(w, b[i * NF + k] - y[i * NF + k], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < NF; ++k)
#pragma unroll
    for (int o = kRLanes / 2; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  if (j < nc && sub == 0) {
    const uint8_t fl = cflag[j];
    if (fl & 1)
      for (int k = 0; k < dim; ++k) acc[k] = T(0);
    if (fl & 2) acc[dim] = T(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) bc[j * NF + k] = acc[k];
  }
}

// x[i] += sum over the prolongation list of fine node i of w xc[j]; nothing
// in the constrained rows of the fine level
template <typename T, int NF>
__global__ void __launch_bounds__(kB) k_prolong_add(int64_t nf_nodes, int dim, const int32_t *__restrict__ pptr,
                                                    const int32_t *__restrict__ pcol, const float *__restrict__ pw,
                                                    const T *__restrict__ xc, const uint8_t *__restrict__ fflag,
                                                    T *__restrict__ x) {
  for (int64_t i = blockIdx.x * int64_t(kB) + threadIdx.x; i < nf_nodes; i += int64_t(gridDim.x) * kB) {
    T acc[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) acc[k] = T(0);
    for (int e = pptr[i]; e < pptr[i + 1]; ++e) {
      const int64_t j = pcol[e];
      const T w = T(pw[e]);
#pragma unroll
      for (int k = 0; k < NF; ++k) acc[k] = fma(w, xc[j * NF + k], acc[k]);
    }
    const uint8_t fl = fflag[i];
    if (fl & 1)
      for (int k = 0; k < dim; ++k) acc[k] = T(0);
    if (fl & 2) acc[dim] = T(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) x[i * NF + k] += acc[k];
  }
}

// ---------------------------------------------------------------- host: hierarchy
struct Leaf {
  uint64_t key;
  uint8_t level;
  uint32_t a[3];
};

// leaves of a built mesh, back in Morton order
std::vector<Leaf> mesh_leaves(const chns_mesh *m) {
  const std::vector<uint8_t> lev = download(m->level, size_t(m->n_elem));
  const std::vector<uint32_t> anc = download(m->anchor, size_t(m->n_elem) * m->dim);
  std::vector<Leaf> out(m->n_elem);
  for (int64_t e = 0; e < m->n_elem; ++e) {
    Leaf &l = out[e];
    l.level = lev[e];
    l.a[0] = l.a[1] = l.a[2] = 0;
    for (int d = 0; d < m->dim; ++d) l.a[d] = anc[e * m->dim + d];
    l.key = morton(l.a, m->dim, m->max_level);
  }
  std::sort(out.begin(), out.end(), [](const Leaf &x, const Leaf &y) { return x.key < y.key; });
  return out;
}

// merge every family of leaves at level lmax into its parent (Morton order
// keeps a family contiguous, its first child carrying the parent's anchor)
std::vector<Leaf> coarsen(const std::vector<Leaf> &in, int dim, int max_level, int lmax) {
  std::vector<Leaf> out;
  out.reserve(in.size());
  const uint32_t ps = uint32_t(1) << (max_level - (lmax - 1));
  for (const Leaf &l : in) {
    if (l.level != lmax) {
      out.push_back(l);
      continue;
    }
    bool first = true;
    for (int d = 0; d < dim; ++d)
      if (l.a[d] % ps != 0) first = false;
    if (!first) continue;
    Leaf p = l;
    p.level = uint8_t(lmax - 1);
    out.push_back(p);
  }
  return out;
}

// Host lists of one problem instance: P (coarse -> fine nodes) as pptr
// (n_fine + 1), pcol, pw; the injection coarse node -> fine node at its
// position.  Local node numbers of F and C.
struct TransferLists {
  std::vector<int32_t> pptr, pcol, inj;
  std::vector<float> pw;
};

chns_status transfer_lists(const chns_mesh *F, const chns_mesh *C, TransferLists &T) {
  const int dim = F->dim, nc = 1 << dim;
  const int ml = F->max_level;
  const int64_t top = int64_t(1) << ml;
  // coarse independent nodes and hanging nodes by position
  KeyMap cnode(size_t(C->n_nodes) + 16);
  for (int64_t j = 0; j < C->n_nodes; ++j) cnode.insert(pack(&C->node_xyz[j * dim], dim), j);
  const std::vector<int32_t> cconn = download(C->conn, size_t(C->n_elem) * nc);
  const std::vector<uint8_t> clev = download(C->level, size_t(C->n_elem));
  const std::vector<uint32_t> canc = download(C->anchor, size_t(C->n_elem) * dim);
  const std::vector<int32_t> chang = download(C->hang, size_t(C->n_hang) * 4);
  KeyMap chpos(size_t(C->n_hang) + 16);
  KeyMap cleaf(size_t(C->n_elem) + 16);
  int lmin = 64, lmax = 0;
  for (int64_t e = 0; e < C->n_elem; ++e) {
    int64_t x[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) x[d] = canc[e * dim + d];
    cleaf.insert(okey(clev[e], x, dim, ml), e);
    lmin = std::min<int>(lmin, clev[e]);
    lmax = std::max<int>(lmax, clev[e]);
    const int64_t s = int64_t(1) << (ml - clev[e]);
    for (int c = 0; c < nc; ++c) {
      const int32_t v = cconn[e * nc + c];
      if (v >= 0) continue;
      int64_t y[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) y[d] = x[d] + (((c >> d) & 1) ? s : 0);
      chpos.insert(pack(y, dim), -v - 1);
    }
  }
  // prolongation lists, fine node by fine node
  std::vector<int32_t> pptr(size_t(F->n_nodes) + 1, 0), pcol;
  std::vector<float> pw;
  pcol.reserve(size_t(F->n_nodes) * 4);
  pw.reserve(size_t(F->n_nodes) * 4);
  for (int64_t i = 0; i < F->n_nodes; ++i) {
    const int64_t *x = &F->node_xyz[i * dim];
    int64_t e = -1, a[3] = {0, 0, 0}, s = 0;
    for (int l = lmax; l >= lmin && e < 0; --l) {
      s = int64_t(1) << (ml - l);
      for (int d = 0; d < dim; ++d) a[d] = std::min(x[d] / s * s, top - s);
      e = cleaf.find(okey(l, a, dim, ml));
    }
    if (e < 0) { set_error("multigrid: fine node %lld lies in no coarse leaf", (long long)i); return CHNS_ERR_MESH; }
    int32_t ids[32];
    double ws[32];
    int cnt = 0;
    auto add = [&](int32_t id, double w) {
      for (int k = 0; k < cnt; ++k)
        if (ids[k] == id) { ws[k] += w; return; }
      ids[cnt] = id;
      ws[cnt++] = w;
    };
    for (int c = 0; c < nc; ++c) {
      double w = 1.0;
      int64_t y[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        const double t = double(x[d] - a[d]) / double(s);
        w *= ((c >> d) & 1) ? t : 1.0 - t;
        y[d] = a[d] + (((c >> d) & 1) ? s : 0);
      }
      if (w == 0.0) continue;
      const int64_t id = cnode.find(pack(y, dim));
      if (id >= 0) {
        add((int32_t)id, w);
      } else {
        const int64_t h = chpos.find(pack(y, dim));
        if (h < 0) { set_error("multigrid: coarse corner is neither a node nor hanging"); return CHNS_ERR_MESH; }
        const int32_t *p = &chang[size_t(h) * 4];
        const int np = p[2] < 0 ? 2 : 4;
        for (int k = 0; k < np; ++k) add(p[k], w / np);
      }
    }
    // fixed order within a list: increasing coarse node
    for (int k = 1; k < cnt; ++k)
      for (int q = k; q > 0 && ids[q - 1] > ids[q]; --q) {
        std::swap(ids[q - 1], ids[q]);
        std::swap(ws[q - 1], ws[q]);
      }
    for (int k = 0; k < cnt; ++k) {
      pcol.push_back(ids[k]);
      pw.push_back(float(ws[k]));
    }
    pptr[i + 1] = (int32_t)pcol.size();
  }
  // injection: coarse node j -> the fine node at its position
  KeyMap fnode(size_t(F->n_nodes) + 16);
  for (int64_t i = 0; i < F->n_nodes; ++i) fnode.insert(pack(&F->node_xyz[i * dim], dim), i);
  std::vector<int32_t> inj(C->n_nodes);
  for (int64_t j = 0; j < C->n_nodes; ++j) {
    const int64_t i = fnode.find(pack(&C->node_xyz[j * dim], dim));
    if (i < 0) { set_error("multigrid: coarse node %lld is not a fine node", (long long)j); return CHNS_ERR_MESH; }
    inj[j] = (int32_t)i;
  }
  T.pptr.swap(pptr);
  T.pcol.swap(pcol);
  T.pw.swap(pw);
  T.inj.swap(inj);
  return CHNS_OK;
}

// identity lists of an instance that is already at the bottom level
void identity_lists(int64_t n, TransferLists &T) {
  T.pptr.resize(n + 1);
  T.pcol.resize(n);
  T.pw.assign(n, 1.0f);
  T.inj.resize(n);
  for (int64_t i = 0; i <= n; ++i) T.pptr[i] = (int32_t)i;
  for (int64_t i = 0; i < n; ++i) T.pcol[i] = T.inj[i] = (int32_t)i;
}

// concatenate the instances' lists (node offsets of the fine and coarse
// union levels), form the restriction P^T (lists in increasing fine node
// order) and upload
chns_status upload_transfer(const std::vector<TransferLists> &parts, const std::vector<int64_t> &foff,
                            const std::vector<int64_t> &coff, MgLevel &L) {
  const int64_t nfine = foff.back(), ncoarse = coff.back();
  std::vector<int32_t> pptr(size_t(nfine) + 1, 0), pcol;
  std::vector<int32_t> inj(static_cast<size_t>(ncoarse), 0);
  std::vector<float> pw;
  for (size_t q = 0; q < parts.size(); ++q) {
    const TransferLists &T = parts[q];
    for (int64_t i = 0; i + 1 < (int64_t)T.pptr.size(); ++i) {
      for (int32_t e = T.pptr[i]; e < T.pptr[i + 1]; ++e) {
        pcol.push_back(int32_t(T.pcol[e] + coff[q]));
        pw.push_back(T.pw[e]);
      }
      pptr[size_t(foff[q] + i) + 1] = (int32_t)pcol.size();
    }
    for (size_t j = 0; j < T.inj.size(); ++j) inj[coff[q] + j] = int32_t(T.inj[j] + foff[q]);
  }
  std::vector<int32_t> rptr(size_t(ncoarse) + 1, 0);
  for (int32_t j : pcol) rptr[size_t(j) + 1]++;
  for (int64_t j = 0; j < ncoarse; ++j) rptr[j + 1] += rptr[j];
  std::vector<int32_t> rcol(pcol.size()), fill(rptr.begin(), rptr.end() - 1);
  std::vector<float> rw(pcol.size());
  for (int64_t i = 0; i < nfine; ++i)
    for (int32_t e = pptr[i]; e < pptr[i + 1]; ++e) {
      const int32_t j = pcol[e];
      rcol[fill[j]] = (int32_t)i;
      rw[fill[j]++] = pw[e];
    }
  TRY_MG(upload(&L.pptr, pptr));
  TRY_MG(upload(&L.pcol, pcol));
  TRY_MG(upload(&L.pw, pw));
  TRY_MG(upload(&L.rptr, rptr));
  TRY_MG(upload(&L.rcol, rcol));
  TRY_MG(upload(&L.rw, rw));
  TRY_MG(upload(&L.inj, inj));
  L.nnz = (int64_t)pcol.size();
  return CHNS_OK;
}

// one level coarser: every family of leaves at the mesh's finest leaf level
// merged (nullptr with CHNS_OK when the mesh is already at or below `bottom`)
chns_status coarser_mesh(const chns_mesh *m, int bottom, chns_mesh **out) {
  *out = nullptr;
  std::vector<Leaf> cur = mesh_leaves(m);
  int lmax = 0;
  for (const Leaf &l : cur) lmax = std::max<int>(lmax, l.level);
  if (lmax <= bottom) return CHNS_OK;
  std::vector<Leaf> nxt = coarsen(cur, m->dim, m->max_level, lmax);
  std::vector<uint8_t> lev(nxt.size());
  std::vector<uint32_t> anc(nxt.size() * m->dim);
  for (size_t e = 0; e < nxt.size(); ++e) {
    lev[e] = nxt[e].level;
    for (int d = 0; d < m->dim; ++d) anc[e * m->dim + d] = nxt[e].a[d];
  }
  chns_mesh *c = new chns_mesh;
  chns_status s = build_mesh(m->dim, (int64_t)nxt.size(), lev.data(), anc.data(), m->max_level, m->lo, m->hi, c);
  if (s == CHNS_OK) s = build_gather(c);
  if (s != CHNS_OK) {
    chns_mesh_destroy(c);
    return s;
  }
  *out = c;
  return CHNS_OK;
}

void free_level(MgLevel &L, bool own_mesh) {
  cudaFree(L.pptr); cudaFree(L.pcol); cudaFree(L.pw);
  cudaFree(L.rptr); cudaFree(L.rcol); cudaFree(L.rw);
  cudaFree(L.inj);
  L.pptr = L.pcol = L.rptr = L.rcol = L.inj = nullptr;
  L.pw = L.rw = nullptr;
  for (int k = 0; k < 2; ++k) {
    L.ut[k].release();
    L.dl[k].release();
    L.binv[k].release();
  }
  L.x.release(); L.b.release(); L.y.release();
  if (own_mesh && L.mesh) chns_mesh_destroy(L.mesh);
  L.mesh = nullptr;
}

}  // namespace

void mg_release(Multigrid *g) {
  if (!g) return;
  for (size_t l = 0; l < g->lv.size(); ++l) free_level(g->lv[l], l > 0);
  delete g;
}

chns_status mg_setup(chns_mesh *m, int bottom) {
  // instances: the mesh itself, or the problem instances of a batch union
  std::vector<const chns_mesh *> inst = m->n_inst > 1 ? m->inst_meshes : std::vector<const chns_mesh *>{m};
  if ((int)inst.size() != m->n_inst) { set_error("multigrid: union mesh without its instance meshes"); return CHNS_ERR_ARG; }
  int minl = 64;
  for (const chns_mesh *q : inst) minl = std::min(minl, q->min_level);
  bottom = std::max(1, std::min(bottom, minl));
  if (m->mg && m->mg->bottom_level == bottom) return CHNS_OK;
  mg_release(m->mg);
  m->mg = new Multigrid;
  Multigrid &G = *m->mg;
  G.bottom_level = bottom;
  G.lv.resize(1);
  G.lv[0].mesh = m;
  // per instance: its meshes level by level (level 0 not owned)
  const size_t ni = inst.size();
  std::vector<std::vector<chns_mesh *>> chain(ni);
  std::vector<size_t> owned;  // chain[0] entries already owned by a level
  auto release_chains = [&]() {
    for (auto &c : chain)
      for (size_t l = 1; l < c.size(); ++l)
        if (c[l]) chns_mesh_destroy(c[l]);
    chain.clear();
  };
  auto fail = [&](chns_status s) {
    for (size_t l : owned) chain[0][l] = nullptr;
    release_chains();
    mg_release(m->mg);
    m->mg = nullptr;
    return s;
  };
  size_t depth = 0;
  for (size_t q = 0; q < ni; ++q) {
    chain[q].push_back(const_cast<chns_mesh *>(inst[q]));
    while (true) {
      chns_mesh *c = nullptr;
      chns_status s = coarser_mesh(chain[q].back(), bottom, &c);
      if (s != CHNS_OK) return fail(s);
      if (!c) break;
      chain[q].push_back(c);
    }
    depth = std::max(depth, chain[q].size() - 1);
  }
  // single instance: the chain's coarse meshes become the levels' meshes
  // (ownership moves to the level as it is pushed); a union: each level is
  // the union of the instances' meshes of that level (an instance already at
  // the bottom repeats its bottom mesh, with identity transfers)
  for (size_t l = 1; l <= depth; ++l) {
    MgLevel L;
    std::vector<const chns_mesh *> ms(ni);
    std::vector<TransferLists> parts(ni);
    for (size_t q = 0; q < ni; ++q) {
      const size_t lf = std::min(l - 1, chain[q].size() - 1), lc = std::min(l, chain[q].size() - 1);
      ms[q] = chain[q][lc];
      chns_status s = CHNS_OK;
      if (lf == lc) identity_lists(chain[q][lc]->n_nodes, parts[q]);
      else s = transfer_lists(chain[q][lf], chain[q][lc], parts[q]);
      if (s != CHNS_OK) return fail(s);
    }
    chns_status s = CHNS_OK;
    if (ni == 1) {
      L.mesh = chain[0][l];
    } else {
      L.mesh = new chns_mesh;
      s = build_union(ms, L.mesh);
      if (s == CHNS_OK) s = build_gather(L.mesh);
      if (s == CHNS_OK) s = copy_coef_tables(m, L.mesh);
    }
    const chns_mesh *F = G.lv[l - 1].mesh;
    if (s == CHNS_OK) s = upload_transfer(parts, F->inst_node_start, L.mesh->inst_node_start, L);
    if (s != CHNS_OK) {
      if (ni == 1) L.mesh = nullptr;  // still owned by the chain
      free_level(L, true);
      return fail(s);
    }
    G.lv.push_back(L);
    if (ni == 1) owned.push_back(l);
  }
  for (size_t l : owned) chain[0][l] = nullptr;  // now owned by the levels
  release_chains();
  // the bottom level is solved exactly: coarse grid = the bottom mesh itself
  chns_mesh *b = G.lv.back().mesh;
  if (!b->uniform || b->min_level != bottom) {
    set_error("multigrid: the coarsest mesh is not uniform at level %d", bottom);
    mg_release(m->mg);
    m->mg = nullptr;
    return CHNS_ERR_MESH;
  }
  chns_status s = coarse_setup(b, bottom);
  if (s != CHNS_OK) {
    mg_release(m->mg);
    m->mg = nullptr;
  }
  return s;
}

template <typename T>
static void launch_inject(const chns_mesh *c, const int32_t *inj, const T *utf, const T *dlf, T *utc, T *dlc,
                          cudaStream_t st) {
  if (c->nf == 5) k_inject<T, 5><<<grid_n(c->n_nodes), kB, 0, st>>>(c->n_nodes, inj, utf, dlf, utc, dlc);
  else k_inject<T, 6><<<grid_n(c->n_nodes), kB, 0, st>>>(c->n_nodes, inj, utf, dlf, utc, dlc);
  note_launches(1);
}

template <typename T>
static chns_status jv_level(void *ctx, const T *w, T *y);

namespace {
template <typename T>
struct LevelCtx {
  chns_mesh *m;
  const PhysCoef *pc;
  const T *ut, *dl;
  cudaStream_t st;
};
}  // namespace

template <typename T>
static chns_status jv_level(void *ctx, const T *w, T *y) {
  LevelCtx<T> *c = static_cast<LevelCtx<T> *>(ctx);
  return jacvec_prepared<T>(c->m, *c->pc, c->ut, c->dl, w, y, c->st);
}

template <typename T>
constexpr int prec_index() { return sizeof(T) == 8 ? 1 : 0; }

template <typename T>
chns_status mg_update_state(chns_mesh *m, const T *ut0, const T *dl0, cudaStream_t st) {
  Multigrid &G = *m->mg;
  constexpr int P = prec_index<T>();
  const T *uf = ut0, *df = dl0;
  for (size_t l = 1; l < G.lv.size(); ++l) {
    MgLevel &L = G.lv[l];
    chns_mesh *c = L.mesh;
    TRY_MG(L.ut[P].ensure(sizeof(T) * c->n_nodes * c->nf));
    TRY_MG(L.dl[P].ensure(sizeof(T) * c->n_nodes * (c->dim + 1)));
    launch_inject<T>(c, L.inj, uf, df, L.ut[P].as<T>(), L.dl[P].as<T>(), st);
    uf = L.ut[P].as<T>();
    df = L.dl[P].as<T>();
  }
  return check_launch();
}

template <typename T>
chns_status mg_build(chns_mesh *m, const PhysCoef &pc, const T *ut0, const T *dl0, double omega, int smooth,
                     cudaStream_t st, bool keep_other) {
  Multigrid &G = *m->mg;
  constexpr int P = prec_index<T>();
  G.omega = omega;
  G.smooth = smooth;
  G.ready[P] = false;
  if (!keep_other) G.ready[1 - P] = false;
  TRY_MG(mg_update_state<T>(m, ut0, dl0, st));
  const size_t nl = G.lv.size();
  for (size_t l = 0; l < nl; ++l) {
    MgLevel &L = G.lv[l];
    chns_mesh *c = L.mesh;
    const T *ut = l == 0 ? ut0 : L.ut[P].as<T>();
    const T *dl = l == 0 ? dl0 : L.dl[P].as<T>();
    const int64_t n = c->n_nodes * c->nf;
    TRY_MG(L.x.ensure(sizeof(double) * n + 16));
    TRY_MG(L.b.ensure(sizeof(double) * n + 16));
    TRY_MG(L.y.ensure(sizeof(double) * n + 16));
    T *E = nullptr;
    TRY_MG(ensure_ebuf<T>(c, &E));  // before any graph capture: nothing allocates inside a V-cycle
    if (sizeof(T) == sizeof(float) && G.autotune && l > 0 && !c->jv_tuned)
      TRY_MG(autotune_jacvec(c, pc, reinterpret_cast<const float *>(ut), reinterpret_cast<const float *>(dl), st));
    if (l + 1 < nl) {
      TRY_MG(build_block_jacobi<T>(c, pc, ut, dl, L.binv[P], st, omega));
    } else {
      // bottom: dense inverse of the level's own operator (coarse grid = this mesh)
      TRY_MG(c->ws.wv.ensure(sizeof(T) * n));
      TRY_MG(c->ws.yv.ensure(sizeof(T) * n));
      LevelCtx<T> ctx{c, &pc, ut, dl, st};
      TRY_MG(coarse_build<T>(c, &jv_level<T>, &ctx, c->ws.wv.as<T>(), c->ws.yv.as<T>(), st));
    }
  }
  G.ready[P] = true;
  ++G.generation;
  return check_launch();
}

template <typename T>
chns_status mg_apply(chns_mesh *m, const PhysCoef &pc, const T *ut0, const T *dl0, const T *v, T *z,
                     cudaStream_t st) {
  Multigrid &G = *m->mg;
  const int nl = (int)G.lv.size();
  const int nu = std::max(1, G.smooth);
  auto X = [&](int l) -> T * { return l == 0 ? z : G.lv[l].x.as<T>(); };
  auto B = [&](int l) -> const T * { return l == 0 ? v : G.lv[l].b.as<T>(); };
  constexpr int P = prec_index<T>();
  auto UT = [&](int l) -> const T * { return l == 0 ? ut0 : G.lv[l].ut[P].as<T>(); };
  auto DL = [&](int l) -> const T * { return l == 0 ? dl0 : G.lv[l].dl[P].as<T>(); };
  auto smooth_k = [&](int l, const T *y) {
    chns_mesh *c = G.lv[l].mesh;
    const T *Bi = G.lv[l].binv[P].as<T>();
    if (c->nf == 5) k_smooth<T, 5><<<grid_n(c->n_nodes), kB, 0, st>>>(c->n_nodes, Bi, B(l), y, X(l));
    else k_smooth<T, 6><<<grid_n(c->n_nodes), kB, 0, st>>>(c->n_nodes, Bi, B(l), y, X(l));
    note_launches(1);
  };
  // down
  for (int l = 0; l + 1 < nl; ++l) {
    chns_mesh *c = G.lv[l].mesh;
    T *y = G.lv[l].y.as<T>();
    smooth_k(l, nullptr);
    for (int s = 1; s < nu; ++s) {
      TRY_MG(jacvec_prepared<T>(c, pc, UT(l), DL(l), X(l), y, st));
      smooth_k(l, y);
    }
    TRY_MG(jacvec_prepared<T>(c, pc, UT(l), DL(l), X(l), y, st));
    const MgLevel &Lc = G.lv[l + 1];
    chns_mesh *cc = Lc.mesh;
    T *bc = G.lv[l + 1].b.as<T>();
    const unsigned gr = (unsigned)((cc->n_nodes * kRLanes + kB - 1) / kB);  // every coarse node one pass
    if (c->nf == 5)
      k_restrict_res<T, 5><<<gr, kB, 0, st>>>(cc->n_nodes, c->dim, Lc.rptr, Lc.rcol, Lc.rw, B(l), y, cc->nflag, bc);
    else
      k_restrict_res<T, 6><<<gr, kB, 0, st>>>(cc->n_nodes, c->dim, Lc.rptr, Lc.rcol, Lc.rw, B(l), y, cc->nflag, bc);
    note_launches(1);
  }
  // bottom: exact solve
  precond_apply<T>(G.lv[nl - 1].mesh, nullptr, true, B(nl - 1), X(nl - 1), st);
  // up
  for (int l = nl - 2; l >= 0; --l) {
    chns_mesh *c = G.lv[l].mesh;
    const MgLevel &Lc = G.lv[l + 1];
    T *y = G.lv[l].y.as<T>();
    if (c->nf == 5)
      k_prolong_add<T, 5><<<grid_n(c->n_nodes), kB, 0, st>>>(c->n_nodes, c->dim, Lc.pptr, Lc.pcol, Lc.pw, X(l + 1),
                                                             c->nflag, X(l));
    else
      k_prolong_add<T, 6><<<grid_n(c->n_nodes), kB, 0, st>>>(c->n_nodes, c->dim, Lc.pptr, Lc.pcol, Lc.pw, X(l + 1),
                                                             c->nflag, X(l));
    note_launches(1);
    for (int s = 0; s < nu; ++s) {
      TRY_MG(jacvec_prepared<T>(c, pc, UT(l), DL(l), X(l), y, st));
      smooth_k(l, y);
    }
  }
  return CHNS_OK;
}

template chns_status mg_update_state<float>(chns_mesh *, const float *, const float *, cudaStream_t);
template chns_status mg_update_state<double>(chns_mesh *, const double *, const double *, cudaStream_t);
template chns_status mg_build<float>(chns_mesh *, const PhysCoef &, const float *, const float *, double, int,
                                     cudaStream_t, bool);
template chns_status mg_build<double>(chns_mesh *, const PhysCoef &, const double *, const double *, double, int,
                                      cudaStream_t, bool);
template chns_status mg_apply<float>(chns_mesh *, const PhysCoef &, const float *, const float *, const float *,
                                     float *, cudaStream_t);
template chns_status mg_apply<double>(chns_mesh *, const PhysCoef &, const double *, const double *, const double *,
                                      double *, cudaStream_t);

}  // namespace chns
