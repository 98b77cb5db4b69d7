// Mesh construction from octree leaves (Sec. 4 "Meshing", "Handling hanging
// nodes", "2:1 Balancing"): validation, node numbering, hanging-node
// constraints, element and node colourings, upload to the device.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <thread>

#include "chns_internal.h"
#include "host_util.h"

namespace chns {

namespace {
thread_local std::string g_last_error;
}

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char *last_error() { return g_last_error.c_str(); }

namespace {
std::atomic<uint64_t> g_launches{0};
}
thread_local int *t_capture_sink = nullptr;
void note_launches(int n) {
  if (t_capture_sink) *t_capture_sink += n;  // captured into a graph: counted per replay
  else g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed);
}
void set_capture_sink(int *sink) { t_capture_sink = sink; }
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

chns_status DevBuf::ensure(size_t n) {
  if (n <= bytes && p) return CHNS_OK;
  release();
  if (n == 0) return CHNS_OK;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    set_error("cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CHNS_ERR_OOM : CHNS_ERR_CUDA;
  }
  bytes = n;
  return CHNS_OK;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

void Workspace::StepGraphs::clear() {
  for (auto g : exec)
    if (g) cudaGraphExecDestroy(g);
  for (auto e : jv) cudaEventDestroy(e);
  exec.clear();
  launches.clear();
  jv.clear();
  key.clear();
}

Workspace::~Workspace() {
  kg[0].clear();
  kg[1].clear();
  if (cap) cudaStreamDestroy(cap);
  for (auto e : ev) cudaEventDestroy(e);
  for (auto e : tev) cudaEventDestroy(e);
  if (hpinned) cudaFreeHost(hpinned);
}

chns_status build_mesh(int dim, int64_t n, const uint8_t *level, const uint32_t *anchor,
                       int max_level, const double lo[3], const double hi[3], chns_mesh *m) {
  if (dim != 2 && dim != 3) { set_error("dim must be 2 or 3"); return CHNS_ERR_ARG; }
  if (n <= 0 || !level || !anchor) { set_error("no leaves"); return CHNS_ERR_ARG; }
  if (max_level < 0 || max_level > 20) { set_error("max_level must be in [0, 20]"); return CHNS_ERR_ARG; }
  if (n > (int64_t(1) << 31) / 8) { set_error("too many leaves"); return CHNS_ERR_ARG; }
  m->dim = dim;
  m->max_level = max_level;
  m->nc = 1 << dim;
  m->nf = dim + 3;
  m->n_elem = n;
  for (int a = 0; a < 3; ++a) {
    m->lo[a] = lo ? lo[a] : 0.0;
    m->hi[a] = hi ? hi[a] : 1.0;
    if (a < dim && !(m->hi[a] > m->lo[a])) { set_error("empty box"); return CHNS_ERR_ARG; }
  }
  const int nc = m->nc;
  const int64_t top = int64_t(1) << max_level;

  // --- leaves: alignment, Morton order, exact tiling of the box
  uint64_t expect = 0;
  bool uniform = true;
  for (int64_t e = 0; e < n; ++e) {
    int l = level[e];
    if (l > max_level) { set_error("leaf %lld: level %d > max_level", (long long)e, l); return CHNS_ERR_MESH; }
    if (l != level[0]) uniform = false;
    int64_t s = int64_t(1) << (max_level - l);
    for (int a = 0; a < dim; ++a) {
      int64_t x = anchor[e * dim + a];
      if (x % s != 0 || x + s > top) {
        set_error("leaf %lld: anchor not aligned to its level or outside the box", (long long)e);
        return CHNS_ERR_MESH;
      }
    }
    uint64_t k = morton(anchor + e * dim, dim, max_level);
    if (k != expect) {
      set_error("leaves are not in Morton order or do not tile the box (leaf %lld)", (long long)e);
      return CHNS_ERR_MESH;
    }
    expect = k + (uint64_t(1) << (dim * (max_level - l)));
  }
  if (expect != (uint64_t(1) << (dim * max_level))) {
    set_error("leaves do not cover the box");
    return CHNS_ERR_MESH;
  }
  m->uniform = uniform;
  m->min_level = max_level;
  for (int64_t e = 0; e < n; ++e) m->min_level = std::min<int>(m->min_level, level[e]);

  // --- 2:1 balance across faces, edges and corners: every same-level
  // neighbour of a leaf has its parent among the leaves or their ancestors.
  {
    KeyMap oct(size_t(n) * 2);
    for (int64_t e = 0; e < n; ++e) {
      int64_t x[3];
      for (int a = 0; a < dim; ++a) x[a] = anchor[e * dim + a];
      int l = level[e];
      oct.insert(okey(l, x, dim, max_level), 1);
      while (l > 0) {
        --l;
        int64_t s = int64_t(1) << (max_level - l);
        for (int a = 0; a < dim; ++a) x[a] = (x[a] / s) * s;
        if (!oct.insert(okey(l, x, dim, max_level), 1).second) break;
      }
    }
    // the parents of the 3^dim - 1 neighbour cells: per axis the cells at
    // a - s, a, a + s inside the box have at most two distinct parents, so
    // at most 2^dim parents to look up (the leaf's own is always present);
    // leaves checked on host threads, the first unbalanced one reported
    std::atomic<int64_t> first_bad{n};
    parallel_for(n, 16384, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1 && e < first_bad.load(std::memory_order_relaxed); ++e) {
      int l = level[e];
      if (l <= 1) continue;
      int64_t s = int64_t(1) << (max_level - l);
      int64_t ps = s * 2;
      int64_t cand[3][2] = {{0, 0}, {0, 0}, {0, 0}};
      int nc3[3] = {1, 1, 1};
      for (int a = 0; a < dim; ++a) {
        const int64_t x0 = anchor[e * dim + a];
        int cnt = 0;
        for (int o = -1; o <= 1; ++o) {
          const int64_t x = x0 + o * s;
          if (x < 0 || x >= top) continue;
          const int64_t p = (x / ps) * ps;
          if (cnt == 0 || cand[a][cnt - 1] != p) cand[a][cnt++] = p;
        }
        nc3[a] = cnt;
      }
      bool ok = true;
      for (int i0 = 0; i0 < nc3[0] && ok; ++i0)
        for (int i1 = 0; i1 < nc3[1] && ok; ++i1)
          for (int i2 = 0; i2 < nc3[2] && ok; ++i2) {
            int64_t x[3] = {cand[0][i0], cand[1][i1], cand[2][i2]};
            if (oct.find(okey(l - 1, x, dim, max_level)) < 0) ok = false;
          }
      if (!ok) {
        int64_t cur = first_bad.load();
        while (e < cur && !first_bad.compare_exchange_weak(cur, e)) {
        }
        break;
      }
    }
    });
    if (first_bad.load() < n) {
      set_error("mesh is not 2:1 balanced at leaf %lld", (long long)first_bad.load());
      return CHNS_ERR_MESH;
    }
  }

  // --- nodes: unique corners in first-appearance order.  The corner keys are
  // split into shards by a hash; each shard's map is filled by one thread
  // scanning all corners in order, so it keeps every key's first corner; the
  // node ids then follow the first corners in corner order.
  const int64_t n_slots = n * nc;
  std::vector<uint64_t> ckey(static_cast<size_t>(n_slots));
  parallel_for(n, 16384, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e) {
      int64_t s = int64_t(1) << (max_level - level[e]);
      for (int c = 0; c < nc; ++c) {
        int64_t x[3];
        for (int a = 0; a < dim; ++a) x[a] = anchor[e * dim + a] + (((c >> a) & 1) ? s : 0);
        ckey[e * nc + c] = pack(x, dim);
      }
    }
  });
  const int n_shards = int(std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>(std::thread::hardware_concurrency(), 64), n_slots / 65536 + 1)));
  auto shard_of = [n_shards](uint64_t k) {
    k ^= k >> 31;
    k *= 0x7fb5d329728ea185ull;
    k ^= k >> 27;
    return int((k >> 32) % uint64_t(n_shards));
  };
  std::vector<KeyMap> shard;
  shard.reserve(n_shards);
  for (int t = 0; t < n_shards; ++t) shard.emplace_back(size_t(n) * (dim == 2 ? 2 : 3) / n_shards + 64);
  parallel_for(n_shards, 1, [&](int64_t t0, int64_t t1) {
    for (int64_t t = t0; t < t1; ++t)
      for (int64_t k = 0; k < n_slots; ++k)
        if (shard_of(ckey[k]) == t) shard[t].insert(ckey[k], k);
  });
  std::vector<int32_t> first(static_cast<size_t>(n_slots));
  parallel_for(n_slots, 65536, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) first[k] = (int32_t)shard[shard_of(ckey[k])].find(ckey[k]);
  });
  std::vector<int64_t> all_xyz;
  std::vector<int32_t> corner_all(static_cast<size_t>(n_slots));
  all_xyz.reserve(size_t(n) * (dim == 2 ? 2 : 3) * dim);
  for (int64_t k = 0; k < n_slots; ++k) {
    if (first[k] == k) {
      corner_all[k] = (int32_t)(all_xyz.size() / dim);
      const int64_t e = k / nc;
      const int c = int(k % nc);
      const int64_t s = int64_t(1) << (max_level - level[e]);
      for (int a = 0; a < dim; ++a) all_xyz.push_back(anchor[e * dim + a] + (((c >> a) & 1) ? s : 0));
    } else {
      corner_all[k] = corner_all[first[k]];
    }
  }
  // node id of a point key, -1 if no leaf has a corner there
  auto node_find = [&](uint64_t key) -> int64_t {
    const int64_t f = shard[shard_of(key)].find(key);
    return f < 0 ? -1 : corner_all[f];
  };
  const int64_t n_all = (int64_t)(all_xyz.size() / dim);

  // --- hanging nodes: a node at the midpoint of an edge, or the centre of a
  // face, of some leaf; constrained to the mean of that edge's / face's corners
  std::vector<int32_t> hang_of(n_all, -1);
  std::vector<int32_t> hang_par;  // 4 per hanging node, all-node ids
  for (int64_t e = 0; e < n; ++e) {
    if (level[e] >= max_level) continue;
    int64_t s = int64_t(1) << (max_level - level[e]);
    int npat = dim == 2 ? 9 : 27;
    for (int pat = 0; pat < npat; ++pat) {
      int ch[3], t = pat, nhalf = 0;
      for (int a = 0; a < dim; ++a) { ch[a] = t % 3; t /= 3; nhalf += ch[a] == 1; }
      if (nhalf == 0 || nhalf == dim) continue;
      int64_t x[3];
      for (int a = 0; a < dim; ++a) x[a] = anchor[e * dim + a] + ch[a] * (s / 2);
      int64_t id = node_find(pack(x, dim));
      if (id < 0) continue;
      int32_t par[4] = {-1, -1, -1, -1};
      for (int b = 0; b < (1 << nhalf); ++b) {
        int64_t y[3];
        int bit = 0;
        for (int a = 0; a < dim; ++a) {
          if (ch[a] == 1) y[a] = anchor[e * dim + a] + (((b >> bit++) & 1) ? s : 0);
          else y[a] = anchor[e * dim + a] + (ch[a] == 2 ? s : 0);
        }
        int64_t pid = node_find(pack(y, dim));
        if (pid < 0) { set_error("hanging node parent missing (mesh not conforming)"); return CHNS_ERR_MESH; }
        par[b] = (int32_t)pid;
      }
      std::sort(par, par + (1 << nhalf));
      if (hang_of[id] < 0) {
        hang_of[id] = (int32_t)(hang_par.size() / 4);
        hang_par.insert(hang_par.end(), par, par + 4);
      } else {
        const int32_t *q = &hang_par[size_t(hang_of[id]) * 4];
        for (int b = 0; b < 4; ++b)
          if (q[b] != par[b]) { set_error("inconsistent hanging-node constraint"); return CHNS_ERR_MESH; }
      }
    }
  }
  const int64_t n_hang = (int64_t)(hang_par.size() / 4);
  for (int64_t h = 0; h < n_hang * 4; ++h)
    if (hang_par[h] >= 0 && hang_of[hang_par[h]] >= 0) {
      set_error("hanging node constrained by another hanging node (mesh not 2:1 balanced)");
      return CHNS_ERR_MESH;
    }

  // --- independent node numbering (first-appearance order)
  std::vector<int32_t> indep_id(n_all, -1);
  int64_t n_nodes = 0;
  std::vector<int64_t> node_xyz;
  node_xyz.reserve(size_t(n_all - n_hang) * dim);
  for (int64_t i = 0; i < n_all; ++i)
    if (hang_of[i] < 0) {
      indep_id[i] = (int32_t)n_nodes++;
      for (int a = 0; a < dim; ++a) node_xyz.push_back(all_xyz[i * dim + a]);
    }
  std::vector<int32_t> hang_dev(size_t(n_hang) * 4);
  for (int64_t h = 0; h < n_hang * 4; ++h) hang_dev[h] = hang_par[h] >= 0 ? indep_id[hang_par[h]] : -1;
  std::vector<int32_t> conn(size_t(n) * nc);
  for (int64_t k = 0; k < n * nc; ++k) {
    int32_t id = corner_all[k];
    conn[k] = hang_of[id] >= 0 ? -(hang_of[id] + 1) : indep_id[id];
  }
  std::vector<int32_t> wall;
  m->origin = -1;
  for (int64_t i = 0; i < n_nodes; ++i) {
    bool w = false, org = true;
    for (int a = 0; a < dim; ++a) {
      int64_t c = node_xyz[i * dim + a];
      if (c == 0 || c == top) w = true;
      if (c != 0) org = false;
    }
    if (w) wall.push_back((int32_t)i);
    if (org) m->origin = i;
  }

  // --- expanded footprints (independent nodes an element reads / writes)
  auto footprint = [&](int64_t e, int32_t *out) {
    int k = 0;
    for (int c = 0; c < nc; ++c) {
      int32_t v = conn[e * nc + c];
      if (v >= 0) out[k++] = v;
      else
        for (int b = 0; b < 4; ++b) {
          int32_t p = hang_dev[size_t(-v - 1) * 4 + b];
          if (p >= 0) out[k++] = p;
        }
    }
    std::sort(out, out + k);
    return int(std::unique(out, out + k) - out);
  };

  // footprints of all elements (CSR) and the node -> elements incidence over
  // them, in increasing element order (non-uniform meshes only)
  std::vector<int64_t> fp_start, inc_start;
  std::vector<int32_t> fp_node, inc_elem;
  if (!uniform) {
    fp_start.assign(size_t(n) + 1, 0);
    parallel_for(n, 16384, [&](int64_t e0, int64_t e1) {
      int32_t fp[32];
      for (int64_t e = e0; e < e1; ++e) fp_start[e + 1] = footprint(e, fp);
    });
    for (int64_t e = 0; e < n; ++e) fp_start[e + 1] += fp_start[e];
    fp_node.resize(size_t(fp_start[n]));
    // through a local buffer: before de-duplication a footprint can hold
    // more entries than its slot in fp_node
    parallel_for(n, 16384, [&](int64_t e0, int64_t e1) {
      int32_t fp[32];
      for (int64_t e = e0; e < e1; ++e) {
        const int k = footprint(e, fp);
        std::copy(fp, fp + k, &fp_node[size_t(fp_start[e])]);
      }
    });
    inc_start.assign(size_t(n_nodes) + 1, 0);
    for (int64_t k = 0; k < fp_start[n]; ++k) inc_start[fp_node[k] + 1]++;
    for (int64_t i = 0; i < n_nodes; ++i) inc_start[i + 1] += inc_start[i];
    inc_elem.resize(size_t(inc_start[n_nodes]));
    std::vector<int64_t> fill(inc_start.begin(), inc_start.end() - 1);
    for (int64_t e = 0; e < n; ++e)
      for (int64_t k = fp_start[e]; k < fp_start[e + 1]; ++k) inc_elem[fill[fp_node[k]]++] = (int32_t)e;
  }

  // --- element colouring: same colour => disjoint footprints
  std::vector<int> ecol(n);
  int n_col = 0;
  if (uniform) {
    int64_t s = int64_t(1) << (max_level - level[0]);
    for (int64_t e = 0; e < n; ++e) {
      int c = 0;
      for (int a = 0; a < dim; ++a) c |= int((anchor[e * dim + a] / s) & 1) << a;
      ecol[e] = c;
    }
    n_col = nc;
  } else {
    std::vector<int64_t> mark(256, -1);
    std::fill(ecol.begin(), ecol.end(), -1);
    for (int64_t e = 0; e < n; ++e) {
      for (int64_t k = fp_start[e]; k < fp_start[e + 1]; ++k)
        for (int64_t t = inc_start[fp_node[k]]; t < inc_start[fp_node[k] + 1]; ++t) {
          int c = ecol[inc_elem[t]];
          if (c >= 0) mark[c] = e;
        }
      int c = 0;
      while (c < 256 && mark[c] == e) ++c;
      if (c == 256) { set_error("element colouring needs more than 256 colours"); return CHNS_ERR_MESH; }
      ecol[e] = c;
      n_col = std::max(n_col, c + 1);
    }
  }
  // elements sorted by colour, Morton order within a colour (counting sort)
  m->n_colours = n_col;
  m->colour_start.assign(n_col + 1, 0);
  for (int64_t e = 0; e < n; ++e) m->colour_start[ecol[e] + 1]++;
  for (int c = 0; c < n_col; ++c) m->colour_start[c + 1] += m->colour_start[c];
  std::vector<int64_t> order(n);
  {
    std::vector<int64_t> at(m->colour_start.begin(), m->colour_start.end() - 1);
    for (int64_t e = 0; e < n; ++e) order[at[ecol[e]]++] = e;
  }
  std::vector<int32_t> conn_s(size_t(n) * nc);
  std::vector<uint8_t> lev_s(n);
  std::vector<uint32_t> anc_s(size_t(n) * dim);
  for (int64_t i = 0; i < n; ++i) {
    int64_t e = order[i];
    for (int c = 0; c < nc; ++c) conn_s[i * nc + c] = conn[e * nc + c];
    lev_s[i] = level[e];
    for (int a = 0; a < dim; ++a) anc_s[i * dim + a] = anchor[e * dim + a];
  }

  // --- node colouring: nodes of one colour never share an element footprint
  // (probing of the nodal diagonal blocks)
  std::vector<int> ncol(n_nodes, -1);
  int n_ncol = 0;
  if (uniform) {
    int64_t s = int64_t(1) << (max_level - level[0]);
    for (int64_t i = 0; i < n_nodes; ++i) {
      int c = 0;
      for (int a = 0; a < dim; ++a) c |= int((node_xyz[i * dim + a] / s) & 1) << a;
      ncol[i] = c;
    }
    n_ncol = nc;
  } else {
    std::vector<int64_t> mark(256, -1);
    for (int64_t a = 0; a < n_nodes; ++a) {
      for (int64_t t = inc_start[a]; t < inc_start[a + 1]; ++t) {
        const int32_t el = inc_elem[t];
        for (int64_t k = fp_start[el]; k < fp_start[el + 1]; ++k) {
          int c = ncol[fp_node[k]];
          if (c >= 0) mark[c] = a;
        }
      }
      int c = 0;
      while (c < 256 && mark[c] == a) ++c;
      if (c == 256) { set_error("node colouring needs more than 256 colours"); return CHNS_ERR_MESH; }
      ncol[a] = c;
      n_ncol = std::max(n_ncol, c + 1);
    }
  }
  m->n_node_colours = n_ncol;
  m->node_colour_start.assign(n_ncol + 1, 0);
  for (int64_t i = 0; i < n_nodes; ++i) m->node_colour_start[ncol[i] + 1]++;
  for (int c = 0; c < n_ncol; ++c) m->node_colour_start[c + 1] += m->node_colour_start[c];
  // nodes grouped by colour, increasing index within a colour (counting sort)
  std::vector<int32_t> nperm(n_nodes);
  {
    std::vector<int64_t> at(m->node_colour_start.begin(), m->node_colour_start.end() - 1);
    for (int64_t i = 0; i < n_nodes; ++i) nperm[at[ncol[i]]++] = (int32_t)i;
  }

  m->n_nodes = n_nodes;
  m->n_hang = n_hang;
  m->n_wall = (int64_t)wall.size();
  m->node_xyz = std::move(node_xyz);
  m->leaf_level.assign(level, level + n);
  m->leaf_anchor.assign(anchor, anchor + n * dim);

  chns_status st;
  CHNS_CUDA_TRY(cudaGetDevice(&m->device));
  if ((st = upload(&m->conn, conn_s)) != CHNS_OK) return st;
  if ((st = upload(&m->level, lev_s)) != CHNS_OK) return st;
  if ((st = upload(&m->anchor, anc_s)) != CHNS_OK) return st;
  if ((st = upload(&m->hang, hang_dev)) != CHNS_OK) return st;
  if ((st = upload(&m->wall, wall)) != CHNS_OK) return st;
  {
    std::vector<int32_t> pins;
    if (m->origin >= 0) pins.push_back((int32_t)m->origin);
    m->n_pins = (int64_t)pins.size();
    if ((st = upload(&m->pins, pins)) != CHNS_OK) return st;
  }
  m->n_inst = 1;
  m->inst_node_start = {0, n_nodes};
  m->inst_max_level = {max_level};
  if ((st = upload(&m->node_perm, nperm)) != CHNS_OK) return st;
  return CHNS_OK;
}


// Node gather lists of a built mesh (single or union): for every node, the
// (element, corner) slots whose element-local J.w contribution it receives,
// directly (weight 1) or as a parent of a hanging corner (1/2 on an edge,
// 1/4 on a face), in increasing slot order so that the sums are taken in a
// fixed order; and the constrained-row flags of the nodes.
chns_status build_gather(chns_mesh *m) {
  const int nc = 1 << m->dim;
  const int64_t ns = m->n_elem * nc;
  if (ns >= (int64_t(1) << 30)) { set_error("mesh too large for the node gather"); return CHNS_ERR_ARG; }
  const std::vector<int32_t> conn = download(m->conn, size_t(ns));
  const std::vector<int32_t> hang = download(m->hang, size_t(m->n_hang) * 4);
  const std::vector<int32_t> wall = download(m->wall, size_t(m->n_wall));
  const std::vector<int32_t> pins = download(m->pins, size_t(m->n_pins));
  std::vector<int64_t> cnt(size_t(m->n_nodes) + 1, 0);
  auto each = [&](auto &&fn) {
    for (int64_t s = 0; s < ns; ++s) {
      const int32_t v = conn[s];
      if (v >= 0) {
        fn(v, s, 0);
      } else {
        const int32_t *p = &hang[size_t(-v - 1) * 4];
        const int code = p[2] < 0 ? 1 : 2;
        for (int k = 0; k < (p[2] < 0 ? 2 : 4); ++k) fn(p[k], s, code);
      }
    }
  };
  each([&](int32_t i, int64_t, int) { cnt[size_t(i) + 1]++; });
  for (int64_t i = 0; i < m->n_nodes; ++i) cnt[i + 1] += cnt[i];
  if (cnt[m->n_nodes] >= (int64_t(1) << 31)) { set_error("mesh too large for the node gather"); return CHNS_ERR_ARG; }
  std::vector<int32_t> gptr(cnt.begin(), cnt.end()), gent(size_t(cnt[m->n_nodes]));
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  each([&](int32_t i, int64_t s, int code) { gent[fill[i]++] = int32_t(uint32_t(s) | (uint32_t(code) << 30)); });
  std::vector<uint8_t> nflag(size_t(m->n_nodes), 0);
  for (int32_t i : wall) nflag[i] |= 1;
  for (int32_t i : pins) nflag[i] |= 2;
  chns_status st;
  if ((st = upload(&m->gptr, gptr)) != CHNS_OK) return st;
  if ((st = upload(&m->gent, gent)) != CHNS_OK) return st;
  if ((st = upload(&m->nflag, nflag)) != CHNS_OK) return st;
  return CHNS_OK;
}

// Host-side validation of a built mesh (single or union) against its device
// arrays: hanging constraints, colouring, node gather lists.
chns_status validate_mesh(const chns_mesh *m) {
  const int nc = 1 << m->dim;
  const int64_t ns = m->n_elem * nc;
  const std::vector<int32_t> conn = download(m->conn, size_t(ns));
  const std::vector<int32_t> hang = download(m->hang, size_t(m->n_hang) * 4);
  const std::vector<int32_t> gptr = download(m->gptr, size_t(m->n_nodes) + 1);
  const std::vector<int32_t> gent = download(m->gent, size_t(gptr.empty() ? 0 : gptr.back()));
  if (cudaGetLastError() != cudaSuccess) { set_error("validate: reading the mesh back failed"); return CHNS_ERR_CUDA; }
  // hanging constraints: 2 (edge) or 4 (face) distinct independent parents
  for (int64_t h = 0; h < m->n_hang; ++h) {
    const int32_t *p = &hang[size_t(h) * 4];
    const int np = p[2] < 0 ? 2 : 4;
    if (p[2] < 0 && p[3] >= 0) { set_error("hanging node %lld: malformed parent list", (long long)h); return CHNS_ERR_MESH; }
    for (int k = 0; k < np; ++k) {
      if (p[k] < 0 || p[k] >= m->n_nodes) { set_error("hanging node %lld: parent out of range", (long long)h); return CHNS_ERR_MESH; }
      for (int l = 0; l < k; ++l)
        if (p[l] == p[k]) { set_error("hanging node %lld: repeated parent", (long long)h); return CHNS_ERR_MESH; }
    }
  }
  for (int64_t s = 0; s < ns; ++s)
    if (conn[s] >= m->n_nodes || (conn[s] < 0 && -conn[s] - 1 >= m->n_hang)) {
      set_error("slot %lld: node index out of range", (long long)s);
      return CHNS_ERR_MESH;
    }
  // colouring: elements of one colour have disjoint expanded footprints
  if (m->colour_start.size() != size_t(m->n_colours) + 1 || m->colour_start.back() != m->n_elem) {
    set_error("colour ranges do not cover the elements");
    return CHNS_ERR_MESH;
  }
  std::vector<int64_t> owner(size_t(m->n_nodes), -1);
  std::vector<int> owner_col(size_t(m->n_nodes), -1);
  for (int c = 0; c < m->n_colours; ++c)
    for (int64_t e = m->colour_start[c]; e < m->colour_start[c + 1]; ++e)
      for (int k = 0; k < nc; ++k) {
        const int32_t v = conn[e * nc + k];
        int32_t fp[4] = {v, -1, -1, -1};
        if (v < 0) std::memcpy(fp, &hang[size_t(-v - 1) * 4], sizeof(fp));
        for (int q = 0; q < 4 && fp[q] >= 0; ++q) {
          const int32_t i = fp[q];
          if (owner_col[i] == c && owner[i] != e) {
            set_error("colour %d: elements %lld and %lld both reach node %d", c, (long long)owner[i],
                      (long long)e, i);
            return CHNS_ERR_MESH;
          }
          owner_col[i] = c;
          owner[i] = e;
        }
      }
  // gather lists: exactly the slots reaching each node, increasing, weighted
  std::vector<std::vector<uint32_t>> want(size_t(m->n_nodes));
  for (int64_t s = 0; s < ns; ++s) {
    const int32_t v = conn[s];
    if (v >= 0) {
      want[v].push_back(uint32_t(s));
    } else {
      const int32_t *p = &hang[size_t(-v - 1) * 4];
      const uint32_t code = p[2] < 0 ? 1u : 2u;
      for (int k = 0; k < (p[2] < 0 ? 2 : 4); ++k) want[p[k]].push_back(uint32_t(s) | (code << 30));
    }
  }
  for (int64_t i = 0; i < m->n_nodes; ++i) {
    const int64_t b = gptr[i], e = gptr[i + 1];
    if (e - b != (int64_t)want[i].size()) {
      set_error("node %lld: gather list has %lld slots, %zu reach it", (long long)i, (long long)(e - b), want[i].size());
      return CHNS_ERR_MESH;
    }
    for (int64_t t = b; t < e; ++t) {
      if (uint32_t(gent[t]) != want[i][t - b]) { set_error("node %lld: gather entry %lld differs", (long long)i, (long long)(t - b)); return CHNS_ERR_MESH; }
      if (t > b && (uint32_t(gent[t]) & 0x3fffffffu) <= (uint32_t(gent[t - 1]) & 0x3fffffffu)) {
        set_error("node %lld: gather list not in increasing slot order", (long long)i);
        return CHNS_ERR_MESH;
      }
    }
  }
  return CHNS_OK;
}

// One mesh holding several independent problems of the same dimension: the
// instances' nodes and elements are concatenated (instance order), element
// colour c of the union is colour c of every instance (instances share no
// node), and each element records its instance so the element kernels can
// look up that instance's coefficients.
chns_status build_union(const std::vector<const chns_mesh *> &ms, chns_mesh *u) {
  if (ms.empty()) { set_error("empty batch"); return CHNS_ERR_ARG; }
  const int dim = ms[0]->dim, nc = 1 << dim;
  if (ms.size() > 65535) { set_error("too many instances"); return CHNS_ERR_ARG; }
  u->dim = dim;
  u->nc = nc;
  u->nf = dim + 3;
  u->n_inst = (int)ms.size();
  u->max_level = 0;
  u->min_level = 1 << 30;
  int n_col = 0, n_ncol = 0;
  int64_t n_elem = 0, n_nodes = 0, n_hang = 0, n_wall = 0;
  for (auto *m : ms) {
    if (m->dim != dim) { set_error("a batch group must have one dimension"); return CHNS_ERR_ARG; }
    n_col = std::max(n_col, m->n_colours);
    n_ncol = std::max(n_ncol, m->n_node_colours);
    n_elem += m->n_elem;
    n_nodes += m->n_nodes;
    n_hang += m->n_hang;
    n_wall += m->n_wall;
    u->max_level = std::max(u->max_level, m->max_level);
    u->min_level = std::min(u->min_level, m->min_level);
  }
  if (n_elem > (int64_t(1) << 31) / 8 || n_nodes >= (int64_t(1) << 31)) { set_error("batch too large"); return CHNS_ERR_ARG; }
  u->n_elem = n_elem;
  u->n_nodes = n_nodes;
  u->n_hang = n_hang;
  u->n_wall = n_wall;
  u->n_colours = n_col;
  u->n_node_colours = n_ncol;
  for (int a = 0; a < 3; ++a) { u->lo[a] = ms[0]->lo[a]; u->hi[a] = ms[0]->hi[a]; }
  std::vector<int64_t> node_off(ms.size() + 1, 0), hang_off(ms.size() + 1, 0);
  for (size_t i = 0; i < ms.size(); ++i) {
    node_off[i + 1] = node_off[i] + ms[i]->n_nodes;
    hang_off[i + 1] = hang_off[i] + ms[i]->n_hang;
  }
  u->inst_node_start = node_off;
  u->inst_max_level.clear();
  u->inst_meshes = ms;
  // uniform when every instance is uniform at one level (a multigrid bottom)
  u->uniform = true;
  for (auto *m : ms)
    if (!m->uniform || m->min_level != ms[0]->min_level) u->uniform = false;
  // elements colour by colour, instance by instance
  std::vector<int32_t> conn;
  std::vector<uint8_t> lev;
  std::vector<uint32_t> anc;
  std::vector<uint16_t> einst;
  conn.reserve(size_t(n_elem) * nc);
  lev.reserve(n_elem);
  anc.reserve(size_t(n_elem) * dim);
  einst.reserve(n_elem);
  std::vector<std::vector<int32_t>> hconn(ms.size());
  std::vector<std::vector<uint8_t>> hlev(ms.size());
  std::vector<std::vector<uint32_t>> hanc(ms.size());
  for (size_t i = 0; i < ms.size(); ++i) {
    hconn[i] = download(ms[i]->conn, size_t(ms[i]->n_elem) * nc);
    hlev[i] = download(ms[i]->level, size_t(ms[i]->n_elem));
    hanc[i] = download(ms[i]->anchor, size_t(ms[i]->n_elem) * dim);
    u->inst_max_level.push_back(ms[i]->max_level);
  }
  u->colour_start.assign(n_col + 1, 0);
  for (int c = 0; c < n_col; ++c) {
    for (size_t i = 0; i < ms.size(); ++i) {
      const chns_mesh *m = ms[i];
      if (c >= m->n_colours) continue;
      for (int64_t e = m->colour_start[c]; e < m->colour_start[c + 1]; ++e) {
        for (int k = 0; k < nc; ++k) {
          int32_t v = hconn[i][e * nc + k];
          conn.push_back(v >= 0 ? int32_t(v + node_off[i]) : int32_t(v - hang_off[i]));
        }
        lev.push_back(hlev[i][e]);
        for (int a = 0; a < dim; ++a) anc.push_back(hanc[i][e * dim + a]);
        einst.push_back((uint16_t)i);
      }
    }
    u->colour_start[c + 1] = (int64_t)lev.size();
  }
  std::vector<int32_t> hang, wall, pins, nperm, ninst(n_nodes);
  for (size_t i = 0; i < ms.size(); ++i) {
    auto h = download(ms[i]->hang, size_t(ms[i]->n_hang) * 4);
    for (int32_t v : h) hang.push_back(v >= 0 ? int32_t(v + node_off[i]) : v);
    auto w = download(ms[i]->wall, size_t(ms[i]->n_wall));
    for (int32_t v : w) wall.push_back(int32_t(v + node_off[i]));
    if (ms[i]->origin >= 0) pins.push_back(int32_t(ms[i]->origin + node_off[i]));
    for (int64_t k = node_off[i]; k < node_off[i + 1]; ++k) ninst[k] = (int32_t)i;
    for (int64_t k = 0; k < ms[i]->n_nodes * dim; ++k) u->node_xyz.push_back(ms[i]->node_xyz[k]);
  }
  // node colours: colour c of the union = colour c of every instance
  u->node_colour_start.assign(n_ncol + 1, 0);
  std::vector<std::vector<int32_t>> hperm(ms.size());
  for (size_t i = 0; i < ms.size(); ++i) hperm[i] = download(ms[i]->node_perm, size_t(ms[i]->n_nodes));
  for (int c = 0; c < n_ncol; ++c) {
    for (size_t i = 0; i < ms.size(); ++i) {
      const chns_mesh *m = ms[i];
      if (c >= m->n_node_colours) continue;
      for (int64_t k = m->node_colour_start[c]; k < m->node_colour_start[c + 1]; ++k)
        nperm.push_back(int32_t(hperm[i][k] + node_off[i]));
    }
    u->node_colour_start[c + 1] = (int64_t)nperm.size();
  }
  u->n_pins = (int64_t)pins.size();
  u->origin = -1;
  chns_status st;
  CHNS_CUDA_TRY(cudaGetDevice(&u->device));
  if ((st = upload(&u->conn, conn)) != CHNS_OK) return st;
  if ((st = upload(&u->level, lev)) != CHNS_OK) return st;
  if ((st = upload(&u->anchor, anc)) != CHNS_OK) return st;
  if ((st = upload(&u->hang, hang)) != CHNS_OK) return st;
  if ((st = upload(&u->wall, wall)) != CHNS_OK) return st;
  if ((st = upload(&u->pins, pins)) != CHNS_OK) return st;
  if ((st = upload(&u->node_perm, nperm)) != CHNS_OK) return st;
  if ((st = upload(&u->elem_inst, einst)) != CHNS_OK) return st;
  if ((st = upload(&u->node_inst, ninst)) != CHNS_OK) return st;
  return CHNS_OK;
}

}  // namespace chns
