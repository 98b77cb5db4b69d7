// Host-side remeshing (Sec. 4, "Refinement", "2:1 Balancing", "Intergrid
// transfers"): split marked leaves, merge marked families, restore 2:1 balance
// across faces, edges and corners, mark leaves against the diffuse interface
// of a nodal phi field, and carry a nodal Q1 field (hanging constraints
// included) from one leaf set to the points of another.  The octree work is
// host code, like the mesh construction it feeds; no device memory is touched.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "chns_internal.h"
#include "host_util.h"

using namespace chns;

namespace {

struct Oct {
  uint8_t level;
  uint32_t a[3];
};

// A set of octants keyed by (level, anchor), with tombstones for split ones.
struct OctSet {
  int dim, max_level;
  KeyMap map;
  std::vector<Oct> oct;
  std::vector<uint8_t> alive;
  OctSet(int d, int ml, size_t expected) : dim(d), max_level(ml), map(expected * 2 + 64) {}
  uint64_t key(int level, const uint32_t *a) const {
    int64_t x[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) x[k] = a[k];
    return okey(level, x, dim, max_level);
  }
  // insert (or revive) an octant, returns its index
  int64_t add(const Oct &o) {
    auto r = map.insert(key(o.level, o.a), (int64_t)oct.size());
    if (r.second) {
      oct.push_back(o);
      alive.push_back(1);
      return r.first;
    }
    alive[r.first] = 1;
    return r.first;
  }
  int64_t find(int level, const uint32_t *a) const {
    const int64_t i = map.find(key(level, a));
    return (i >= 0 && alive[i]) ? i : -1;
  }
  // the live octant of level <= from_level whose cell holds the
  // max-level-resolution point p (lower-left convention), -1 if none
  int64_t containing(const int64_t *p, int from_level) const {
    for (int l = from_level; l >= 0; --l) {
      const int64_t s = int64_t(1) << (max_level - l);
      uint32_t a[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) a[k] = uint32_t(p[k] / s * s);
      const int64_t i = find(l, a);
      if (i >= 0) return i;
    }
    return -1;
  }
};

void children(const Oct &o, int dim, int max_level, std::vector<Oct> &out) {
  const uint32_t hs = uint32_t(1) << (max_level - o.level - 1);
  for (int c = 0; c < (1 << dim); ++c) {
    Oct ch = o;
    ch.level = uint8_t(o.level + 1);
    for (int k = 0; k < dim; ++k) ch.a[k] = o.a[k] + (((c >> k) & 1) ? hs : 0);
    out.push_back(ch);
  }
}

bool args_ok(int dim, int max_level) { return (dim == 2 || dim == 3) && max_level >= 0 && max_level <= 20; }

// Leaves must be aligned to their level, in Morton order and tile the box
// (the same contract as chns_mesh_create, without the balance requirement).
chns_status check_tiling(int dim, int max_level, int64_t n, const uint8_t *level, const uint32_t *anchor) {
  const int64_t top = int64_t(1) << max_level;
  uint64_t expect = 0;
  for (int64_t e = 0; e < n; ++e) {
    const int l = level[e];
    if (l > max_level) { set_error("leaf %lld: level %d > max_level", (long long)e, l); return CHNS_ERR_MESH; }
    const int64_t s = int64_t(1) << (max_level - l);
    for (int k = 0; k < dim; ++k) {
      const int64_t x = anchor[e * dim + k];
      if (x % s != 0 || x + s > top) {
        set_error("leaf %lld: anchor not aligned to its level or outside the box", (long long)e);
        return CHNS_ERR_MESH;
      }
    }
    if (morton(anchor + e * dim, dim, max_level) != expect) {
      set_error("leaves are not in Morton order or do not tile the box (leaf %lld)", (long long)e);
      return CHNS_ERR_MESH;
    }
    expect += uint64_t(1) << (dim * (max_level - l));
  }
  if (expect != (uint64_t(1) << (dim * max_level))) { set_error("leaves do not cover the box"); return CHNS_ERR_MESH; }
  return CHNS_OK;
}

struct LeafList {
  std::vector<uint8_t> level;
  std::vector<uint32_t> anchor;
  int64_t n() const { return (int64_t)level.size(); }
};

// One adaptation pass.  Marks: +1 split (below max_level), -1 merge into the
// parent when all 2^dim members of the family are leaves marked -1 (above
// level 0), 0 keep.  Then 2:1 balance by splitting: leaves are visited finest
// level first; every same-size cell next to a leaf (across a face, an edge or
// a corner) must lie in a leaf at most one level coarser, else that leaf is
// split, and its children join the coarser levels still to be visited.  The
// result is the coarsest balanced refinement of the marked tree, in Morton
// order.
void adapt_pass(int dim, int max_level, const LeafList &in, const int8_t *mark, LeafList &res) {
  const int64_t n = in.n();
  const int64_t top = int64_t(1) << max_level;
  OctSet src(dim, max_level, size_t(n));
  for (int64_t e = 0; e < n; ++e) {
    Oct o;
    o.level = in.level[e];
    o.a[0] = o.a[1] = o.a[2] = 0;
    for (int k = 0; k < dim; ++k) o.a[k] = in.anchor[e * dim + k];
    src.add(o);
  }
  OctSet out(dim, max_level, size_t(n) * 2);
  std::vector<Oct> kids;
  for (int64_t e = 0; e < n; ++e) {
    const Oct &o = src.oct[e];
    const int m = mark ? mark[e] : 0;
    if (m > 0 && o.level < max_level) {
      kids.clear();
      children(o, dim, max_level, kids);
      for (const Oct &c : kids) out.add(c);
    } else if (m < 0 && o.level > 0) {
      const uint32_t ps = uint32_t(1) << (max_level - o.level + 1);
      Oct p = o;
      p.level = uint8_t(o.level - 1);
      for (int k = 0; k < dim; ++k) p.a[k] = o.a[k] / ps * ps;
      kids.clear();
      children(p, dim, max_level, kids);
      bool all = true;
      for (const Oct &c : kids) {
        const int64_t i = src.find(c.level, c.a);
        if (i < 0 || mark[i] >= 0) all = false;
      }
      out.add(all ? p : o);
    } else {
      out.add(o);
    }
  }
  std::vector<std::vector<int64_t>> by_level(size_t(max_level) + 1);
  for (int64_t i = 0; i < (int64_t)out.oct.size(); ++i) by_level[out.oct[i].level].push_back(i);
  const int nnb = dim == 2 ? 9 : 27;
  for (int l = max_level; l >= 2; --l) {
    for (size_t t = 0; t < by_level[l].size(); ++t) {
      const int64_t i = by_level[l][t];
      if (!out.alive[i]) continue;
      const Oct o = out.oct[i];
      const int64_t s = int64_t(1) << (max_level - l);
      for (int q = 0; q < nnb; ++q) {
        int64_t p[3] = {0, 0, 0};
        int tq = q;
        bool self = true, inside = true;
        for (int k = 0; k < dim; ++k) {
          const int off = tq % 3 - 1;
          tq /= 3;
          if (off) self = false;
          p[k] = int64_t(o.a[k]) + off * s;
          if (p[k] < 0 || p[k] >= top) inside = false;
        }
        if (self || !inside) continue;
        while (true) {
          const int64_t c = out.containing(p, l);
          if (c < 0 || out.oct[c].level >= l - 1) break;  // finer, same or one coarser
          const Oct big = out.oct[c];
          out.alive[c] = 0;
          kids.clear();
          children(big, dim, max_level, kids);
          for (const Oct &ch : kids) by_level[ch.level].push_back(out.add(ch));
        }
      }
    }
  }
  std::vector<std::pair<uint64_t, int64_t>> order;
  for (int64_t i = 0; i < (int64_t)out.oct.size(); ++i)
    if (out.alive[i]) order.push_back({morton(out.oct[i].a, dim, max_level), i});
  std::sort(order.begin(), order.end());
  res.level.resize(order.size());
  res.anchor.resize(order.size() * dim);
  for (size_t e = 0; e < order.size(); ++e) {
    const Oct &o = out.oct[order[e].second];
    res.level[e] = o.level;
    for (int k = 0; k < dim; ++k) res.anchor[e * dim + k] = o.a[k];
  }
}

// A nodal Q1 field on a leaf set: values at the independent nodes, hanging
// nodes interpolated from the corners of the coarser edge or face they lie on
// (Sec. 4, "Handling hanging nodes"); evaluated at any point of the box.
struct Field {
  int dim, max_level, nf, lmax = 0;
  int64_t top;
  OctSet leaves;
  KeyMap node;
  const double *U;
  Field(int d, int ml, int64_t n_leaves, const uint8_t *level, const uint32_t *anchor, int64_t n_nodes,
        const int64_t *xyz, int nf_, const double *U_)
      : dim(d), max_level(ml), nf(nf_), top(int64_t(1) << ml), leaves(d, ml, size_t(n_leaves)),
        node(size_t(n_nodes) + 16), U(U_) {
    for (int64_t e = 0; e < n_leaves; ++e) {
      Oct o;
      o.level = level[e];
      o.a[0] = o.a[1] = o.a[2] = 0;
      for (int k = 0; k < d; ++k) o.a[k] = anchor[e * d + k];
      lmax = std::max<int>(lmax, o.level);
      leaves.add(o);
    }
    for (int64_t i = 0; i < n_nodes; ++i) node.insert(pack(&xyz[i * d], d), i);
  }
  // value at a corner y of a leaf of size s
  bool corner(const int64_t *y, int64_t s, double *val) const {
    const int64_t id = node.find(pack(y, dim));
    if (id >= 0) {
      for (int k = 0; k < nf; ++k) val[k] = U[id * nf + k];
      return true;
    }
    int ax[3], na = 0;
    for (int a = 0; a < dim; ++a)
      if ((y[a] / s) % 2 != 0) ax[na++] = a;
    if (na == 0 || na == 3) return false;
    for (int k = 0; k < nf; ++k) val[k] = 0.0;
    for (int b = 0; b < (1 << na); ++b) {
      int64_t z[3] = {y[0], y[1], dim > 2 ? y[2] : 0};
      for (int t = 0; t < na; ++t) z[ax[t]] += ((b >> t) & 1) ? s : -s;
      const int64_t pid = node.find(pack(z, dim));
      if (pid < 0) return false;
      for (int k = 0; k < nf; ++k) val[k] += U[pid * nf + k] / double(1 << na);
    }
    return true;
  }
  // multilinear interpolation in the leaf holding x
  chns_status eval(const int64_t *x, double *out, double *cv) const {
    for (int k = 0; k < dim; ++k)
      if (x[k] < 0 || x[k] > top) { set_error("point outside the box"); return CHNS_ERR_ARG; }
    int64_t a[3] = {0, 0, 0}, s = 0;
    int64_t e = -1;
    for (int l = lmax; l >= 0 && e < 0; --l) {
      s = int64_t(1) << (max_level - l);
      uint32_t ua[3] = {0, 0, 0};
      for (int k = 0; k < dim; ++k) {
        a[k] = std::min(x[k] / s * s, top - s);
        ua[k] = uint32_t(a[k]);
      }
      e = leaves.find(l, ua);
    }
    if (e < 0) { set_error("a point lies in no source leaf"); return CHNS_ERR_MESH; }
    for (int k = 0; k < nf; ++k) out[k] = 0.0;
    for (int c = 0; c < (1 << dim); ++c) {
      double w = 1.0;
      int64_t y[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        const double t = double(x[d] - a[d]) / double(s);
        w *= ((c >> d) & 1) ? t : 1.0 - t;
        y[d] = a[d] + (((c >> d) & 1) ? s : 0);
      }
      if (w == 0.0) continue;
      if (!corner(y, s, cv)) {
        set_error("a source leaf corner is neither a node nor a hanging node of the source mesh");
        return CHNS_ERR_MESH;
      }
      for (int k = 0; k < nf; ++k) out[k] += w * cv[k];
    }
    return CHNS_OK;
  }
};

// Interface marks of the leaves (level, anchor) against the field's phi
// component: a leaf meets the interface when phi at one of its corners has
// |phi| <= band, or its corners carry both signs of phi (the corner test of
// Sec. 4 "Refinement", applied to the diffuse interface); it aims at
// level_max then, else at level_min.
chns_status mark_pass(const Field &f, int phi_index, double band, int level_min, int level_max,
                      const LeafList &cur, std::vector<int8_t> &mark) {
  const int dim = f.dim;
  const int64_t n = cur.n();
  mark.assign(size_t(n), 0);
  std::vector<double> val(size_t(f.nf)), cv(size_t(f.nf));
  for (int64_t e = 0; e < n; ++e) {
    const int l = cur.level[e];
    const int64_t s = int64_t(1) << (f.max_level - l);
    bool near = false, pos = false, neg = false;
    for (int c = 0; c < (1 << dim) && !near; ++c) {
      int64_t y[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) y[d] = int64_t(cur.anchor[e * dim + d]) + (((c >> d) & 1) ? s : 0);
      const chns_status st = f.eval(y, val.data(), cv.data());
      if (st != CHNS_OK) return st;
      const double phi = val[size_t(phi_index)];
      if (!(std::fabs(phi) <= band)) {
        if (phi > 0) pos = true;
        else if (phi < 0) neg = true;
        else { set_error("phi is not finite"); return CHNS_ERR_NONFINITE; }
      } else {
        near = true;
      }
    }
    const int target = (near || (pos && neg)) ? level_max : level_min;
    mark[e] = l < target ? 1 : (l > target ? -1 : 0);
  }
  return CHNS_OK;
}

chns_status hand_out(const LeafList &r, int dim, int64_t *n_out, uint8_t **level_out, uint32_t **anchor_out) {
  const int64_t m = r.n();
  uint8_t *lv = static_cast<uint8_t *>(std::malloc(size_t(m)));
  uint32_t *an = static_cast<uint32_t *>(std::malloc(sizeof(uint32_t) * size_t(m) * dim));
  if (!lv || !an) {
    std::free(lv);
    std::free(an);
    set_error("host allocation failed");
    return CHNS_ERR_OOM;
  }
  std::memcpy(lv, r.level.data(), size_t(m));
  std::memcpy(an, r.anchor.data(), sizeof(uint32_t) * size_t(m) * dim);
  *n_out = m;
  *level_out = lv;
  *anchor_out = an;
  return CHNS_OK;
}

}  // namespace

extern "C" {

chns_status chns_leaves_adapt(int dim, int max_level, int64_t n, const uint8_t *level, const uint32_t *anchor,
                              const int8_t *mark, int64_t *n_out, uint8_t **level_out, uint32_t **anchor_out) {
  if (!args_ok(dim, max_level) || n <= 0 || !level || !anchor || !n_out || !level_out || !anchor_out) {
    set_error("invalid arguments");
    return CHNS_ERR_ARG;
  }
  *n_out = 0;
  *level_out = nullptr;
  *anchor_out = nullptr;
  chns_status st = check_tiling(dim, max_level, n, level, anchor);
  if (st != CHNS_OK) return st;
  LeafList in, res;
  in.level.assign(level, level + n);
  in.anchor.assign(anchor, anchor + n * dim);
  adapt_pass(dim, max_level, in, mark, res);
  return hand_out(res, dim, n_out, level_out, anchor_out);
}

chns_status chns_leaves_transfer(int dim, int max_level, int64_t n_leaves, const uint8_t *level,
                                 const uint32_t *anchor, int64_t n_nodes, const int64_t *xyz, int nf,
                                 const double *U, int64_t n_points, const int64_t *points, double *out) {
  if (!args_ok(dim, max_level) || n_leaves <= 0 || !level || !anchor || n_nodes <= 0 || !xyz || nf <= 0 ||
      !U || n_points < 0 || (n_points > 0 && (!points || !out))) {
    set_error("invalid arguments");
    return CHNS_ERR_ARG;
  }
  chns_status st = check_tiling(dim, max_level, n_leaves, level, anchor);
  if (st != CHNS_OK) return st;
  Field f(dim, max_level, n_leaves, level, anchor, n_nodes, xyz, nf, U);
  std::vector<double> cv(static_cast<size_t>(nf));
  for (int64_t j = 0; j < n_points; ++j)
    if ((st = f.eval(&points[j * dim], &out[j * nf], cv.data())) != CHNS_OK) return st;
  return CHNS_OK;
}

chns_status chns_leaves_mark_interface(int dim, int max_level, int64_t n_src, const uint8_t *src_level,
                                       const uint32_t *src_anchor, int64_t n_nodes, const int64_t *xyz,
                                       int nf, const double *U, int phi_index, double band, int level_min,
                                       int level_max, int64_t n, const uint8_t *level,
                                       const uint32_t *anchor, int8_t *mark) {
  if (!args_ok(dim, max_level) || n_src <= 0 || !src_level || !src_anchor || n_nodes <= 0 || !xyz ||
      nf <= 0 || !U || phi_index < 0 || phi_index >= nf || !(band >= 0.0) || level_min < 0 ||
      level_max < level_min || level_max > max_level || n <= 0 || !level || !anchor || !mark) {
    set_error("invalid arguments");
    return CHNS_ERR_ARG;
  }
  chns_status st = check_tiling(dim, max_level, n_src, src_level, src_anchor);
  if (st == CHNS_OK) st = check_tiling(dim, max_level, n, level, anchor);
  if (st != CHNS_OK) return st;
  Field f(dim, max_level, n_src, src_level, src_anchor, n_nodes, xyz, nf, U);
  LeafList cur;
  cur.level.assign(level, level + n);
  cur.anchor.assign(anchor, anchor + n * dim);
  std::vector<int8_t> mk;
  if ((st = mark_pass(f, phi_index, band, level_min, level_max, cur, mk)) != CHNS_OK) return st;
  std::memcpy(mark, mk.data(), size_t(n));
  return CHNS_OK;
}

chns_status chns_leaves_remesh(int dim, int max_level, int64_t n_src, const uint8_t *src_level,
                               const uint32_t *src_anchor, int64_t n_nodes, const int64_t *xyz, int nf,
                               const double *U, int phi_index, double band, int level_min, int level_max,
                               int64_t *n_out, uint8_t **level_out, uint32_t **anchor_out, int *passes) {
  if (!args_ok(dim, max_level) || n_src <= 0 || !src_level || !src_anchor || n_nodes <= 0 || !xyz ||
      nf <= 0 || !U || phi_index < 0 || phi_index >= nf || !(band >= 0.0) || level_min < 0 ||
      level_max < level_min || level_max > max_level || !n_out || !level_out || !anchor_out) {
    set_error("invalid arguments");
    return CHNS_ERR_ARG;
  }
  *n_out = 0;
  *level_out = nullptr;
  *anchor_out = nullptr;
  chns_status st = check_tiling(dim, max_level, n_src, src_level, src_anchor);
  if (st != CHNS_OK) return st;
  Field f(dim, max_level, n_src, src_level, src_anchor, n_nodes, xyz, nf, U);
  LeafList cur, nxt;
  cur.level.assign(src_level, src_level + n_src);
  cur.anchor.assign(src_anchor, src_anchor + n_src * dim);
  std::vector<int8_t> mk;
  int it = 0;
  // every pass moves each leaf one level toward its target; a merge that the
  // balance undoes leaves the set unchanged, which ends the loop
  const int max_passes = 2 * max_level + 2;
  for (; it < max_passes; ++it) {
    if ((st = mark_pass(f, phi_index, band, level_min, level_max, cur, mk)) != CHNS_OK) return st;
    if (std::all_of(mk.begin(), mk.end(), [](int8_t v) { return v == 0; })) break;
    adapt_pass(dim, max_level, cur, mk.data(), nxt);
    if (nxt.level == cur.level && nxt.anchor == cur.anchor) break;
    std::swap(cur, nxt);
  }
  if (passes) *passes = it;
  return hand_out(cur, dim, n_out, level_out, anchor_out);
}

void chns_leaves_free(void *p) { std::free(p); }

chns_status chns_mesh_leaves(const chns_mesh *m, uint8_t *level, uint32_t *anchor) {
  if (!m || !level || !anchor) { set_error("null argument"); return CHNS_ERR_ARG; }
  if (m->n_inst != 1 || (int64_t)m->leaf_level.size() != m->n_elem) {
    set_error("the mesh holds no leaf list (a batched union mesh)");
    return CHNS_ERR_ARG;
  }
  std::memcpy(level, m->leaf_level.data(), m->leaf_level.size());
  std::memcpy(anchor, m->leaf_anchor.data(), sizeof(uint32_t) * m->leaf_anchor.size());
  return CHNS_OK;
}

}  // extern "C"
