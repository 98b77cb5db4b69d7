// Host-side remeshing (Sec. 4, "Refinement", "2:1 Balancing", "Intergrid
// transfers"): split marked leaves, merge marked families, restore 2:1 balance
// across faces, edges and corners, mark leaves against the diffuse interface
// of a nodal phi field, and carry a nodal Q1 field (hanging constraints
// included) from one leaf set to the points of another.  The octree work is
// host code, like the mesh construction it feeds; no device memory is touched.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "chns_internal.h"
#include "host_util.h"

using namespace chns;

namespace {

struct Oct {
  uint8_t level;
  uint32_t a[3];
};

enum : uint8_t { kLeaf = 1, kInternal = 2 };

// A set of octants keyed by (level, anchor): leaves, and the internal octants
// (ancestors of leaves) where the balance needs them.
struct OctSet {
  int dim, max_level;
  KeyMap map;
  std::vector<Oct> oct;
  std::vector<uint8_t> kind;
  OctSet(int d, int ml, size_t expected) : dim(d), max_level(ml), map(expected + 64) {
    oct.reserve(expected);
    kind.reserve(expected);
  }
  uint64_t key(int level, const uint32_t *a) const {
    int64_t x[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) x[k] = a[k];
    return okey(level, x, dim, max_level);
  }
  // insert an octant of the given kind (an existing one takes that kind)
  int64_t add(const Oct &o, uint8_t k = kLeaf) {
    auto r = map.insert(key(o.level, o.a), (int64_t)oct.size());
    if (r.second) {
      oct.push_back(o);
      kind.push_back(k);
    } else {
      kind[r.first] = k;
    }
    return r.first;
  }
  int64_t lookup(int level, const uint32_t *a) const { return map.find(key(level, a)); }
  int64_t find(int level, const uint32_t *a) const {
    const int64_t i = lookup(level, a);
    return (i >= 0 && kind[i] == kLeaf) ? i : -1;
  }
};

Oct parent_of(const Oct &o, int dim, int max_level) {
  const uint32_t ps = uint32_t(1) << (max_level - o.level + 1);
  Oct p = o;
  p.level = uint8_t(o.level - 1);
  for (int k = 0; k < dim; ++k) p.a[k] = o.a[k] / ps * ps;
  return p;
}

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

// (key, value) pairs in increasing key order; keys below 2^bits and
// distinct (LSD radix sort, 16-bit digits)
void radix_sort(std::vector<std::pair<uint64_t, int64_t>> &v, int bits) {
  std::vector<std::pair<uint64_t, int64_t>> tmp(v.size());
  std::vector<size_t> count(size_t(1) << 16);
  for (int shift = 0; shift < bits; shift += 16) {
    std::fill(count.begin(), count.end(), 0);
    for (const auto &x : v) ++count[(x.first >> shift) & 0xffff];
    size_t sum = 0;
    for (auto &c : count) {
      const size_t t = c;
      c = sum;
      sum += t;
    }
    for (const auto &x : v) tmp[count[(x.first >> shift) & 0xffff]++] = x;
    v.swap(tmp);
  }
}

struct LeafList {
  std::vector<uint8_t> level;
  std::vector<uint32_t> anchor;
  int64_t n() const { return (int64_t)level.size(); }
};

// One adaptation pass.  Marks: +1 split (below max_level), -1 merge into the
// parent when all 2^dim members of the family are leaves marked -1 (above
// level 0), 0 keep.  Then 2:1 balance by splitting.  Every ancestor of a leaf
// is kept as an internal octant, so the leaves inside an octant q are finer
// than q exactly when q is internal.  Leaves are visited finest level first:
// a leaf of level l is out of balance when a same-size cell next to it
// (across a face, an edge or a corner) lies in a leaf of level <= l - 2, i.e.
// when one of the level-(l-2) octants holding those cells (at most 2^dim of
// them) is a leaf or lies inside one.  That leaf is split; its children join
// the coarser levels still to be visited.  The result is the coarsest
// balanced refinement of the marked tree, in Morton order.
void adapt_pass(int dim, int max_level, const LeafList &in, const int8_t *mark, LeafList &res) {
  const int64_t n = in.n();
  const int64_t top = int64_t(1) << max_level;
  auto leaf_at = [&](int64_t e) {
    Oct o;
    o.level = in.level[e];
    o.a[0] = o.a[1] = o.a[2] = 0;
    for (int k = 0; k < dim; ++k) o.a[k] = in.anchor[e * dim + k];
    return o;
  };
  bool any_merge = false;
  if (mark)
    for (int64_t e = 0; e < n && !any_merge; ++e) any_merge = mark[e] < 0;
  OctSet src(dim, max_level, any_merge ? size_t(n) : 0);
  if (any_merge)
    for (int64_t e = 0; e < n; ++e) src.add(leaf_at(e));
  OctSet out(dim, max_level, size_t(n) + size_t(n) / 4);
  std::vector<Oct> kids;
  for (int64_t e = 0; e < n; ++e) {
    const Oct o = leaf_at(e);
    const int m = mark ? mark[e] : 0;
    if (m > 0 && o.level < max_level) {
      kids.clear();
      children(o, dim, max_level, kids);
      for (const Oct &c : kids) out.add(c);
    } else if (m < 0 && o.level > 0) {
      const Oct p = parent_of(o, dim, max_level);
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
  // ancestors of the leaves as internal octants
  const int64_t n_leaves = (int64_t)out.oct.size();
  for (int64_t i = 0; i < n_leaves; ++i) {
    Oct o = out.oct[i];
    while (o.level > 0) {
      o = parent_of(o, dim, max_level);
      if (out.lookup(o.level, o.a) >= 0) break;
      out.add(o, kInternal);
    }
  }
  std::vector<std::vector<int64_t>> by_level(size_t(max_level) + 1);
  for (int64_t i = 0; i < n_leaves; ++i) by_level[out.oct[i].level].push_back(i);
  auto split = [&](int64_t c) {
    const Oct big = out.oct[c];
    out.kind[c] = kInternal;
    kids.clear();
    children(big, dim, max_level, kids);
    for (const Oct &ch : kids) by_level[ch.level].push_back(out.add(ch));
  };
  for (int l = max_level; l >= 2; --l) {
    const int64_t s = int64_t(1) << (max_level - l);
    const int64_t S = 4 * s;  // size of a level-(l-2) octant
    for (size_t t = 0; t < by_level[l].size(); ++t) {
      const int64_t i = by_level[l][t];
      if (out.kind[i] != kLeaf) continue;
      const Oct o = out.oct[i];
      // per axis, the level-(l-2) octants holding the cells at a - s, a, a + s
      int64_t cand[3][2];
      int nc[3] = {1, 1, 1};
      for (int k = 0; k < 3; ++k) cand[k][0] = cand[k][1] = 0;
      for (int k = 0; k < dim; ++k) {
        const int64_t a = o.a[k];
        int cnt = 0;
        for (int off = -1; off <= 1; ++off) {
          const int64_t p = a + off * s;
          if (p < 0 || p >= top) continue;
          const int64_t q = p / S * S;
          if (cnt == 0 || cand[k][cnt - 1] != q) cand[k][cnt++] = q;
        }
        nc[k] = cnt;
      }
      for (int i0 = 0; i0 < nc[0]; ++i0)
        for (int i1 = 0; i1 < nc[1]; ++i1)
          for (int i2 = 0; i2 < nc[2]; ++i2) {
            uint32_t q[3] = {uint32_t(cand[0][i0]), uint32_t(cand[1][i1]), uint32_t(cand[2][i2])};
            while (true) {
              const int64_t j = out.lookup(l - 2, q);
              if (j >= 0 && out.kind[j] == kInternal) break;
              if (j >= 0) {  // a leaf of level l - 2
                split(j);
                break;
              }
              // inside a coarser leaf: the nearest ancestor present is that leaf
              Oct a;
              a.level = uint8_t(l - 2);
              for (int k = 0; k < 3; ++k) a.a[k] = q[k];
              int64_t c = -1;
              while (a.level > 0 && c < 0) {
                a = parent_of(a, dim, max_level);
                c = out.lookup(a.level, a.a);
              }
              if (c < 0 || out.kind[c] != kLeaf) break;  // not reachable for a tiling
              split(c);
            }
          }
    }
  }
  std::vector<std::pair<uint64_t, int64_t>> order;
  order.reserve(out.oct.size());
  for (int64_t i = 0; i < (int64_t)out.oct.size(); ++i)
    if (out.kind[i] == kLeaf) order.push_back({morton(out.oct[i].a, dim, max_level), i});
  radix_sort(order, dim * max_level);
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
// (Sec. 4, "Handling hanging nodes"); components [k0, k0 + kn) evaluated at
// any point of the box.
struct Field {
  int dim, max_level, nf, k0, kn, lmax = 0;
  int64_t top;
  OctSet leaves;
  KeyMap node;
  const double *U;
  Field(int d, int ml, int64_t n_leaves, const uint8_t *level, const uint32_t *anchor, int64_t n_nodes,
        const int64_t *xyz, int nf_, const double *U_, int k0_, int kn_)
      : dim(d), max_level(ml), nf(nf_), k0(k0_), kn(kn_), top(int64_t(1) << ml),
        leaves(d, ml, size_t(n_leaves)), node(size_t(n_nodes) + 16), U(U_) {
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
      for (int k = 0; k < kn; ++k) val[k] = U[id * nf + k0 + k];
      return true;
    }
    int ax[3], na = 0;
    for (int a = 0; a < dim; ++a)
      if ((y[a] / s) % 2 != 0) ax[na++] = a;
    if (na == 0 || na == 3) return false;
    for (int k = 0; k < kn; ++k) val[k] = 0.0;
    for (int b = 0; b < (1 << na); ++b) {
      int64_t z[3] = {y[0], y[1], dim > 2 ? y[2] : 0};
      for (int t = 0; t < na; ++t) z[ax[t]] += ((b >> t) & 1) ? s : -s;
      const int64_t pid = node.find(pack(z, dim));
      if (pid < 0) return false;
      for (int k = 0; k < kn; ++k) val[k] += U[pid * nf + k0 + k] / double(1 << na);
    }
    return true;
  }
  // the leaf whose cell holds the finest cell at x (clamped into the box),
  // searched from level `hint` outwards; its anchor and size in a, *s
  int64_t locate(const int64_t *x, int hint, int64_t *a, int64_t *s) const {
    hint = std::min(std::max(hint, 0), lmax);
    for (int r = 0; r <= lmax; ++r) {
      for (int sgn = 0; sgn < 2; ++sgn) {
        const int l = sgn ? hint + r : hint - r;
        if ((sgn && r == 0) || l < 0 || l > lmax) continue;
        const int64_t sz = int64_t(1) << (max_level - l);
        uint32_t ua[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) ua[k] = uint32_t(std::min(x[k], top - 1) / sz * sz);
        const int64_t e = leaves.find(l, ua);
        if (e >= 0) {
          for (int k = 0; k < dim; ++k) a[k] = ua[k];
          *s = sz;
          return e;
        }
      }
    }
    return -1;
  }
  // multilinear interpolation at x in the leaf (a, s); cv: kn scratch values
  chns_status interp(const int64_t *a, int64_t s, const int64_t *x, double *out, double *cv) const {
    for (int k = 0; k < kn; ++k) out[k] = 0.0;
    for (int c = 0; c < (1 << dim); ++c) {
      double w = 1.0;
      int64_t y[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        const double t = double(x[d] - a[d]) / double(s);
        w *= ((c >> d) & 1) ? t : 1.0 - t;
        y[d] = a[d] + (((c >> d) & 1) ? s : 0);
      }
      if (w == 0.0) continue;
      if (!corner(y, s, cv)) return CHNS_ERR_MESH;
      for (int k = 0; k < kn; ++k) out[k] += w * cv[k];
    }
    return CHNS_OK;
  }
  chns_status eval(const int64_t *x, int hint, double *out, double *cv) const {
    for (int k = 0; k < dim; ++k)
      if (x[k] < 0 || x[k] > top) return CHNS_ERR_ARG;
    int64_t a[3] = {0, 0, 0}, s = 0;
    if (locate(x, hint, a, &s) < 0) return CHNS_ERR_MESH;
    return interp(a, s, x, out, cv);
  }
  // the field at the 2^dim corners of the leaf (level l, anchor) into
  // vals[c * kn + k]; one source leaf serves all corners when it holds the leaf
  chns_status leaf_corners(int l, const uint32_t *anchor, double *vals, double *cv) const {
    const int64_t s = int64_t(1) << (max_level - l);
    int64_t x0[3] = {0, 0, 0}, a[3] = {0, 0, 0}, sa = 0;
    for (int d = 0; d < dim; ++d) x0[d] = anchor[d];
    const bool inside = locate(x0, l, a, &sa) >= 0 && sa >= s;
    for (int c = 0; c < (1 << dim); ++c) {
      int64_t y[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) y[d] = x0[d] + (((c >> d) & 1) ? s : 0);
      const chns_status st = inside ? interp(a, sa, y, &vals[c * kn], cv) : eval(y, l, &vals[c * kn], cv);
      if (st != CHNS_OK) return st;
    }
    return CHNS_OK;
  }
};

void field_error(chns_status st) {
  if (st == CHNS_ERR_ARG) set_error("point outside the box");
  else if (st == CHNS_ERR_MESH)
    set_error("a source leaf corner is neither a node nor a hanging node of the source mesh, or a point lies in no source leaf");
  else if (st == CHNS_ERR_NONFINITE) set_error("phi is not finite");
}

// Interface marks of the leaves against the field's single component (phi):
// a leaf meets the interface when phi at one of its corners has |phi| <=
// band, or its corners carry both signs of phi (the corner test of Sec. 4
// "Refinement", applied to the diffuse interface); it aims at level_max then,
// else at level_min.
chns_status mark_pass(const Field &f, double band, int level_min, int level_max, const LeafList &cur,
                      std::vector<int8_t> &mark) {
  const int dim = f.dim;
  const int64_t n = cur.n();
  mark.assign(size_t(n), 0);
  std::atomic<int> fail{0};
  parallel_for(n, 4096, [&](int64_t b, int64_t e_end) {
    double phi[8], cv[1];
    for (int64_t e = b; e < e_end; ++e) {
      const int l = cur.level[e];
      chns_status st = f.leaf_corners(l, &cur.anchor[size_t(e) * dim], phi, cv);
      bool near = false, pos = false, neg = false;
      for (int c = 0; c < (1 << dim) && st == CHNS_OK; ++c) {
        if (std::fabs(phi[c]) <= band) near = true;
        else if (phi[c] > 0) pos = true;
        else if (phi[c] < 0) neg = true;
        else st = CHNS_ERR_NONFINITE;
      }
      if (st != CHNS_OK) {
        int expected = 0;
        fail.compare_exchange_strong(expected, int(st));
        return;
      }
      const int target = (near || (pos && neg)) ? level_max : level_min;
      mark[e] = l < target ? 1 : (l > target ? -1 : 0);
    }
  });
  if (fail.load()) {
    field_error(chns_status(fail.load()));
    return chns_status(fail.load());
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

// runs fn, turning a host allocation failure into CHNS_ERR_OOM
template <class F>
chns_status guarded(F fn) {
  try {
    return fn();
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return CHNS_ERR_OOM;
  } catch (...) {
    set_error("unexpected host exception");
    return CHNS_ERR_ARG;
  }
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
  return guarded([&] {
    LeafList in, res;
    in.level.assign(level, level + n);
    in.anchor.assign(anchor, anchor + n * dim);
    adapt_pass(dim, max_level, in, mark, res);
    return hand_out(res, dim, n_out, level_out, anchor_out);
  });
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
  return guarded([&] {
    Field f(dim, max_level, n_leaves, level, anchor, n_nodes, xyz, nf, U, 0, nf);
    std::atomic<int> fail{0};
    parallel_for(n_points, 4096, [&](int64_t b, int64_t e) {
      std::vector<double> cv(static_cast<size_t>(nf));
      for (int64_t j = b; j < e; ++j) {
        const chns_status sj = f.eval(&points[j * dim], f.lmax, &out[j * nf], cv.data());
        if (sj != CHNS_OK) {
          int expected = 0;
          fail.compare_exchange_strong(expected, int(sj));
          return;
        }
      }
    });
    if (fail.load()) field_error(chns_status(fail.load()));
    return chns_status(fail.load());
  });
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
  return guarded([&] {
    Field f(dim, max_level, n_src, src_level, src_anchor, n_nodes, xyz, nf, U, phi_index, 1);
    LeafList cur;
    cur.level.assign(level, level + n);
    cur.anchor.assign(anchor, anchor + n * dim);
    std::vector<int8_t> mk;
    const chns_status s2 = mark_pass(f, band, level_min, level_max, cur, mk);
    if (s2 == CHNS_OK) std::memcpy(mark, mk.data(), size_t(n));
    return s2;
  });
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
  return guarded([&] {
    Field f(dim, max_level, n_src, src_level, src_anchor, n_nodes, xyz, nf, U, phi_index, 1);
    LeafList cur, nxt;
    cur.level.assign(src_level, src_level + n_src);
    cur.anchor.assign(src_anchor, src_anchor + n_src * dim);
    std::vector<int8_t> mk;
    int it = 0;
    // every pass moves each leaf one level toward its target; a merge that the
    // balance undoes leaves the set unchanged, which ends the loop
    const int max_passes = 2 * max_level + 2;
    for (; it < max_passes; ++it) {
      const chns_status s2 = mark_pass(f, band, level_min, level_max, cur, mk);
      if (s2 != CHNS_OK) return s2;
      if (std::all_of(mk.begin(), mk.end(), [](int8_t v) { return v == 0; })) break;
      adapt_pass(dim, max_level, cur, mk.data(), nxt);
      if (nxt.level == cur.level && nxt.anchor == cur.anchor) break;
      std::swap(cur, nxt);
    }
    if (passes) *passes = it;
    return hand_out(cur, dim, n_out, level_out, anchor_out);
  });
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
