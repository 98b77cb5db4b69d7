// Builds a mesh with the library's host builder (mesh.cpp, CUDA calls stood
// in by host memory), runs the library's own validation, and writes what the
// tests compare: status, counts, independent node coordinates, hanging
// parents (as coordinates), element colours.  Test infrastructure only.
//   mesh_host <leaves.bin> <out.bin>
// leaves.bin: int64 n, int32 dim, int32 max_level, uint8 level[n],
// uint32 anchor[n*dim].
#include <cstdint>
#include <cstdio>
#include <vector>

#include "chns_internal.h"

namespace chns {
chns_status build_mesh(int dim, int64_t n, const uint8_t *level, const uint32_t *anchor, int max_level,
                       const double lo[3], const double hi[3], chns_mesh *m);
chns_status build_gather(chns_mesh *m);
chns_status validate_mesh(const chns_mesh *m);
const char *last_error();
}  // namespace chns

int main(int argc, char **argv) {
  if (argc != 3) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t n = 0;
  int32_t dim = 0, ml = 0;
  if (std::fread(&n, 8, 1, f) != 1 || std::fread(&dim, 4, 1, f) != 1 || std::fread(&ml, 4, 1, f) != 1) return 2;
  std::vector<uint8_t> lv(static_cast<size_t>(n));
  std::vector<uint32_t> an(size_t(n) * dim);
  if (std::fread(lv.data(), 1, lv.size(), f) != lv.size() || std::fread(an.data(), 4, an.size(), f) != an.size())
    return 2;
  std::fclose(f);
  chns_mesh *m = new chns_mesh;
  chns_status s = chns::build_mesh(dim, n, lv.data(), an.data(), ml, nullptr, nullptr, m);
  if (s == CHNS_OK) s = chns::build_gather(m);
  int32_t sv = s;
  chns_status v = s == CHNS_OK ? chns::validate_mesh(m) : CHNS_OK;
  int32_t vv = v;
  FILE *o = std::fopen(argv[2], "wb");
  if (!o) return 2;
  std::fwrite(&sv, 4, 1, o);
  std::fwrite(&vv, 4, 1, o);
  if (s != CHNS_OK || v != CHNS_OK) {
    std::fprintf(stderr, "%s\n", chns::last_error());
    std::fclose(o);
    return 0;
  }
  const int nc = 1 << dim;
  int64_t head[5] = {m->n_nodes, m->n_hang, m->n_colours, m->origin, m->n_wall};
  std::fwrite(head, 8, 5, o);
  std::fwrite(m->node_xyz.data(), 8, m->node_xyz.size(), o);
  // hanging parents of every hanging corner, as node coordinates, one record
  // per (element, corner) slot: the corner's coordinates and its parents'
  std::vector<int64_t> rec;
  for (int64_t e = 0; e < m->n_elem; ++e)
    for (int c = 0; c < nc; ++c) {
      const int32_t id = m->conn[e * nc + c];
      if (id >= 0) continue;
      const int64_t s_ = int64_t(1) << (ml - m->level[e]);
      for (int a = 0; a < dim; ++a) rec.push_back(int64_t(m->anchor[e * dim + a]) + (((c >> a) & 1) ? s_ : 0));
      for (int b = 0; b < 4; ++b) {
        const int32_t p = m->hang[size_t(-id - 1) * 4 + b];
        for (int a = 0; a < dim; ++a) rec.push_back(p >= 0 ? m->node_xyz[size_t(p) * dim + a] : -1);
      }
    }
  const int64_t nrec = int64_t(rec.size());
  std::fwrite(&nrec, 8, 1, o);
  std::fwrite(rec.data(), 8, rec.size(), o);
  std::fwrite(m->colour_start.data(), 8, m->colour_start.size(), o);
  std::fclose(o);
  return 0;
}
