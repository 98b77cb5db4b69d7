// Runs the library's host remeshing calls (octree.cpp) from a standalone
// executable, so that a test can build them with AddressSanitizer and compare
// their output with the shared library's.  Test infrastructure only.
//   octree_host adapt    <in.bin> <out.bin>   in: leaves, int8 mark[n]
//   octree_host remesh   <in.bin> <out.bin>   in: leaves, int64 n_nodes, int32 nf,
//                                                 int64 xyz[n_nodes*dim], double U[n_nodes*nf],
//                                                 int32 level_min, level_max, double band
//   octree_host transfer <in.bin> <out.bin>   in: as remesh without the last three,
//                                                 then int64 n_points, int64 points[n_points*dim]
// leaves: int64 n, int32 dim, int32 max_level, uint8 level[n], uint32 anchor[n*dim]
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "chns.h"

namespace {
FILE *in_f;
template <class T>
bool rd(T *p, size_t n) { return std::fread(p, sizeof(T), n, in_f) == n; }
}  // namespace

int main(int argc, char **argv) {
  if (argc != 4) return 2;
  const std::string mode = argv[1];
  in_f = std::fopen(argv[2], "rb");
  if (!in_f) return 2;
  int64_t n = 0;
  int32_t dim = 0, ml = 0;
  if (!rd(&n, 1) || !rd(&dim, 1) || !rd(&ml, 1)) return 2;
  std::vector<uint8_t> lv(static_cast<size_t>(n));
  std::vector<uint32_t> an(static_cast<size_t>(n) * dim);
  if (!rd(lv.data(), lv.size()) || !rd(an.data(), an.size())) return 2;
  FILE *o = std::fopen(argv[3], "wb");
  if (!o) return 2;
  int32_t st = 0;
  if (mode == "adapt") {
    std::vector<int8_t> mark(static_cast<size_t>(n));
    if (!rd(mark.data(), mark.size())) return 2;
    int64_t m = 0;
    uint8_t *lo = nullptr;
    uint32_t *ao = nullptr;
    st = chns_leaves_adapt(dim, ml, n, lv.data(), an.data(), mark.data(), &m, &lo, &ao);
    std::fwrite(&st, 4, 1, o);
    if (st == 0) {
      std::fwrite(&m, 8, 1, o);
      std::fwrite(lo, 1, size_t(m), o);
      std::fwrite(ao, 4, size_t(m) * dim, o);
      chns_leaves_free(lo);
      chns_leaves_free(ao);
    }
  } else {
    int64_t nn = 0;
    int32_t nf = 0;
    if (!rd(&nn, 1) || !rd(&nf, 1)) return 2;
    std::vector<int64_t> xyz(static_cast<size_t>(nn) * dim);
    std::vector<double> U(static_cast<size_t>(nn) * nf);
    if (!rd(xyz.data(), xyz.size()) || !rd(U.data(), U.size())) return 2;
    if (mode == "remesh") {
      int32_t lmin = 0, lmax = 0;
      double band = 0;
      if (!rd(&lmin, 1) || !rd(&lmax, 1) || !rd(&band, 1)) return 2;
      int64_t m = 0;
      uint8_t *lo = nullptr;
      uint32_t *ao = nullptr;
      int passes = 0;
      st = chns_leaves_remesh(dim, ml, n, lv.data(), an.data(), nn, xyz.data(), nf, U.data(), dim + 1, band, lmin,
                              lmax, &m, &lo, &ao, &passes);
      std::fwrite(&st, 4, 1, o);
      if (st == 0) {
        std::fwrite(&m, 8, 1, o);
        std::fwrite(&passes, 4, 1, o);
        std::fwrite(lo, 1, size_t(m), o);
        std::fwrite(ao, 4, size_t(m) * dim, o);
        chns_leaves_free(lo);
        chns_leaves_free(ao);
      }
    } else if (mode == "transfer") {
      int64_t np = 0;
      if (!rd(&np, 1)) return 2;
      std::vector<int64_t> pts(static_cast<size_t>(np) * dim);
      if (!rd(pts.data(), pts.size())) return 2;
      std::vector<double> out(static_cast<size_t>(np) * nf);
      st = chns_leaves_transfer(dim, ml, n, lv.data(), an.data(), nn, xyz.data(), nf, U.data(), np, pts.data(),
                                out.data());
      std::fwrite(&st, 4, 1, o);
      if (st == 0) std::fwrite(out.data(), 8, out.size(), o);
    } else {
      return 2;
    }
  }
  std::fclose(o);
  std::fclose(in_f);
  return 0;
}
