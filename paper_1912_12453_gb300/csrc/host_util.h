// Host-side helpers shared by the mesh builder and the multigrid hierarchy:
// an open-addressing hash map, integer point / octant keys, Morton keys, and
// device upload / download of std::vectors.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "chns_internal.h"

namespace chns {

// Open-addressing hash map from a 64-bit key to a 32-bit value.
class KeyMap {
 public:
  explicit KeyMap(size_t expected) {
    size_t cap = 16;
    while (cap < expected * 2) cap <<= 1;
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, 0);
    mask_ = cap - 1;
  }
  // returns (value, inserted)
  std::pair<int64_t, bool> insert(uint64_t key, int64_t value) {
    size_t i = hash(key) & mask_;
    while (true) {
      if (keys_[i] == kEmpty) {
        keys_[i] = key;
        vals_[i] = value;
        ++size_;
        return {value, true};
      }
      if (keys_[i] == key) return {vals_[i], false};
      i = (i + 1) & mask_;
    }
  }
  int64_t find(uint64_t key) const {
    size_t i = hash(key) & mask_;
    while (true) {
      if (keys_[i] == kEmpty) return -1;
      if (keys_[i] == key) return vals_[i];
      i = (i + 1) & mask_;
    }
  }
  size_t size() const { return size_; }

 private:
  static constexpr uint64_t kEmpty = ~uint64_t(0);
  static uint64_t hash(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
  }
  std::vector<uint64_t> keys_;
  std::vector<int64_t> vals_;
  size_t mask_ = 0, size_ = 0;
};

inline uint64_t pack(const int64_t *x, int dim) {
  uint64_t k = 0;
  for (int a = 0; a < dim; ++a) k |= uint64_t(x[a]) << (21 * a);
  return k;
}

// octant key: the doubled coordinates of its centre, 2 x + s (unique per
// octant, < 2^21 per axis for max_level <= 20)
inline uint64_t okey(int level, const int64_t *x, int dim, int max_level) {
  int64_t c[3];
  int64_t s = int64_t(1) << (max_level - level);
  for (int a = 0; a < dim; ++a) c[a] = 2 * x[a] + s;
  return pack(c, dim);
}

inline uint64_t morton(const uint32_t *a, int dim, int max_level) {
  uint64_t k = 0;
  for (int b = 0; b <= max_level; ++b)
    for (int ax = 0; ax < dim; ++ax) k |= uint64_t((a[ax] >> b) & 1u) << (dim * b + ax);
  return k;
}

template <class T>
inline chns_status upload(T **dst, const std::vector<T> &src) {
  if (src.empty()) { *dst = nullptr; return CHNS_OK; }
  CHNS_CUDA_TRY(cudaMalloc((void **)dst, sizeof(T) * src.size()));
  CHNS_CUDA_TRY(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
  return CHNS_OK;
}


template <class T>
inline std::vector<T> download(const T *d, size_t n) {
  std::vector<T> h(n);
  if (n) cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost);
  return h;
}

}  // namespace chns
