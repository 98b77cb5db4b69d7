// Host-side helpers shared by the mesh builder and the multigrid hierarchy:
// an open-addressing hash map, integer point / octant keys, Morton keys, and
// device upload / download of std::vectors.
#pragma once

#include <algorithm>
#include <cstdint>
#include <thread>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "chns_internal.h"

namespace chns {

// Open-addressing hash map from a 64-bit key to a 64-bit value (linear
// probing; key and value side by side, one cache line per probe).
class KeyMap {
 public:
  explicit KeyMap(size_t expected) {
    size_t cap = 16;
    while (cap < expected * 2) cap <<= 1;
    slots_.assign(cap, Slot{kEmpty, 0});
    mask_ = cap - 1;
  }
  // returns (value, inserted); the table doubles when it is half full
  std::pair<int64_t, bool> insert(uint64_t key, int64_t value) {
    if (2 * (size_ + 1) > slots_.size()) grow();
    size_t i = hash(key) & mask_;
    while (true) {
      Slot &sl = slots_[i];
      if (sl.key == kEmpty) {
        sl.key = key;
        sl.val = value;
        ++size_;
        return {value, true};
      }
      if (sl.key == key) return {sl.val, false};
      i = (i + 1) & mask_;
    }
  }
  int64_t find(uint64_t key) const {
    size_t i = hash(key) & mask_;
    while (true) {
      const Slot &sl = slots_[i];
      if (sl.key == kEmpty) return -1;
      if (sl.key == key) return sl.val;
      i = (i + 1) & mask_;
    }
  }
  size_t size() const { return size_; }

 private:
  struct Slot {
    uint64_t key;
    int64_t val;
  };
  void grow() {
    std::vector<Slot> old = std::move(slots_);
    slots_.assign(old.size() * 2, Slot{kEmpty, 0});
    mask_ = slots_.size() - 1;
    for (const Slot &o : old) {
      if (o.key == kEmpty) continue;
      size_t i = hash(o.key) & mask_;
      while (slots_[i].key != kEmpty) i = (i + 1) & mask_;
      slots_[i] = o;
    }
  }
  static constexpr uint64_t kEmpty = ~uint64_t(0);
  static uint64_t hash(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
  }
  std::vector<Slot> slots_;
  size_t mask_ = 0, size_ = 0;
};

// fn(begin, end) over [0, n) split across host threads; a thread that cannot
// be started leaves its range to the calling thread
template <class F>
inline void parallel_for(int64_t n, int64_t grain, F fn) {
  const int64_t hw = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), 64));
  const int nt = int(std::max<int64_t>(1, std::min<int64_t>(hw, (n + grain - 1) / grain)));
  if (nt <= 1) {
    fn(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  int started = 0;
  try {
    for (int t = 1; t < nt; ++t) {
      th.emplace_back([&fn, n, nt, t] { fn(n * t / nt, n * (t + 1) / nt); });
      ++started;
    }
  } catch (...) {
  }
  fn(int64_t(0), n / nt);
  for (int t = started + 1; t < nt; ++t) fn(n * t / nt, n * (t + 1) / nt);
  for (auto &x : th) x.join();
}

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

// Morton key: bit b of coordinate ax goes to bit dim*b + ax.  Coordinates
// are at most 2^20 (max_level <= 20), so bits 0..20 of each are spread: every
// bit moves to a multiple of dim by shift-and-mask steps of halving width.
inline uint64_t spread2(uint64_t x) {  // bits 0..31 -> even bits
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
inline uint64_t spread3(uint64_t x) {  // bits 0..20 -> every third bit
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
inline uint64_t morton(const uint32_t *a, int dim, int /*max_level*/) {
  if (dim == 2) return spread2(a[0]) | (spread2(a[1]) << 1);
  return spread3(a[0]) | (spread3(a[1]) << 1) | (spread3(a[2]) << 2);
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
