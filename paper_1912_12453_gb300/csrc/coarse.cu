// Two-level additive preconditioner for the Krylov solve of Sec. 3.5:
//   z = B^{-1} v + P A_c^{-1} R v
// B: nodal block-Jacobi (vector.cu); P: trilinear interpolation of all fields
// from the nodes of a uniform coarse octree level L_c to the mesh nodes;
// R = P^T; A_c = R J P, the Galerkin projection of the Jacobian.  Nodal
// block-Jacobi alone leaves the smooth pressure modes of the VMS saddle
// point unresolved (they couple across the whole domain); the coarse space
// carries them.
//
// A_c is probed: the image J P e_c of a coarse hat lives within H + h of its
// coarse node c (H, h: coarse and mesh spacing), so the hats of one field
// whose nodes share the residues of their coordinates mod 3 (27 colours in
// 3D, 9 in 2D) are applied together, and each mesh row is credited to the
// nearest coarse node of the probed colour.  Exact when h <= H/2, i.e. every
// leaf at least one level finer than L_c.  All reductions run in a fixed
// order (one block per coarse node); nothing is atomic.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "chns_internal.h"
#include "coarse.h"

namespace chns {

namespace {

constexpr int kB = 256;
constexpr unsigned FULL = 0xffffffffu;

inline unsigned grid_n(int64_t n) {
  int64_t b = (n + kB - 1) / kB;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 8);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

struct CGeo {
  int dim, nf, nc1;   // nc1 = 2^Lc + 1 coarse nodes per axis
  int64_t n_nodes;
  int64_t ncn_inst;   // coarse nodes per instance
  int64_t nc0;        // coarse unknowns per instance
  int64_t ncell_inst; // coarse cells per instance, (nc1 - 1)^dim
};

// 16 bytes of T
template <typename T>
struct alignas(16) V16 {
  T a[16 / sizeof(T)];
};

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  return v;
}

// cell (lowest corner, per axis) and fraction of a position in coarse units
__device__ __forceinline__ void locate(const CGeo &g, const float *pos, int *b, float *t) {
  for (int a = 0; a < g.dim; ++a) {
    int c = (int)floorf(pos[a]);
    c = c < 0 ? 0 : (c > g.nc1 - 2 ? g.nc1 - 2 : c);
    b[a] = c;
    t[a] = pos[a] - float(c);
  }
}

__device__ __forceinline__ int lin(const CGeo &g, const int *c) {
  int idx = 0;
  for (int a = g.dim - 1; a >= 0; --a) idx = idx * g.nc1 + c[a];
  return idx;
}

// probing vector: field f = sum of the coarse hats of colour k; other fields 0
template <typename T, int NF, int DIM>
__global__ void __launch_bounds__(kB) k_probe_coarse(CGeo g, const float *__restrict__ pos, int k, int f,
                                                     T *__restrict__ w) {
  int kk[3] = {k % 3, (k / 3) % 3, k / 9};
  for (int64_t i = blockIdx.x * int64_t(kB) + threadIdx.x; i < g.n_nodes; i += int64_t(gridDim.x) * kB) {
    int b[3];
    float t[3];
    locate(g, pos + i * g.dim, b, t);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < (1 << DIM); ++c) {
      double wc = 1.0;
      bool in = true;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        int ca = b[a] + ((c >> a) & 1);
        if (ca % 3 != kk[a]) in = false;
        wc *= ((c >> a) & 1) ? double(t[a]) : 1.0 - double(t[a]);
      }
      if (in) s += wc;
    }
#pragma unroll
    for (int q = 0; q < NF; ++q) w[i * NF + q] = q == f ? T(s) : T(0);
  }
}

// owner coordinates (residue kk mod 3, within two coarse steps of the row
// node cpc) of slot s: bit a set = positive offset along axis a
__device__ __forceinline__ bool slot_owner(const CGeo &g, const int *cpc, const int *kk, int s, int *oc) {
  bool ok = true;
  for (int a = 0; a < g.dim; ++a) {
    oc[a] = -1;
    for (int d = -2; d <= 2; ++d) {
      int o = cpc[a] + d;
      if (o < 0 || o >= g.nc1 || o % 3 != kk[a]) continue;
      if ((d > 0) == (((s >> a) & 1) == 1)) oc[a] = o;
    }
    if (oc[a] < 0) ok = false;
  }
  return ok;
}

constexpr int kChunks = 16;

// Block (c', sl) takes the sl-th of kChunks slices of the restriction list of
// coarse row node c' and, for the probed colour k, sums P[i, c'] y[i, q] per
// owner slot (the owner of mesh node i: the nearest coarse node of colour k).
// Sums in T within the block (fixed order), one partial per slice.
template <typename T, int NF>
__global__ void __launch_bounds__(kB) k_gather_coarse(CGeo g, const int64_t *__restrict__ rstart,
                                                      const int32_t *__restrict__ rnode,
                                                      const float *__restrict__ rw, const float *__restrict__ pos,
                                                      int k, const T *__restrict__ y, double *__restrict__ part) {
  const int cp = blockIdx.x, sl = blockIdx.y;
  int cpc[3] = {0, 0, 0}, kk[3] = {k % 3, (k / 3) % 3, k / 9};
  {
    int r = int(cp % g.ncn_inst);
    for (int a = 0; a < g.dim; ++a) { cpc[a] = r % g.nc1; r /= g.nc1; }
  }
  T acc[8][NF];
#pragma unroll
  for (int s = 0; s < 8; ++s)
#pragma unroll
    for (int q = 0; q < NF; ++q) acc[s][q] = T(0);
  const int64_t b0 = rstart[cp], len = rstart[cp + 1] - b0;
  const int64_t lo = b0 + len * sl / kChunks, hi = b0 + len * (sl + 1) / kChunks;
  for (int64_t e = lo + threadIdx.x; e < hi; e += kB) {
    const int64_t i = rnode[e];
    const T wgt = T(rw[e]);
    int slot = 0;
    bool ok = true;
    for (int a = 0; a < g.dim; ++a) {
      const float p = pos[i * g.dim + a];
      int o = kk[a] + 3 * (int)floorf((p - float(kk[a])) / 3.0f + 0.5f);
      if (o < 0 || o >= g.nc1) ok = false;
      if (o > cpc[a]) slot |= 1 << a;
    }
    if (!ok) continue;
    T yq[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) yq[q] = y[i * NF + q];
#pragma unroll
    for (int s = 0; s < 8; ++s)
      if (s == slot)
#pragma unroll
        for (int q = 0; q < NF; ++q) acc[s][q] = fma(wgt, yq[q], acc[s][q]);
  }
  __shared__ T red[kB / 32][8 * NF];
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 8; ++s)
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      const T v = warp_sum_t(acc[s][q]);
      if (ln == 0) red[wid][s * NF + q] = v;
    }
  __syncthreads();
  for (int t = threadIdx.x; t < 8 * NF; t += kB) {
    T v = T(0);
#pragma unroll
    for (int w = 0; w < kB / 32; ++w) v += red[w][t];
    part[(int64_t(cp) * kChunks + sl) * 8 * NF + t] = double(v);
  }
}

// A[(c', q), (owner(s), f)] = sum of the slices, in slice order
__global__ void k_gather_sum(CGeo g, int k, int f, const double *__restrict__ part, double *__restrict__ A,
                             int64_t ldA, int64_t ncn) {
  const int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x;
  const int nf = g.nf;
  if (t >= ncn * 8 * nf) return;
  const int cp = int(t / (8 * nf)), s = int((t / nf) % 8), q = int(t % nf);
  if (s >= (1 << g.dim)) return;
  const int64_t inst = cp / g.ncn_inst, lcp = cp % g.ncn_inst;
  int cpc[3] = {0, 0, 0}, kk[3] = {k % 3, (k / 3) % 3, k / 9}, oc[3];
  {
    int r = int(lcp);
    for (int a = 0; a < g.dim; ++a) { cpc[a] = r % g.nc1; r /= g.nc1; }
  }
  if (!slot_owner(g, cpc, kk, s, oc)) return;
  double v = 0.0;
  for (int sl = 0; sl < kChunks; ++sl) v += part[((int64_t(cp) * kChunks + sl) * 8 + s) * nf + q];
  double *Ai = A + inst * g.nc0 * ldA;
  Ai[(lcp * nf + q) * ldA + int64_t(lin(g, oc)) * nf + f] = v;
}

constexpr int kPiece = 1024;

// rc = R v = P^T v, node by node.  The mesh nodes of each coarse cell are
// stored together (cnodes) and cut into pieces; block p sums, for each of
// its cell's 2^d corners, w_corner(i) v[i, q] over the piece, in T within
// the block (fixed order; no FP64 instruction on the FP32 path, where the
// FP64 pipe is the narrow one).  The weights are those of k_block_prolong,
// so R is exactly P^T.
template <typename T, int NF, int DIM>
__global__ void __launch_bounds__(kB) k_restrict_cells(CGeo g, const float *__restrict__ pos,
                                                       const int32_t *__restrict__ cnodes,
                                                       const int32_t *__restrict__ piece_cell,
                                                       const int32_t *__restrict__ piece_begin,
                                                       const T *__restrict__ v, T *__restrict__ part) {
  constexpr int NC = 1 << DIM;
  const int p = blockIdx.x;
  float base[3] = {0.f, 0.f, 0.f};
  {
    int r = int(piece_cell[p] % g.ncell_inst);
#pragma unroll
    for (int a = 0; a < DIM; ++a) { base[a] = float(r % (g.nc1 - 1)); r /= (g.nc1 - 1); }
  }
  T acc[NC][NF];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < NF; ++q) acc[c][q] = T(0);
  const int e1 = piece_begin[p + 1];
  for (int e = piece_begin[p] + threadIdx.x; e < e1; e += kB) {
    const int64_t i = cnodes[e];
    T t[DIM], x[NF];
#pragma unroll
    for (int a = 0; a < DIM; ++a) t[a] = T(pos[i * DIM + a] - base[a]);
#pragma unroll
    for (int q = 0; q < NF; ++q) x[q] = v[i * NF + q];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T wc = T(1);
#pragma unroll
      for (int a = 0; a < DIM; ++a) wc *= ((c >> a) & 1) ? t[a] : T(1) - t[a];
#pragma unroll
      for (int q = 0; q < NF; ++q) acc[c][q] = fma(wc, x[q], acc[c][q]);
    }
  }
  __shared__ T red[kB / 32][NC * NF];
  const int wid = threadIdx.x >> 5, ln = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      const T sum = warp_sum_t(acc[c][q]);
      if (ln == 0) red[wid][c * NF + q] = sum;
    }
  __syncthreads();
  for (int k = threadIdx.x; k < NC * NF; k += kB) {
    T sum = T(0);
#pragma unroll
    for (int w = 0; w < kB / 32; ++w) sum += red[w][k];
    part[int64_t(p) * NC * NF + k] = sum;
  }
}

// rc[c', q]: the corner sums of the cells around coarse node c' -- the
// (piece, corner) entries listed for c' (corner by corner, each cell's
// pieces in order) -- one warp per coarse unknown, lanes over the entries
template <typename T>
__global__ void k_restrict_sum(int64_t nc, int nf, const int32_t *__restrict__ sptr,
                               const int32_t *__restrict__ sent, const T *__restrict__ part, T *__restrict__ rc) {
  const int64_t t = (blockIdx.x * int64_t(kB) + threadIdx.x) >> 5;
  const int ln = threadIdx.x & 31;
  if (t >= nc) return;
  const int64_t cp = t / nf;
  const int q = int(t % nf);
  T sum = T(0);
  for (int e = sptr[cp] + ln; e < sptr[cp + 1]; e += 32) sum += part[int64_t(sent[e]) * nf + q];
  sum = warp_sum_t(sum);
  if (ln == 0) rc[t] = sum;
}

// zc = A_c^{-1} rc, one warp per row, in precision T; row r of instance i at
// Minv + i * inst_stride + (r % nc0) * ld
template <typename T>
__global__ void k_coarse_matvec(const T *__restrict__ Minv, int64_t ld, int64_t inst_stride, int64_t nc,
                                int64_t nc0, const T *__restrict__ rc, T *__restrict__ zc) {
  const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int ln = threadIdx.x & 31;
  if (r >= nc) return;
  const int64_t inst = r / nc0, lr = r % nc0;
  const T *row = Minv + inst * inst_stride + lr * ld;
  const T *x = rc + inst * nc0;
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);  // four chains for load parallelism
  int64_t c = ln;
  for (; c + 96 < nc0; c += 128) {
    s0 = fma(row[c], x[c], s0);
    s1 = fma(row[c + 32], x[c + 32], s1);
    s2 = fma(row[c + 64], x[c + 64], s2);
    s3 = fma(row[c + 96], x[c + 96], s3);
  }
  for (; c < nc0; c += 32) s0 = fma(row[c], x[c], s0);
  T s = (s0 + s1) + (s2 + s3);
  s = warp_sum_t(s);
  if (ln == 0) zc[r] = s;
}

// z = Binv v + P zc  (nodal block-Jacobi plus the prolonged coarse
// correction; zc == nullptr: block-Jacobi only; Binv == nullptr: the coarse
// correction only)
template <typename T, int NF, int DIM>
__global__ void __launch_bounds__(kB) k_block_prolong(CGeo g, const float *__restrict__ pos,
                                                      const int32_t *__restrict__ node_inst,
                                                      const T *__restrict__ Binv, const T *__restrict__ v,
                                                      const T *__restrict__ zc, T *__restrict__ z) {
  for (int64_t i = blockIdx.x * int64_t(kB) + threadIdx.x; i < g.n_nodes; i += int64_t(gridDim.x) * kB) {
    T x[NF], acc[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) { x[q] = v[i * NF + q]; acc[q] = T(0); }
    if (zc) {
      int b[3];
      float tf[3];
      locate(g, pos + i * DIM, b, tf);
      const int64_t cbase = node_inst ? int64_t(node_inst[i]) * g.ncn_inst : 0;
      T t[DIM];
#pragma unroll
      for (int a = 0; a < DIM; ++a) t[a] = T(tf[a]);
#pragma unroll
      for (int c = 0; c < (1 << DIM); ++c) {
        T wc = T(1);
        int64_t idx = 0;
#pragma unroll
        for (int a = DIM - 1; a >= 0; --a) idx = idx * g.nc1 + b[a] + ((c >> a) & 1);
#pragma unroll
        for (int a = 0; a < DIM; ++a) wc *= ((c >> a) & 1) ? t[a] : T(1) - t[a];
        const T *zp = zc + (cbase + idx) * NF;
#pragma unroll
        for (int q = 0; q < NF; ++q) acc[q] = fma(wc, zp[q], acc[q]);
      }
    }
    if (!Binv) {  // coarse correction only
#pragma unroll
      for (int r = 0; r < NF; ++r) z[i * NF + r] = acc[r];
      continue;
    }
    T B[NF * NF];
    if constexpr ((NF * NF * sizeof(T)) % 16 == 0) {
      constexpr int L = 16 / sizeof(T);
      const V16<T> *Bv = reinterpret_cast<const V16<T> *>(Binv + i * NF * NF);
#pragma unroll
      for (int k = 0; k < NF * NF / L; ++k) {
        const V16<T> b = Bv[k];
#pragma unroll
        for (int l = 0; l < L; ++l) B[k * L + l] = b.a[l];
      }
    } else {
#pragma unroll
      for (int k = 0; k < NF * NF; ++k) B[k] = Binv[i * NF * NF + k];
    }
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      T s = acc[r];
#pragma unroll
      for (int c = 0; c < NF; ++c) s = fma(B[r * NF + c], x[c], s);
      z[i * NF + r] = s;
    }
  }
}

// A -> B elementwise with a type change (n values)
template <typename A, typename B>
__global__ void k_copy_cast(const A *__restrict__ x, int64_t n, B *__restrict__ y) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n; t += int64_t(gridDim.x) * kB) y[t] = B(x[t]);
}

// In-place Gauss-Jordan inversion of each instance's n x n block (row-major)
// with partial pivoting: pivot step k swaps the row of the largest |a_rk|,
// r >= k, into row k (recorded in piv), scales row k by d = 1/a_kk and puts
// d on the diagonal, and eliminates column k from the other rows, whose
// column k becomes -a_rk d; the recorded row interchanges are undone as
// column interchanges at the end.  No [A | I] copy: the working set is n^2
// values (76.5 MB in float at n = 4374, inside L2).
template <typename T>
__global__ void k_gj_pivot(T *__restrict__ Mall, int64_t n, int64_t k, T *__restrict__ colall,
                           int32_t *__restrict__ pivall, int *__restrict__ bad) {
  T *M = Mall + int64_t(blockIdx.x) * n * n;
  T *col = colall + int64_t(blockIdx.x) * n;
  __shared__ T bv[1024];
  __shared__ int64_t bi[1024];
  __shared__ T pv;
  T best = T(-1);
  int64_t arg = k;
  for (int64_t r = k + threadIdx.x; r < n; r += blockDim.x) {
    const T v = fabs(M[r * n + k]);
    if (v > best) { best = v; arg = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      if (bv[threadIdx.x + s] > bv[threadIdx.x] ||
          (bv[threadIdx.x + s] == bv[threadIdx.x] && bi[threadIdx.x + s] < bi[threadIdx.x])) {
        bv[threadIdx.x] = bv[threadIdx.x + s];
        bi[threadIdx.x] = bi[threadIdx.x + s];
      }
    }
    __syncthreads();
  }
  const int64_t p = bi[0];
  if (threadIdx.x == 0) {
    pv = M[p * n + k];
    pivall[int64_t(blockIdx.x) * n + k] = int32_t(p);
  }
  __syncthreads();
  if (!(fabs(pv) > T(0))) {
    if (threadIdx.x == 0) *bad = 1;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) col[r] = T(0);
    return;
  }
  const T d = T(1) / pv;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const T a = M[k * n + j], b = M[p * n + j];
    if (p != k) M[p * n + j] = a;
    M[k * n + j] = j == k ? d : b * d;
  }
  __syncthreads();
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) col[r] = r == k ? T(0) : M[r * n + k];
}

// elimination of column k: thread = one column j (coalesced along rows of
// the row-major block), block y = a range of kRowsGJ rows, z = instance
constexpr int kRowsGJ = 32;
template <typename T>
__global__ void __launch_bounds__(kB) k_gj_elim(T *__restrict__ Mall, int64_t n, int64_t k,
                                                const T *__restrict__ colall) {
  T *M = Mall + int64_t(blockIdx.z) * n * n;
  const T *col = colall + int64_t(blockIdx.z) * n;
  const int64_t j = blockIdx.x * int64_t(kB) + threadIdx.x;
  if (j >= n) return;
  const T d = M[k * n + k];
  const T rk = M[k * n + j];
  const int64_t r0 = int64_t(blockIdx.y) * kRowsGJ, r1 = r0 + kRowsGJ < n ? r0 + kRowsGJ : n;
  for (int64_t r = r0; r < r1; ++r) {
    if (r == k) continue;
    const T fr = col[r];
    T *a = M + r * n + j;
    if (j == k) *a = -fr * d;
    else if (fr != T(0)) *a = fma(-fr, rk, *a);
  }
}

// undo the row interchanges as column interchanges, last first (a thread per row)
template <typename T>
__global__ void k_gj_unswap(T *__restrict__ Mall, int64_t n, const int32_t *__restrict__ pivall, int n_inst) {
  for (int64_t t = blockIdx.x * int64_t(kB) + threadIdx.x; t < n * n_inst; t += int64_t(gridDim.x) * kB) {
    const int64_t inst = t / n, r = t % n;
    T *row = Mall + inst * n * n + r * n;
    const int32_t *piv = pivall + inst * n;
    for (int64_t k = n - 1; k >= 0; --k) {
      const int64_t p = piv[k];
      if (p != k) {
        const T x = row[k];
        row[k] = row[p];
        row[p] = x;
      }
    }
  }
}

template <typename T>
void gauss_jordan(T *M, int64_t n, int n_inst, T *col, int32_t *piv, int *bad, cudaStream_t st) {
  const dim3 ge((unsigned)((n + kB - 1) / kB), (unsigned)((n + kRowsGJ - 1) / kRowsGJ), (unsigned)n_inst);
  for (int64_t k = 0; k < n; ++k) {
    k_gj_pivot<T><<<n_inst, 1024, 0, st>>>(M, n, k, col, piv, bad);
    k_gj_elim<T><<<ge, kB, 0, st>>>(M, n, k, col);
  }
  k_gj_unswap<T><<<grid_n(n * n_inst), kB, 0, st>>>(M, n, piv, n_inst);
  note_launches(int(2 * n + 1));
}

}  // namespace

// ---------------------------------------------------------------- host side
Coarse::~Coarse() { release(); }

void Coarse::release() {
  cudaFree(pos);
  cudaFree(rstart);
  cudaFree(rnode);
  cudaFree(rw);
  cudaFree(cnodes);
  cudaFree(piece_cell);
  cudaFree(piece_begin);
  cudaFree(cell_piece);
  cudaFree(sptr);
  cudaFree(sent);
  sptr = sent = nullptr;
  pos = nullptr;
  rstart = nullptr;
  rnode = nullptr;
  rw = nullptr;
  cnodes = piece_cell = piece_begin = cell_piece = nullptr;
  ncell_inst = ncell = n_pieces = 0;
  M.release();
  Minv32.release();
  piv.release();
  vec.release();
  rpart.release();
  level = -1;
  ready = false;
}

chns_status coarse_setup(chns_mesh *m, int Lc) {
  Coarse &C = m->coarse;
  if (C.level == Lc && C.pos) return CHNS_OK;
  C.release();
  // a uniform mesh may be its own coarse grid (P = I, A_c = J: an exact solve)
  const int lc_max = m->uniform ? m->min_level : m->min_level - 1;
  if (Lc < 1 || Lc > lc_max) {
    set_error("coarse level %d must be in [1, %d] (below the coarsest leaf level, or equal on a uniform mesh)",
              Lc, lc_max);
    return CHNS_ERR_ARG;
  }
  const int dim = m->dim, nf = m->nf, ni = m->n_inst;
  const int nc1 = (1 << Lc) + 1;
  int64_t ncn = 1;
  for (int a = 0; a < dim; ++a) ncn *= nc1;
  std::vector<float> pos(size_t(m->n_nodes) * dim);
  std::vector<int> base(size_t(m->n_nodes) * dim);
  std::vector<int64_t> cbase(m->n_nodes);  // first coarse node of the node's instance
  for (int q = 0; q < ni; ++q) {
    const double scale = std::ldexp(1.0, Lc - m->inst_max_level[q]);
    for (int64_t i = m->inst_node_start[q]; i < m->inst_node_start[q + 1]; ++i) {
      cbase[i] = int64_t(q) * ncn;
      for (int a = 0; a < dim; ++a) {
        double p = double(m->node_xyz[i * dim + a]) * scale;
        pos[i * dim + a] = float(p);
        int b = (int)std::floor(p);
        base[i * dim + a] = std::min(std::max(b, 0), nc1 - 2);
      }
    }
  }
  auto corners = [&](int64_t i, auto &&fn) {
    for (int c = 0; c < (1 << dim); ++c) {
      double w = 1.0;
      int64_t idx = 0;
      for (int a = dim - 1; a >= 0; --a) {
        int ca = base[i * dim + a] + ((c >> a) & 1);
        double t = double(pos[i * dim + a]) - base[i * dim + a];
        w *= ((c >> a) & 1) ? t : 1.0 - t;
        idx = idx * nc1 + ca;
      }
      if (w != 0.0) fn(cbase[i] + idx, w);
    }
  };
  const int64_t ncn_all = ncn * ni;
  std::vector<int64_t> cnt(ncn_all + 1, 0);
  for (int64_t i = 0; i < m->n_nodes; ++i) corners(i, [&](int64_t idx, double) { cnt[idx + 1]++; });
  for (int64_t c = 0; c < ncn_all; ++c) cnt[c + 1] += cnt[c];
  std::vector<int32_t> rnode(cnt[ncn_all]);
  std::vector<float> rw(cnt[ncn_all]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t i = 0; i < m->n_nodes; ++i)
    corners(i, [&](int64_t idx, double w) {
      rnode[fill[idx]] = (int32_t)i;
      rw[fill[idx]++] = (float)w;
    });
  CHNS_CUDA_TRY(cudaMalloc(&C.pos, sizeof(float) * pos.size()));
  CHNS_CUDA_TRY(cudaMemcpy(C.pos, pos.data(), sizeof(float) * pos.size(), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.rstart, sizeof(int64_t) * cnt.size()));
  CHNS_CUDA_TRY(cudaMemcpy(C.rstart, cnt.data(), sizeof(int64_t) * cnt.size(), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.rnode, sizeof(int32_t) * std::max<size_t>(rnode.size(), 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.rnode, rnode.data(), sizeof(int32_t) * rnode.size(), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.rw, sizeof(float) * std::max<size_t>(rw.size(), 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.rw, rw.data(), sizeof(float) * rw.size(), cudaMemcpyHostToDevice));
  // nodes grouped by coarse cell (stable: node order within a cell), pieces
  int64_t ncell_inst = 1;
  for (int a = 0; a < dim; ++a) ncell_inst *= (nc1 - 1);
  const int64_t ncell = ncell_inst * ni;
  std::vector<int64_t> ccnt(ncell + 1, 0);
  std::vector<int64_t> cell_of(m->n_nodes);
  for (int64_t i = 0; i < m->n_nodes; ++i) {
    int64_t c = 0;
    for (int a = dim - 1; a >= 0; --a) c = c * (nc1 - 1) + base[i * dim + a];
    cell_of[i] = cbase[i] / ncn * ncell_inst + c;
    ccnt[cell_of[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) ccnt[c + 1] += ccnt[c];
  std::vector<int32_t> cnodes(m->n_nodes);
  {
    std::vector<int64_t> f(ccnt.begin(), ccnt.end() - 1);
    for (int64_t i = 0; i < m->n_nodes; ++i) cnodes[f[cell_of[i]]++] = (int32_t)i;
  }
  std::vector<int32_t> piece_cell, piece_begin, cell_piece(ncell + 1, 0);
  for (int64_t c = 0; c < ncell; ++c) {
    cell_piece[c] = (int32_t)piece_cell.size();
    for (int64_t b = ccnt[c]; b < ccnt[c + 1]; b += kPiece) {
      piece_cell.push_back((int32_t)c);
      piece_begin.push_back((int32_t)b);
    }
  }
  cell_piece[ncell] = (int32_t)piece_cell.size();
  piece_begin.push_back((int32_t)m->n_nodes);
  // restriction-sum lists: for coarse node c', entries piece * 2^dim + corner
  // of the cells around it (corner of c' in that cell), corner by corner
  std::vector<int32_t> sptr(ncn_all + 1, 0), sent;
  for (int64_t cp = 0; cp < ncn_all; ++cp) {
    const int64_t inst = cp / ncn;
    int cc[3] = {0, 0, 0};
    {
      int64_t r = cp % ncn;
      for (int a = 0; a < dim; ++a) { cc[a] = int(r % nc1); r /= nc1; }
    }
    for (int s = 0; s < (1 << dim); ++s) {
      int64_t cell = 0;
      bool ok = true;
      for (int a = dim - 1; a >= 0; --a) {
        const int ca = cc[a] - ((s >> a) & 1);
        if (ca < 0 || ca > nc1 - 2) ok = false;
        cell = cell * (nc1 - 1) + ca;
      }
      if (!ok) continue;
      const int64_t gc = inst * ncell_inst + cell;
      for (int32_t p = cell_piece[gc]; p < cell_piece[gc + 1]; ++p) sent.push_back(p * (1 << dim) + s);
    }
    sptr[cp + 1] = (int32_t)sent.size();
  }
  const int64_t np = (int64_t)piece_cell.size();
  CHNS_CUDA_TRY(cudaMalloc(&C.cnodes, sizeof(int32_t) * std::max<size_t>(cnodes.size(), 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.cnodes, cnodes.data(), sizeof(int32_t) * cnodes.size(), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.piece_cell, sizeof(int32_t) * std::max<int64_t>(np, 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.piece_cell, piece_cell.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.piece_begin, sizeof(int32_t) * (np + 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.piece_begin, piece_begin.data(), sizeof(int32_t) * (np + 1), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.sptr, sizeof(int32_t) * sptr.size()));
  CHNS_CUDA_TRY(cudaMemcpy(C.sptr, sptr.data(), sizeof(int32_t) * sptr.size(), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.sent, sizeof(int32_t) * std::max<size_t>(sent.size(), 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.sent, sent.data(), sizeof(int32_t) * sent.size(), cudaMemcpyHostToDevice));
  CHNS_CUDA_TRY(cudaMalloc(&C.cell_piece, sizeof(int32_t) * (ncell + 1)));
  CHNS_CUDA_TRY(cudaMemcpy(C.cell_piece, cell_piece.data(), sizeof(int32_t) * (ncell + 1), cudaMemcpyHostToDevice));
  C.ncell_inst = ncell_inst;
  C.ncell = ncell;
  C.n_pieces = np;
  C.level = Lc;
  C.nc1 = nc1;
  C.n_inst = ni;
  C.ncn_inst = ncn;
  C.nc0 = ncn * nf;
  C.ncn = ncn_all;
  C.nc = ncn_all * nf;
  TRY_CHNS(C.M.ensure(sizeof(double) * C.nc0 * C.nc0 * ni));
  TRY_CHNS(C.piv.ensure(sizeof(int32_t) * C.nc0 * ni));
  TRY_CHNS(C.Minv32.ensure(sizeof(float) * C.nc0 * C.nc0 * ni));
  TRY_CHNS(C.vec.ensure(sizeof(double) * (3 * C.nc + 8 + C.ncn * kChunks * 8 * nf)));
  TRY_CHNS(C.rpart.ensure(sizeof(double) * std::max<int64_t>(np, 1) * (1 << dim) * nf));
  return CHNS_OK;
}

template <typename T>
chns_status coarse_build(chns_mesh *m, JvFn<T> jv, void *ctx, T *w, T *y, cudaStream_t st) {
  Coarse &C = m->coarse;
  const int nf = m->nf, dim = m->dim;
  CGeo g{dim, nf, C.nc1, m->n_nodes, C.ncn_inst, C.nc0, C.ncell_inst};
  double *M = C.M.as<double>();
  const int64_t nc0 = C.nc0, nn = nc0 * nc0 * C.n_inst;
  CHNS_CUDA_TRY(cudaMemsetAsync(M, 0, sizeof(double) * nn, st));
  const int ncol = dim == 2 ? 9 : 27;
  double *part = C.vec.as<double>() + 3 * C.nc + 8;
  for (int k = 0; k < ncol; ++k)
    for (int f = 0; f < nf; ++f) {
      if (dim == 2) k_probe_coarse<T, 5, 2><<<grid_n(m->n_nodes), kB, 0, st>>>(g, C.pos, k, f, w);
      else k_probe_coarse<T, 6, 3><<<grid_n(m->n_nodes), kB, 0, st>>>(g, C.pos, k, f, w);
      note_launches(1);
      TRY_CHNS(jv(ctx, w, y));
      dim3 gr((unsigned)C.ncn, kChunks);
      if (nf == 5)
        k_gather_coarse<T, 5><<<gr, kB, 0, st>>>(g, C.rstart, C.rnode, C.rw, C.pos, k, y, part);
      else
        k_gather_coarse<T, 6><<<gr, kB, 0, st>>>(g, C.rstart, C.rnode, C.rw, C.pos, k, y, part);
      k_gather_sum<<<(unsigned)((C.ncn * 8 * nf + kB - 1) / kB), kB, 0, st>>>(g, k, f, part, M, nc0, C.ncn);
      note_launches(2);
    }
  // A_c^{-1} per instance, in the element precision: the FP32 path inverts
  // in float (A_c is ill-conditioned along a pressure direction only, which
  // float resolves: per-field errors of the applied inverse ~1e-6 at
  // cond(A_c) ~ 1e9), the FP64 path in double.  Both copies are kept: M in
  // double, Minv32 in float.
  void *colv = C.vec.as<double>() + 2 * C.nc;  // nc0 per instance
  int *bad = reinterpret_cast<int *>(C.vec.as<double>() + 3 * C.nc);
  int32_t *piv = C.piv.as<int32_t>();
  float *M32 = C.Minv32.as<float>();
  CHNS_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
  if (sizeof(T) == sizeof(float)) {
    k_copy_cast<double, float><<<grid_n(nn), kB, 0, st>>>(M, nn, M32);
    gauss_jordan<float>(M32, nc0, C.n_inst, static_cast<float *>(colv), piv, bad, st);
    k_copy_cast<float, double><<<grid_n(nn), kB, 0, st>>>(M32, nn, M);
  } else {
    gauss_jordan<double>(M, nc0, C.n_inst, static_cast<double *>(colv), piv, bad, st);
    k_copy_cast<double, float><<<grid_n(nn), kB, 0, st>>>(M, nn, M32);
  }
  note_launches(2);
  int hbad = 0;
  CHNS_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHNS_CUDA_TRY(cudaStreamSynchronize(st));
  if (hbad) { set_error("singular coarse operator"); return CHNS_ERR_KRYLOV; }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error("coarse build: %s", cudaGetErrorString(e)); return CHNS_ERR_CUDA; }
  C.ready = true;
  return CHNS_OK;
}
template chns_status coarse_build<float>(chns_mesh *, JvFn<float>, void *, float *, float *, cudaStream_t);
template chns_status coarse_build<double>(chns_mesh *, JvFn<double>, void *, double *, double *, cudaStream_t);

// z = B^{-1} v (+ P A_c^{-1} R v when the coarse space is ready and wanted)
template <typename T>
void precond_apply(chns_mesh *m, const T *Binv, bool coarse, const T *v, T *z, cudaStream_t st) {
  Coarse &C = m->coarse;
  const bool use = coarse && C.ready;
  CGeo g{m->dim, m->nf, C.nc1, m->n_nodes, C.ncn_inst, C.nc0, C.ncell_inst};
  T *rc = nullptr, *zc = nullptr;
  if (use) {
    rc = reinterpret_cast<T *>(C.vec.as<double>());
    zc = reinterpret_cast<T *>(C.vec.as<double>() + C.nc);
    T *part = reinterpret_cast<T *>(C.rpart.as<double>());
    const unsigned np = (unsigned)C.n_pieces;
    const unsigned gs = (unsigned)((C.nc * 32 + kB - 1) / kB);
    if (m->dim == 2)
      k_restrict_cells<T, 5, 2><<<np, kB, 0, st>>>(g, C.pos, C.cnodes, C.piece_cell, C.piece_begin, v, part);
    else
      k_restrict_cells<T, 6, 3><<<np, kB, 0, st>>>(g, C.pos, C.cnodes, C.piece_cell, C.piece_begin, v, part);
    k_restrict_sum<T><<<gs, kB, 0, st>>>(C.nc, m->nf, C.sptr, C.sent, part, rc);
    const unsigned gm = (unsigned)((C.nc * 32 + kB - 1) / kB);
    if (sizeof(T) == sizeof(float))
      k_coarse_matvec<T><<<gm, kB, 0, st>>>(reinterpret_cast<const T *>(C.Minv32.as<float>()), C.nc0,
                                            C.nc0 * C.nc0, C.nc, C.nc0, rc, zc);
    else
      k_coarse_matvec<T><<<gm, kB, 0, st>>>(reinterpret_cast<const T *>(C.M.as<double>()), C.nc0,
                                            C.nc0 * C.nc0, C.nc, C.nc0, rc, zc);
    note_launches(3);
  }
  const int32_t *ni = (use && m->n_inst > 1) ? m->node_inst : nullptr;
  if (m->dim == 2) k_block_prolong<T, 5, 2><<<grid_n(m->n_nodes), kB, 0, st>>>(g, C.pos, ni, Binv, v, zc, z);
  else k_block_prolong<T, 6, 3><<<grid_n(m->n_nodes), kB, 0, st>>>(g, C.pos, ni, Binv, v, zc, z);
  note_launches(1);
}
template void precond_apply<float>(chns_mesh *, const float *, bool, const float *, float *, cudaStream_t);
template void precond_apply<double>(chns_mesh *, const double *, bool, const double *, double *, cudaStream_t);

}  // namespace chns
