// Element kernels of the matrix-free CN-VMS CHNS operator (Sec. 3.4 fully
// discrete form, Sec. 3.1 time averages) on Q1 leaves with hanging nodes
// (Sec. 4), and the small node kernels around them.
//
// Thread mapping: an element owns 2^D consecutive lanes of a warp.  Lane c is
// corner c of the element while gathering and scattering, and Gauss point c
// (xi_a = +-1/sqrt(3) by bit a of c) while evaluating the physics.  Moving
// between the two uses the tensor-product structure of Q1 with the 2-point
// Gauss rule: per axis a butterfly between the lanes that differ in that
// axis' bit (one warp shuffle), which gives values, gradients and mixed second
// derivatives at all Gauss points, and its transpose, which contracts the
// Gauss-point coefficients with N_a and grad N_a.
//
// The Jacobian-vector product evaluates the same Gauss-point physics on dual
// numbers (value, derivative along w).
#include <algorithm>
#include <cstdint>

#include "chns_internal.h"
#include "kernels.h"

namespace chns {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- dual numbers
template <typename T>
struct Dl {
  T v, d;
  __device__ __forceinline__ Dl() {}
  __device__ __forceinline__ Dl(T a) : v(a), d(T(0)) {}
  __device__ __forceinline__ Dl(T a, T b) : v(a), d(b) {}
};
template <typename T> __device__ __forceinline__ Dl<T> operator+(Dl<T> a, Dl<T> b) { return Dl<T>(a.v + b.v, a.d + b.d); }
template <typename T> __device__ __forceinline__ Dl<T> operator-(Dl<T> a, Dl<T> b) { return Dl<T>(a.v - b.v, a.d - b.d); }
template <typename T> __device__ __forceinline__ Dl<T> operator-(Dl<T> a) { return Dl<T>(-a.v, -a.d); }
template <typename T> __device__ __forceinline__ Dl<T> operator*(Dl<T> a, Dl<T> b) { return Dl<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <typename T> __device__ __forceinline__ Dl<T> operator+(Dl<T> a, T b) { return Dl<T>(a.v + b, a.d); }
template <typename T> __device__ __forceinline__ Dl<T> operator-(Dl<T> a, T b) { return Dl<T>(a.v - b, a.d); }
template <typename T> __device__ __forceinline__ Dl<T> operator*(Dl<T> a, T b) { return Dl<T>(a.v * b, a.d * b); }
template <typename T> __device__ __forceinline__ Dl<T> operator*(T b, Dl<T> a) { return Dl<T>(a.v * b, a.d * b); }
template <typename T> __device__ __forceinline__ T val(Dl<T> a) { return a.v; }
__device__ __forceinline__ float val(float a) { return a; }
__device__ __forceinline__ double val(double a) { return a; }

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float rcp_(float x) { return 1.0f / x; }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
template <typename T> __device__ __forceinline__ Dl<T> rcp_(Dl<T> a) {
  T r = rcp_(a.v);
  return Dl<T>(r, -a.d * r * r);
}
// rad^(-1/2) and its derivative -1/2 rad^(-3/2) rad'
template <typename T> __device__ __forceinline__ Dl<T> rsqrt_(Dl<T> a) {
  T r = rsqrt_(a.v);
  return Dl<T>(r, T(-0.5) * a.d * r * r * r);
}

// ---------------------------------------------------------------- butterflies
template <typename T>
struct Stage {
  T ca, cb;      // (1 + g)/2, (1 - g)/2 with g = 1/sqrt(3)
  T sh[3];       // (+1 or -1 by lane bit) / h_a : physical derivative of the 1D hat
};

template <typename T>
__device__ __forceinline__ void st_vd(T u, int m, T ca, T cb, T sh, T &v, T &d) {
  T o = __shfl_xor_sync(FULL, u, m);
  v = ca * u + cb * o;
  d = sh * (u - o);
}
template <typename T>
__device__ __forceinline__ T st_v(T u, int m, T ca, T cb) {
  T o = __shfl_xor_sync(FULL, u, m);
  return ca * u + cb * o;
}

// value only
template <int D, typename T>
__device__ __forceinline__ T ip_v(T u, const Stage<T> &s) {
  T a = st_v(u, 1, s.ca, s.cb);
  a = st_v(a, 2, s.ca, s.cb);
  if (D == 3) a = st_v(a, 4, s.ca, s.cb);
  return a;
}

// value and gradient
template <int D, typename T>
__device__ __forceinline__ void ip_vg(T u, const Stage<T> &s, T &v, T *g) {
  T A, Bx;
  st_vd(u, 1, s.ca, s.cb, s.sh[0], A, Bx);
  if (D == 2) {
    st_vd(A, 2, s.ca, s.cb, s.sh[1], v, g[1]);
    g[0] = st_v(Bx, 2, s.ca, s.cb);
  } else {
    T AA, AB;
    st_vd(A, 2, s.ca, s.cb, s.sh[1], AA, AB);
    T BA = st_v(Bx, 2, s.ca, s.cb);
    st_vd(AA, 4, s.ca, s.cb, s.sh[2], v, g[2]);
    g[1] = st_v(AB, 4, s.ca, s.cb);
    g[0] = st_v(BA, 4, s.ca, s.cb);
  }
}

// value, gradient and mixed second derivatives (xy; xy, xz, yz in 3D); the
// pure second derivatives of Q1 vanish on an axis-aligned box
template <int D, typename T>
__device__ __forceinline__ void ip_full(T u, const Stage<T> &s, T &v, T *g, T *hs) {
  T A, Bx;
  st_vd(u, 1, s.ca, s.cb, s.sh[0], A, Bx);
  if (D == 2) {
    st_vd(A, 2, s.ca, s.cb, s.sh[1], v, g[1]);
    st_vd(Bx, 2, s.ca, s.cb, s.sh[1], g[0], hs[0]);
  } else {
    T AA, AB, BA, BB;
    st_vd(A, 2, s.ca, s.cb, s.sh[1], AA, AB);
    st_vd(Bx, 2, s.ca, s.cb, s.sh[1], BA, BB);
    st_vd(AA, 4, s.ca, s.cb, s.sh[2], v, g[2]);
    st_vd(AB, 4, s.ca, s.cb, s.sh[2], g[1], hs[2]);
    st_vd(BA, 4, s.ca, s.cb, s.sh[2], g[0], hs[1]);
    hs[0] = st_v(BB, 4, s.ca, s.cb);
  }
}

// transpose: r_node = sum_gp N_node(gp) S(gp) + grad N_node(gp) . V(gp)
template <int D, typename T>
__device__ __forceinline__ T contract(T S, const T *V, const Stage<T> &s) {
  T X = s.ca * S + s.sh[0] * V[0] + __shfl_xor_sync(FULL, s.cb * S - s.sh[0] * V[0], 1);
  T Y1 = s.ca * V[1] + __shfl_xor_sync(FULL, s.cb * V[1], 1);
  if (D == 2) {
    return s.ca * X + s.sh[1] * Y1 + __shfl_xor_sync(FULL, s.cb * X - s.sh[1] * Y1, 2);
  } else {
    T Y2 = s.ca * V[2] + __shfl_xor_sync(FULL, s.cb * V[2], 1);
    T X2 = s.ca * X + s.sh[1] * Y1 + __shfl_xor_sync(FULL, s.cb * X - s.sh[1] * Y1, 2);
    T Z2 = s.ca * Y2 + __shfl_xor_sync(FULL, s.cb * Y2, 2);
    return s.ca * X2 + s.sh[2] * Z2 + __shfl_xor_sync(FULL, s.cb * X2 - s.sh[2] * Z2, 4);
  }
}

// ---------------------------------------------------------------- node gather / scatter
// Node blocks are N consecutive values at p = base + node * N: for even N the
// block starts on a 2-element boundary (float2 / double2 loads), for N = 4
// floats on a 16-byte boundary (float4).
template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

template <int N, typename T>
__device__ __forceinline__ void load_block(const T *__restrict__ p, T *out) {
  if constexpr (N == 4 && sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else if constexpr (N % 2 == 0) {
    using P = typename Pair<T>::type;
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      const P v = __ldg(reinterpret_cast<const P *>(p) + k);
      out[2 * k] = v.x;
      out[2 * k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = __ldg(p + k);
  }
}

// corner value through the hanging constraint: mean of 2 or 4 parents
template <int N, typename T>
__device__ __forceinline__ void gather(int cn, const int32_t *__restrict__ hang,
                                       const T *__restrict__ src, T *out) {
  if (cn >= 0) {
    load_block<N>(src + (int64_t)cn * N, out);
  } else {
    const int4 p = reinterpret_cast<const int4 *>(hang)[-cn - 1];
    T a[N], b[N];
    load_block<N>(src + (int64_t)p.x * N, a);
    load_block<N>(src + (int64_t)p.y * N, b);
    if (p.z < 0) {
#pragma unroll
      for (int k = 0; k < N; ++k) out[k] = T(0.5) * (a[k] + b[k]);
    } else {
      T c[N], d[N];
      load_block<N>(src + (int64_t)p.z * N, c);
      load_block<N>(src + (int64_t)p.w * N, d);
#pragma unroll
      for (int k = 0; k < N; ++k) out[k] = T(0.25) * ((a[k] + b[k]) + (c[k] + d[k]));
    }
  }
}

template <int N, typename T, typename O>
__device__ __forceinline__ void add_block(O *__restrict__ p, const T *r, T wgt) {
  if constexpr (N % 2 == 0) {
    using P = typename Pair<O>::type;
    P *q = reinterpret_cast<P *>(p);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      P v = q[k];
      v.x += O(wgt * r[2 * k]);
      v.y += O(wgt * r[2 * k + 1]);
      q[k] = v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) p[k] += O(wgt * r[k]);
  }
}

template <int N, typename T>
__device__ __forceinline__ void store_block(T *__restrict__ p, const T *r) {
  if constexpr (N % 2 == 0) {
    using P = typename Pair<T>::type;
    P *q = reinterpret_cast<P *>(p);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      P v;
      v.x = r[2 * k];
      v.y = r[2 * k + 1];
      q[k] = v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) p[k] = r[k];
  }
}

// non-atomic: elements of one launch (one colour) touch disjoint nodes
template <int N, typename T, typename O>
__device__ __forceinline__ void scatter(int cn, const int32_t *__restrict__ hang, O *__restrict__ dst,
                                        const T *r) {
  if (cn >= 0) {
    add_block<N>(dst + (int64_t)cn * N, r, T(1));
  } else {
    const int4 p = reinterpret_cast<const int4 *>(hang)[-cn - 1];
    T wgt = p.z < 0 ? T(0.5) : T(0.25);
    add_block<N>(dst + (int64_t)p.x * N, r, wgt);
    add_block<N>(dst + (int64_t)p.y * N, r, wgt);
    if (p.z >= 0) {
      add_block<N>(dst + (int64_t)p.z * N, r, wgt);
      add_block<N>(dst + (int64_t)p.w * N, r, wgt);
    }
  }
}

// ---------------------------------------------------------------- Gauss-point physics
template <int D, typename S>
struct GpIn {
  S vt[D], dvt[D][D];  // v~ and d_j v~_i (dvt[i][j])
  S pt, dpt[D];        // p~
  S phit, dphit[D], hphit[3];  // phi~, gradient, mixed second derivatives
  S mut, dmut[D];      // mu~
  S dv[D];             // v^{k+1} - v^k
  S dphi;              // phi^{k+1} - phi^k
  S phin, dphin[D];    // phi^{k+1} and its gradient
  S f[D + 3];          // forcing at t_{k+1/2}
};

template <typename T>
struct KCoef {
  T inv_dt, four_dt2, alpha, beta, gamma, xi, jc;
  T inv_Pe, inv_We, inv_Re, inv_Fr, CnWe, inv_PeCn, Cn2, C_I;
  T g[3];
  T ext[3];  // box extent per axis
};

template <int D> __device__ __forceinline__ int hidx(int i, int j) {
  // index of the mixed derivative d_i d_j (i != j) in hphit
  return D == 2 ? 0 : (i + j - 1);
}

// Weak-form coefficients at one Gauss point: the row of test function N_a
// receives W (N_a Sq[k] + sum_j d_j N_a Vq[k][j]) for equation k.  floored:
// whether the tau_m radicand was raised to 4/dt^2.
template <int D, typename T, typename S>
__device__ __forceinline__ void gp_physics(const KCoef<T> &c, const T *G, T CI_GG, T inv_trG,
                                           const GpIn<D, S> &q, S *Sq, S (*Vq)[D], bool &floored) {
  // phi* clip (Eq. phi_for_density) and mixture properties at t_{k+1}
  const T pn = val(q.phin);
  const bool inside = fabs(pn) <= T(1);
  S phis = inside ? q.phin : S(pn > T(0) ? T(1) : T(-1));
  S rho = c.alpha * phis + c.beta;
  S eta = c.gamma * phis + c.xi;
  S inv_rho = rcp_(rho);
  S deta[D];
#pragma unroll
  for (int k = 0; k < D; ++k) deta[k] = inside ? c.gamma * q.dphin[k] : S(T(0));
  // thermodynamic-consistency flux
  S J[D];
#pragma unroll
  for (int i = 0; i < D; ++i) J[i] = c.jc * q.dmut[i];
  // tau_m, tau_c with G = diag(4/h^2); radicand floored at 4/dt^2
  S vGv = S(T(0)), vGJ = S(T(0));
#pragma unroll
  for (int i = 0; i < D; ++i) {
    vGv = vGv + G[i] * (q.vt[i] * q.vt[i]);
    vGJ = vGJ + G[i] * (q.vt[i] * J[i]);
  }
  S visc = eta * inv_rho * c.inv_Re;
  S rad = vGv + vGJ * inv_rho * c.inv_Pe + CI_GG * (visc * visc) + c.four_dt2;
  floored = val(rad) < c.four_dt2;
  if (floored) rad = S(c.four_dt2);
  S tau = rsqrt_(rad);
  S tau_c = inv_trG * rcp_(tau);
  // strong residuals
  S Rm[D], conv[D], flux[D];
  S divv = S(T(0));
#pragma unroll
  for (int i = 0; i < D; ++i) {
    S cv = S(T(0)), fl = S(T(0)), cap = S(T(0)), vs = S(T(0));
#pragma unroll
    for (int j = 0; j < D; ++j) {
      cv = cv + q.vt[j] * q.dvt[i][j];
      fl = fl + J[j] * q.dvt[i][j];
      vs = vs + deta[j] * q.dvt[i][j];
      if (j != i) cap = cap + q.hphit[hidx<D>(i, j)] * q.dphit[j];
    }
    conv[i] = cv;
    flux[i] = fl;
    divv = divv + q.dvt[i][i];
    Rm[i] = rho * (q.dv[i] * c.inv_dt + cv) + fl * c.inv_Pe + c.CnWe * cap + q.dpt[i] * c.inv_We -
            vs * c.inv_Re - rho * (c.g[i] * c.inv_Fr) - q.f[i];
  }
  S Rc = divv - q.f[D];
  // momentum rows
  S tR[D];
#pragma unroll
  for (int j = 0; j < D; ++j) tR[j] = tau * Rm[j];
  S diag = (rho * tau_c * Rc - q.pt) * c.inv_We;
  S etaRe = eta * c.inv_Re;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    S cross = S(T(0));
#pragma unroll
    for (int j = 0; j < D; ++j) cross = cross + tR[j] * q.dvt[i][j];
    Sq[i] = rho * (q.dv[i] * c.inv_dt + conv[i]) - cross + flux[i] * c.inv_Pe -
            rho * (c.g[i] * c.inv_Fr) - q.f[i];
    S b = tR[i] * inv_rho;  // tau R_i / rho
#pragma unroll
    for (int j = 0; j < D; ++j)
      Vq[i][j] = q.vt[j] * tR[i] - tR[j] * b + c.inv_Pe * J[j] * b -
                 c.CnWe * (q.dphit[i] * q.dphit[j]) + etaRe * q.dvt[i][j];
    Vq[i][i] = Vq[i][i] + diag;
  }
  // continuity row with PSPG
  Sq[D] = divv - q.f[D];
#pragma unroll
  for (int i = 0; i < D; ++i) Vq[D][i] = tR[i] * inv_rho;
  // Cahn-Hilliard row
  Sq[D + 1] = q.dphi * c.inv_dt - q.f[D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) Vq[D + 1][i] = c.inv_PeCn * q.dmut[i] - q.vt[i] * q.phit;
  // chemical-potential row, psi'(phi~) = phi~^3 - phi~
  Sq[D + 2] = q.phit * q.phit * q.phit - q.phit - q.mut - q.f[D + 2];
#pragma unroll
  for (int i = 0; i < D; ++i) Vq[D + 2][i] = c.Cn2 * q.dphit[i];
}

template <int D, typename T>
struct Interp {  // one state interpolated at the lane's Gauss point
  T vt[D], dvt[D][D], pt, dpt[D], phit, dphit[D], hphit[3], mut, dmut[D];
};

template <int D, typename T>
__device__ __forceinline__ void interp_state(const T *u, const Stage<T> &s, Interp<D, T> &I) {
#pragma unroll
  for (int i = 0; i < D; ++i) ip_vg<D>(u[i], s, I.vt[i], I.dvt[i]);
  ip_vg<D>(u[D], s, I.pt, I.dpt);
  I.hphit[1] = I.hphit[2] = T(0);
  ip_full<D>(u[D + 1], s, I.phit, I.dphit, I.hphit);
  ip_vg<D>(u[D + 2], s, I.mut, I.dmut);
}

template <typename T>
KCoef<T> kcoef(const PhysCoef &p) {
  KCoef<T> c;
  c.inv_dt = T(p.inv_dt); c.four_dt2 = T(p.four_dt2);
  c.alpha = T(p.alpha); c.beta = T(p.beta); c.gamma = T(p.gamma); c.xi = T(p.xi); c.jc = T(p.jc);
  c.inv_Pe = T(p.inv_Pe); c.inv_We = T(p.inv_We); c.inv_Re = T(p.inv_Re); c.inv_Fr = T(p.inv_Fr);
  c.CnWe = T(p.CnWe); c.inv_PeCn = T(p.inv_PeCn); c.Cn2 = T(p.Cn2); c.C_I = T(p.C_I);
  for (int a = 0; a < 3; ++a) {
    c.g[a] = T(p.g[a]);
    c.ext[a] = T(p.ext[a]);
  }
  return c;
}

// ---------------------------------------------------------------- the element kernel
// MODE 0: residual (output O = double), MODE 1: J.w into the element-local
// slots (O = T), MODE 2: count of the Gauss points whose tau_m radicand is
// floored (O = unsigned long long, one counter), MODE 3: J.w scattered into
// the node vector (O = T; one launch per element colour).  BS, MINB: block
// size and minimum resident blocks per SM (the register budget).
template <int D, typename T, int MODE, bool HASF, typename O, int BS = 128, int MINB = 6>
__global__ void __launch_bounds__(BS, MINB) k_element(
    const int32_t *__restrict__ conn, const uint8_t *__restrict__ level,
    const int32_t *__restrict__ hang, int64_t e_begin, int64_t e_end,
    const T *__restrict__ ut, const T *__restrict__ dl, const T *__restrict__ w,
    const T *__restrict__ f, O *__restrict__ out, KCoef<T> c0, const KCoef<T> *__restrict__ tab,
    const uint16_t *__restrict__ einst) {
  constexpr int NC = 1 << D, NF = D + 3, ND = D + 1;
  const int lc = threadIdx.x & (NC - 1);
  int64_t e = e_begin + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> D);
  const bool active = e < e_end;
  if (!active) e = e_end - 1;  // keep the lanes alive for the shuffles
  const int cn = conn[e * NC + lc];
  // batched meshes: the coefficients of the element's own problem instance
  const KCoef<T> c = tab ? tab[einst[e]] : c0;

  // gather the corner's nodal blocks
  T u[NF], d[ND];
  gather<NF>(cn, hang, ut, u);
  gather<ND>(cn, hang, dl, d);
  T wn[NF];
  if (MODE == 1 || MODE == 3) gather<NF>(cn, hang, w, wn);
  T fn[NF];
  if (HASF) gather<NF>(cn, hang, f, fn);

  // geometry of this leaf
  const T scale = T(1) / T(1u << level[e]);
  const T *ext = c.ext;
  Stage<T> s;
  s.ca = T(0.5) + T(0.28867513459481288225);  // (1 + 1/sqrt(3)) / 2
  s.cb = T(0.5) - T(0.28867513459481288225);
  T G[D], trG = T(0), GG = T(0), W = T(1);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T h = ext[a] * scale;
    s.sh[a] = ((lc >> a) & 1) ? T(1) / h : T(-1) / h;
    G[a] = T(4) / (h * h);
    trG += G[a];
    GG += G[a] * G[a];
    W *= T(0.5) * h;
  }
  const T CI_GG = c.C_I * GG, inv_trG = T(1) / trG;

  // interpolate to the lane's Gauss point
  Interp<D, T> A;
  interp_state<D>(u, s, A);
  T dvq[D], dphiq, dphig[D];
#pragma unroll
  for (int i = 0; i < D; ++i) dvq[i] = ip_v<D>(d[i], s);
  ip_vg<D>(d[D], s, dphiq, dphig);
  T fq[NF];
#pragma unroll
  for (int k = 0; k < NF; ++k) fq[k] = HASF ? ip_v<D>(fn[k], s) : T(0);

  T r[NF];
  bool floored = false;
  if (MODE == 0 || MODE == 2) {
    GpIn<D, T> q;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      q.vt[i] = A.vt[i];
      q.dv[i] = dvq[i];
      q.dpt[i] = A.dpt[i];
      q.dphit[i] = A.dphit[i];
      q.dmut[i] = A.dmut[i];
      q.dphin[i] = A.dphit[i] + T(0.5) * dphig[i];
#pragma unroll
      for (int j = 0; j < D; ++j) q.dvt[i][j] = A.dvt[i][j];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) q.hphit[k] = A.hphit[k];
    q.pt = A.pt;
    q.phit = A.phit;
    q.mut = A.mut;
    q.dphi = dphiq;
    q.phin = A.phit + T(0.5) * dphiq;
#pragma unroll
    for (int k = 0; k < NF; ++k) q.f[k] = fq[k];
    T Sq[NF], Vq[NF][D];
    gp_physics<D, T, T>(c, G, CI_GG, inv_trG, q, Sq, Vq, floored);
    if constexpr (MODE == 2) {
      const unsigned b = __ballot_sync(FULL, floored && active);
      if ((threadIdx.x & 31) == 0 && b) atomicAdd(reinterpret_cast<unsigned long long *>(out), (unsigned long long)__popc(b));
      return;
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      T Vk[D];
#pragma unroll
      for (int j = 0; j < D; ++j) Vk[j] = W * Vq[k][j];
      r[k] = contract<D>(W * Sq[k], Vk, s);
    }
  } else {
    // perturbation U_new + e w: v~, p~, phi~, mu~ move by w/2, increments by w
    Interp<D, T> B;
    interp_state<D>(wn, s, B);
    GpIn<D, Dl<T>> q;
    const T hf = T(0.5);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      q.vt[i] = Dl<T>(A.vt[i], hf * B.vt[i]);
      q.dv[i] = Dl<T>(dvq[i], B.vt[i]);
      q.dpt[i] = Dl<T>(A.dpt[i], hf * B.dpt[i]);
      q.dphit[i] = Dl<T>(A.dphit[i], hf * B.dphit[i]);
      q.dmut[i] = Dl<T>(A.dmut[i], hf * B.dmut[i]);
      q.dphin[i] = Dl<T>(A.dphit[i] + hf * dphig[i], B.dphit[i]);
#pragma unroll
      for (int j = 0; j < D; ++j) q.dvt[i][j] = Dl<T>(A.dvt[i][j], hf * B.dvt[i][j]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) q.hphit[k] = Dl<T>(A.hphit[k], hf * B.hphit[k]);
    q.pt = Dl<T>(A.pt, hf * B.pt);
    q.phit = Dl<T>(A.phit, hf * B.phit);
    q.mut = Dl<T>(A.mut, hf * B.mut);
    q.dphi = Dl<T>(dphiq, B.phit);
    q.phin = Dl<T>(A.phit + hf * dphiq, B.phit);
#pragma unroll
    for (int k = 0; k < NF; ++k) q.f[k] = Dl<T>(fq[k]);
    Dl<T> Sq[NF], Vq[NF][D];
    gp_physics<D, T, Dl<T>>(c, G, CI_GG, inv_trG, q, Sq, Vq, floored);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      T Vk[D];
#pragma unroll
      for (int j = 0; j < D; ++j) Vk[j] = W * Vq[k][j].d;
      r[k] = contract<D>(W * Sq[k].d, Vk, s);
    }
  }
  if constexpr (MODE == 1) {
    // J.w: element-local output, slot (e, corner); k_gather_nodes sums the
    // slots of each node in a fixed order
    if (active) store_block<NF>(reinterpret_cast<T *>(out) + (e * NC + lc) * NF, r);
  } else if constexpr (MODE == 0 || MODE == 3) {
    // Lanes of one element may reach the same node: a hanging corner's parents
    // can be corners of the element or parents of its other hanging corner.
    // Warps that hold a hanging corner scatter one corner index at a time.
    if (__any_sync(FULL, cn < 0)) {
#pragma unroll 1
      for (int k = 0; k < NC; ++k) {
        if (active && lc == k) scatter<NF>(cn, hang, out, r);
        __syncwarp();
      }
    } else if (active) {
      scatter<NF>(cn, hang, out, r);
    }
  }
}

// ---------------------------------------------------------------- node kernels
// v~ = (U_new + U_old)/2 for all fields; increments of v and phi
template <int D, typename T>
__global__ void k_prep(const double *__restrict__ Un, const double *__restrict__ Uo, int64_t n,
                       T *__restrict__ ut, T *__restrict__ dl) {
  constexpr int NF = D + 3, ND = D + 1;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double a[NF], b[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) { a[k] = Un[i * NF + k]; b[k] = Uo[i * NF + k]; }
#pragma unroll
    for (int k = 0; k < NF; ++k) ut[i * NF + k] = T(0.5 * (a[k] + b[k]));
#pragma unroll
    for (int k = 0; k < D; ++k) dl[i * ND + k] = T(a[k] - b[k]);
    dl[i * ND + D] = T(a[D + 1] - b[D + 1]);
  }
}

// y[i] = sum over the slots of node i of weight * E[slot] (fixed order), then
// the constrained rows: y = w on wall velocities and the pinned pressure.
// The slots of a node are fetched eight at a time (independent loads), then
// added in list order.
template <int D, typename T>
__global__ void __launch_bounds__(256) k_gather_nodes(const int32_t *__restrict__ gptr,
                                                      const int32_t *__restrict__ gent,
                                                      const uint8_t *__restrict__ nflag, int64_t n_nodes,
                                                      const T *__restrict__ E, const T *__restrict__ w,
                                                      T *__restrict__ y, uint32_t fmask) {
  constexpr int NF = D + 3, G = 8;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n_nodes; i += int64_t(gridDim.x) * blockDim.x) {
    T acc[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) acc[k] = T(0);
    const int p0 = gptr[i], p1 = gptr[i + 1];
    for (int pb = p0; pb < p1; pb += G) {
      uint32_t ent[G];
#pragma unroll
      for (int g = 0; g < G; ++g) ent[g] = pb + g < p1 ? uint32_t(gent[pb + g]) : 0xffffffffu;
      T v[G][NF];
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (ent[g] != 0xffffffffu) load_block<NF>(E + int64_t(ent[g] & 0x3fffffffu) * NF, v[g]);
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (ent[g] != 0xffffffffu) {
          const uint32_t code = ent[g] >> 30;
          const T wt = code == 0 ? T(1) : (code == 1 ? T(0.5) : T(0.25));
#pragma unroll
          for (int k = 0; k < NF; ++k) acc[k] = fma(wt, v[g][k], acc[k]);
        }
    }
    const uint8_t fl = nflag[i];
    if (fl & 1)
#pragma unroll
      for (int k = 0; k < D; ++k) acc[k] = w[i * NF + k];
    if (fl & 2) acc[D] = w[i * NF + D];
    if (fmask != 0xffu)
#pragma unroll
      for (int k = 0; k < NF; ++k)
        if (!((fmask >> k) & 1u)) acc[k] = w[i * NF + k];
    store_block<NF>(y + i * NF, acc);
  }
}

// J.w by colour scatter: the constrained rows and the rows of fields outside
// fmask become y = w (as k_gather_nodes does after its sums)
template <int D, typename T>
__global__ void k_fix_rows(const uint8_t *__restrict__ nflag, int64_t n_nodes, const T *__restrict__ w,
                           T *__restrict__ y, uint32_t fmask) {
  constexpr int NF = D + 3;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n_nodes; i += int64_t(gridDim.x) * blockDim.x) {
    const uint8_t fl = nflag[i];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const bool keep = ((fmask >> k) & 1u) && !((fl & 1) && k < D) && !((fl & 2) && k == D);
      if (!keep) y[i * NF + k] = w[i * NF + k];
    }
  }
}

// constrained rows of the residual: wall velocities and the pinned pressure
__global__ void k_dirichlet_res(const int32_t *__restrict__ wall, int64_t n_wall, const int32_t *__restrict__ pins,
                                int64_t n_pins, int dim, const double *__restrict__ Un,
                                const double *__restrict__ bc, double *__restrict__ F) {
  const int nf = dim + 3;
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n_wall) {
    int64_t b = int64_t(wall[i]) * nf;
    for (int k = 0; k < dim; ++k) F[b + k] = Un[b + k] - (bc ? bc[b + k] : 0.0);
  }
  if (i < n_pins) {
    int64_t b = int64_t(pins[i]) * nf + dim;
    F[b] = Un[b] - (bc ? bc[b] : 0.0);
  }
}

// ---------------------------------------------------------------- diagnostics
// per block: energy, integral of phi, volume with phi < 0 (2^D Gauss rule)
template <int D>
__global__ void __launch_bounds__(256) k_energy(
    const int32_t *__restrict__ conn, const uint8_t *__restrict__ level,
    const uint32_t *__restrict__ anchor, const int32_t *__restrict__ hang, int64_t n_elem,
    const double *__restrict__ U, KCoef<double> c, double ext0, double ext1, double ext2,
    double lo0, double lo1, double lo2, double inv_top, double *__restrict__ partial) {
  constexpr int NC = 1 << D, NF = D + 3;
  const int lc = threadIdx.x & (NC - 1);
  int64_t e = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> D;
  const bool active = e < n_elem;
  if (!active) e = n_elem - 1;
  const int cn = conn[e * NC + lc];
  double u[NF];
  gather<NF>(cn, hang, U, u);
  const double ext[3] = {ext0, ext1, ext2}, lo[3] = {lo0, lo1, lo2};
  const double scale = 1.0 / double(1u << level[e]);
  Stage<double> s;
  s.ca = 0.5 + 0.28867513459481288225;
  s.cb = 0.5 - 0.28867513459481288225;
  double W = 1.0, zg = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double h = ext[a] * scale;
    s.sh[a] = ((lc >> a) & 1) ? 1.0 / h : -1.0 / h;
    W *= 0.5 * h;
    double xi = ((lc >> a) & 1) ? 0.57735026918962576451 : -0.57735026918962576451;
    double x = lo[a] + ext[a] * double(anchor[e * D + a]) * inv_top + 0.5 * (1.0 + xi) * h;
    zg -= c.g[a] * x;
  }
  double v2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double vi = ip_v<D>(u[i], s);
    v2 += vi * vi;
  }
  double phi, dphi[D];
  ip_vg<D>(u[D + 1], s, phi, dphi);
  double g2 = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) g2 += dphi[i] * dphi[i];
  double phis = fabs(phi) <= 1.0 ? phi : (phi > 0 ? 1.0 : -1.0);
  double rho = c.alpha * phis + c.beta;
  double psi = 0.25 * (phi * phi - 1.0) * (phi * phi - 1.0);
  double E = 0.0, M = 0.0, Lt = 0.0;
  if (active) {
    // Cn^2/2 |grad phi|^2 / (Cn We) = Cn/(2 We) |grad phi|^2 ; psi/(Cn We)
    E = W * (0.5 * rho * v2 + c.CnWe / (c.Cn2) * psi + 0.5 * c.CnWe * g2 + rho * zg * c.inv_Fr);
    M = W * phi;
    Lt = phi < 0.0 ? W : 0.0;
  }
  // deterministic block reduction
  __shared__ double sh[3][256 / 32];
  for (int o = 16; o > 0; o >>= 1) {
    E += __shfl_down_sync(FULL, E, o);
    M += __shfl_down_sync(FULL, M, o);
    Lt += __shfl_down_sync(FULL, Lt, o);
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][wid] = E; sh[1][wid] = M; sh[2][wid] = Lt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, d = 0;
    for (int k = 0; k < int(blockDim.x >> 5); ++k) { a += sh[0][k]; b += sh[1][k]; d += sh[2][k]; }
    partial[blockIdx.x * 3 + 0] = a;
    partial[blockIdx.x * 3 + 1] = b;
    partial[blockIdx.x * 3 + 2] = d;
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers
PhysCoef make_coef(const chns_params &p, const double *lo, const double *hi) {
  PhysCoef c;
  c.dt = p.dt;
  c.inv_dt = 1.0 / p.dt;
  c.four_dt2 = 4.0 / (p.dt * p.dt);
  c.alpha = 0.5 * (1.0 - p.rho_ratio);
  c.beta = 0.5 * (1.0 + p.rho_ratio);
  c.gamma = 0.5 * (1.0 - p.eta_ratio);
  c.xi = 0.5 * (1.0 + p.eta_ratio);
  c.jc = 0.5 * (p.rho_ratio - 1.0);
  c.inv_Pe = 1.0 / p.Pe;
  c.inv_We = 1.0 / p.We;
  c.inv_Re = 1.0 / p.Re;
  c.inv_Fr = 1.0 / p.Fr;
  c.CnWe = p.Cn / p.We;
  c.inv_PeCn = 1.0 / (p.Pe * p.Cn);
  c.Cn2 = p.Cn * p.Cn;
  c.C_I = p.C_I;
  for (int a = 0; a < 3; ++a) {
    c.g[a] = p.gravity[a];
    c.ext[a] = hi[a] - lo[a];
    c.lo[a] = lo[a];
  }
  c.fmask = 0xffu;
  return c;
}

namespace {
constexpr int kBlock = 256;
inline unsigned grid_for(int64_t threads) { return (unsigned)((threads + kBlock - 1) / kBlock); }
// element kernels: 128 threads (16 leaves in 3D), 6 blocks per SM (measured
// slightly ahead of 256 x 3 on the uniform and the adaptive meshes)
constexpr int kElemBlock = 128;
// FP64 element kernels: 3 blocks of 128 threads per SM (up to 170 registers)
constexpr int kFp64MinBlocks = 3;
inline unsigned grid_elem(int64_t threads) { return (unsigned)((threads + kElemBlock - 1) / kElemBlock); }
inline unsigned grid_nodes(int64_t n) {
  int64_t b = (n + kBlock - 1) / kBlock;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}
}  // namespace

template <typename T>
void launch_prep(const chns_mesh *m, const double *Un, const double *Uo, T *ut, T *dl, cudaStream_t st) {
  if (m->dim == 2) { k_prep<2, T><<<grid_nodes(m->n_nodes), kBlock, 0, st>>>(Un, Uo, m->n_nodes, ut, dl); note_launches(1); }
  else { k_prep<3, T><<<grid_nodes(m->n_nodes), kBlock, 0, st>>>(Un, Uo, m->n_nodes, ut, dl); note_launches(1); }
}
template void launch_prep<float>(const chns_mesh *, const double *, const double *, float *, float *, cudaStream_t);
template void launch_prep<double>(const chns_mesh *, const double *, const double *, double *, double *, cudaStream_t);

namespace {
template <int D, typename T, int MODE, bool HASF, typename O>
void element_pass(const chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, const T *w,
                  const T *f, O *out, cudaStream_t st, int colour_lo, int colour_hi) {
  KCoef<T> c = kcoef<T>(pc);
  constexpr int MINB = sizeof(T) == 8 ? kFp64MinBlocks : 6;
  for (int col = colour_lo; col < colour_hi; ++col) {
    int64_t b = m->colour_start[col], e = m->colour_start[col + 1];
    if (e <= b) continue;
    k_element<D, T, MODE, HASF, O, 128, MINB><<<grid_elem((e - b) << D), kElemBlock, 0, st>>>(
        m->conn, m->level, m->hang, b, e, ut, dl, w, f, out, c,
        reinterpret_cast<const KCoef<T> *>(sizeof(T) == 8 ? m->coef64 : m->coef32), m->elem_inst);
    note_launches(1);
  }
}
}  // namespace

void launch_residual(const chns_mesh *m, const PhysCoef &pc, const double *ut, const double *dl,
                     const double *f, double *F, cudaStream_t st) {
  if (m->dim == 2) {
    if (f) element_pass<2, double, 0, true, double>(m, pc, ut, dl, nullptr, f, F, st, 0, m->n_colours);
    else element_pass<2, double, 0, false, double>(m, pc, ut, dl, nullptr, nullptr, F, st, 0, m->n_colours);
  } else {
    if (f) element_pass<3, double, 0, true, double>(m, pc, ut, dl, nullptr, f, F, st, 0, m->n_colours);
    else element_pass<3, double, 0, false, double>(m, pc, ut, dl, nullptr, nullptr, F, st, 0, m->n_colours);
  }
}

// J.w schedules (chosen per mesh by the autotuner, FP32 only; FP64 always
// uses schedule 0):
//   0: all elements at once into the element-local buffer E (n_elem * 2^dim
//      * nf values of T), 128-thread blocks, 6 per SM; then the node gather
//      with the constrained rows (no colouring, no output zeroing)
//   1: as 0 with 256-thread blocks, 3 per SM
//   2: as 0 with 64-thread blocks, 12 per SM
//   3: as 0 with 128-thread blocks, 8 per SM (at most 64 registers)
//   4: element colours one launch after another, each element adding its
//      contributions into y (disjoint nodes within a colour; no E buffer),
//      then the constrained rows
//   5: as 0 with 128-thread blocks, 5 per SM (up to 102 registers)
//   6: as 0 with 128-thread blocks, 4 per SM (up to 128 registers)
template <int D, typename T, int BS, int MINB>
static void jv_elemlocal(const chns_mesh *m, const KCoef<T> &c, const KCoef<T> *tab, const T *ut, const T *dl,
                         const T *w, T *E, T *y, uint32_t fmask, cudaStream_t st) {
  const int64_t threads = m->n_elem << D;
  k_element<D, T, 1, false, T, BS, MINB><<<(unsigned)((threads + BS - 1) / BS), BS, 0, st>>>(
      m->conn, m->level, m->hang, 0, m->n_elem, ut, dl, w, nullptr, E, c, tab, m->elem_inst);
  k_gather_nodes<D, T><<<grid_nodes(m->n_nodes), kBlock, 0, st>>>(m->gptr, m->gent, m->nflag, m->n_nodes, E, w, y,
                                                                  fmask);
  note_launches(2);
}

template <int D, typename T>
static void jv_colours(const chns_mesh *m, const KCoef<T> &c, const KCoef<T> *tab, const T *ut, const T *dl,
                       const T *w, T *y, uint32_t fmask, cudaStream_t st) {
  cudaMemsetAsync(y, 0, sizeof(T) * m->n_nodes * (D + 3), st);
  for (int col = 0; col < m->n_colours; ++col) {
    const int64_t b = m->colour_start[col], e = m->colour_start[col + 1];
    if (e <= b) continue;
    k_element<D, T, 3, false, T><<<grid_elem((e - b) << D), kElemBlock, 0, st>>>(
        m->conn, m->level, m->hang, b, e, ut, dl, w, nullptr, y, c, tab, m->elem_inst);
    note_launches(1);
  }
  k_fix_rows<D, T><<<grid_nodes(m->n_nodes), kBlock, 0, st>>>(m->nflag, m->n_nodes, w, y, fmask);
  note_launches(1);
}

template <int D, typename T>
static void jv_dispatch(const chns_mesh *m, int variant, const KCoef<T> &c, const KCoef<T> *tab, const T *ut,
                        const T *dl, const T *w, T *E, T *y, uint32_t fmask, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    switch (variant) {
      case 1: jv_elemlocal<D, T, 256, 3>(m, c, tab, ut, dl, w, E, y, fmask, st); return;
      case 2: jv_elemlocal<D, T, 64, 12>(m, c, tab, ut, dl, w, E, y, fmask, st); return;
      case 3: jv_elemlocal<D, T, 128, 8>(m, c, tab, ut, dl, w, E, y, fmask, st); return;
      case 4: jv_colours<D, T>(m, c, tab, ut, dl, w, y, fmask, st); return;
      case 5: jv_elemlocal<D, T, 128, 5>(m, c, tab, ut, dl, w, E, y, fmask, st); return;
      case 6: jv_elemlocal<D, T, 128, 4>(m, c, tab, ut, dl, w, E, y, fmask, st); return;
      default: break;
    }
  }
  if constexpr (sizeof(T) == 8) {
    // FP64: bound by the narrow FP64 pipe, so occupancy matters less than
    // the register spills a 6-blocks-per-SM budget causes
    jv_elemlocal<D, T, 128, kFp64MinBlocks>(m, c, tab, ut, dl, w, E, y, fmask, st);
  } else {
    jv_elemlocal<D, T, 128, 6>(m, c, tab, ut, dl, w, E, y, fmask, st);
  }
}

template <typename T>
void launch_jacvec(const chns_mesh *m, const PhysCoef &pc, const T *ut, const T *dl, const T *w, T *E, T *y,
                   cudaStream_t st, int variant) {
  KCoef<T> c = kcoef<T>(pc);
  const KCoef<T> *tab = reinterpret_cast<const KCoef<T> *>(sizeof(T) == 8 ? m->coef64 : m->coef32);
  if (variant < 0) variant = sizeof(T) == 4 ? m->jv_variant : 0;
  if (m->dim == 2) jv_dispatch<2, T>(m, variant, c, tab, ut, dl, w, E, y, pc.fmask, st);
  else jv_dispatch<3, T>(m, variant, c, tab, ut, dl, w, E, y, pc.fmask, st);
}
template void launch_jacvec<float>(const chns_mesh *, const PhysCoef &, const float *, const float *,
                                   const float *, float *, float *, cudaStream_t, int);
template void launch_jacvec<double>(const chns_mesh *, const PhysCoef &, const double *, const double *,
                                    const double *, double *, double *, cudaStream_t, int);

// Gauss points with a floored tau_m radicand, added to *count (all elements
// in one launch, FP64 physics as in the residual)
void launch_tau_floor_count(const chns_mesh *m, const PhysCoef &pc, const double *ut, const double *dl,
                            unsigned long long *count, cudaStream_t st) {
  KCoef<double> c = kcoef<double>(pc);
  const KCoef<double> *tab = reinterpret_cast<const KCoef<double> *>(m->coef64);
  if (m->dim == 2)
    k_element<2, double, 2, false, unsigned long long><<<grid_elem(m->n_elem << 2), kElemBlock, 0, st>>>(
        m->conn, m->level, m->hang, 0, m->n_elem, ut, dl, nullptr, nullptr, count, c, tab, m->elem_inst);
  else
    k_element<3, double, 2, false, unsigned long long><<<grid_elem(m->n_elem << 3), kElemBlock, 0, st>>>(
        m->conn, m->level, m->hang, 0, m->n_elem, ut, dl, nullptr, nullptr, count, c, tab, m->elem_inst);
  note_launches(1);
}

void launch_dirichlet_res(const chns_mesh *m, const double *Un, const double *bc, double *F, cudaStream_t st) {
  int64_t n = std::max<int64_t>(std::max(m->n_wall, m->n_pins), 1);
  k_dirichlet_res<<<grid_for(n), kBlock, 0, st>>>(m->wall, m->n_wall, m->pins, m->n_pins, m->dim, Un, bc, F);
  note_launches(1);
}

chns_status upload_coef_tables(chns_mesh *m, const std::vector<PhysCoef> &pcs, cudaStream_t st) {
  const size_t n = pcs.size();
  if (!m->coef32) {
    CHNS_CUDA_TRY(cudaMalloc(&m->coef32, sizeof(KCoef<float>) * n));
    CHNS_CUDA_TRY(cudaMalloc(&m->coef64, sizeof(KCoef<double>) * n));
  }
  std::vector<KCoef<float>> a(n);
  std::vector<KCoef<double>> b(n);
  for (size_t i = 0; i < n; ++i) {
    a[i] = kcoef<float>(pcs[i]);
    b[i] = kcoef<double>(pcs[i]);
  }
  CHNS_CUDA_TRY(cudaMemcpyAsync(m->coef32, a.data(), sizeof(KCoef<float>) * n, cudaMemcpyHostToDevice, st));
  CHNS_CUDA_TRY(cudaMemcpyAsync(m->coef64, b.data(), sizeof(KCoef<double>) * n, cudaMemcpyHostToDevice, st));
  CHNS_CUDA_TRY(cudaStreamSynchronize(st));
  return CHNS_OK;
}

// the per-instance coefficient tables of src, copied to dst (same instances)
chns_status copy_coef_tables(const chns_mesh *src, chns_mesh *dst) {
  if (!src->coef32) { set_error("union mesh without coefficient tables"); return CHNS_ERR_ARG; }
  const size_t n = (size_t)src->n_inst;
  if (!dst->coef32) {
    CHNS_CUDA_TRY(cudaMalloc(&dst->coef32, sizeof(KCoef<float>) * n));
    CHNS_CUDA_TRY(cudaMalloc(&dst->coef64, sizeof(KCoef<double>) * n));
  }
  CHNS_CUDA_TRY(cudaMemcpy(dst->coef32, src->coef32, sizeof(KCoef<float>) * n, cudaMemcpyDeviceToDevice));
  CHNS_CUDA_TRY(cudaMemcpy(dst->coef64, src->coef64, sizeof(KCoef<double>) * n, cudaMemcpyDeviceToDevice));
  return CHNS_OK;
}

int64_t energy_blocks(const chns_mesh *m) { return (int64_t)grid_for(m->n_elem << m->dim); }

void launch_energy(const chns_mesh *m, const PhysCoef &pc, const double *U, double *partial,
                   cudaStream_t st) {
  KCoef<double> c = kcoef<double>(pc);
  double inv_top = 1.0 / double(int64_t(1) << m->max_level);
  unsigned g = grid_for(m->n_elem << m->dim);
  if (m->dim == 2)
    k_energy<2><<<g, kBlock, 0, st>>>(m->conn, m->level, m->anchor, m->hang, m->n_elem, U, c, pc.ext[0],
                                      pc.ext[1], pc.ext[2], pc.lo[0], pc.lo[1], pc.lo[2], inv_top, partial);
  else
    k_energy<3><<<g, kBlock, 0, st>>>(m->conn, m->level, m->anchor, m->hang, m->n_elem, U, c, pc.ext[0],
                                      pc.ext[1], pc.ext[2], pc.lo[0], pc.lo[1], pc.lo[2], inv_top, partial);
  note_launches(1);
}

}  // namespace chns
