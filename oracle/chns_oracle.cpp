// CHNS oracle: a plain, slow FP64 CPU implementation of the fully discrete
// Crank-Nicolson VMS Cahn-Hilliard-Navier-Stokes residual (Sec. 3.1 time
// scheme, Sec. 3.4 fully discrete VMS form) on cG(1) elements over the leaves
// of a 2:1 balanced octree (Sec. 4), and of its exact Jacobian-vector product.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
// baseline leg of the benchmark load this library.  It shares no code with the
// CUDA path.
//
// Structure (deliberately unoptimised):
//   * mesh: corners of all leaves -> sorted unique node list; a node lying at an
//     edge midpoint or face centre of another leaf is hanging and is replaced by
//     the mean of that edge's / face's corners (conforming cG(1), Sec. 4
//     "Handling hanging nodes").  The constraint is stored as an explicit
//     sparse matrix P: each element corner owns a list of (independent node,
//     weight) pairs.
//   * element residual: per Gauss point, evaluate the Q1 basis directly,
//     interpolate U^{k+1} and U^k, form the time averages of Sec. 3.1, the
//     phase-dependent properties with the phi* clip (Eq. phi_for_density),
//     tau_m / tau_c and the strong residuals R_m, R_c (Sec. 3.4), then add the
//     weak terms one by one in the order the paper lists them.
//   * J.w: the same element routine evaluated on dual numbers seeded with w,
//     i.e. the definition J.w = d/de F(U^{k+1} + e w) |_{e=0}.
//   * Dirichlet velocity rows on the walls and a pressure pin at the origin
//     node replace the corresponding weak rows.
//
// Readings of the paper that this file encodes (all listed with their reasons
// in the design notes): nondimensional flux coefficient (rho_r - 1)/2; G =
// diag(4/h_i^2); Delta t in tau_m is the time step; tau_m uses the time
// averaged velocity and flux and rho, eta of phi*^{k+1}; a tau_m radicand
// below 4/dt^2 is raised to 4/dt^2 (zero derivative); the PSPG term of the
// continuity row enters with a plus sign; the cross-stress term is
// -(w_i, tau_m R_m,j d_j v_i); the forcing, when given, is subtracted inside
// R_m and R_c as well as from the Galerkin rows; at |phi| = 1 the clip takes
// its interior branch.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline double sqrt(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

// ---------------------------------------------------------------- parameters
struct Params {
  int dim;
  double dt, Cn, Re, We, Pe, Fr, rho_r, eta_r, C_I, g[3];
};

Params unpack(const double* p) {
  Params q;
  q.dim = (int)p[0];
  q.dt = p[1]; q.Cn = p[2]; q.Re = p[3]; q.We = p[4]; q.Pe = p[5]; q.Fr = p[6];
  q.rho_r = p[7]; q.eta_r = p[8]; q.C_I = p[9];
  q.g[0] = p[10]; q.g[1] = p[11]; q.g[2] = p[12];
  return q;
}

// ---------------------------------------------------------------- mesh
struct Mesh {
  int dim = 0, max_level = 0, nc = 0, nf = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int64_t n_elem = 0;
  std::vector<int> level;
  std::vector<int64_t> anchor;          // n_elem * dim
  int64_t n_nodes = 0;                  // independent nodes
  std::vector<int64_t> node_xyz;        // n_nodes * dim integer coordinates
  std::vector<int64_t> P_start;         // n_elem * nc + 1
  std::vector<int64_t> P_node;
  std::vector<double> P_w;
  std::vector<uint8_t> on_wall;         // n_nodes
  int64_t origin = -1;
  int64_t n_hanging = 0;
  std::string err;
  // element colours for the threaded J.w (built on first use): elements of
  // one colour share no independent node through P
  std::vector<std::vector<int64_t>> colour_elems;
};

// canonical key: z slowest, x fastest
int64_t pkey(const int64_t* x, int dim, int64_t M) {
  int64_t k = 0;
  for (int a = dim - 1; a >= 0; --a) k = k * (M + 1) + x[a];
  return k;
}

bool build_mesh(Mesh& m) {
  const int dim = m.dim;
  const int64_t M = int64_t(1) << m.max_level;
  m.nc = 1 << dim;
  m.nf = dim + 3;
  // every corner of every leaf
  std::vector<int64_t> all;
  all.reserve(m.n_elem * m.nc);
  for (int64_t e = 0; e < m.n_elem; ++e) {
    int64_t s = int64_t(1) << (m.max_level - m.level[e]);
    for (int c = 0; c < m.nc; ++c) {
      int64_t x[3];
      for (int a = 0; a < dim; ++a) x[a] = m.anchor[e * dim + a] + (((c >> a) & 1) ? s : 0);
      all.push_back(pkey(x, dim, M));
    }
  }
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  auto is_node = [&](int64_t k) { return std::binary_search(all.begin(), all.end(), k); };
  // hanging nodes: nodes at an edge midpoint / face centre of some leaf
  std::map<int64_t, std::vector<int64_t>> hang;  // key -> parent keys
  for (int64_t e = 0; e < m.n_elem; ++e) {
    if (m.level[e] >= m.max_level) continue;
    int64_t s = int64_t(1) << (m.max_level - m.level[e]);
    int npat = 1;
    for (int a = 0; a < dim; ++a) npat *= 3;
    for (int pat = 0; pat < npat; ++pat) {
      int choice[3], t = pat, nhalf = 0;
      for (int a = 0; a < dim; ++a) { choice[a] = t % 3; t /= 3; if (choice[a] == 1) ++nhalf; }
      if (nhalf == 0 || nhalf == dim) continue;  // corners and the element centre
      int64_t x[3];
      for (int a = 0; a < dim; ++a) x[a] = m.anchor[e * dim + a] + choice[a] * (s / 2);
      int64_t k = pkey(x, dim, M);
      if (!is_node(k)) continue;
      std::vector<int64_t> par;
      for (int b = 0; b < (1 << nhalf); ++b) {
        int64_t y[3];
        int bit = 0;
        for (int a = 0; a < dim; ++a) {
          if (choice[a] == 1) { y[a] = m.anchor[e * dim + a] + (((b >> bit) & 1) ? s : 0); ++bit; }
          else y[a] = m.anchor[e * dim + a] + (choice[a] == 2 ? s : 0);
        }
        par.push_back(pkey(y, dim, M));
      }
      std::sort(par.begin(), par.end());
      auto it = hang.find(k);
      if (it == hang.end()) hang[k] = par;
      else if (it->second != par) { m.err = "inconsistent hanging constraint"; return false; }
    }
  }
  m.n_hanging = (int64_t)hang.size();
  std::vector<int64_t> indep;
  indep.reserve(all.size());
  for (int64_t k : all) if (!hang.count(k)) indep.push_back(k);
  for (auto& h : hang)
    for (int64_t p : h.second)
      if (!std::binary_search(indep.begin(), indep.end(), p)) {
        m.err = "hanging node constrained by a hanging node (mesh not 2:1 balanced)";
        return false;
      }
  m.n_nodes = (int64_t)indep.size();
  m.node_xyz.resize(m.n_nodes * dim);
  m.on_wall.assign(m.n_nodes, 0);
  for (int64_t i = 0; i < m.n_nodes; ++i) {
    int64_t k = indep[i];
    bool wall = false;
    for (int a = 0; a < dim; ++a) {
      int64_t c = k % (M + 1);
      k /= (M + 1);
      m.node_xyz[i * dim + a] = c;
      if (c == 0 || c == M) wall = true;
    }
    m.on_wall[i] = wall;
  }
  int64_t zero[3] = {0, 0, 0};
  m.origin = std::lower_bound(indep.begin(), indep.end(), pkey(zero, dim, M)) - indep.begin();
  auto index_of = [&](int64_t k) {
    return (int64_t)(std::lower_bound(indep.begin(), indep.end(), k) - indep.begin());
  };
  // constraint matrix P, one row list per element corner
  m.P_start.assign(m.n_elem * m.nc + 1, 0);
  m.P_node.clear();
  m.P_w.clear();
  for (int64_t e = 0; e < m.n_elem; ++e) {
    int64_t s = int64_t(1) << (m.max_level - m.level[e]);
    for (int c = 0; c < m.nc; ++c) {
      int64_t x[3];
      for (int a = 0; a < dim; ++a) x[a] = m.anchor[e * dim + a] + (((c >> a) & 1) ? s : 0);
      int64_t k = pkey(x, dim, M);
      auto it = hang.find(k);
      if (it == hang.end()) {
        m.P_node.push_back(index_of(k));
        m.P_w.push_back(1.0);
      } else {
        double w = 1.0 / (double)it->second.size();
        for (int64_t p : it->second) { m.P_node.push_back(index_of(p)); m.P_w.push_back(w); }
      }
      m.P_start[e * m.nc + c + 1] = (int64_t)m.P_node.size();
    }
  }
  return true;
}

// ---------------------------------------------------------------- Q1 basis
// Reference element [-1,1]^d, corner c has sign s_a = +1 if bit a of c is set.
// Physical element: box of edge h_a, x_a = x0_a + (1 + xi_a) h_a / 2.
struct Basis {
  double N[8];
  double dN[8][3];      // physical first derivatives
  double ddN[8][3][3];  // physical second derivatives
};

void eval_basis(int dim, const double* xi, const double* h, Basis& B) {
  int nc = 1 << dim;
  for (int c = 0; c < nc; ++c) {
    double f[3], df[3];
    for (int a = 0; a < dim; ++a) {
      double s = ((c >> a) & 1) ? 1.0 : -1.0;
      f[a] = 0.5 * (1.0 + s * xi[a]);
      df[a] = 0.5 * s * 2.0 / h[a];  // d f_a / d x_a
    }
    double N = 1.0;
    for (int a = 0; a < dim; ++a) N *= f[a];
    B.N[c] = N;
    for (int i = 0; i < 3; ++i) {
      B.dN[c][i] = 0.0;
      for (int j = 0; j < 3; ++j) B.ddN[c][i][j] = 0.0;
    }
    for (int i = 0; i < dim; ++i) {
      double g = df[i];
      for (int a = 0; a < dim; ++a) if (a != i) g *= f[a];
      B.dN[c][i] = g;
      for (int j = 0; j < dim; ++j) {
        if (j == i) { B.ddN[c][i][j] = 0.0; continue; }  // f_a is linear in x_a
        double q = df[i] * df[j];
        for (int a = 0; a < dim; ++a) if (a != i && a != j) q *= f[a];
        B.ddN[c][i][j] = q;
      }
    }
  }
}

// interpolated field at a Gauss point
template <class T>
struct Field {
  T u;
  T du[3];
  T ddu[3][3];
};

template <class T>
Field<T> interp(int dim, const Basis& B, const T* nodal, int stride, int comp) {
  Field<T> F;
  F.u = T(0.0);
  for (int i = 0; i < 3; ++i) { F.du[i] = T(0.0); for (int j = 0; j < 3; ++j) F.ddu[i][j] = T(0.0); }
  int nc = 1 << dim;
  for (int c = 0; c < nc; ++c) {
    T v = nodal[c * stride + comp];
    F.u += v * T(B.N[c]);
    for (int i = 0; i < dim; ++i) {
      F.du[i] += v * T(B.dN[c][i]);
      for (int j = 0; j < dim; ++j) F.ddu[i][j] += v * T(B.ddN[c][i][j]);
    }
  }
  return F;
}

// ---------------------------------------------------------------- element residual
// un, uo: local nodal values (nc x nf) of U^{k+1}, U^k; f: local nodal forcing
// at t_{k+1/2} or null.  r: local residual (nc x nf), overwritten.
// floors (nullable): incremented once per Gauss point whose tau_m radicand is
// raised to 4/dt^2 (the reading of an unbounded radicand, see the header);
// margin (nullable): lowered to |radicand dt^2 / 4 - 1| where smaller.
template <class T>
void element_residual(const Mesh& m, const Params& P, int64_t e, const T* un, const T* uo,
                      const double* f, T* r, int64_t* floors = nullptr, double* margin = nullptr) {
  const int dim = m.dim, nc = m.nc, nf = m.nf;
  const int IP = dim, IPHI = dim + 1, IMU = dim + 2;
  double h[3];
  for (int a = 0; a < dim; ++a) h[a] = (m.hi[a] - m.lo[a]) / double(int64_t(1) << m.level[e]);
  double detJ = 1.0;
  for (int a = 0; a < dim; ++a) detJ *= 0.5 * h[a];
  // density / viscosity maps rho = alpha phi + beta, eta = gamma phi + xi (Sec. 2)
  const double alpha = 0.5 * (1.0 - P.rho_r), beta = 0.5 * (1.0 + P.rho_r);
  const double gamma = 0.5 * (1.0 - P.eta_r), xi_ = 0.5 * (1.0 + P.eta_r);
  // G_ij = d xi_k/d x_i d xi_k/d x_j = diag(4/h^2)
  double G[3] = {0, 0, 0}, trG = 0.0, GG = 0.0;
  for (int a = 0; a < dim; ++a) { G[a] = 4.0 / (h[a] * h[a]); trG += G[a]; GG += G[a] * G[a]; }
  const double dt = P.dt;
  for (int i = 0; i < nc * nf; ++i) r[i] = T(0.0);

  const double gp = 1.0 / std::sqrt(3.0);
  for (int q = 0; q < nc; ++q) {
    double xi[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) xi[a] = ((q >> a) & 1) ? gp : -gp;
    Basis B;
    eval_basis(dim, xi, h, B);
    const double W = detJ;  // Gauss weights are 1

    // fields at both time levels
    Field<T> vn[3], vo[3];
    for (int i = 0; i < dim; ++i) { vn[i] = interp(dim, B, un, nf, i); vo[i] = interp(dim, B, uo, nf, i); }
    Field<T> pn = interp(dim, B, un, nf, IP), po = interp(dim, B, uo, nf, IP);
    Field<T> phin = interp(dim, B, un, nf, IPHI), phio = interp(dim, B, uo, nf, IPHI);
    Field<T> mun = interp(dim, B, un, nf, IMU), muo = interp(dim, B, uo, nf, IMU);
    double fq[6] = {0, 0, 0, 0, 0, 0};
    if (f) {
      for (int k = 0; k < nf; ++k) {
        double s = 0.0;
        for (int c = 0; c < nc; ++c) s += f[c * nf + k] * B.N[c];
        fq[k] = s;
      }
    }

    // Crank-Nicolson time averages (Sec. 3.1)
    T vt[3], dvt[3][3], dv[3];
    for (int i = 0; i < dim; ++i) {
      vt[i] = T(0.5) * (vn[i].u + vo[i].u);
      dv[i] = vn[i].u - vo[i].u;
      for (int j = 0; j < dim; ++j) dvt[i][j] = T(0.5) * (vn[i].du[j] + vo[i].du[j]);
    }
    T lap_vt[3];
    for (int i = 0; i < dim; ++i) {
      lap_vt[i] = T(0.0);
      for (int k = 0; k < dim; ++k) lap_vt[i] += T(0.5) * (vn[i].ddu[k][k] + vo[i].ddu[k][k]);
    }
    T pt = T(0.5) * (pn.u + po.u), dpt[3];
    T phit = T(0.5) * (phin.u + phio.u), dphit[3], ddphit[3][3];
    T dmut[3], mut = T(0.5) * (mun.u + muo.u);
    for (int i = 0; i < dim; ++i) {
      dpt[i] = T(0.5) * (pn.du[i] + po.du[i]);
      dphit[i] = T(0.5) * (phin.du[i] + phio.du[i]);
      dmut[i] = T(0.5) * (mun.du[i] + muo.du[i]);
      for (int j = 0; j < dim; ++j) ddphit[i][j] = T(0.5) * (phin.ddu[i][j] + phio.ddu[i][j]);
    }
    T dphi = phin.u - phio.u;
    T lap_phit = T(0.0);
    for (int k = 0; k < dim; ++k) lap_phit += ddphit[k][k];

    // phi* (Eq. phi_for_density) and the mixture properties at t_{k+1}
    bool inside = std::fabs(val(phin.u)) <= 1.0;
    T phis = inside ? phin.u : T(val(phin.u) > 0 ? 1.0 : -1.0);
    T rho = T(alpha) * phis + T(beta);
    T eta = T(gamma) * phis + T(xi_);
    T deta[3];
    for (int k = 0; k < dim; ++k) deta[k] = inside ? T(gamma) * phin.du[k] : T(0.0);

    // thermodynamic-consistency flux J = (rho_- - rho_+)/2 grad mu, nondimensional
    T J[3];
    for (int i = 0; i < dim; ++i) J[i] = T(0.5 * (P.rho_r - 1.0)) * dmut[i];

    // stabilisation parameters (Sec. 3.4)
    T vGv = T(0.0), vGJ = T(0.0);
    for (int i = 0; i < dim; ++i) { vGv += vt[i] * T(G[i]) * vt[i]; vGJ += vt[i] * T(G[i]) * J[i]; }
    T visc = eta / (rho * T(P.Re));
    T rad = T(4.0 / (dt * dt)) + vGv + vGJ / (rho * T(P.Pe)) + T(P.C_I) * visc * visc * T(GG);
    if (margin) *margin = std::min(*margin, std::fabs(val(rad) * dt * dt / 4.0 - 1.0));
    if (val(rad) < 4.0 / (dt * dt)) {
      rad = T(4.0 / (dt * dt));
      if (floors) ++*floors;
    }
    T tau_m = T(1.0) / sqrt(rad);
    T tau_c = T(1.0) / (T(trG) * tau_m);

    // strong residuals R_m, R_c (Sec. 3.4) with CN time derivative
    T Rm[3];
    for (int i = 0; i < dim; ++i) {
      T conv = T(0.0), flux = T(0.0), capil = T(0.0), visc_t = T(0.0);
      for (int j = 0; j < dim; ++j) {
        conv += vt[j] * dvt[i][j];
        flux += J[j] * dvt[i][j];
        capil += ddphit[i][j] * dphit[j];
      }
      capil += dphit[i] * lap_phit;
      for (int k = 0; k < dim; ++k) visc_t += deta[k] * dvt[i][k];
      visc_t += eta * lap_vt[i];
      Rm[i] = rho * dv[i] / T(dt) + rho * conv + flux / T(P.Pe) + T(P.Cn / P.We) * capil +
              dpt[i] / T(P.We) - visc_t / T(P.Re) - rho * T(P.g[i] / P.Fr) - T(fq[i]);
    }
    T divv = T(0.0);
    for (int i = 0; i < dim; ++i) divv += dvt[i][i];
    T Rc = divv - T(fq[IP]);

    T dpsi = phit * phit * phit - phit;  // psi'(phi~) with psi = (phi^2 - 1)^2 / 4

    for (int a = 0; a < nc; ++a) {
      const double Na = B.N[a];
      const double* dNa = B.dN[a];
      // momentum rows
      for (int i = 0; i < dim; ++i) {
        T s = T(0.0);
        s += T(Na) * rho * dv[i] / T(dt);                                   // (w, rho dv/dt)
        T conv = T(0.0), flux = T(0.0), cross = T(0.0);
        for (int j = 0; j < dim; ++j) {
          conv += vt[j] * dvt[i][j];
          flux += J[j] * dvt[i][j];
          cross += tau_m * Rm[j] * dvt[i][j];
        }
        s += T(Na) * rho * conv;                                            // (w, rho v.grad v)
        s = s - T(Na) * cross;                                              // -(w, tau R_m,j d_j v_i)
        for (int j = 0; j < dim; ++j) {
          s += T(dNa[j]) * vt[j] * tau_m * Rm[i];                           // (d_j w, v_j tau R_m,i)
          s = s - T(dNa[j]) * tau_m * tau_m / rho * Rm[j] * Rm[i];          // -(d_j w, tau^2/rho R_j R_i)
        }
        s += T(Na) * flux / T(P.Pe);                                        // (1/Pe)(w, J.grad v)
        for (int j = 0; j < dim; ++j)
          s += T(dNa[j]) * J[j] * tau_m / rho * Rm[i] / T(P.Pe);            // (1/Pe)(d_j w, J_j tau/rho R_i)
        for (int j = 0; j < dim; ++j)
          s = s - T(P.Cn / P.We) * T(dNa[j]) * dphit[i] * dphit[j];         // -(Cn/We)(d_j w, d_i phi d_j phi)
        s = s - T(dNa[i]) * pt / T(P.We);                                   // -(1/We)(d_i w, p)
        s += T(dNa[i]) * rho * tau_c * Rc / T(P.We);                        // (1/We)(d_i w, rho tau_c R_c)
        for (int k = 0; k < dim; ++k) s += T(dNa[k]) * eta * dvt[i][k] / T(P.Re);  // (1/Re)(d_k w, eta d_k v_i)
        s = s - T(Na) * rho * T(P.g[i] / P.Fr);                             // -(w, rho g_i / Fr)
        s = s - T(Na) * T(fq[i]);                                           // forcing
        r[a * nf + i] += T(W) * s;
      }
      // continuity row (solenoidality with PSPG)
      {
        T s = T(Na) * divv;                                                 // (q, div v)
        for (int i = 0; i < dim; ++i) s += T(dNa[i]) * tau_m / rho * Rm[i]; // +(d_i q, tau/rho R_m,i)
        s = s - T(Na) * T(fq[IP]);
        r[a * nf + IP] += T(W) * s;
      }
      // Cahn-Hilliard row
      {
        T s = T(Na) * dphi / T(dt);                                         // (q, dphi/dt)
        for (int i = 0; i < dim; ++i) {
          s = s - T(dNa[i]) * vt[i] * phit;                                 // -(d_i q, v_i phi)
          s += T(dNa[i]) * dmut[i] / T(P.Pe * P.Cn);                        // (1/(Pe Cn))(d_i q, d_i mu)
        }
        s = s - T(Na) * T(fq[IPHI]);
        r[a * nf + IPHI] += T(W) * s;
      }
      // chemical potential row
      {
        T s = T(0.0) - T(Na) * mut + T(Na) * dpsi;                          // -(q, mu) + (q, psi')
        for (int i = 0; i < dim; ++i) s += T(P.Cn * P.Cn) * T(dNa[i]) * dphit[i];  // Cn^2 (d_i q, d_i phi)
        s = s - T(Na) * T(fq[IMU]);
        r[a * nf + IMU] += T(W) * s;
      }
    }
  }
}

// local gather through P
template <class T>
void gather(const Mesh& m, int64_t e, const double* U, const double* w, T* loc);

template <>
void gather<double>(const Mesh& m, int64_t e, const double* U, const double*, double* loc) {
  for (int c = 0; c < m.nc; ++c)
    for (int k = 0; k < m.nf; ++k) {
      double s = 0.0;
      for (int64_t t = m.P_start[e * m.nc + c]; t < m.P_start[e * m.nc + c + 1]; ++t)
        s += m.P_w[t] * U[m.P_node[t] * m.nf + k];
      loc[c * m.nf + k] = s;
    }
}

template <>
void gather<Dual>(const Mesh& m, int64_t e, const double* U, const double* w, Dual* loc) {
  for (int c = 0; c < m.nc; ++c)
    for (int k = 0; k < m.nf; ++k) {
      double s = 0.0, sd = 0.0;
      for (int64_t t = m.P_start[e * m.nc + c]; t < m.P_start[e * m.nc + c + 1]; ++t) {
        s += m.P_w[t] * U[m.P_node[t] * m.nf + k];
        if (w) sd += m.P_w[t] * w[m.P_node[t] * m.nf + k];
      }
      loc[c * m.nf + k] = Dual(s, sd);
    }
}

void scatter(const Mesh& m, int64_t e, const double* loc, double* F) {
  for (int c = 0; c < m.nc; ++c)
    for (int64_t t = m.P_start[e * m.nc + c]; t < m.P_start[e * m.nc + c + 1]; ++t)
      for (int k = 0; k < m.nf; ++k) F[m.P_node[t] * m.nf + k] += m.P_w[t] * loc[c * m.nf + k];
}

// constrained rows: velocity on walls (Dirichlet), pressure at the origin node
template <class F>
void for_constrained_rows(const Mesh& m, F fn) {
  for (int64_t i = 0; i < m.n_nodes; ++i)
    if (m.on_wall[i])
      for (int k = 0; k < m.dim; ++k) fn(i * m.nf + k);
  fn(m.origin * m.nf + m.dim);
}

}  // namespace

// ============================================================== C interface
extern "C" {

void* oracle_mesh_create(int dim, int64_t n_leaves, const uint8_t* level, const uint32_t* anchor,
                         int max_level, const double* lo, const double* hi, char* err, int errlen) {
  Mesh* m = new Mesh;
  m->dim = dim;
  m->max_level = max_level;
  m->n_elem = n_leaves;
  for (int a = 0; a < 3; ++a) { m->lo[a] = lo ? lo[a] : 0.0; m->hi[a] = hi ? hi[a] : 1.0; }
  m->level.resize(n_leaves);
  m->anchor.resize(n_leaves * dim);
  for (int64_t e = 0; e < n_leaves; ++e) {
    m->level[e] = level[e];
    for (int a = 0; a < dim; ++a) m->anchor[e * dim + a] = anchor[e * dim + a];
  }
  if (!build_mesh(*m)) {
    if (err && errlen > 0) { std::strncpy(err, m->err.c_str(), errlen - 1); err[errlen - 1] = 0; }
    delete m;
    return nullptr;
  }
  return m;
}

void oracle_mesh_destroy(void* h) { delete (Mesh*)h; }

void oracle_mesh_info(void* h, int64_t* out) {
  Mesh* m = (Mesh*)h;
  out[0] = m->n_nodes;
  out[1] = m->n_nodes * m->nf;
  out[2] = m->n_hanging;
  out[3] = m->origin;
  out[4] = m->n_elem;
}

void oracle_mesh_nodes(void* h, int64_t* xyz, uint8_t* wall) {
  Mesh* m = (Mesh*)h;
  std::memcpy(xyz, m->node_xyz.data(), sizeof(int64_t) * m->node_xyz.size());
  if (wall) std::memcpy(wall, m->on_wall.data(), m->n_nodes);
}

// element corner -> (node, weight) lists (the constraint matrix P)
int64_t oracle_mesh_P(void* h, int64_t* start, int64_t* node, double* w) {
  Mesh* m = (Mesh*)h;
  if (start) {
    std::memcpy(start, m->P_start.data(), sizeof(int64_t) * m->P_start.size());
    std::memcpy(node, m->P_node.data(), sizeof(int64_t) * m->P_node.size());
    std::memcpy(w, m->P_w.data(), sizeof(double) * m->P_w.size());
  }
  return (int64_t)m->P_node.size();
}

// F(U_new; U_old).  f (forcing, nodal at t_{k+1/2}) and g (prescribed values of
// the constrained rows) may be null.
void oracle_residual(void* h, const double* prm, const double* Un, const double* Uo, const double* f,
                     const double* g, double* F) {
  Mesh& m = *(Mesh*)h;
  Params P = unpack(prm);
  const int L = m.nc * m.nf;
  std::fill(F, F + m.n_nodes * m.nf, 0.0);
  std::vector<double> un(L), uo(L), fl(L), r(L);
  for (int64_t e = 0; e < m.n_elem; ++e) {
    gather<double>(m, e, Un, nullptr, un.data());
    gather<double>(m, e, Uo, nullptr, uo.data());
    if (f) gather<double>(m, e, f, nullptr, fl.data());
    element_residual<double>(m, P, e, un.data(), uo.data(), f ? fl.data() : nullptr, r.data());
    scatter(m, e, r.data(), F);
  }
  for_constrained_rows(m, [&](int64_t row) { F[row] = Un[row] - (g ? g[row] : 0.0); });
}

// y = J(U_new; U_old) w, J = dF/dU_new
void oracle_jacvec(void* h, const double* prm, const double* Un, const double* Uo, const double* w,
                   double* y) {
  Mesh& m = *(Mesh*)h;
  Params P = unpack(prm);
  const int L = m.nc * m.nf;
  std::fill(y, y + m.n_nodes * m.nf, 0.0);
  std::vector<Dual> un(L), uo(L), r(L);
  std::vector<double> rd(L);
  for (int64_t e = 0; e < m.n_elem; ++e) {
    gather<Dual>(m, e, Un, w, un.data());
    gather<Dual>(m, e, Uo, nullptr, uo.data());
    element_residual<Dual>(m, P, e, un.data(), uo.data(), nullptr, r.data());
    for (int i = 0; i < L; ++i) rd[i] = r[i].d;
    scatter(m, e, rd.data(), y);
  }
  for_constrained_rows(m, [&](int64_t row) { y[row] = w[row]; });
}

// Sparse Jacobian as COO triplets (duplicates summed by the caller).  Returns
// the triplet count; call with null outputs to size the buffers.
int64_t oracle_jacobian_coo(void* h, const double* prm, const double* Un, const double* Uo,
                            int64_t* I, int64_t* Jc, double* V) {
  Mesh& m = *(Mesh*)h;
  Params P = unpack(prm);
  const int L = m.nc * m.nf;
  std::vector<uint8_t> constrained(m.n_nodes * m.nf, 0);
  for_constrained_rows(m, [&](int64_t row) { constrained[row] = 1; });
  int64_t cnt = 0;
  std::vector<Dual> un(L), uo(L), r(L);
  for (int64_t e = 0; e < m.n_elem; ++e) {
    gather<Dual>(m, e, Un, nullptr, un.data());
    gather<Dual>(m, e, Uo, nullptr, uo.data());
    for (int cs = 0; cs < m.nc; ++cs)
      for (int ks = 0; ks < m.nf; ++ks) {
        for (int i = 0; i < L; ++i) un[i].d = 0.0;
        un[cs * m.nf + ks].d = 1.0;  // seed the local (corner, field) value
        element_residual<Dual>(m, P, e, un.data(), uo.data(), nullptr, r.data());
        for (int64_t ts = m.P_start[e * m.nc + cs]; ts < m.P_start[e * m.nc + cs + 1]; ++ts) {
          int64_t col = m.P_node[ts] * m.nf + ks;
          for (int c = 0; c < m.nc; ++c)
            for (int64_t t = m.P_start[e * m.nc + c]; t < m.P_start[e * m.nc + c + 1]; ++t)
              for (int k = 0; k < m.nf; ++k) {
                int64_t row = m.P_node[t] * m.nf + k;
                if (constrained[row]) continue;
                if (I) { I[cnt] = row; Jc[cnt] = col; V[cnt] = m.P_w[t] * m.P_w[ts] * r[c * m.nf + k].d; }
                ++cnt;
              }
        }
      }
  }
  for (int64_t row = 0; row < m.n_nodes * m.nf; ++row)
    if (constrained[row]) {
      if (I) { I[cnt] = row; Jc[cnt] = row; V[cnt] = 1.0; }
      ++cnt;
    }
  return cnt;
}

// Number of Gauss points (over all leaves) whose tau_m radicand is raised to
// 4/dt^2, evaluated as in oracle_residual (double precision); margin
// (nullable): the smallest |radicand dt^2 / 4 - 1| over all Gauss points, how
// far the closest one is from the floor decision.
int64_t oracle_tau_floor_count(void* h, const double* prm, const double* Un, const double* Uo, double* margin) {
  Mesh& m = *(Mesh*)h;
  Params P = unpack(prm);
  const int L = m.nc * m.nf;
  std::vector<double> un(L), uo(L), r(L);
  int64_t floors = 0;
  double mg = 1e300;
  for (int64_t e = 0; e < m.n_elem; ++e) {
    gather<double>(m, e, Un, nullptr, un.data());
    gather<double>(m, e, Uo, nullptr, uo.data());
    element_residual<double>(m, P, e, un.data(), uo.data(), nullptr, r.data(), &floors, &mg);
  }
  if (margin) *margin = mg;
  return floors;
}

// oracle_jacvec on several host threads (the CPU baseline on all cores): the
// same element routine, elements grouped by a greedy colouring in element
// order so that elements of one colour write disjoint rows; the colours run
// one after another, the elements of a colour are split among the threads.
// Within a row the contributions arrive in colour order instead of element
// order, so results agree with oracle_jacvec to rounding.
void oracle_jacvec_threads(void* h, const double* prm, const double* Un, const double* Uo, const double* w,
                           double* y, int n_threads) {
  Mesh& m = *(Mesh*)h;
  Params P = unpack(prm);
  const int L = m.nc * m.nf;
  if (m.colour_elems.empty()) {
    std::vector<std::vector<int64_t>> node_elems(m.n_nodes);
    for (int64_t e = 0; e < m.n_elem; ++e)
      for (int64_t t = m.P_start[e * m.nc]; t < m.P_start[(e + 1) * m.nc]; ++t) node_elems[m.P_node[t]].push_back(e);
    std::vector<int> col(m.n_elem, -1);
    std::vector<int64_t> seen(1024, -1);
    for (int64_t e = 0; e < m.n_elem; ++e) {
      for (int64_t t = m.P_start[e * m.nc]; t < m.P_start[(e + 1) * m.nc]; ++t)
        for (int64_t o : node_elems[m.P_node[t]])
          if (col[o] >= 0) seen[col[o]] = e;
      int c = 0;
      while (c < (int)seen.size() && seen[c] == e) ++c;
      if (c == (int)seen.size()) seen.push_back(-1);
      col[e] = c;
      if ((int)m.colour_elems.size() <= c) m.colour_elems.resize(c + 1);
      m.colour_elems[c].push_back(e);
    }
  }
  std::fill(y, y + m.n_nodes * m.nf, 0.0);
  if (n_threads < 1) n_threads = 1;
  for (const auto& elems : m.colour_elems) {
    auto work = [&](int tid) {
      std::vector<Dual> un(L), uo(L), r(L);
      std::vector<double> rd(L);
      const int64_t n = (int64_t)elems.size();
      for (int64_t k = n * tid / n_threads; k < n * (tid + 1) / n_threads; ++k) {
        const int64_t e = elems[k];
        gather<Dual>(m, e, Un, w, un.data());
        gather<Dual>(m, e, Uo, nullptr, uo.data());
        element_residual<Dual>(m, P, e, un.data(), uo.data(), nullptr, r.data());
        for (int i = 0; i < L; ++i) rd[i] = r[i].d;
        scatter(m, e, rd.data(), y);
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < n_threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
  }
  for_constrained_rows(m, [&](int64_t row) { y[row] = w[row]; });
}

// Diagnostics with the same 2^d Gauss rule: out[0] energy (Eq. energy_functional,
// gravity potential (1/Fr) rho z with z = -g.x), out[1] integral of phi,
// out[2] volume where phi < 0.
void oracle_energy_mass(void* h, const double* prm, const double* U, double* out) {
  Mesh& m = *(Mesh*)h;
  Params P = unpack(prm);
  const int dim = m.dim, nf = m.nf, nc = m.nc;
  const double alpha = 0.5 * (1.0 - P.rho_r), beta = 0.5 * (1.0 + P.rho_r);
  std::vector<double> u(nc * nf);
  double E = 0.0, mass = 0.0, light = 0.0;
  const double gp = 1.0 / std::sqrt(3.0);
  for (int64_t e = 0; e < m.n_elem; ++e) {
    gather<double>(m, e, U, nullptr, u.data());
    double h[3], x0[3], detJ = 1.0;
    for (int a = 0; a < dim; ++a) {
      h[a] = (m.hi[a] - m.lo[a]) / double(int64_t(1) << m.level[e]);
      x0[a] = m.lo[a] + (m.hi[a] - m.lo[a]) * double(m.anchor[e * dim + a]) / double(int64_t(1) << m.max_level);
      detJ *= 0.5 * h[a];
    }
    for (int q = 0; q < nc; ++q) {
      double xi[3] = {0, 0, 0}, x[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) {
        xi[a] = ((q >> a) & 1) ? gp : -gp;
        x[a] = x0[a] + 0.5 * (1.0 + xi[a]) * h[a];
      }
      Basis B;
      eval_basis(dim, xi, h, B);
      Field<double> phi = interp<double>(dim, B, u.data(), nf, dim + 1);
      double v2 = 0.0;
      for (int i = 0; i < dim; ++i) { double vi = interp<double>(dim, B, u.data(), nf, i).u; v2 += vi * vi; }
      double phis = std::fabs(phi.u) <= 1.0 ? phi.u : (phi.u > 0 ? 1.0 : -1.0);
      double rho = alpha * phis + beta;
      double g2 = 0.0, zg = 0.0;
      for (int i = 0; i < dim; ++i) { g2 += phi.du[i] * phi.du[i]; zg -= P.g[i] * x[i]; }
      double psi = 0.25 * (phi.u * phi.u - 1.0) * (phi.u * phi.u - 1.0);
      E += detJ * (0.5 * rho * v2 + (psi + 0.5 * P.Cn * P.Cn * g2) / (P.Cn * P.We) + rho * zg / P.Fr);
      mass += detJ * phi.u;
      if (phi.u < 0.0) light += detJ;
    }
  }
  out[0] = E;
  out[1] = mass;
  out[2] = light;
}

}  // extern "C"
