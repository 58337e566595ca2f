// Test infrastructure only: a plain, slow FP64 CPU oracle for the discontinuous
// Galerkin residual of the charge-conservation Nernst-Planck (CNP) model.
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it;
// the CUDA library never links, includes or calls anything here.
//
// What it computes (Sec. 3.3 "Scheme", Eq. NPDG and Eq. chargeDG): for every
// element K and every basis function phi_i of K, the residual row
//   R_{f,K,i} = volume integral over K + sum over the faces of K of the face
//   integrals, tested with phi_i restricted to K (so on an interior face
//   v^- = phi_i, v^+ = 0, [[v]] = phi_i n^-, {grad v} = grad phi_i / 2).
// Everything is evaluated by full tensor Gauss-Legendre quadrature (q points
// per direction): every basis function is evaluated at every point as the
// product of its 1D Lagrange factors; there is no sum factorisation.
//
// Fields: f = 0 is the potential Phi (charge-conservation rows, Eq. chargeDG),
// f = k (k = 1..m-1) is the concentration c_k (mass-conservation rows, Eq. NPDG);
// c_m is eliminated by Eq. substitution (Sec. 2.2).
//
// Derivatives: the residual code is templated on its scalar. With a forward
// dual number it gives J(u)v exactly (up to rounding); seeding one local column
// at a time assembles the Jacobian (used for J^T w on small meshes).
//
// Readings of places where the paper is silent or ambiguous (each one is also
// stated where it is used):
//  * kappa = sum_{k<m} z_k (z_k mu_k - z_m mu_m) F^2 c_k (Eq. charge2; the
//    short-hand in Sec. 3.2 drops the c_k factor).
//  * On an interior face q_k is two-valued; the upwind term is read as
//    {c q}.n + |{q}.n|/2 (c^- - c^+), with d|x|/dx = 0 at x = 0.
//  * The outlet term uses (q_k . n) c_k, as in Eq. NPDG.
//  * delta_p = C_IP p^2 / h with h the element diagonal; an interior face uses
//    the mean of the two diagonals.
//  * DIRICHLET faces (used for manufactured solutions) take the Nitsche form of
//    the interior-face terms with the given exterior state g.
//  * Butler-Volmer (Eq. bv): the reductant is the solid electrode metal, so
//    (c_r/c_r^*)^gamma = 1; g_k = J_n/(n F) for the oxidant, g = z_ox J_n / n.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual pow(Dual a, double g) {
  return Dual(std::pow(a.v, g), g * std::pow(a.v, g - 1.0) * a.d);
}
// |x| with derivative sign(x), sign(0) = 0
inline Dual absval(Dual a) {
  double s = (a.v > 0) ? 1.0 : ((a.v < 0) ? -1.0 : 0.0);
  return Dual(std::fabs(a.v), s * a.d);
}
inline double absval(double a) { return std::fabs(a); }
inline double value_of(double a) { return a; }
inline double value_of(Dual a) { return a.v; }
using std::exp;
using std::pow;

// ---------------------------------------------------------------- 1D rules
// Legendre polynomial P_n and its derivative at x by the three-term recurrence.
void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *P = p1;
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

// Gauss-Legendre: the q roots of P_q and weights 2 / ((1 - x^2) P_q'(x)^2).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0); w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP; legendre(q, t, &P, &dP);
      double dt = P / dP; t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, dP; legendre(q, t, &P, &dP);
    x[q - 1 - i] = t;
    w[q - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

// Gauss-Lobatto-Legendre nodes for n = p+1 points: -1, the roots of P_p', +1.
// Interior roots by Newton on P_p'(x), with P_p'' from the Legendre ODE
// (1 - x^2) P'' = 2 x P' - p (p+1) P.
void gauss_lobatto(int n, std::vector<double>& x) {
  x.assign(n, 0.0);
  if (n == 1) { x[0] = 0.0; return; }
  int p = n - 1;
  x[0] = -1.0; x[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP; legendre(p, t, &P, &dP);
      double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P; t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
}

// All n Lagrange basis values L_j(x) and derivatives L_j'(x) on the nodes xn.
void lagrange1d(const std::vector<double>& xn, double x, double* L, double* dL) {
  int n = (int)xn.size();
  for (int j = 0; j < n; ++j) {
    double prod = 1.0, der = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == j) continue;
      prod *= (x - xn[k]) / (xn[j] - xn[k]);
    }
    for (int l = 0; l < n; ++l) {
      if (l == j) continue;
      double t = 1.0 / (xn[j] - xn[l]);
      for (int k = 0; k < n; ++k) {
        if (k == j || k == l) continue;
        t *= (x - xn[k]) / (xn[j] - xn[k]);
      }
      der += t;
    }
    L[j] = prod; dL[j] = der;
  }
}

// ---------------------------------------------------------------- problem
enum { TAG_INTERIOR = 0, TAG_WALL = 1, TAG_INLET = 2, TAG_OUTLET = 3, TAG_DIRICHLET = 4,
       TAG_ELECTRODE0 = 5 };
constexpr int MAXF = 4;

struct Problem {
  int dim = 3, ne[3] = {1, 1, 1}, E = 1;
  std::vector<double> xv[3];
  std::vector<uint8_t> tag[6];
  int side_off[7] = {0};  // first boundary-face index of each side
  int NBF = 0;
  int m = 2, NF = 2;
  double z[MAXF] = {0}, D[MAXF] = {0}, cin[MAXF] = {0}, F = 1, RT = 1;
  int vel_kind = 0; double vp[8] = {0};
  int bv_ox = -1; double J0 = 0, a1 = 0.5, a2 = 0.5, nel = 1, gam = 1, cref = 1, phiapp[4] = {0};
  int J0axis = -1; double J0lo = 0, J0hi = 1;
  int p = 1, n = 2, q = 3, Np = 8, Nq = 27, Nfq = 9; double cip = 10.0;
  std::vector<double> xgl, wgl, xnode;
  // parameter carrying the unit tangent in a dual evaluation, -1 none;
  // theta = (D_1..D_m, c_in_1..c_in_{m-1}, phi_app_0..phi_app_3)
  int theta_seed = -1;
};

inline int side_axis(int s) { return s / 2; }

// The other axes of a face normal to axis a, in increasing order.
void other_axes(int dim, int a, int* b) {
  int k = 0;
  for (int c = 0; c < dim; ++c) if (c != a) b[k++] = c;
}

void velocity(const Problem& P, const double* x, double* uv) {
  uv[0] = uv[1] = uv[2] = 0.0;
  if (P.vel_kind == 0) {
    uv[0] = P.vp[0]; uv[1] = P.vp[1]; uv[2] = P.vp[2];
  } else {
    // plate (Poiseuille) flow: u_A = 6 u_avg s (H - s) / H^2, s = x_N - y0 (Sec. 5.2)
    int A = (int)P.vp[0], N = (int)P.vp[1];
    double s = x[N] - P.vp[2], H = P.vp[3], uavg = P.vp[4];
    uv[A] = 6.0 * uavg * s * (H - s) / (H * H);
  }
}

double exchange_current(const Problem& P, const double* x) {
  if (P.J0axis < 0) return P.J0;
  // J_0 = 3/5 Jbar [2 - ((t - w/2)/(w/2))^2], t measured from J0lo over width w (Sec. 5.2)
  double w = P.J0hi - P.J0lo, t = x[P.J0axis] - P.J0lo;
  double r = (t - 0.5 * w) / (0.5 * w);
  return 0.6 * P.J0 * (2.0 - r * r);
}

struct ElemGeom { double lo[3], h[3], diag; };
ElemGeom elem_geom(const Problem& P, int e, int* idx) {
  ElemGeom g;
  idx[0] = e % P.ne[0];
  idx[1] = (e / P.ne[0]) % P.ne[1];
  idx[2] = e / (P.ne[0] * P.ne[1]);
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (a < P.dim) {
      g.lo[a] = P.xv[a][idx[a]];
      g.h[a] = P.xv[a][idx[a] + 1] - P.xv[a][idx[a]];
      d2 += g.h[a] * g.h[a];
    } else { g.lo[a] = 0.0; g.h[a] = 1.0; }
  }
  g.diag = std::sqrt(d2);
  return g;
}

// Basis values and physical gradients of all Np functions of an element at the
// reference point xi, each as a product of 1D Lagrange factors.
void basis_at(const Problem& P, const ElemGeom& g, const double* xi, double* phi,
              double* gphi) {
  double L[3][16], dL[3][16];
  for (int a = 0; a < 3; ++a) {
    if (a < P.dim) lagrange1d(P.xnode, xi[a], L[a], dL[a]);
    else { L[a][0] = 1.0; dL[a][0] = 0.0; }
  }
  int nz = (P.dim == 3) ? P.n : 1;
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < P.n; ++iy)
      for (int ix = 0; ix < P.n; ++ix) {
        int i = ix + P.n * (iy + P.n * iz);
        phi[i] = L[0][ix] * L[1][iy] * L[2][iz];
        gphi[3 * i + 0] = dL[0][ix] * L[1][iy] * L[2][iz] * (2.0 / g.h[0]);
        gphi[3 * i + 1] = L[0][ix] * dL[1][iy] * L[2][iz] * (2.0 / g.h[1]);
        gphi[3 * i + 2] = (P.dim == 3) ? L[0][ix] * L[1][iy] * dL[2][iz] * (2.0 / g.h[2]) : 0.0;
      }
}

template <class T>
struct PointState { T val[MAXF]; T grad[MAXF][3]; };

template <class T>
void state_at(const Problem& P, int e, const double* phi, const double* gphi,
              const T* u, PointState<T>& s) {
  for (int f = 0; f < P.NF; ++f) {
    const T* uf = u + ((size_t)f * P.E + e) * P.Np;
    T v = T(0.0), g0 = T(0.0), g1 = T(0.0), g2 = T(0.0);
    for (int i = 0; i < P.Np; ++i) {
      v += uf[i] * T(phi[i]);
      g0 += uf[i] * T(gphi[3 * i + 0]);
      g1 += uf[i] * T(gphi[3 * i + 1]);
      g2 += uf[i] * T(gphi[3 * i + 2]);
    }
    s.val[f] = v; s.grad[f][0] = g0; s.grad[f][1] = g1; s.grad[f][2] = g2;
  }
}

// Physical coefficients as scalars of type T (a dual number carries the unit
// tangent of the seeded parameter). mu_k = D_k / RT (Eq. NE);
// a_k = F z_k (D_k - D_m); kappa = sum_{k<m} z_k (z_k mu_k - z_m mu_m) F^2 c_k (Eq. charge2).
template <class T> T seeded(double v, bool on);
template <> double seeded<double>(double v, bool) { return v; }
template <> Dual seeded<Dual>(double v, bool on) { return Dual(v, on ? 1.0 : 0.0); }

template <class T> T D_of(const Problem& P, int k) { return seeded<T>(P.D[k], P.theta_seed == k); }
template <class T> T mig_of(const Problem& P, int k) {  // z_k mu_k F
  return T(P.z[k] * P.F / P.RT) * D_of<T>(P, k);
}
template <class T> T a_of(const Problem& P, int k) {
  return T(P.F * P.z[k]) * (D_of<T>(P, k) - D_of<T>(P, P.m - 1));
}
template <class T> T kc_of(const Problem& P, int k) {  // coefficient of c_k in kappa
  return T(P.z[k] * P.F * P.F / P.RT) * (T(P.z[k]) * D_of<T>(P, k) - T(P.z[P.m - 1]) * D_of<T>(P, P.m - 1));
}
template <class T> T cin_of(const Problem& P, int k) {
  return seeded<T>(P.cin[k], P.theta_seed == P.m + k);
}
template <class T> T phiapp_of(const Problem& P, int j) {
  return seeded<T>(P.phiapp[j], P.theta_seed == 2 * P.m - 1 + j);
}

template <class T>
T kappa_of(const Problem& P, const T* val) {
  T kap = T(0.0);
  for (int k = 0; k < P.m - 1; ++k) kap += kc_of<T>(P, k) * val[k + 1];
  return kap;
}

// Butler-Volmer current J_n (Eq. bv) at a point of electrode j.
template <class T>
T bv_current(const Problem& P, int j, const double* x, const T* val) {
  int ox = P.bv_ox, m = P.m;
  T co;
  if (ox < m - 1) co = val[ox + 1];
  else {  // the oxidant is the eliminated species: Eq. substitution
    T s = T(0.0);
    for (int k = 0; k < m - 1; ++k) s += T(P.z[k]) * val[k + 1];
    co = T(-1.0 / P.z[m - 1]) * s;
  }
  double fac = P.nel * P.F / P.RT;
  T eta = phiapp_of<T>(P, j) - val[0];
  T ratio = co * T(1.0 / P.cref);
  T ratio_g = (P.gam == 1.0) ? ratio : pow(ratio, P.gam);
  return T(exchange_current(P, x)) * (exp(T(P.a1 * fac) * eta) - ratio_g * exp(T(-P.a2 * fac) * eta));
}

// ---------------------------------------------------------------- element rows
// out[f * Np + i] = R_{f,K,i} (all fields, all basis functions of element K).
template <class T>
void element_rows(const Problem& P, int K, const T* u, const double* src, const double* dirv,
                  T* out) {
  const int NF = P.NF, Np = P.Np, q = P.q, dim = P.dim;
  for (int r = 0; r < NF * Np; ++r) out[r] = T(0.0);
  int idx[3];
  ElemGeom g = elem_geom(P, K, idx);
  std::vector<double> phi(Np), phiN(Np), gphi(3 * Np), gphiN(3 * Np);

  // ---- volume terms: Eq. NPDG and Eq. chargeDG volume integrals
  double detJ = 1.0;
  for (int a = 0; a < dim; ++a) detJ *= 0.5 * g.h[a];
  int qz = (dim == 3) ? q : 1;
  for (int kz = 0; kz < qz; ++kz)
    for (int ky = 0; ky < q; ++ky)
      for (int kx = 0; kx < q; ++kx) {
        double xi[3] = {P.xgl[kx], P.xgl[ky], (dim == 3) ? P.xgl[kz] : 0.0};
        double w = P.wgl[kx] * P.wgl[ky] * ((dim == 3) ? P.wgl[kz] : 1.0) * detJ;
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = g.lo[a] + 0.5 * (xi[a] + 1.0) * g.h[a];
        basis_at(P, g, xi, phi.data(), gphi.data());
        PointState<T> s; state_at(P, K, phi.data(), gphi.data(), u, s);
        double uv[3]; velocity(P, x, uv);
        int pt = kx + q * (ky + q * kz);
        // flux vectors G_f multiplying grad phi_i, and scalars S_f multiplying phi_i
        T G[MAXF][3], S[MAXF];
        T kap = kappa_of(P, s.val);
        for (int d = 0; d < 3; ++d) {
          T gch = kap * s.grad[0][d];
          for (int k = 0; k < P.m - 1; ++k) gch += a_of<T>(P, k) * s.grad[k + 1][d];
          G[0][d] = gch;
        }
        for (int k = 0; k < P.m - 1; ++k) {
          for (int d = 0; d < 3; ++d) {
            T qk = T(uv[d]) - mig_of<T>(P, k) * s.grad[0][d];
            G[k + 1][d] = D_of<T>(P, k) * s.grad[k + 1][d] - s.val[k + 1] * qk;
          }
        }
        for (int f = 0; f < NF; ++f)
          S[f] = src ? T(-src[((size_t)f * P.E + K) * P.Nq + pt]) : T(0.0);
        for (int f = 0; f < NF; ++f)
          for (int i = 0; i < Np; ++i)
            out[f * Np + i] += T(w) * (G[f][0] * T(gphi[3 * i]) + G[f][1] * T(gphi[3 * i + 1]) +
                                       G[f][2] * T(gphi[3 * i + 2]) + S[f] * T(phi[i]));
      }

  // ---- face terms
  for (int s = 0; s < 2 * dim; ++s) {
    int a = side_axis(s), hi = s & 1;
    double nrm = hi ? 1.0 : -1.0;  // outward normal n = nrm * e_a
    int b[2] = {0, 0}; other_axes(dim, a, b);
    bool boundary = hi ? (idx[a] == P.ne[a] - 1) : (idx[a] == 0);
    int tag = TAG_INTERIOR, bface = -1, Kn = -1;
    ElemGeom gn{};
    if (boundary) {
      int loc = (dim == 3) ? idx[b[0]] + P.ne[b[0]] * idx[b[1]] : idx[b[0]];
      tag = P.tag[s][loc];
      bface = P.side_off[s] + loc;
    } else {
      int stride = (a == 0) ? 1 : ((a == 1) ? P.ne[0] : P.ne[0] * P.ne[1]);
      Kn = K + (hi ? stride : -stride);
      int idxn[3]; gn = elem_geom(P, Kn, idxn);
    }
    if (tag == TAG_WALL) continue;
    double area = 1.0;
    for (int c = 0; c < dim - 1; ++c) area *= 0.5 * g.h[b[c]];
    double delta = (P.p == 0) ? 0.0
                 : P.cip * P.p * P.p / (boundary ? g.diag : 0.5 * (g.diag + gn.diag));
    int q2 = (dim == 3) ? q : 1;
    for (int k2 = 0; k2 < q2; ++k2)
      for (int k1 = 0; k1 < q; ++k1) {
        double xi[3] = {0, 0, 0}, xin[3] = {0, 0, 0};
        xi[a] = nrm; xin[a] = -nrm;
        xi[b[0]] = xin[b[0]] = P.xgl[k1];
        double w = P.wgl[k1] * area;
        if (dim == 3) { xi[b[1]] = xin[b[1]] = P.xgl[k2]; w *= P.wgl[k2]; }
        int fpt = k1 + q * k2;
        double x[3];
        for (int c = 0; c < 3; ++c) x[c] = g.lo[c] + 0.5 * (xi[c] + 1.0) * g.h[c];
        if (dim == 2) x[2] = 0.0;
        basis_at(P, g, xi, phi.data(), gphi.data());
        PointState<T> sm; state_at(P, K, phi.data(), gphi.data(), u, sm);
        double uv[3]; velocity(P, x, uv);
        double un = uv[a] * nrm;
        T dnm[MAXF];  // normal derivatives on the K side, n = n^-
        for (int f = 0; f < NF; ++f) dnm[f] = sm.grad[f][a] * T(nrm);
        T S[MAXF], Tn[MAXF];  // coefficients of phi_i and of grad phi_i . n
        for (int f = 0; f < NF; ++f) { S[f] = T(0.0); Tn[f] = T(0.0); }
        if (tag == TAG_INTERIOR) {
          basis_at(P, gn, xin, phiN.data(), gphiN.data());
          PointState<T> sp; state_at(P, Kn, phiN.data(), gphiN.data(), u, sp);
          T dnp[MAXF];
          for (int f = 0; f < NF; ++f) dnp[f] = sp.grad[f][a] * T(nrm);
          // mass conservation rows, interior faces of Eq. NPDG
          for (int k = 0; k < P.m - 1; ++k) {
            int f = k + 1;
            T Dk = D_of<T>(P, k), mk = mig_of<T>(P, k);
            T jc = sm.val[f] - sp.val[f];
            T qnm = T(un) - mk * dnm[0];
            T qnp = T(un) - mk * dnp[0];
            T qavg = T(0.5) * (qnm + qnp);
            Tn[f] += T(-0.5) * Dk * jc;
            S[f] += T(-0.5) * Dk * (dnm[f] + dnp[f]) + Dk * T(delta) * jc
                  + T(0.5) * (sm.val[f] * qnm + sp.val[f] * qnp) + T(0.5) * absval(qavg) * jc;
          }
          // charge conservation rows, interior faces of Eq. chargeDG
          T kapm = kappa_of(P, sm.val), kapp = kappa_of(P, sp.val);
          T jphi = sm.val[0] - sp.val[0];
          for (int k = 0; k < P.m - 1; ++k) {
            int f = k + 1; T ak = a_of<T>(P, k);
            Tn[0] += T(-0.5) * ak * (sm.val[f] - sp.val[f]);
            S[0] += T(-0.5) * ak * (dnm[f] + dnp[f]);
          }
          Tn[0] += T(-0.5) * kapm * jphi;
          S[0] += T(-0.5) * (kapm * dnm[0] + kapp * dnp[0])
                + T(0.5 * delta) * (kapm + kapp) * jphi;
        } else if (tag == TAG_INLET) {
          for (int k = 0; k < P.m - 1; ++k) S[k + 1] += T(un) * cin_of<T>(P, k);
        } else if (tag == TAG_OUTLET) {
          for (int k = 0; k < P.m - 1; ++k) {
            T qn = T(un) - mig_of<T>(P, k) * dnm[0];
            S[k + 1] += qn * sm.val[k + 1];
          }
        } else if (tag >= TAG_ELECTRODE0) {
          T Jn = bv_current(P, tag - TAG_ELECTRODE0, x, sm.val);
          if (P.bv_ox < P.m - 1) S[P.bv_ox + 1] += T(-1.0 / (P.nel * P.F)) * Jn;
          S[0] += T(-P.z[P.bv_ox] / P.nel) * Jn;
        } else if (tag == TAG_DIRICHLET) {
          double gv[MAXF];
          for (int f = 0; f < NF; ++f)
            gv[f] = dirv ? dirv[((size_t)f * P.NBF + bface) * P.Nfq + fpt] : 0.0;
          for (int k = 0; k < P.m - 1; ++k) {
            int f = k + 1;
            T Dk = D_of<T>(P, k), mk = mig_of<T>(P, k);
            T jc = sm.val[f] - T(gv[f]);
            T qn = T(un) - mk * dnm[0];
            Tn[f] += -Dk * jc;
            S[f] += -Dk * dnm[f] + Dk * T(delta) * jc
                  + T(0.5) * (sm.val[f] + T(gv[f])) * qn + T(0.5) * absval(qn) * jc;
          }
          T kap = kappa_of(P, sm.val);
          T jphi = sm.val[0] - T(gv[0]);
          for (int k = 0; k < P.m - 1; ++k) {
            int f = k + 1; T ak = a_of<T>(P, k);
            Tn[0] += -ak * (sm.val[f] - T(gv[f]));
            S[0] += -ak * dnm[f];
          }
          Tn[0] += T(-1.0) * kap * jphi;
          S[0] += T(-1.0) * kap * dnm[0] + T(delta) * kap * jphi;
        }
        for (int f = 0; f < NF; ++f)
          for (int i = 0; i < Np; ++i) {
            double dn = gphi[3 * i + a] * nrm;
            out[f * Np + i] += T(w) * (S[f] * T(phi[i]) + Tn[f] * T(dn));
          }
      }
  }
}

Problem* build_problem(int dim, const int* ne, const double* coords, const unsigned char* tags,
                       int m, const double* z, const double* D, const double* cin, double F,
                       double RT, int vel_kind, const double* vp, int bv_ox, const double* bvp,
                       int p, int q, double cip) {
  Problem* P = new Problem();
  P->dim = dim;
  P->E = 1;
  size_t off = 0;
  for (int a = 0; a < 3; ++a) {
    P->ne[a] = (a < dim) ? ne[a] : 1;
    P->E *= P->ne[a];
    if (a < dim) { P->xv[a].assign(coords + off, coords + off + P->ne[a] + 1); off += P->ne[a] + 1; }
  }
  size_t toff = 0;
  P->NBF = 0;
  for (int s = 0; s < 2 * dim; ++s) {
    int a = s / 2, b[2] = {0, 0}; other_axes(dim, a, b);
    int nf = (dim == 3) ? P->ne[b[0]] * P->ne[b[1]] : P->ne[b[0]];
    P->tag[s].assign(tags + toff, tags + toff + nf);
    toff += nf;
    P->side_off[s] = P->NBF;
    P->NBF += nf;
  }
  P->side_off[2 * dim] = P->NBF;
  P->m = m; P->NF = m;
  for (int k = 0; k < m; ++k) { P->z[k] = z[k]; P->D[k] = D[k]; P->cin[k] = cin[k]; }
  P->F = F; P->RT = RT;
  P->vel_kind = vel_kind;
  for (int i = 0; i < 8; ++i) P->vp[i] = vp[i];
  P->bv_ox = bv_ox;
  // bvp: J0, alpha1, alpha2, n, gamma, c_ref, phi_app[4], J0axis, J0lo, J0hi
  P->J0 = bvp[0]; P->a1 = bvp[1]; P->a2 = bvp[2]; P->nel = bvp[3]; P->gam = bvp[4];
  P->cref = bvp[5];
  for (int j = 0; j < 4; ++j) P->phiapp[j] = bvp[6 + j];
  P->J0axis = (int)bvp[10]; P->J0lo = bvp[11]; P->J0hi = bvp[12];
  P->p = p; P->n = p + 1; P->q = q; P->cip = cip;
  P->Np = 1; P->Nq = 1; P->Nfq = 1;
  for (int a = 0; a < dim; ++a) { P->Np *= P->n; P->Nq *= q; }
  for (int a = 0; a < dim - 1; ++a) P->Nfq *= q;
  gauss_legendre(q, P->xgl, P->wgl);
  gauss_lobatto(P->n, P->xnode);
  return P;
}

int neighbours(const Problem& P, int K, int* out) {
  int idx[3]; elem_geom(P, K, idx);
  int cnt = 0;
  int stride[3] = {1, P.ne[0], P.ne[0] * P.ne[1]};
  for (int a = 0; a < P.dim; ++a) {
    if (idx[a] > 0) out[cnt++] = K - stride[a];
    if (idx[a] < P.ne[a] - 1) out[cnt++] = K + stride[a];
  }
  return cnt;
}

}  // namespace

// ---------------------------------------------------------------- C entry points
extern "C" {

void* oracle_create(int dim, const int* ne, const double* coords, const unsigned char* tags, int m,
                    const double* z, const double* D, const double* cin, double F, double RT,
                    int vel_kind, const double* vp, int bv_ox, const double* bvp, int p, int q,
                    double cip) {
  if (dim < 2 || dim > 3 || m < 2 || m > MAXF || p < 0 || p > 8 || q < 1 || q > 15) return nullptr;
  return build_problem(dim, ne, coords, tags, m, z, D, cin, F, RT, vel_kind, vp, bv_ox, bvp, p, q,
                       cip);
}

void oracle_destroy(void* h) { delete static_cast<Problem*>(h); }

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// 1D rules, for the pins on the rules themselves.
void oracle_rules(int p, int q, double* xg, double* wg, double* xn) {
  std::vector<double> a, b, c;
  gauss_legendre(q, a, b);
  gauss_lobatto(p + 1, c);
  for (int i = 0; i < q; ++i) { xg[i] = a[i]; wg[i] = b[i]; }
  for (int i = 0; i <= p; ++i) xn[i] = c[i];
}

// Physical coordinates of the volume quadrature points [E][Nq][3] and of the
// boundary-face quadrature points [NBF][Nfq][3] (either may be NULL).
void oracle_quad_points(void* h, double* xq, double* xbq) {
  const Problem& P = *static_cast<Problem*>(h);
  for (int e = 0; e < P.E; ++e) {
    int idx[3]; ElemGeom g = elem_geom(P, e, idx);
    int qz = (P.dim == 3) ? P.q : 1;
    for (int kz = 0; kz < qz; ++kz)
      for (int ky = 0; ky < P.q; ++ky)
        for (int kx = 0; kx < P.q; ++kx) {
          int pt = kx + P.q * (ky + P.q * kz);
          double xi[3] = {P.xgl[kx], P.xgl[ky], P.dim == 3 ? P.xgl[kz] : -1.0};
          if (!xq) continue;
          for (int a = 0; a < 3; ++a)
            xq[((size_t)e * P.Nq + pt) * 3 + a] =
                (a < P.dim) ? g.lo[a] + 0.5 * (xi[a] + 1.0) * g.h[a] : 0.0;
        }
  }
  if (!xbq) return;
  for (int s = 0; s < 2 * P.dim; ++s) {
    int a = s / 2, hi = s & 1, b[2] = {0, 0}; other_axes(P.dim, a, b);
    int nb0 = P.ne[b[0]], nb1 = (P.dim == 3) ? P.ne[b[1]] : 1;
    for (int j1 = 0; j1 < nb1; ++j1)
      for (int j0 = 0; j0 < nb0; ++j0) {
        int loc = j0 + nb0 * j1, bf = P.side_off[s] + loc;
        int q2 = (P.dim == 3) ? P.q : 1;
        for (int k2 = 0; k2 < q2; ++k2)
          for (int k1 = 0; k1 < P.q; ++k1) {
            int fpt = k1 + P.q * k2;
            double* o = xbq + ((size_t)bf * P.Nfq + fpt) * 3;
            o[0] = o[1] = o[2] = 0.0;
            o[a] = hi ? P.xv[a][P.ne[a]] : P.xv[a][0];
            double l0 = P.xv[b[0]][j0], h0 = P.xv[b[0]][j0 + 1] - l0;
            o[b[0]] = l0 + 0.5 * (P.xgl[k1] + 1.0) * h0;
            if (P.dim == 3) {
              double l1 = P.xv[b[1]][j1], h1 = P.xv[b[1]][j1 + 1] - l1;
              o[b[1]] = l1 + 0.5 * (P.xgl[k2] + 1.0) * h1;
            }
          }
      }
  }
}

// Nodal coordinates of every degree of freedom of one field: [E][Np][3].
void oracle_node_points(void* h, double* xn) {
  const Problem& P = *static_cast<Problem*>(h);
  for (int e = 0; e < P.E; ++e) {
    int idx[3]; ElemGeom g = elem_geom(P, e, idx);
    int nz = (P.dim == 3) ? P.n : 1;
    for (int iz = 0; iz < nz; ++iz)
      for (int iy = 0; iy < P.n; ++iy)
        for (int ix = 0; ix < P.n; ++ix) {
          int i = ix + P.n * (iy + P.n * iz);
          int ii[3] = {ix, iy, iz};
          for (int a = 0; a < 3; ++a)
            xn[((size_t)e * P.Np + i) * 3 + a] =
                (a < P.dim) ? g.lo[a] + 0.5 * (P.xnode[ii[a]] + 1.0) * g.h[a] : 0.0;
        }
  }
}

// Values of every field at the volume quadrature points, vals[NF][E][Nq], and
// the quadrature weights times the Jacobian determinant, jxw[E][Nq] (for L2 norms).
void oracle_eval_quad(void* h, const double* u, double* vals, double* jxw) {
  const Problem& P = *static_cast<Problem*>(h);
  std::vector<double> phi(P.Np), gphi(3 * P.Np);
  for (int e = 0; e < P.E; ++e) {
    int idx[3]; ElemGeom g = elem_geom(P, e, idx);
    double detJ = 1.0;
    for (int a = 0; a < P.dim; ++a) detJ *= 0.5 * g.h[a];
    int qz = (P.dim == 3) ? P.q : 1;
    for (int kz = 0; kz < qz; ++kz)
      for (int ky = 0; ky < P.q; ++ky)
        for (int kx = 0; kx < P.q; ++kx) {
          int pt = kx + P.q * (ky + P.q * kz);
          double xi[3] = {P.xgl[kx], P.xgl[ky], P.dim == 3 ? P.xgl[kz] : 0.0};
          basis_at(P, g, xi, phi.data(), gphi.data());
          PointState<double> s; state_at(P, e, phi.data(), gphi.data(), u, s);
          for (int f = 0; f < P.NF; ++f) vals[((size_t)f * P.E + e) * P.Nq + pt] = s.val[f];
          jxw[(size_t)e * P.Nq + pt] =
              detJ * P.wgl[kx] * P.wgl[ky] * (P.dim == 3 ? P.wgl[kz] : 1.0);
        }
  }
}

// r = R(u) on the rows of the listed elements (all elements if elems == NULL);
// other rows of r are left untouched. Layout of u, r: [NF][E][Np].
int oracle_residual(void* h, const double* u, const double* src, const double* dirv,
                    const int* elems, int n_elems, double* r) {
  const Problem& P = *static_cast<Problem*>(h);
  int n = elems ? n_elems : P.E;
#pragma omp parallel
  {
    std::vector<double> out(P.NF * P.Np);
#pragma omp for schedule(dynamic, 4)
    for (int t = 0; t < n; ++t) {
      int K = elems ? elems[t] : t;
      element_rows<double>(P, K, u, src, dirv, out.data());
      for (int f = 0; f < P.NF; ++f)
        for (int i = 0; i < P.Np; ++i) r[((size_t)f * P.E + K) * P.Np + i] = out[f * P.Np + i];
    }
  }
  return 0;
}

// jv = J(u) v (forward dual numbers) on the rows of the listed elements.
int oracle_jvp(void* h, const double* u, const double* v, const double* src, const double* dirv,
               const int* elems, int n_elems, double* jv) {
  const Problem& P = *static_cast<Problem*>(h);
  size_t N = (size_t)P.NF * P.E * P.Np;
  std::vector<Dual> ud(N);
  for (size_t i = 0; i < N; ++i) ud[i] = Dual(u[i], v[i]);
  int n = elems ? n_elems : P.E;
#pragma omp parallel
  {
    std::vector<Dual> out(P.NF * P.Np);
#pragma omp for schedule(dynamic, 4)
    for (int t = 0; t < n; ++t) {
      int K = elems ? elems[t] : t;
      element_rows<Dual>(P, K, ud.data(), src, dirv, out.data());
      for (int f = 0; f < P.NF; ++f)
        for (int i = 0; i < P.Np; ++i) jv[((size_t)f * P.E + K) * P.Np + i] = out[f * P.Np + i].d;
    }
  }
  return 0;
}

// (J(u)^T w)_c for the listed global columns c: each column J e_c is evaluated
// with one dual sweep over the rows of the column's element and its face
// neighbours (the only rows it touches), then dotted with w.
int oracle_vjp_entries(void* h, const double* u, const double* w, const double* src,
                       const double* dirv, const long long* cols, int n_cols, double* out) {
  const Problem& P = *static_cast<Problem*>(h);
  size_t N = (size_t)P.NF * P.E * P.Np;
#pragma omp parallel
  {
    std::vector<Dual> ud(N);
    for (size_t i = 0; i < N; ++i) ud[i] = Dual(u[i], 0.0);
    std::vector<Dual> rows(P.NF * P.Np);
#pragma omp for schedule(dynamic, 1)
    for (int t = 0; t < n_cols; ++t) {
      long long c = cols[t];
      int Kc = (int)((c / P.Np) % P.E);
      ud[c].d = 1.0;
      int nb[7]; int cnt = neighbours(P, Kc, nb);  // up to 2*dim neighbours + itself
      nb[cnt++] = Kc;
      double acc = 0.0;
      for (int j = 0; j < cnt; ++j) {
        int K = nb[j];
        element_rows<Dual>(P, K, ud.data(), src, dirv, rows.data());
        for (int f = 0; f < P.NF; ++f)
          for (int i = 0; i < P.Np; ++i)
            acc += rows[f * P.Np + i].d * w[((size_t)f * P.E + K) * P.Np + i];
      }
      ud[c].d = 0.0;
      out[t] = acc;
    }
  }
  return 0;
}

// dR/dtheta_j on every row, exactly: one dual sweep with the unit tangent on
// parameter j of theta = (D_1..D_m, c_in_1..c_in_{m-1}, phi_app_0..phi_app_3).
int oracle_param_jacobian(void* h, const double* u, const double* src, const double* dirv,
                          int j, double* out) {
  Problem P = *static_cast<Problem*>(h);
  if (j < 0 || j >= 2 * P.m + 3) return -1;
  P.theta_seed = j;
  size_t N = (size_t)P.NF * P.E * P.Np;
  std::vector<Dual> ud(N);
  for (size_t i = 0; i < N; ++i) ud[i] = Dual(u[i], 0.0);
#pragma omp parallel
  {
    std::vector<Dual> rows(P.NF * P.Np);
#pragma omp for schedule(dynamic, 4)
    for (int K = 0; K < P.E; ++K) {
      element_rows<Dual>(P, K, ud.data(), src, dirv, rows.data());
      for (int f = 0; f < P.NF; ++f)
        for (int i = 0; i < P.Np; ++i) out[((size_t)f * P.E + K) * P.Np + i] = rows[f * P.Np + i].d;
    }
  }
  return 0;
}

// Assembled Jacobian in COO form. For every row element K, every column element
// K' in {K} and its face neighbours, and every local column, one dual sweep of
// the rows of K. Entries that are exactly zero are dropped. Returns the number
// of entries, or -1 if cap is too small.
long long oracle_jacobian_coo(void* h, const double* u, const double* src, const double* dirv,
                              long long* ri, long long* ci, double* vals, long long cap) {
  const Problem& P = *static_cast<Problem*>(h);
  size_t N = (size_t)P.NF * P.E * P.Np;
  int nb_loc = P.NF * P.Np;
  long long total = 0;
  bool overflow = false;
#pragma omp parallel
  {
    std::vector<Dual> ud(N);
    for (size_t i = 0; i < N; ++i) ud[i] = Dual(u[i], 0.0);
    std::vector<Dual> rows(nb_loc);
    std::vector<long long> lr, lc; std::vector<double> lv;
#pragma omp for schedule(dynamic, 1)
    for (int K = 0; K < P.E; ++K) {
      int nb[7]; int cnt = neighbours(P, K, nb);
      nb[cnt++] = K;
      for (int j = 0; j < cnt; ++j) {
        int Kc = nb[j];
        for (int g = 0; g < P.NF; ++g)
          for (int l = 0; l < P.Np; ++l) {
            long long col = ((long long)g * P.E + Kc) * P.Np + l;
            ud[col].d = 1.0;
            element_rows<Dual>(P, K, ud.data(), src, dirv, rows.data());
            ud[col].d = 0.0;
            for (int f = 0; f < P.NF; ++f)
              for (int i = 0; i < P.Np; ++i) {
                double val = rows[f * P.Np + i].d;
                if (val != 0.0) {
                  lr.push_back(((long long)f * P.E + K) * P.Np + i);
                  lc.push_back(col);
                  lv.push_back(val);
                }
              }
          }
      }
    }
#pragma omp critical
    {
      long long base = total;
      total += (long long)lv.size();
      if (total > cap) overflow = true;
      else
        for (size_t t = 0; t < lv.size(); ++t) {
          ri[base + t] = lr[t]; ci[base + t] = lc[t]; vals[base + t] = lv[t];
        }
    }
  }
  return overflow ? -1 : total;
}

}  // extern "C"
