// Shared definitions for the CNP discontinuous Galerkin kernels (sm_103a).
//
// Data layout in device memory (all vectors caller-owned):
//   u[b][f][e][i]  b = operating point (batch), f = field (0 = Phi, k = c_k),
//                  e = element (lexicographic, x fastest), i = tensor
//                  Gauss-Lobatto node (lexicographic, x fastest).
// Element geometry is a structured box mesh with per-axis vertex coordinates.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "enp_df.cuh"

namespace enp {

constexpr int kMaxSpecies = 4;
constexpr int kMaxP = 4;
constexpr int kMaxN = kMaxP + 1;
constexpr int kMaxQ = kMaxP + 2;

// kBlockCol: column blockIdx.y of every element-diagonal block of J(u): the
// J v pass with v = the local unit vector e_col in every element and the
// neighbour's tangent set to zero, written to blk[e][row][col].
// kParam: dR/dtheta_j for every parameter j (grid.y = batch * n_theta), the
// residual evaluated with forward-tangent coefficients seeded on theta_j.
enum OpMode : int { kResidual = 0, kJvp = 1, kVjp = 2, kBlockCol = 3, kParam = 4 };

enum FaceTag : int { kInterior = 0, kWall = 1, kInlet = 2, kOutlet = 3, kDirichlet = 4, kElectrode0 = 5 };

// Arithmetic of the FP64-accurate operator (R, J v, J^T w, block columns,
// dR/dtheta on hexahedra): native FP64, or double-float on the FP32 pipe.
enum Arith : int { kArithF64 = 0, kArithDF = 1 };

// Physical coefficients in the arithmetic type T of a kernel, converted once on
// the host so that the pointwise code does no FP64 conversions in FP32 kernels.
template <class T>
struct PhysT {
  T D[kMaxSpecies], cin[kMaxSpecies], mig[kMaxSpecies], acoef[kMaxSpecies], kcoef[kMaxSpecies],
      z[kMaxSpecies], zratio[kMaxSpecies];   // zratio_k = -z_k / z_m
  T neg_inv_zm;                               // -1 / z_m
  T vp[8], vel_coef;
  T J0, e1, e2, gam, gam1, inv_cref, ox_species_scale, ox_charge_scale, phiapp[4];
  T J0lo, J0half, J0inv_half;                 // profile: r = (x - lo - half) / half
  T cip;
  // derivatives of the coefficients with respect to the diffusivities (dR/dtheta):
  // dmig_k/dD_k = z_k F/RT, da_k/dD_k = F z_k (and -F z_k for D_m),
  // dkappa_k/dD_k = z_k^2 F^2/RT, dkappa_k/dD_m = -z_k z_m F^2/RT
  T dmig[kMaxSpecies], da[kMaxSpecies], dkc_own[kMaxSpecies], dkc_m[kMaxSpecies];
  int vel_kind, velA, velN, bv_ox, J0axis;
};

// Everything the operator kernels read besides the vectors. Passed by value.
struct OpParams {
  int dim, ne[3], E, NF, m, p, n, q, Np, Nq, Nfq, NBF;
  int side_off[7];
  const double* xv[3];        // device: per-axis vertex coordinates
  const float* xvf[3];        // the same in FP32, for FP32 kernels
  const float2* xvdf[3];      // the same as double-float pairs (hi, lo)
  const uint8_t* btag;        // device: boundary tags, side-major
  // physics (Sec. 2): mu_k = D_k / RT; migration coefficient z_k mu_k F;
  // a_k = F z_k (D_k - D_m); kappa_k so that kappa = sum_k kappa_k c_k (Eq. charge2)
  double D[kMaxSpecies], cin[kMaxSpecies], mig[kMaxSpecies], acoef[kMaxSpecies],
      kcoef[kMaxSpecies], z[kMaxSpecies];
  double F;
  int vel_kind;               // 0 constant, 1 plate (Poiseuille)
  double vp[8];
  double vel_coef;            // plate flow: 6 u_avg / H^2
  // Butler-Volmer (Eq. bv), nondimensional exponent factors alpha_i n F / RT
  int bv_ox;                  // species index of the oxidant, -1 none
  double J0, e1, e2, gam, inv_cref, ox_species_scale, ox_charge_scale, phiapp[4];
  int J0axis;
  double J0lo, J0hi;
  double cip;                 // C_IP of delta_p = C_IP p^2 / h
  const double* src;          // device [NF][E][Nq] or null
  const double* dirv;         // device [NF][NBF][Nfq] or null
  const double* phiapp_batch; // device [batch][4] or null (per-operating-point phi_app)
  long long batch_stride;     // entries per operating point (NF * E * Np)
  PhysT<double> pd;           // the coefficients above, in each kernel arithmetic type
  PhysT<float> pf;
  PhysT<df> pdf;
  int arith;                  // Arith of the FP64-accurate operator
  double RT;
  int batch;                  // operating points
  int n_theta;                // parameters of dR/dtheta: D_1..D_m, c_in_1..c_in_{m-1}, phi_app_0..3
  // hexahedra: faces of direction a are planes ia = 0..ne[a] times the cells of
  // the other two axes, numbered from foff[a] (foff[3] = all faces); the face
  // kernel leaves per face and side the lifted face coefficients in fbuf,
  // [batch][face][side][value, normal derivative][NF][n^2], in the kernel's type
  long long foff[4];
  void* fbuf;
  long long fbuf_stride;      // entries per operating point
};

template <class R> __host__ __device__ __forceinline__ const PhysT<R>& phys(const OpParams& p);
// Vertex coordinate i of axis a in the kernel's arithmetic type.
template <class R> __device__ __forceinline__ R vertex(const OpParams& p, int a, int i);
template <> __device__ __forceinline__ double vertex<double>(const OpParams& p, int a, int i) { return p.xv[a][i]; }
template <> __device__ __forceinline__ float vertex<float>(const OpParams& p, int a, int i) { return p.xvf[a][i]; }
template <> __device__ __forceinline__ df vertex<df>(const OpParams& p, int a, int i) {
  const float2 c = p.xvdf[a][i];
  return df(c.x, c.y);
}
template <> __host__ __device__ __forceinline__ const PhysT<df>& phys<df>(const OpParams& p) { return p.pdf; }
template <> __host__ __device__ __forceinline__ const PhysT<double>& phys<double>(const OpParams& p) { return p.pd; }
template <> __host__ __device__ __forceinline__ const PhysT<float>& phys<float>(const OpParams& p) { return p.pf; }

// Basis tables for one polynomial degree, built on the host.
struct Tables {
  double B[kMaxQ * kMaxN];    // B[a][i] = L_i(xg_a): Lagrange-GLL basis at Gauss points
  double Dq[kMaxQ * kMaxQ];   // Dq[a][b] = l_b'(xg_a): collocation derivative on Gauss points
  double wq[kMaxQ];           // Gauss weights
  double xq[kMaxQ];           // Gauss points
  double dL[2 * kMaxN];       // dL[s][i] = L_i'(-1 or +1)
};

// Forward tangent scalar: value and one directional derivative.
template <class R>
struct Tan {
  R v, d;
  __device__ __forceinline__ Tan() {}
  __device__ __forceinline__ Tan(R a) : v(a), d(R(0)) {}
  __device__ __forceinline__ Tan(R a, R b) : v(a), d(b) {}
};
template <class R> __device__ __forceinline__ Tan<R> operator+(Tan<R> a, Tan<R> b) { return Tan<R>(a.v + b.v, a.d + b.d); }
template <class R> __device__ __forceinline__ Tan<R> operator-(Tan<R> a, Tan<R> b) { return Tan<R>(a.v - b.v, a.d - b.d); }
template <class R> __device__ __forceinline__ Tan<R> operator*(Tan<R> a, Tan<R> b) { return Tan<R>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class R> __device__ __forceinline__ Tan<R> operator*(R a, Tan<R> b) { return Tan<R>(a * b.v, a * b.d); }
template <class R> __device__ __forceinline__ Tan<R> operator*(Tan<R> b, R a) { return Tan<R>(a * b.v, a * b.d); }
template <class R> __device__ __forceinline__ Tan<R> operator+(Tan<R> a, R b) { return Tan<R>(a.v + b, a.d); }
template <class R> __device__ __forceinline__ Tan<R> operator-(Tan<R> a, R b) { return Tan<R>(a.v - b, a.d); }
template <class R> __device__ __forceinline__ Tan<R> operator-(R a, Tan<R> b) { return Tan<R>(a - b.v, -b.d); }
template <class R> __device__ __forceinline__ Tan<R> operator-(Tan<R> a) { return Tan<R>(-a.v, -a.d); }
template <class R> __device__ __forceinline__ Tan<R>& operator+=(Tan<R>& a, Tan<R> b) { a.v += b.v; a.d += b.d; return a; }

__device__ __forceinline__ double absv(double x) { return fabs(x); }
__device__ __forceinline__ float absv(float x) { return fabsf(x); }
template <class R> __device__ __forceinline__ Tan<R> absv(Tan<R> x) {
  R s = x.v > R(0) ? R(1) : (x.v < R(0) ? R(-1) : R(0));  // d|x|/dx = 0 at x = 0
  return Tan<R>(absv(x.v), s * x.d);
}
__device__ __forceinline__ double sqrtv(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrtv(float x) { return sqrtf(x); }
__device__ __forceinline__ double expv(double x) { return exp(x); }
__device__ __forceinline__ float expv(float x) { return expf(x); }
template <class R> __device__ __forceinline__ Tan<R> expv(Tan<R> x) { R e = expv(x.v); return Tan<R>(e, e * x.d); }
__device__ __forceinline__ double powv(double x, double g) { return pow(x, g); }
__device__ __forceinline__ float powv(float x, float g) { return powf(x, g); }
template <class R> __device__ __forceinline__ Tan<R> powv(Tan<R> x, R g) {
  R pv = powv(x.v, g);
  return Tan<R>(pv, g * powv(x.v, g - R(1)) * x.d);
}
template <class R> __device__ __forceinline__ R valof(R x) { return x; }
template <class R> __device__ __forceinline__ R valof(Tan<R> x) { return x.v; }

__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }

// Apply a small dense matrix along one direction of a 3D array held in shared
// memory by one warp. Input extents (E0, E1, E2), E0 fastest; the contracted
// direction DIR has extent COLS in the input and ROWS in the output.
//   TRANS = false: out(r) = sum_c M[r * COLS + c] in(c)      (M stored ROWS x COLS)
//   TRANS = true:  out(r) = sum_c M[c * ROWS + r] in(c)      (M stored COLS x ROWS)
//   ACC:           out += instead of out =
template <int E0, int E1, int E2, int DIR, int ROWS, bool TRANS, bool ACC, class R>
__device__ __forceinline__ void apply1d(const R* __restrict__ M, const R* __restrict__ in,
                                        R* __restrict__ out, int lane) {
  constexpr int O0 = DIR == 0 ? ROWS : E0;
  constexpr int O1 = DIR == 1 ? ROWS : E1;
  constexpr int O2 = DIR == 2 ? ROWS : E2;
  constexpr int COLS = DIR == 0 ? E0 : (DIR == 1 ? E1 : E2);
  constexpr int NOUT = O0 * O1 * O2;
  constexpr int IS = DIR == 0 ? 1 : (DIR == 1 ? E0 : E0 * E1);  // input stride along DIR
#pragma unroll 1
  for (int o = lane; o < NOUT; o += 32) {
    const int i0 = o % O0, i1 = (o / O0) % O1, i2 = o / (O0 * O1);
    const int r = DIR == 0 ? i0 : (DIR == 1 ? i1 : i2);
    const int base = (DIR == 0 ? 0 : i0) + E0 * ((DIR == 1 ? 0 : i1) + E1 * (DIR == 2 ? 0 : i2));
    R acc = ACC ? out[o] : R(0);
#pragma unroll
    for (int c = 0; c < COLS; ++c) {
      const R m = TRANS ? M[c * ROWS + r] : M[r * COLS + c];
      acc = mad(m, in[base + c * IS], acc);
    }
    out[o] = acc;
  }
}

}  // namespace enp
