// The CNP discontinuous Galerkin operator on sm_103a: residual R(u), J(u)v and
// J(u)^T w of Eq. NPDG and Eq. chargeDG (Sec. 3.3), for tensor-product quads
// (DIM = 2) and hexahedra (DIM = 3) with a Gauss-Lobatto nodal basis of degree
// P and Q = P + 2 Gauss points per direction.
//
// One warp owns one element. It stages the element's nodal values in shared
// memory, evaluates values and gradients at the Q^DIM Gauss points by sum
// factorisation (B along each axis, then the collocation derivative Dq), forms
// the pointwise fluxes, and applies the transposed contractions to get the
// element's rows. Each face of the element is then evaluated from this
// element's side: both traces (value and normal derivative at the face Gauss
// points) are computed, the numerical fluxes formed, and tested with this
// element's basis only. Every row is written by exactly one warp: no atomics,
// and results do not depend on scheduling.
#pragma once
#include "enp_common.cuh"

namespace enp {


template <int DIM, int P, int NF>
struct Shape {
  static constexpr int N = P + 1, Q = P + 2;
  static constexpr int NN = DIM == 3 ? N * N * N : N * N;  // nodes per field
  static constexpr int NQ = DIM == 3 ? Q * Q * Q : Q * Q;  // volume points
  static constexpr int FN = DIM == 3 ? N * N : N;          // nodes on a face
  static constexpr int FQ = DIM == 3 ? Q * Q : Q;          // points on a face
  static constexpr int N2 = DIM == 3 ? N : 1, Q2 = DIM == 3 ? Q : 1;
  static constexpr int NS = NF - 1;                        // unknown species
  static constexpr int TMP = Q * Q * N;                    // contraction scratch
};

// Shared-memory footprint of one warp (in elements of type R).
template <int DIM, int P, int NF, int MODE>
struct WarpSmem {
  using S = Shape<DIM, P, NF>;
  static constexpr int NV = MODE == kResidual ? 1 : 2;           // vectors carried (block mode: 2)
  static constexpr int kNodes = NV * NF * S::NN;                   // own element data
  static constexpr int kOut = NF * S::NN;                          // element rows
  static constexpr int kTmp = 2 * S::TMP;
  static constexpr int kPoints = NV * NF * (1 + DIM) * S::NQ;      // volume point data
  static constexpr int kFace = NV * NF * S::NN                     // neighbour data
                               + 2 * NV * NF * 2 * S::FQ           // traces, both sides
                               + 2 * NF * S::FQ;                   // face fluxes
  static constexpr int kWork = kPoints > kFace ? kPoints : kFace;
  static constexpr int total = kNodes + kOut + kTmp + kWork;
};

// Table block staged once per thread block.
template <int P>
struct TabSmem {
  static constexpr int N = P + 1, Q = P + 2;
  static constexpr int total = Q * N + Q * Q + Q + Q + 2 * N;
};

// ----------------------------------------------------------------- physics
// Component i (0..2) of a 3-vector held in registers, selected rather than
// indexed, so that a run-time i keeps the vector out of local memory.
template <class R>
__device__ __forceinline__ R pick3(const R* v, int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

template <class R>
__device__ __forceinline__ void velocity(const PhysT<R>& p, const R* x, R* uv) {
  if (p.vel_kind == 0) {
    uv[0] = p.vp[0]; uv[1] = p.vp[1]; uv[2] = p.vp[2];
  } else {  // plate flow u_A = 6 u_avg s (H - s) / H^2 (Sec. 5.2)
    const int A = p.velA;
    const R s = pick3(x, p.velN) - p.vp[2], H = p.vp[3];
    const R ua = p.vel_coef * s * (H - s);
    uv[0] = A == 0 ? ua : R(0);
    uv[1] = A == 1 ? ua : R(0);
    uv[2] = A == 2 ? ua : R(0);
  }
}

// J_0 = 3/5 Jbar [2 - ((t - w/2)/(w/2))^2] (Sec. 5.2), or constant.
template <class C, class R>
__device__ __forceinline__ C exchange_current(const PhysT<C>& p, const R* x) {
  if (p.J0axis < 0) return p.J0;
  const C r = (pick3(x, p.J0axis) - p.J0lo - p.J0half) * p.J0inv_half;
  return R(0.6) * p.J0 * (R(2) - r * r);
}

// Volume flux at one point (Eq. NPDG and Eq. chargeDG volume terms): the
// coefficient Sf of phi_i and the vector Gf multiplying grad phi_i.
template <int NF, int DIM, class S, class R, class C = R>
__device__ __forceinline__ void volume_flux(const PhysT<C>& p, const S* c, const S (*g)[3],
                                            const R* uv, S* Sf, S (*Gf)[3]) {
  S kap = S(R(0));
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) kap += p.kcoef[k] * c[k + 1];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    S acc = kap * g[0][d];
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) acc += p.acoef[k] * g[k + 1][d];
    Gf[0][d] = acc;
  }
#pragma unroll
  for (int k = 0; k < NF - 1; ++k)
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const S qk = uv[d] - p.mig[k] * g[0][d];
      Gf[k + 1][d] = p.D[k] * g[k + 1][d] - c[k + 1] * qk;
    }
#pragma unroll
  for (int f = 0; f < NF; ++f) Sf[f] = S(R(0));
}

// Adjoint of the linearised volume flux: given the test-side values W_f and
// gradients GW_f (the w field at the point), the coefficients of phi_j and
// grad phi_j for the columns (J^T w).
template <int NF, int DIM, class R>
__device__ __forceinline__ void volume_flux_adjoint(const PhysT<R>& p, const R* c, const R (*g)[3],
                                                    const R* uv, const R (*GW)[3], R* chat,
                                                    R (*ghat)[3]) {
  R kap = R(0);
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) kap += p.kcoef[k] * c[k + 1];
  R g0GW0 = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) g0GW0 += g[0][d] * GW[0][d];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R acc = kap * GW[0][d];
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) acc += p.mig[k] * c[k + 1] * GW[k + 1][d];
    ghat[0][d] = acc;
  }
  chat[0] = R(0);
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) {
    R qG = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      qG += (uv[d] - p.mig[k] * g[0][d]) * GW[k + 1][d];
      ghat[k + 1][d] = p.acoef[k] * GW[0][d] + p.D[k] * GW[k + 1][d];
    }
    chat[k + 1] = p.kcoef[k] * g0GW0 - qG;
  }
}

// Own-row flux on an interior face (Eq. NPDG / Eq. chargeDG face integrals over
// Gamma_I, tested with this element's basis: [[v]] = phi_i n, {grad v} = grad phi_i / 2).
// cm, dm: values and normal derivatives (along n = this element's outward
// normal) on this side; cp, dp on the other side. Returns the coefficient Sf
// of phi_i and Tf of grad phi_i . n. Upwind reading: {c q}.n + |{q}.n|/2 [[c]].
template <int NF, class S, class R, class C = R>
__device__ __forceinline__ void face_interior_flux(const PhysT<C>& p, const S* cm, const S* dm,
                                                   const S* cp, const S* dp, R un, R delta,
                                                   S* Sf, S* Tf) {
  S kapm = S(R(0)), kapp = S(R(0));
  S T0 = S(R(0)), S0 = S(R(0));
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) {
    const int f = k + 1;
    const C Dk = p.D[k], mg = p.mig[k], ak = p.acoef[k];
    const S jc = cm[f] - cp[f];
    const S qnm = un - mg * dm[0];
    const S qnp = un - mg * dp[0];
    const S qa = R(0.5) * (qnm + qnp);
    Tf[f] = R(-0.5) * Dk * jc;
    Sf[f] = R(-0.5) * Dk * (dm[f] + dp[f]) + (Dk * delta) * jc +
            R(0.5) * (cm[f] * qnm + cp[f] * qnp) + R(0.5) * absv(qa) * jc;
    kapm += p.kcoef[k] * cm[f];
    kapp += p.kcoef[k] * cp[f];
    T0 += R(-0.5) * ak * jc;
    S0 += R(-0.5) * ak * (dm[f] + dp[f]);
  }
  const S jphi = cm[0] - cp[0];
  Tf[0] = T0 + R(-0.5) * kapm * jphi;
  Sf[0] = S0 + R(-0.5) * (kapm * dm[0] + kapp * dp[0]) + (R(0.5) * delta) * (kapm + kapp) * jphi;
}

// The same interior flux for both sides of the face at once: (Sf, Tf) for the
// minus side as above, and for the plus side (its own outward normal -n) the
// value coefficient -Sf and the normal-derivative coefficient TfP. Only the
// potential's T term differs from -Tf: it carries the plus side's kappa.
template <int NF, class S, class R, class C = R>
__device__ __forceinline__ void face_interior_flux2(const PhysT<C>& p, const S* cm, const S* dm,
                                                    const S* cp, const S* dp, R un, R delta,
                                                    S* Sf, S* Tf, S* TfP) {
  S kapm = S(R(0)), kapp = S(R(0));
  S T0 = S(R(0)), S0 = S(R(0));
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) {
    const int f = k + 1;
    const C Dk = p.D[k], mg = p.mig[k], ak = p.acoef[k];
    const S jc = cm[f] - cp[f];
    const S qnm = un - mg * dm[0];
    const S qnp = un - mg * dp[0];
    const S qa = R(0.5) * (qnm + qnp);
    Tf[f] = R(-0.5) * Dk * jc;
    TfP[f] = -Tf[f];
    Sf[f] = R(-0.5) * Dk * (dm[f] + dp[f]) + (Dk * delta) * jc +
            R(0.5) * (cm[f] * qnm + cp[f] * qnp) + R(0.5) * absv(qa) * jc;
    kapm += p.kcoef[k] * cm[f];
    kapp += p.kcoef[k] * cp[f];
    T0 += R(-0.5) * ak * jc;
    S0 += R(-0.5) * ak * (dm[f] + dp[f]);
  }
  const S jphi = cm[0] - cp[0];
  Tf[0] = T0 + R(-0.5) * kapm * jphi;
  TfP[0] = -(T0 + R(-0.5) * kapp * jphi);
  Sf[0] = S0 + R(-0.5) * (kapm * dm[0] + kapp * dp[0]) + (R(0.5) * delta) * (kapm + kapp) * jphi;
}

// Adjoint of the linearised interior own-row flux with respect to both sides,
// given the weighted test traces Sh (value) and Th (normal derivative).
// Accumulates into (acm, adm) for this side and (acp, adp) for the other side.
template <int NF, class R>
__device__ __forceinline__ void face_interior_adjoint(const PhysT<R>& p, const R* cm, const R* dm,
                                                      const R* cp, const R* dp, R un, R delta,
                                                      const R* Sh, const R* Th, R* acm, R* adm,
                                                      R* acp, R* adp) {
  R kapm = R(0), kapp = R(0);
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) { kapm += p.kcoef[k] * cm[k + 1]; kapp += p.kcoef[k] * cp[k + 1]; }
  const R jphi = cm[0] - cp[0];
  const R S0 = Sh[0], T0 = Th[0];
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) {
    const int f = k + 1;
    const R Dk = p.D[k], mg = p.mig[k], ak = p.acoef[k], kc = p.kcoef[k];
    const R jc = cm[f] - cp[f];
    const R qnm = un - mg * dm[0], qnp = un - mg * dp[0];
    const R qa = R(0.5) * (qnm + qnp);
    const R sg = qa > R(0) ? R(1) : (qa < R(0) ? R(-1) : R(0));
    const R Sf = Sh[f], Tf = Th[f];
    // species rows
    acm[f] += R(-0.5) * Dk * Tf + (Dk * delta + R(0.5) * qnm + R(0.5) * absv(qa)) * Sf;
    acp[f] += R(0.5) * Dk * Tf + (-Dk * delta + R(0.5) * qnp - R(0.5) * absv(qa)) * Sf;
    adm[f] += R(-0.5) * Dk * Sf;
    adp[f] += R(-0.5) * Dk * Sf;
    const R dq = -mg * sg * jc * R(0.25) * Sf;
    adm[0] += R(-0.5) * mg * cm[f] * Sf + dq;
    adp[0] += R(-0.5) * mg * cp[f] * Sf + dq;
    // charge rows
    acm[f] += R(-0.5) * ak * T0 - R(0.5) * kc * jphi * T0 - R(0.5) * kc * dm[0] * S0 +
              R(0.5) * delta * kc * jphi * S0;
    acp[f] += R(0.5) * ak * T0 - R(0.5) * kc * dp[0] * S0 + R(0.5) * delta * kc * jphi * S0;
    adm[f] += R(-0.5) * ak * S0;
    adp[f] += R(-0.5) * ak * S0;
  }
  acm[0] += R(-0.5) * kapm * T0 + R(0.5) * delta * (kapm + kapp) * S0;
  acp[0] += R(0.5) * kapm * T0 - R(0.5) * delta * (kapm + kapp) * S0;
  adm[0] += R(-0.5) * kapm * S0;
  adp[0] += R(-0.5) * kapp * S0;
}

// Concentration of the Butler-Volmer oxidant (Eq. substitution if it is c_m).
template <int NF, class S, class R, class C = R>
__device__ __forceinline__ S oxidant_conc(const PhysT<C>& p, const S* c) {
  if (p.bv_ox < NF - 1) {  // selected, not indexed: c stays in registers
    S o = c[1];
#pragma unroll
    for (int k = 1; k < NF - 1; ++k)
      if (k == p.bv_ox) o = c[k + 1];
    return o;
  }
  S s = S(R(0));
#pragma unroll
  for (int k = 0; k < NF - 1; ++k) s += p.z[k] * c[k + 1];
  return p.neg_inv_zm * s;
}

// Own-row flux on a boundary face (the boundary integrals of Eq. NPDG and
// Eq. chargeDG; DIRICHLET is the Nitsche form of the interior terms with the
// exterior state g, used for manufactured solutions).
template <int NF, class S, class R, class C = R>
__device__ __forceinline__ void face_boundary_flux(const PhysT<C>& p, int tag, const S* cm,
                                                   const S* dm, const R* g, R un, R delta,
                                                   const R* x, C phiapp, S* Sf, S* Tf) {
#pragma unroll
  for (int f = 0; f < NF; ++f) { Sf[f] = S(R(0)); Tf[f] = S(R(0)); }
  if (tag == kInlet) {
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) Sf[k + 1] = S(un * p.cin[k]);
  } else if (tag == kOutlet) {
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) Sf[k + 1] = (un - p.mig[k] * dm[0]) * cm[k + 1];
  } else if (tag >= kElectrode0) {
    if (p.bv_ox < 0) return;
    const S co = oxidant_conc<NF, S, R, C>(p, cm);
    const S eta = phiapp - cm[0];
    S r = p.inv_cref * co;
    if (valof(p.gam) != R(1)) r = powv(r, valof(p.gam));
    const S Jn = exchange_current(p, x) * (expv(p.e1 * eta) - r * expv((-p.e2) * eta));
#pragma unroll
    for (int k = 0; k < NF - 1; ++k)
      if (k == p.bv_ox) Sf[k + 1] = p.ox_species_scale * Jn;
    Sf[0] = p.ox_charge_scale * Jn;
  } else if (tag == kDirichlet) {
    S kap = S(R(0)), T0 = S(R(0)), S0 = S(R(0));
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
      const int f = k + 1;
      const C Dk = p.D[k], ak = p.acoef[k];
      const S jc = cm[f] - g[f];
      const S qn = un - p.mig[k] * dm[0];
      Tf[f] = (-Dk) * jc;
      Sf[f] = (-Dk) * dm[f] + (Dk * delta) * jc + R(0.5) * (cm[f] + g[f]) * qn +
              R(0.5) * absv(qn) * jc;
      kap += p.kcoef[k] * cm[f];
      T0 += (-ak) * jc;
      S0 += (-ak) * dm[f];
    }
    const S jphi = cm[0] - g[0];
    Tf[0] = T0 - kap * jphi;
    Sf[0] = S0 - kap * dm[0] + delta * (kap * jphi);
  }
}

// Adjoint of the linearised boundary own-row flux (this side only).
template <int NF, class R>
__device__ __forceinline__ void face_boundary_adjoint(const PhysT<R>& p, int tag, const R* cm,
                                                      const R* dm, const R* g, R un, R delta,
                                                      const R* x, R phiapp, const R* Sh,
                                                      const R* Th, R* acm, R* adm) {
  if (tag == kOutlet) {
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
      const R mg = p.mig[k];
      acm[k + 1] += (un - mg * dm[0]) * Sh[k + 1];
      adm[0] += -mg * cm[k + 1] * Sh[k + 1];
    }
  } else if (tag >= kElectrode0) {
    if (p.bv_ox < 0) return;
    const R co = oxidant_conc<NF, R, R>(p, cm);
    const R eta = phiapp - cm[0];
    const R E1 = expv(p.e1 * eta), E2 = expv((-p.e2) * eta);
    R r = p.inv_cref * co, drdc = p.inv_cref;
    if (valof(p.gam) != R(1)) {
      const R rb = r;
      r = powv(rb, p.gam);
      drdc = p.gam * powv(rb, p.gam1) * p.inv_cref;
    }
    const R J0 = exchange_current(p, x);
    const R dJdphi = J0 * (-p.e1 * E1 - r * p.e2 * E2);
    const R dJdco = -J0 * E2 * drdc;
    R Jh = p.ox_charge_scale * Sh[0];
#pragma unroll
    for (int k = 0; k < NF - 1; ++k)
      if (k == p.bv_ox) Jh += p.ox_species_scale * Sh[k + 1];
    acm[0] += Jh * dJdphi;
    if (p.bv_ox < NF - 1) {
#pragma unroll
      for (int k = 0; k < NF - 1; ++k)
        if (k == p.bv_ox) acm[k + 1] += Jh * dJdco;
    } else {
#pragma unroll
      for (int k = 0; k < NF - 1; ++k) acm[k + 1] += Jh * dJdco * p.zratio[k];
    }
  } else if (tag == kDirichlet) {
    R kap = R(0);
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) kap += p.kcoef[k] * cm[k + 1];
    const R jphi = cm[0] - g[0];
    const R S0 = Sh[0], T0 = Th[0];
#pragma unroll
    for (int k = 0; k < NF - 1; ++k) {
      const int f = k + 1;
      const R Dk = p.D[k], mg = p.mig[k], ak = p.acoef[k], kc = p.kcoef[k];
      const R jc = cm[f] - g[f];
      const R qn = un - mg * dm[0];
      const R sg = qn > R(0) ? R(1) : (qn < R(0) ? R(-1) : R(0));
      acm[f] += -Dk * Th[f] + (Dk * delta + R(0.5) * qn + R(0.5) * absv(qn)) * Sh[f];
      adm[f] += -Dk * Sh[f];
      adm[0] += -mg * (R(0.5) * (cm[f] + g[f]) + R(0.5) * sg * jc) * Sh[f];
      acm[f] += -ak * T0 - kc * jphi * T0 - kc * dm[0] * S0 + delta * kc * jphi * S0;
      adm[f] += -ak * S0;
    }
    acm[0] += -kap * T0 + delta * kap * S0;
    adm[0] += -kap * S0;
  }
}

// ----------------------------------------------------------------- helpers
// Index of the element node with layer k along axis a and in-face indices
// (j1, j2) along the other axes (lower axis first).
template <int DIM, int N>
__device__ __forceinline__ int face_node(int a, int k, int j1, int j2) {
  if (DIM == 2) return a == 0 ? k + N * j1 : j1 + N * k;
  if (a == 0) return k + N * (j1 + N * j2);
  if (a == 1) return j1 + N * (k + N * j2);
  return j1 + N * (j2 + N * k);
}

// Value and normal derivative (reference, along +axis a) of one field at the
// face Gauss points: X nodal data of one field; layer = 0 or N-1; dLs = dL row.
template <int DIM, int P, class R>
__device__ __forceinline__ void face_trace(const R* X, int a, int layer, const R* dLs,
                                           const R* Bt, R* ftmp, R* fval, R* fder, R* ftmp2,
                                           int lane) {
  using S = Shape<DIM, P, 2>;
  constexpr int N = S::N, Q = S::Q;
  for (int j = lane; j < S::FN; j += 32) {
    const int j1 = j % N, j2 = j / N;
    ftmp[j] = X[face_node<DIM, N>(a, layer, j1, j2)];
    R d = R(0);
#pragma unroll
    for (int k = 0; k < N; ++k) d = mad(dLs[k], X[face_node<DIM, N>(a, k, j1, j2)], d);
    ftmp[S::FN + j] = d;
  }
  __syncwarp();
  if (DIM == 3) {
    apply1d<N, N, 1, 0, Q, false, false>(Bt, ftmp, ftmp2, lane);
    apply1d<N, N, 1, 0, Q, false, false>(Bt, ftmp + S::FN, ftmp2 + Q * N, lane);
    __syncwarp();
    apply1d<Q, N, 1, 1, Q, false, false>(Bt, ftmp2, fval, lane);
    apply1d<Q, N, 1, 1, Q, false, false>(Bt, ftmp2 + Q * N, fder, lane);
  } else {
    apply1d<N, 1, 1, 0, Q, false, false>(Bt, ftmp, fval, lane);
    apply1d<N, 1, 1, 0, Q, false, false>(Bt, ftmp + S::FN, fder, lane);
  }
  __syncwarp();
}

// Add the face-point coefficients (Sv of phi_i, Tv of the reference derivative
// of phi_i along +axis a, both weighted) into the element rows RO of one field.
template <int DIM, int P, class R>
__device__ __forceinline__ void face_test(R* RO, int a, int layer, const R* dLs, const R* Bt,
                                          const R* Sv, const R* Tv, R* ftmp, R* ftmp2, int lane) {
  using S = Shape<DIM, P, 2>;
  constexpr int N = S::N, Q = S::Q;
  if (DIM == 3) {
    apply1d<Q, Q, 1, 1, N, true, false>(Bt, Sv, ftmp2, lane);
    apply1d<Q, Q, 1, 1, N, true, false>(Bt, Tv, ftmp2 + Q * N, lane);
    __syncwarp();
    apply1d<Q, N, 1, 0, N, true, false>(Bt, ftmp2, ftmp, lane);
    apply1d<Q, N, 1, 0, N, true, false>(Bt, ftmp2 + Q * N, ftmp + S::FN, lane);
  } else {
    apply1d<Q, 1, 1, 0, N, true, false>(Bt, Sv, ftmp, lane);
    apply1d<Q, 1, 1, 0, N, true, false>(Bt, Tv, ftmp + S::FN, lane);
  }
  __syncwarp();
  for (int j = lane; j < S::FN; j += 32)
    RO[face_node<DIM, N>(a, layer, j % N, j / N)] += ftmp[j];
  __syncwarp();
  for (int t = lane; t < S::FN * N; t += 32) {
    const int j = t % S::FN, k = t / S::FN;
    RO[face_node<DIM, N>(a, k, j % N, j / N)] += dLs[k] * ftmp[S::FN + j];
  }
  __syncwarp();
}

// ----------------------------------------------------------------- kernel
// MODE kResidual: out = R(u).  kJvp: out = J(u) v.  kVjp: out = J(u)^T v.
// Vectors are indexed [batch][field][element][node]; blockIdx.y is the batch item.
template <int DIM, int P, int NF, int MODE, int WPB, class R>
__global__ void __launch_bounds__(WPB * 32)
op_kernel(const OpParams prm, const Tables* __restrict__ tabs, const R* __restrict__ u,
          const R* __restrict__ v, R* __restrict__ out) {
  constexpr bool kBlk = MODE == kBlockCol;
  constexpr int MODEc = kBlk ? kJvp : MODE;  // the arithmetic of the column pass is J v
  const PhysT<R>& ph = phys<R>(prm);
  using S = Shape<DIM, P, NF>;
  using M = WarpSmem<DIM, P, NF, MODE>;
  constexpr int N = S::N, Q = S::Q, NN = S::NN, NQ = S::NQ, FQ = S::FQ;
  constexpr int NV = M::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = reinterpret_cast<R*>(smem_raw);
  // tables
  R* tB = sm;
  R* tDq = tB + Q * N;
  R* tW = tDq + Q * Q;
  R* tX = tW + Q;
  R* tdL = tX + Q;
  for (int t = threadIdx.x; t < Q * N; t += blockDim.x) tB[t] = R(tabs->B[t]);
  for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) tDq[t] = R(tabs->Dq[t]);
  for (int t = threadIdx.x; t < Q; t += blockDim.x) { tW[t] = R(tabs->wq[t]); tX[t] = R(tabs->xq[t]); }
  for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) tdL[t] = R(tabs->dL[t]);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * WPB + warp;
  if (e >= prm.E) return;
  const int col = kBlk ? (int)blockIdx.y : -1;
  const long long boff = kBlk ? 0 : (long long)blockIdx.y * prm.batch_stride;
  const int bidx = kBlk ? 0 : (int)blockIdx.y;
  R* base = sm + TabSmem<P>::total + warp * M::total;
  R* XA = base;                       // [NV][NF][NN] own data (u, then v or w)
  R* RO = XA + M::kNodes;             // [NF][NN] rows
  R* T1 = RO + M::kOut;               // scratch
  R* T2 = T1 + S::TMP;
  R* WK = T2 + S::TMP;                // work area (volume points, then faces)

  // ---- element geometry
  int idx[3];
  idx[0] = e % prm.ne[0];
  idx[1] = (e / prm.ne[0]) % prm.ne[1];
  idx[2] = e / (prm.ne[0] * prm.ne[1]);
  R lo[3], h[3];
  R diag2 = R(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < DIM) {
      lo[a] = vertex<R>(prm, a, idx[a]);
      h[a] = vertex<R>(prm, a, idx[a] + 1) - lo[a];
      diag2 += h[a] * h[a];
    } else { lo[a] = R(0); h[a] = R(1); }
  }
  const R diag = sqrt(diag2);
  R detJ = R(1);
#pragma unroll
  for (int a = 0; a < DIM; ++a) detJ *= R(0.5) * h[a];

  // ---- load own element data
  const long long EN = (long long)prm.E * NN;
  for (int t = lane; t < NF * NN; t += 32) {
    const int f = t / NN, i = t % NN;
    const long long gi = boff + f * EN + (long long)e * NN + i;
    XA[t] = u[gi];
    if (NV == 2) XA[NF * NN + t] = kBlk ? R(t == col ? 1 : 0) : v[gi];
  }
  __syncwarp();

  // ---- volume: values and reference gradients at Gauss points
  // WK layout: [NV][NF][1 + DIM][NQ]
  for (int s = 0; s < NV; ++s)
    for (int f = 0; f < NF; ++f) {
      const R* X = XA + (s * NF + f) * NN;
      R* V = WK + ((s * NF + f) * (1 + DIM)) * NQ;
      if (DIM == 3) {
        apply1d<N, N, N, 0, Q, false, false>(tB, X, T1, lane);
        __syncwarp();
        apply1d<Q, N, N, 1, Q, false, false>(tB, T1, T2, lane);
        __syncwarp();
        apply1d<Q, Q, N, 2, Q, false, false>(tB, T2, V, lane);
        __syncwarp();
        apply1d<Q, Q, Q, 0, Q, false, false>(tDq, V, V + NQ, lane);
        apply1d<Q, Q, Q, 1, Q, false, false>(tDq, V, V + 2 * NQ, lane);
        apply1d<Q, Q, Q, 2, Q, false, false>(tDq, V, V + 3 * NQ, lane);
      } else {
        apply1d<N, N, 1, 0, Q, false, false>(tB, X, T1, lane);
        __syncwarp();
        apply1d<Q, N, 1, 1, Q, false, false>(tB, T1, V, lane);
        __syncwarp();
        apply1d<Q, Q, 1, 0, Q, false, false>(tDq, V, V + NQ, lane);
        apply1d<Q, Q, 1, 1, Q, false, false>(tDq, V, V + 2 * NQ, lane);
      }
      __syncwarp();
    }

  // ---- pointwise volume fluxes; results go to vector slot NV-1
  for (int pt = lane; pt < NQ; pt += 32) {
    const int kx = pt % Q, ky = (pt / Q) % Q, kz = pt / (Q * Q);
    R xp[3] = {lo[0] + R(0.5) * (tX[kx] + R(1)) * h[0], lo[1] + R(0.5) * (tX[ky] + R(1)) * h[1],
               DIM == 3 ? lo[2] + R(0.5) * (tX[kz] + R(1)) * h[2] : R(0)};
    R uv[3];
    velocity(ph, xp, uv);
    const R w = tW[kx] * tW[ky] * (DIM == 3 ? tW[kz] : R(1)) * detJ;
    R sc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) sc[a] = R(2) / h[a];
    R c0[NF], g0[NF][3];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const R* V = WK + (f * (1 + DIM)) * NQ;
      c0[f] = V[pt];
#pragma unroll
      for (int a = 0; a < 3; ++a) g0[f][a] = a < DIM ? V[(1 + a) * NQ + pt] * sc[a] : R(0);
    }
    R outS[NF], outG[NF][3];
    if (MODEc == kResidual) {
      R Sf[NF], Gf[NF][3];
      volume_flux<NF, DIM, R, R>(ph, c0, g0, uv, Sf, Gf);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        outS[f] = Sf[f] - (prm.src ? R(prm.src[((long long)f * prm.E + e) * NQ + pt]) : R(0));
#pragma unroll
        for (int a = 0; a < 3; ++a) outG[f][a] = Gf[f][a];
      }
    } else {
      R c1[NF], g1[NF][3];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const R* V = WK + ((NF + f) * (1 + DIM)) * NQ;
        c1[f] = V[pt];
#pragma unroll
        for (int a = 0; a < 3; ++a) g1[f][a] = a < DIM ? V[(1 + a) * NQ + pt] * sc[a] : R(0);
      }
      if (MODEc == kJvp) {
        Tan<R> ct[NF], gt[NF][3], Sf[NF], Gf[NF][3];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          ct[f] = Tan<R>(c0[f], c1[f]);
#pragma unroll
          for (int a = 0; a < 3; ++a) gt[f][a] = Tan<R>(g0[f][a], g1[f][a]);
        }
        volume_flux<NF, DIM, Tan<R>, R>(ph, ct, gt, uv, Sf, Gf);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          outS[f] = Sf[f].d;
#pragma unroll
          for (int a = 0; a < 3; ++a) outG[f][a] = Gf[f][a].d;
        }
      } else {
        volume_flux_adjoint<NF, DIM, R>(ph, c0, g0, uv, g1, outS, outG);
        (void)c1;
      }
    }
    // write weighted coefficients; gradient slots carry the 2/h chain factor
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      R* V = WK + (((NV - 1) * NF + f) * (1 + DIM)) * NQ;
      V[pt] = w * outS[f];
#pragma unroll
      for (int a = 0; a < DIM; ++a) V[(1 + a) * NQ + pt] = w * sc[a] * outG[f][a];
    }
  }
  __syncwarp();

  // ---- transposed test contraction into the rows
  for (int f = 0; f < NF; ++f) {
    R* V = WK + (((NV - 1) * NF + f) * (1 + DIM)) * NQ;
    R* Rf = RO + f * NN;
    if (DIM == 3) {
      apply1d<Q, Q, Q, 0, Q, true, true>(tDq, V + NQ, V, lane);
      __syncwarp();
      apply1d<Q, Q, Q, 1, Q, true, true>(tDq, V + 2 * NQ, V, lane);
      __syncwarp();
      apply1d<Q, Q, Q, 2, Q, true, true>(tDq, V + 3 * NQ, V, lane);
      __syncwarp();
      apply1d<Q, Q, Q, 2, N, true, false>(tB, V, T2, lane);
      __syncwarp();
      apply1d<Q, Q, N, 1, N, true, false>(tB, T2, T1, lane);
      __syncwarp();
      apply1d<Q, N, N, 0, N, true, false>(tB, T1, Rf, lane);
    } else {
      apply1d<Q, Q, 1, 0, Q, true, true>(tDq, V + NQ, V, lane);
      __syncwarp();
      apply1d<Q, Q, 1, 1, Q, true, true>(tDq, V + 2 * NQ, V, lane);
      __syncwarp();
      apply1d<Q, Q, 1, 1, N, true, false>(tB, V, T1, lane);
      __syncwarp();
      apply1d<Q, N, 1, 0, N, true, false>(tB, T1, Rf, lane);
    }
    __syncwarp();
  }

  // ---- faces
  // WK layout now: XN [NV][NF][NN] neighbour data, TR [2 sides][NV][NF][2][FQ]
  // traces (value, normal derivative), FS [2][NF][FQ] face coefficients (S, T).
  R* XN = WK;
  R* TR = XN + NV * NF * NN;
  R* FSv = TR + 2 * NV * NF * 2 * FQ;
  R* FTv = FSv + NF * FQ;
  const int stride[3] = {1, prm.ne[0], prm.ne[0] * prm.ne[1]};
  for (int s = 0; s < 2 * DIM; ++s) {
    const int a = s >> 1, hi = s & 1;
    const R nrm = hi ? R(1) : R(-1);
    const bool boundary = hi ? (idx[a] == prm.ne[a] - 1) : (idx[a] == 0);
    int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    int tag = kInterior, bface = -1, en = -1;
    R hn = R(0), diagn = R(0);
    if (boundary) {
      const int loc = DIM == 3 ? idx[b0] + prm.ne[b0] * idx[b1] : idx[b0];
      tag = prm.btag[prm.side_off[s] + loc];
      bface = prm.side_off[s] + loc;
      if (tag == kWall || (tag == kInlet && MODEc != kResidual)) continue;
    } else {
      en = e + (hi ? stride[a] : -stride[a]);
      int in[3] = {idx[0], idx[1], idx[2]};
      in[a] += hi ? 1 : -1;
      R d2 = R(0);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const R hc = vertex<R>(prm, c, in[c] + 1) - vertex<R>(prm, c, in[c]);
        d2 += hc * hc;
        if (c == a) hn = hc;
      }
      diagn = sqrt(d2);
      for (int t = lane; t < NF * NN; t += 32) {
        const int f = t / NN, i = t % NN;
        const long long gi = boff + f * EN + (long long)en * NN + i;
        XN[t] = u[gi];
        if (NV == 2) XN[NF * NN + t] = kBlk ? R(0) : v[gi];
      }
      __syncwarp();
    }
    const R* dLs = tdL + hi * N;          // this side's end
    const R* dLo = tdL + (1 - hi) * N;    // other side's end
    const int lay = hi ? N - 1 : 0, layo = hi ? 0 : N - 1;
    for (int vv = 0; vv < NV; ++vv)
      for (int f = 0; f < NF; ++f) {
        R* tv = TR + ((0 * NV + vv) * NF + f) * 2 * FQ;
        face_trace<DIM, P>(XA + (vv * NF + f) * NN, a, lay, dLs, tB, T1, tv, tv + FQ, T2, lane);
        if (!boundary) {
          R* tn = TR + ((1 * NV + vv) * NF + f) * 2 * FQ;
          face_trace<DIM, P>(XN + (vv * NF + f) * NN, a, layo, dLo, tB, T1, tn, tn + FQ, T2, lane);
        }
      }
    // pointwise face fluxes
    R area = R(1);
    if (DIM == 3) area = R(0.25) * h[b0] * h[b1]; else area = R(0.5) * h[b0];
    const R delta = ph.cip * R(P * P) / (boundary ? diag : R(0.5) * (diag + diagn));
    const R sca = R(2) / h[a] * nrm;           // reference -> physical normal derivative, this side
    const R scn = boundary ? R(0) : R(2) / hn * nrm;  // other side, along this side's normal
    const R phiapp = (tag >= kElectrode0)
        ? (prm.phiapp_batch ? R(prm.phiapp_batch[bidx * 4 + (tag - kElectrode0)])
                            : ph.phiapp[tag - kElectrode0])
        : R(0);
    for (int pt = lane; pt < FQ; pt += 32) {
      const int k1 = pt % Q, k2 = DIM == 3 ? pt / Q : 0;
      R xp[3];
      xp[a] = hi ? lo[a] + h[a] : lo[a];
      xp[b0] = lo[b0] + R(0.5) * (tX[k1] + R(1)) * h[b0];
      if (DIM == 3) xp[b1] = lo[b1] + R(0.5) * (tX[k2] + R(1)) * h[b1]; else xp[2] = R(0);
      R uv[3];
      velocity(ph, xp, uv);
      const R un = uv[a] * nrm;
      const R w = tW[k1] * (DIM == 3 ? tW[k2] : R(1)) * area;
      R cm[NF], dm[NF], cp[NF], dp[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const R* tv = TR + (f * 2) * FQ;
        cm[f] = tv[pt]; dm[f] = tv[FQ + pt] * sca;
        if (!boundary) {
          const R* tn = TR + ((NV + 0) * NF + f) * 2 * FQ;
          cp[f] = tn[pt]; dp[f] = tn[FQ + pt] * scn;
        } else { cp[f] = R(0); dp[f] = R(0); }
      }
      R g[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f)
        g[f] = (tag == kDirichlet && prm.dirv)
                   ? R(prm.dirv[((long long)f * prm.NBF + bface) * prm.Nfq + pt]) : R(0);
      R oS[NF], oT[NF];
      if (MODEc == kResidual) {
        if (boundary) face_boundary_flux<NF, R, R>(ph, tag, cm, dm, g, un, delta, xp, phiapp, oS, oT);
        else face_interior_flux<NF, R, R>(ph, cm, dm, cp, dp, un, delta, oS, oT);
      } else {
        R cm1[NF], dm1[NF], cp1[NF], dp1[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const R* tv = TR + ((1 * NF) + f) * 2 * FQ;
          cm1[f] = tv[pt]; dm1[f] = tv[FQ + pt] * sca;
          if (!boundary) {
            const R* tn = TR + ((NV + 1) * NF + f) * 2 * FQ;
            cp1[f] = tn[pt]; dp1[f] = tn[FQ + pt] * scn;
          } else { cp1[f] = R(0); dp1[f] = R(0); }
        }
        if (MODEc == kJvp) {
          Tan<R> tm[NF], tdm[NF], tp[NF], tdp[NF], Sf[NF], Tf[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            tm[f] = Tan<R>(cm[f], cm1[f]); tdm[f] = Tan<R>(dm[f], dm1[f]);
            tp[f] = Tan<R>(cp[f], cp1[f]); tdp[f] = Tan<R>(dp[f], dp1[f]);
          }
          if (boundary) face_boundary_flux<NF, Tan<R>, R>(ph, tag, tm, tdm, g, un, delta, xp, phiapp, Sf, Tf);
          else face_interior_flux<NF, Tan<R>, R>(ph, tm, tdm, tp, tdp, un, delta, Sf, Tf);
#pragma unroll
          for (int f = 0; f < NF; ++f) { oS[f] = Sf[f].d; oT[f] = Tf[f].d; }
        } else {
          // J^T w: this side's state adjoint from this element's rows (test
          // traces cm1/dm1) and from the neighbour's rows (test traces cp1/dp1,
          // flux seen from the neighbour: normal and normal derivatives flip).
          R Sh[NF], Th[NF], acm[NF], adm[NF], acp[NF], adp[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) { Sh[f] = cm1[f]; Th[f] = dm1[f]; acm[f] = adm[f] = acp[f] = adp[f] = R(0); }
          if (boundary) {
            face_boundary_adjoint<NF, R>(ph, tag, cm, dm, g, un, delta, xp, phiapp, Sh, Th, acm, adm);
          } else {
            face_interior_adjoint<NF, R>(ph, cm, dm, cp, dp, un, delta, Sh, Th, acm, adm, acp, adp);
            R ncm[NF], ndm[NF], ncp[NF], ndp[NF], bcm[NF], bdm[NF], bcp[NF], bdp[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              ncm[f] = cp[f]; ndm[f] = -dp[f]; ncp[f] = cm[f]; ndp[f] = -dm[f];
              Sh[f] = cp1[f]; Th[f] = -dp1[f];
              bcm[f] = bdm[f] = bcp[f] = bdp[f] = R(0);
            }
            face_interior_adjoint<NF, R>(ph, ncm, ndm, ncp, ndp, -un, delta, Sh, Th, bcm, bdm, bcp, bdp);
#pragma unroll
            for (int f = 0; f < NF; ++f) { acm[f] += bcp[f]; adm[f] -= bdp[f]; }
          }
#pragma unroll
          for (int f = 0; f < NF; ++f) { oS[f] = acm[f]; oT[f] = adm[f]; }
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        FSv[f * FQ + pt] = w * oS[f];
        FTv[f * FQ + pt] = w * sca * oT[f];
      }
    }
    __syncwarp();
    for (int f = 0; f < NF; ++f)
      face_test<DIM, P>(RO + f * NN, a, lay, dLs, tB, FSv + f * FQ, FTv + f * FQ, T1, T2, lane);
  }

  // ---- write rows
  if (kBlk) {
    const long long nb = NF * NN;
    for (int t = lane; t < NF * NN; t += 32) out[((long long)e * nb + t) * nb + col] = RO[t];
  } else {
    for (int t = lane; t < NF * NN; t += 32) {
      const int f = t / NN, i = t % NN;
      out[boff + f * EN + (long long)e * NN + i] = RO[t];
    }
  }
}

}  // namespace enp
