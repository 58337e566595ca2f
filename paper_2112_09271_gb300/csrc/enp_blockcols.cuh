// Element-diagonal blocks of J(u) on hexahedra, a chunk of block columns per
// thread block (the "element-wise Jacobi" blocks of Sec. 4.2: volume terms and
// the element's own side of every face term, all fields coupled; column j is
// J(u) applied to the element's basis function j with every other element's
// direction zero).
//
// The state-dependent work is done once per (element, chunk): the state's
// values and gradients at the volume Gauss points, and the traces (value and
// reference normal derivative at the face Gauss points) of the element and of
// each neighbour on the six faces. A column's direction is one basis function
// phi_j of one field, so its values and gradients at the points are products of
// the 1D tables (B, and BD = Dq B for derivatives) and need no contraction;
// each column then costs the pointwise linearisation, the transposed volume
// contractions and the lifting of the six faces' terms. The arithmetic per
// point and face is the operator's own (volume_flux, face_interior_flux,
// face_boundary_flux with the forward tangent), so the blocks equal those of
// the block-column pass of op3d_kernel up to rounding order.
#pragma once
#include "enp_operator3d.cuh"

namespace enp {

template <int P, int NF, int NT, int CH>
struct SmemB {
  static constexpr int N = P + 1, Q = P + 2;
  static constexpr int NX = Pad<N>::X;
  static constexpr int NN = N * N * N, NQ = Q * Q * Q, FN = N * N, FQ = Q * Q;
  static constexpr int NNP = NX * N * N, FNP = NX * N;
  static constexpr int kX = NF * NNP;                 // the element's state
  static constexpr int kPU = NF * 4 * NQ;             // state values + gradients at the points
  static constexpr int kTRU = 6 * 2 * NF * 2 * FQ;    // state traces [face][side][f][value, deriv]
  static constexpr int kPO = NF * 4 * NQ;             // a column's point coefficients
  static constexpr int kT2 = NF * Q * Q * N;          // contraction scratch
  static constexpr int kT1 = NF * Q * N * N;
  static constexpr int kRO = NF * NNP;                // a column's rows
  static constexpr int kFC = 6 * 2 * NF * FQ;         // face coefficients [face][S, T][f]
  static constexpr int kG1 = 6 * 2 * NF * Q * N;
  static constexpr int kG2 = 6 * 2 * NF * FNP;
  static constexpr int kCOL = NF * NN * (CH + 1);     // the chunk's columns [row][column], rows padded
  // the neighbour and face-trace scratch of the set-up phase reuse PO/T2/T1
  static constexpr int kSetup = NF * NNP + 2 * NF * 2 * FNP + 2 * NF * 2 * Q * N + 2 * NF * 2 * FQ;
  static constexpr int kColWork = kPO + kT2 + (kT1 > kFC + kG1 + kG2 ? kT1 : kFC + kG1 + kG2);
  static constexpr int kWork = kColWork > kSetup ? kColWork : kSetup;
  static constexpr int total = kX + kPU + kTRU + kRO + kCOL + kWork;
};

// Columns [blockIdx.y * chunk, ...) of the diagonal block of element
// blockIdx.x, written to blk[e][row][col] (nb = NF * N^3).
template <int P, int NF, int CH, class R>
__global__ void __launch_bounds__(kMaxThreads3D)
blockcol3d_kernel(const OpParams prm, const io_t<R>* __restrict__ u, io_t<R>* __restrict__ out) {
  constexpr int NT = tpe3d<P, R>();
  using S = SmemB<P, NF, NT, CH>;
  using TO = TabOff<P>;
  constexpr int N = S::N, Q = S::Q, NN = S::NN, NQ = S::NQ, FN = S::FN, FQ = S::FQ;
  constexpr int NX = S::NX, NNP = S::NNP, FNP = S::FNP;
  constexpr int nb = NF * NN;
  const PhysT<R>& ph = phys<R>(prm);
  extern __shared__ __align__(16) unsigned char smemb_raw[];
  R* XA = reinterpret_cast<R*>(smemb_raw);   // [NF][NNP]
  R* PU = XA + S::kX;                        // [NF][4][NQ]
  R* TRU = PU + S::kPU;                      // [6][2][NF][2][FQ]
  R* RO = TRU + S::kTRU;                     // [NF][NNP]
  R* COL = RO + S::kRO;                      // [nb][CH + 1]: consecutive rows in different banks
  R* WK = COL + S::kCOL;
  const int tid = threadIdx.x;
  const int e = blockIdx.x;
  const int c0 = blockIdx.y * CH;
  const long long EN = (long long)prm.E * NN;
  int idx[3];
  idx[0] = e % prm.ne[0];
  idx[1] = (e / prm.ne[0]) % prm.ne[1];
  idx[2] = e / (prm.ne[0] * prm.ne[1]);
  R lo[3], h[3], sc[3];
  R diag2 = R(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = vertex<R>(prm, a, idx[a]);
    h[a] = vertex<R>(prm, a, idx[a] + 1) - lo[a];
    sc[a] = R(2) / h[a];
    diag2 += h[a] * h[a];
  }
  const R diag = sqrtv(diag2);
  const R detJ = R(0.125) * h[0] * h[1] * h[2];
  const int stride[3] = {1, prm.ne[0], prm.ne[0] * prm.ne[1]};

  // ------------------------------------------------------------ the state
  for (int t = tid; t < NF * NN; t += NT) {
    const int f = t / NN, i = t % NN;
    XA[f * NNP + padded_node<N>(i)] = R(u[f * EN + (long long)e * NN + i]);
  }
  __syncthreads();
  {
    R* T2 = WK;
    R* T1 = WK + S::kT2;
    pencil<P, N, N, N, 0, 0, false, false, NF, NNP, Q * N * N, R, NX>(XA, T1, tid, NT);
    __syncthreads();
    pencil<P, Q, N, N, 1, 0, false, false, NF, Q * N * N, Q * Q * N>(T1, T2, tid, NT);
    __syncthreads();
    pencil<P, Q, Q, N, 2, 0, false, false, NF, Q * Q * N, 4 * NQ>(T2, PU, tid, NT);
    __syncthreads();
    pencil_grad3<P, NF, 4 * NQ>(PU, tid, NT);
    __syncthreads();
  }
  // the six faces: this element's and the neighbour's traces of the state
  {
    R* XN = WK;                            // [NF][NNP]
    R* FL = XN + NF * NNP;                 // [2][NF][2][FNP]
    R* F1 = FL + 2 * NF * 2 * FNP;         // [2][NF][2][Q][N]
    R* TR = F1 + 2 * NF * 2 * Q * N;       // [2][NF][2][FQ]
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      const int a = s >> 1, hi = s & 1;
      const bool boundary = hi ? (idx[a] == prm.ne[a] - 1) : (idx[a] == 0);
      if (!boundary) {
        const int en = e + (hi ? stride[a] : -stride[a]);
        for (int t = tid; t < NF * NN; t += NT) {
          const int f = t / NN, i = t % NN;
          XN[f * NNP + padded_node<N>(i)] = R(u[f * EN + (long long)en * NN + i]);
        }
      }
      __syncthreads();
      const int lay = hi ? N - 1 : 0, layo = hi ? 0 : N - 1;
      const int nsides = boundary ? 1 : 2;
      for (int w = tid; w < nsides * NF * FN; w += NT) {
        const int side = w / (NF * FN), r = w % (NF * FN), f = r / FN, j = r % FN;
        const int j1 = j % N, j2 = j / N;
        const R* X = (side == 0 ? XA : XN) + f * NNP;
        const int L = side == 0 ? lay : layo;
        const int dsel = side == 0 ? hi : 1 - hi;
        R d = R(0);
#pragma unroll
        for (int k = 0; k < N; ++k)
          d = mad(ctab<P, R>(TO::dL + dsel * N + k), X[face_node_pad<N>(a, k, j1, j2)], d);
        R* o = FL + ((side * NF + f) * 2) * FNP;
        const int jp = j1 + NX * j2;
        o[jp] = X[face_node_pad<N>(a, L, j1, j2)];
        o[FNP + jp] = d;
      }
      __syncthreads();
      pencil<P, N, N, 1, 0, 0, false, false, 4 * NF, FNP, Q * N, R, NX>(FL, F1, tid, NT);
      __syncthreads();
      pencil<P, Q, N, 1, 1, 0, false, false, 4 * NF, Q * N, FQ>(F1, TR, tid, NT);
      __syncthreads();
      for (int w = tid; w < 2 * NF * 2 * FQ; w += NT) TRU[s * 2 * NF * 2 * FQ + w] = TR[w];
      __syncthreads();
    }
  }

  // ------------------------------------------------------------ the columns
  R* PO = WK;                        // [NF][4][NQ]
  R* T2 = PO + S::kPO;               // [NF][Q][Q][N]
  R* T1 = T2 + S::kT2;               // [NF][Q][N][N] (test stage), over FC/G1 (faces)
  R* FC = T1;                        // [6][2][NF][FQ]
  R* G1 = FC + S::kFC;               // [6][2][NF][Q][N]
  R* G2 = G1 + S::kG1;               // [6][2][NF][FNP]
  const int ncol = min(CH, nb - c0);
#pragma unroll 1
  for (int cc = 0; cc < ncol; ++cc) {
    const int col = c0 + cc;
    const int fc = col / NN, jn = col % NN;
    const int jc[3] = {jn % N, (jn / N) % N, jn / (N * N)};
    // volume: the linearised flux in direction phi_col at every point
    {
#pragma unroll 1
      for (int pt = tid; pt < NQ; pt += NT) {
        const int kq[3] = {pt % Q, (pt / Q) % Q, pt / (Q * Q)};
        R xp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) xp[a] = lo[a] + R(0.5) * (ctab<P, R>(TO::X + kq[a]) + R(1)) * h[a];
        R uv[3];
        velocity(ph, xp, uv);
        const R w = ctab<P, R>(TO::W + kq[0]) * ctab<P, R>(TO::W + kq[1]) *
                    ctab<P, R>(TO::W + kq[2]) * detJ;
        const R bx = ctab<P, R>(TO::B + kq[0] * N + jc[0]);
        const R by = ctab<P, R>(TO::B + kq[1] * N + jc[1]);
        const R bz = ctab<P, R>(TO::B + kq[2] * N + jc[2]);
        const R dv = bx * by * bz;
        const R dg[3] = {ctab<P, R>(TO::BD + kq[0] * N + jc[0]) * by * bz * sc[0],
                         bx * ctab<P, R>(TO::BD + kq[1] * N + jc[1]) * bz * sc[1],
                         bx * by * ctab<P, R>(TO::BD + kq[2] * N + jc[2]) * sc[2]};
        Tan<R> ct[NF], gt[NF][3], Sf[NF], Gf[NF][3];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const R* V = PU + f * 4 * NQ;
          const bool on = f == fc;
          ct[f] = Tan<R>(V[pt], on ? dv : R(0));
#pragma unroll
          for (int a = 0; a < 3; ++a) gt[f][a] = Tan<R>(V[(1 + a) * NQ + pt] * sc[a], on ? dg[a] : R(0));
        }
        volume_flux<NF, 3, Tan<R>, R>(ph, ct, gt, uv, Sf, Gf);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          R* V = PO + f * 4 * NQ;
          V[pt] = w * Sf[f].d;
#pragma unroll
          for (int a = 0; a < 3; ++a) V[(1 + a) * NQ + pt] = w * sc[a] * Gf[f][a].d;
        }
      }
    }
    // faces: this element's side of the linearised face terms in direction phi_col
#pragma unroll 1
    for (int w = tid; w < 6 * FQ; w += NT) {
      const int s = w / FQ, pt = w % FQ;
      const int a = s >> 1, hi = s & 1;
      const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
      const R nrm = hi ? R(1) : R(-1);
      const bool boundary = hi ? (idx[a] == prm.ne[a] - 1) : (idx[a] == 0);
      int tag = kInterior, bface = -1;
      R hn = h[a], diagn = diag;
      if (boundary) {
        bface = prm.side_off[s] + idx[b0] + prm.ne[b0] * idx[b1];
        tag = prm.btag[bface];
      } else {
        int in3[3] = {idx[0], idx[1], idx[2]};
        in3[a] += hi ? 1 : -1;
        R d2 = R(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const R hc = vertex<R>(prm, c, in3[c] + 1) - vertex<R>(prm, c, in3[c]);
          d2 += hc * hc;
          if (c == a) hn = hc;
        }
        diagn = sqrtv(d2);
      }
      const bool active = !(tag == kWall || tag == kInlet);
      R oS[NF], oT[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) { oS[f] = R(0); oT[f] = R(0); }
      const R sca = sc[a] * nrm;
      if (active) {
        const int k1 = pt % Q, k2 = pt / Q;
        const R delta = ph.cip * R(P * P) / (boundary ? diag : R(0.5) * (diag + diagn));
        const R scn = R(2) / hn * nrm;
        R xp[3];
        xp[a] = hi ? lo[a] + h[a] : lo[a];
        xp[b0] = lo[b0] + R(0.5) * (ctab<P, R>(TO::X + k1) + R(1)) * h[b0];
        xp[b1] = lo[b1] + R(0.5) * (ctab<P, R>(TO::X + k2) + R(1)) * h[b1];
        R uv[3];
        velocity(ph, xp, uv);
        const R un = pick3(uv, a) * nrm;
        const R phiapp = (tag >= kElectrode0)
            ? (prm.phiapp_batch ? R(prm.phiapp_batch[tag - kElectrode0]) : ph.phiapp[tag - kElectrode0])
            : R(0);
        // phi_col's trace: nonzero at one face node (its in-face coordinates),
        // interpolated to the points by the 1D tables
        const int ja = pick3(jc, a), jb0 = pick3(jc, b0), jb1 = pick3(jc, b1);
        const R bb = ctab<P, R>(TO::B + k1 * N + jb0) * ctab<P, R>(TO::B + k2 * N + jb1);
        const R tv = ja == (hi ? N - 1 : 0) ? bb : R(0);
        const R td = ctab<P, R>(TO::dL + hi * N + ja) * bb * sca;
        const R* tr = TRU + s * 2 * NF * 2 * FQ + pt;
        auto trv = [&](int side, int f, int comp) -> R { return tr[((side * NF + f) * 2 + comp) * FQ]; };
        Tan<R> tm[NF], tdm[NF], Sf[NF], Tf[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const bool on = f == fc;
          tm[f] = Tan<R>(trv(0, f, 0), on ? tv : R(0));
          tdm[f] = Tan<R>(trv(0, f, 1) * sca, on ? td : R(0));
        }
        if (boundary) {
          R g[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f)
            g[f] = (tag == kDirichlet && prm.dirv)
                       ? R(prm.dirv[((long long)f * prm.NBF + bface) * prm.Nfq + pt]) : R(0);
          face_boundary_flux<NF, Tan<R>, R>(ph, tag, tm, tdm, g, un, delta, xp, phiapp, Sf, Tf);
        } else {
          Tan<R> tp[NF], tdp[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            tp[f] = Tan<R>(trv(1, f, 0));
            tdp[f] = Tan<R>(trv(1, f, 1) * scn);
          }
          face_interior_flux<NF, Tan<R>, R>(ph, tm, tdm, tp, tdp, un, delta, Sf, Tf);
        }
        const R wq = ctab<P, R>(TO::W + k1) * ctab<P, R>(TO::W + k2) * R(0.25) * h[b0] * h[b1];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          oS[f] = wq * Sf[f].d;
          oT[f] = wq * sca * Tf[f].d;
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        FC[((s * 2 + 0) * NF + f) * FQ + pt] = oS[f];
        FC[((s * 2 + 1) * NF + f) * FQ + pt] = oT[f];
      }
    }
    __syncthreads();
    // the transposed volume contractions (as op3d_kernel) into the rows
    R* PO_ = PO;
    pencil<P, Q, Q, Q, 0, 1, true, true, NF, 4 * NQ, 4 * NQ>(PO_ + NQ, PO_, tid, NT);
    // the faces' terms lifted to the face nodes (both stages over all six faces)
    pencil<P, Q, Q, 1, 1, 0, true, false, 12 * NF, FQ, Q * N>(FC, G1, tid, NT);
    __syncthreads();
    pencil<P, Q, Q, Q, 1, 1, true, true, NF, 4 * NQ, 4 * NQ>(PO_ + 2 * NQ, PO_, tid, NT);
    pencil<P, Q, N, 1, 0, 0, true, false, 12 * NF, Q * N, FNP, R, Q, NX>(G1, G2, tid, NT);
    __syncthreads();
    pencil<P, Q, Q, Q, 2, 1, true, true, NF, 4 * NQ, 4 * NQ>(PO_ + 3 * NQ, PO_, tid, NT);
    __syncthreads();
    pencil<P, Q, Q, Q, 2, 0, true, false, NF, 4 * NQ, Q * Q * N>(PO_, T2, tid, NT);
    __syncthreads();
    R* T1v = PO_;  // the point arrays are dead once T2 holds the z-transposed values
    pencil<P, Q, Q, N, 1, 0, true, false, NF, Q * Q * N, Q * N * N>(T2, T1v, tid, NT);
    __syncthreads();
    pencil<P, Q, N, N, 0, 0, true, false, NF, Q * N * N, NNP, R, Q, NX>(T1v, RO, tid, NT);
    __syncthreads();
    // every row: volume plus its six faces' terms, in side order
    for (int t = tid; t < nb; t += NT) {
      const int f = t / NN, i = t % NN;
      const int c3[3] = {i % N, (i / N) % N, i / (N * N)};
      R acc = RO[f * NNP + padded_node<N>(i)];
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const int a = s >> 1, hi = s & 1;
        const int k = c3[a];
        const int j1 = a == 0 ? c3[1] : c3[0], j2 = a == 2 ? c3[1] : c3[2];
        const int jp = j1 + NX * j2;
        const R sv = G2[((s * 2 + 0) * NF + f) * FNP + jp];
        const R tv = G2[((s * 2 + 1) * NF + f) * FNP + jp];
        R add = ctab<P, R>(TO::dL + hi * N + k) * tv;
        if (k == (hi ? N - 1 : 0)) add += sv;
        acc += add;
      }
      COL[t * (CH + 1) + cc] = acc;
    }
    __syncthreads();
  }
  // the chunk's columns, row by row
  for (int t = tid; t < nb * ncol; t += NT) {
    const int r = t / ncol, cc = t % ncol;
    out[((long long)e * nb + r) * nb + c0 + cc] = to_io(COL[r * (CH + 1) + cc]);
  }
}

}  // namespace enp
