// The CNP DG operator on hexahedra, thread-per-pencil layout (sm_103a).
//
// Same arithmetic as op_kernel (enp_operator.cuh: R(u), J(u)v, J(u)^T w and
// block columns of Eq. NPDG / Eq. chargeDG), organised for throughput:
//  * Q x Q threads per element, EB elements per thread block;
//  * every 1D contraction is done by one thread per pencil: it loads the
//    pencil into registers and forms all outputs with the basis table in
//    __constant__ memory at compile-time indices (the table entries become
//    FMA operands, no loads);
//  * each stage runs over all fields and vectors of the element at once, so a
//    stage costs one __syncthreads;
//  * the pointwise physics (volume and faces) is the one op_kernel uses.
#pragma once
#include <type_traits>

#include "enp_operator.cuh"

#ifndef ENP_DF_MIN_BLOCKS
#define ENP_DF_MIN_BLOCKS 3
#endif

namespace enp {

constexpr int kTabSz = 128;  // per degree: B (Q*N), Dq (Q*Q), dL (2N), wq (Q), xq (Q), BD (Q*N)
static __constant__ double c_tabd[kMaxP + 1][kTabSz];
static __constant__ float c_tabf[kMaxP + 1][kTabSz];
static __constant__ float2 c_tabdf[kMaxP + 1][kTabSz];   // (hi, lo) double-float pairs

// Upload the tables of degree p to this translation unit's constant banks on
// the current device.
static inline cudaError_t upload_const_tables(int p, const Tables& t) {
  const int n = p + 1, q = p + 2;
  double d[kTabSz] = {0};
  float f[kTabSz] = {0};
  float2 w[kTabSz];
  int o = 0;
  for (int i = 0; i < q * n; ++i) d[o++] = t.B[i];
  for (int i = 0; i < q * q; ++i) d[o++] = t.Dq[i];
  for (int i = 0; i < 2 * n; ++i) d[o++] = t.dL[i];
  for (int i = 0; i < q; ++i) d[o++] = t.wq[i];
  for (int i = 0; i < q; ++i) d[o++] = t.xq[i];
  // BD = Dq B: the derivative of each basis function at the Gauss points, as the
  // operator forms gradients (collocation derivative of the interpolant)
  for (int a = 0; a < q; ++a)
    for (int i = 0; i < n; ++i) {
      double sacc = 0.0;
      for (int b = 0; b < q; ++b) sacc += t.Dq[a * q + b] * t.B[b * n + i];
      d[o++] = sacc;
    }
  for (int i = 0; i < kTabSz; ++i) {
    f[i] = (float)d[i];
    const df x(d[i]);
    w[i] = make_float2(x.hi, x.lo);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_tabd, d, sizeof(d), sizeof(d) * p);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tabf, f, sizeof(f), sizeof(f) * p);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tabdf, w, sizeof(w), sizeof(w) * p);
  return e;
}

template <int P, class R>
__device__ __forceinline__ R ctab(int i) {
  if constexpr (std::is_same<R, double>::value) return c_tabd[P][i];
  else if constexpr (std::is_same<R, df>::value) return df(c_tabdf[P][i].x, c_tabdf[P][i].y);
  else return c_tabf[P][i];
}
template <int P> struct TabOff {
  static constexpr int N = P + 1, Q = P + 2;
  static constexpr int B = 0, Dq = Q * N, dL = Q * N + Q * Q, W = dL + 2 * N, X = W + Q;
  static constexpr int BD = X + Q;
  static_assert(BD + Q * N <= kTabSz, "table block too small");
};

// The outputs of one pencil: dst[r * os] = sum_k M[r][k] src[k * is] (+ dst[r * os]
// when ACC), r < ROWS, k < COLS, with M the B table (TAB 0, Q x N, or its
// transpose) or the Dq table (TAB 1, Q x Q); table entries at compile-time
// indices.
template <int P, int TAB, bool TRANS, bool ACC, int COLS, int ROWS, class R>
__device__ __forceinline__ void pencil_rows(const R* __restrict__ src, int is, R* __restrict__ dst,
                                            int os) {
  using T = TabOff<P>;
  R x[COLS];
#pragma unroll
  for (int k = 0; k < COLS; ++k) x[k] = src[k * is];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    if constexpr (std::is_same<R, df>::value) {
      // double-float dot product: the leading parts summed with TwoSum, the
      // product errors, cross terms and sum errors gathered in one binary32
      // term, one renormalisation per output
      float s = 0.f, t = 0.f;
      if (ACC) { s = dst[r * os].hi; t = dst[r * os].lo; }
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        int idx;
        if (TAB == 0) idx = T::B + (TRANS ? k * T::N + r : r * T::N + k);
        else idx = T::Dq + (TRANS ? k * T::Q + r : r * T::Q + k);
        const float2 m = c_tabdf[P][idx];
        const float p = __fmul_rn(m.x, x[k].hi);
        float e = __fmaf_rn(m.x, x[k].hi, -p);
        e = __fmaf_rn(m.x, x[k].lo, e);
        e = __fmaf_rn(m.y, x[k].hi, e);
        if (!ACC && k == 0) {
          s = p;
          t = e;
        } else {
          float s2, err;
          two_sum(s, p, s2, err);
          s = s2;
          t = __fadd_rn(t, __fadd_rn(err, e));
        }
      }
      dst[r * os] = fast_two_sum(s, t);
    } else {
      R acc = ACC ? dst[r * os] : R(0);
#pragma unroll
      for (int k = 0; k < COLS; ++k) {
        int idx;
        if (TAB == 0) idx = T::B + (TRANS ? k * T::N + r : r * T::N + k);
        else idx = T::Dq + (TRANS ? k * T::Q + r : r * T::Q + k);
        acc = mad(ctab<P, R>(idx), x[k], acc);
      }
      dst[r * os] = acc;
    }
  }
}

// One thread per pencil: out = M in along direction DIR of a 3D array with
// input extents (E0, E1, E2); M is the B table (TAB 0, ROWS x COLS = Q x N, or
// its transpose) or the Dq table (TAB 1, Q x Q). CNT arrays (stride IN_ST in
// the input, OUT_ST in the output) are processed, pencils shared over the
// NT threads of the element.
template <int P, int E0, int E1, int E2, int DIR, int TAB, bool TRANS, bool ACC, int CNT,
          int IN_ST, int OUT_ST, class R, int IX = E0, int OX = -1>
__device__ __forceinline__ void pencil(const R* __restrict__ in, R* __restrict__ out, int tid,
                                       int NT) {
  // IX: input row stride along dimension 0 (>= E0, padded arrays); OX: output row
  // stride (default: the output extent of dimension 0).
  using T = TabOff<P>;
  constexpr int COLS = DIR == 0 ? E0 : (DIR == 1 ? E1 : E2);
  constexpr int ROWS = TAB == 0 ? (TRANS ? T::N : T::Q) : T::Q;
  constexpr int O0 = DIR == 0 ? ROWS : E0, O1 = DIR == 1 ? ROWS : E1, O2 = DIR == 2 ? ROWS : E2;
  constexpr int OXX = OX < 0 ? O0 : OX;
  constexpr int IS = DIR == 0 ? 1 : (DIR == 1 ? IX : IX * E1);
  constexpr int OS = DIR == 0 ? 1 : (DIR == 1 ? OXX : OXX * O1);
  constexpr int PA = DIR == 0 ? O1 : O0;          // pencil index ranges over the other dims
  constexpr int PB = DIR == 2 ? O1 : O2;
  constexpr int NP = PA * PB;
  // work item w = c * NP + pp; (c, pp) advance by constant steps (no division
  // per item), and the pencil's position is recomputed only when pp moves
  int c = tid / NP, pp = tid % NP;
  const int dc = NT / NP, dp = NT % NP;
#pragma unroll 1
  for (int w = tid; w < NP * CNT; w += NT) {
    const int ia = pp % PA, ib = pp / PA;
    int ibase, obase;
    if (DIR == 0) { ibase = IX * (ia + E1 * ib); obase = OXX * (ia + O1 * ib); }
    else if (DIR == 1) { ibase = ia + IX * E1 * ib; obase = ia + OXX * O1 * ib; }
    else { ibase = ia + IX * ib; obase = ia + OXX * ib; }
    pencil_rows<P, TAB, TRANS, ACC, COLS, ROWS, R>(in + c * IN_ST + ibase, IS,
                                                    out + c * OUT_ST + obase, OS);
    c += dc;
    pp += dp;
    if (pp >= NP) { pp -= NP; ++c; }
  }
}

// The three reference derivatives at the Q^3 points in one pass: for each of
// CNT arrays (stride ST) of point values V, the arrays V + d Q^3 (d = 1, 2, 3)
// receive Dq V along x, y and z. Work items run over (direction, array,
// pencil), so the three directions share the passes of the block's threads.
template <int P, int CNT, int ST, class R>
__device__ __forceinline__ void pencil_grad3(R* V, int tid, int NT) {
  constexpr int Q = P + 2, NQ = Q * Q * Q, NP = Q * Q, PER = NP * CNT;
#pragma unroll 1
  for (int w = tid; w < 3 * PER; w += NT) {
    const int d = w / PER, r = w - d * PER;
    const int c = r / NP, pp = r - c * NP;
    const int ia = pp % Q, ib = pp / Q;
    // pencil along d: the other two coordinates are (ia, ib) in increasing order
    const int is = d == 0 ? 1 : (d == 1 ? Q : Q * Q);
    const int base = d == 0 ? Q * (ia + Q * ib) : (d == 1 ? ia + Q * Q * ib : ia + Q * ib);
    const R* src = V + c * ST + base;
    pencil_rows<P, 1, false, false, Q, Q, R>(src, is, V + c * ST + (1 + d) * NQ + base, is);
  }
}

// Nodal arrays are stored with the x row padded to an odd length, so that
// threads working on neighbouring x-pencils hit different shared-memory banks.
template <int N> struct Pad { static constexpr int X = (N % 2 == 0) ? N + 1 : N; };
template <int N>
__device__ __forceinline__ int padded_node(int i) {  // lexicographic node -> padded offset
  const int ix = i % N, iyz = i / N;
  return ix + Pad<N>::X * iyz;
}
template <int N>
__device__ __forceinline__ int face_node_pad(int a, int k, int j1, int j2) {
  constexpr int X = Pad<N>::X;
  if (a == 0) return k + X * (j1 + N * j2);
  if (a == 1) return j1 + X * (k + N * j2);
  return j1 + X * (j2 + N * k);
}

// Staging of global values into shared memory with asynchronous copies
// (cp.async), so that all of a stage's loads are in flight at once without
// holding registers. A slot of R receives the raw value of the vector type IO
// (the same bytes for FP32 and FP64; a double into a double-float slot, whose
// 8 bytes it fills, converted in place by stage_finish once the copies landed).
template <class R, class IO>
__device__ __forceinline__ void stage_copy(R* dst, const IO* src) {
  static_assert(sizeof(IO) == sizeof(R) && (sizeof(R) == 4 || sizeof(R) == 8), "slot size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(sizeof(R))
               : "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// After stage_wait, by the thread that issued the copy: the slot's value as R.
template <class R>
__device__ __forceinline__ void stage_finish(R* slot) {
  if constexpr (std::is_same<R, df>::value)
    *slot = df_from_double_dev(*reinterpret_cast<const double*>(slot));
}

// The coefficients as forward tangents seeded on parameter j of
// theta = (D_1..D_m, c_in_1..c_in_{m-1}, phi_app_0..phi_app_3).
template <class R>
__device__ PhysT<Tan<R>> seed_phys(const PhysT<R>& p, int m, int j) {
  PhysT<Tan<R>> q;
  for (int k = 0; k < kMaxSpecies; ++k) {
    q.D[k] = Tan<R>(p.D[k]); q.cin[k] = Tan<R>(p.cin[k]); q.mig[k] = Tan<R>(p.mig[k]);
    q.acoef[k] = Tan<R>(p.acoef[k]); q.kcoef[k] = Tan<R>(p.kcoef[k]); q.z[k] = Tan<R>(p.z[k]);
    q.zratio[k] = Tan<R>(p.zratio[k]);
    q.dmig[k] = Tan<R>(p.dmig[k]); q.da[k] = Tan<R>(p.da[k]);
    q.dkc_own[k] = Tan<R>(p.dkc_own[k]); q.dkc_m[k] = Tan<R>(p.dkc_m[k]);
  }
  q.neg_inv_zm = Tan<R>(p.neg_inv_zm);
  for (int i = 0; i < 8; ++i) q.vp[i] = Tan<R>(p.vp[i]);
  q.vel_coef = Tan<R>(p.vel_coef);
  q.J0 = Tan<R>(p.J0); q.e1 = Tan<R>(p.e1); q.e2 = Tan<R>(p.e2);
  q.gam = Tan<R>(p.gam); q.gam1 = Tan<R>(p.gam1); q.inv_cref = Tan<R>(p.inv_cref);
  q.ox_species_scale = Tan<R>(p.ox_species_scale); q.ox_charge_scale = Tan<R>(p.ox_charge_scale);
  for (int i = 0; i < 4; ++i) q.phiapp[i] = Tan<R>(p.phiapp[i]);
  q.J0lo = Tan<R>(p.J0lo); q.J0half = Tan<R>(p.J0half); q.J0inv_half = Tan<R>(p.J0inv_half);
  q.cip = Tan<R>(p.cip);
  q.vel_kind = p.vel_kind; q.velA = p.velA; q.velN = p.velN; q.bv_ox = p.bv_ox; q.J0axis = p.J0axis;
  if (j < m) {                        // D_j: D, z_j mu_j F, the a_k and kappa coefficients
    if (j < m - 1) { q.D[j].d = R(1); q.mig[j].d = p.dmig[j]; }
    for (int k = 0; k < m - 1; ++k) {
      q.acoef[k].d = (k == j ? p.da[k] : R(0)) - (j == m - 1 ? p.da[k] : R(0));
      q.kcoef[k].d = (k == j ? p.dkc_own[k] : R(0)) + (j == m - 1 ? p.dkc_m[k] : R(0));
    }
  } else if (j < 2 * m - 1) {         // c_in of species j - m
    q.cin[j - m].d = R(1);
  } else {                            // phi_app of electrode j - (2m - 1)
    q.phiapp[j - (2 * m - 1)].d = R(1);
  }
  return q;
}

// Threads per element of the hexahedral kernel: Q x Q (one per pencil) for
// FP64, whose issue rate the FP64 pipe bounds; more for FP32, which is
// latency-bound and needs more warps in flight for the same shared memory.
template <int P, class R>
__host__ __device__ constexpr int tpe3d() {
  if constexpr (std::is_same<R, double>::value) return (P + 2) * (P + 2);
  else return P <= 1 ? 32 : (P == 2 ? 64 : 128);   // FP32 and double-float: the FP32 pipe
}

template <int P, int NF, int MODE, int NT>
struct Smem3 {
  static constexpr int N = P + 1, Q = P + 2;
  static constexpr int NX = Pad<N>::X;                   // padded x row of nodal arrays
  static constexpr int NN = N * N * N, NQ = Q * Q * Q, FN = N * N, FQ = Q * Q;
  static constexpr int NNP = NX * N * N;                 // padded nodal array
  static constexpr int FNP = NX * N;                     // padded face-node array
  static constexpr int NV = (MODE == kResidual || MODE == kParam) ? 1 : 2;
  static constexpr int NA = NV * NF;                     // arrays carried through the volume
  static constexpr int kX = NA * NNP;                    // element data
  static constexpr int kOut = NF * NNP;                  // rows
  static constexpr int kT1 = NA * Q * N * N;             // after the x contraction
  static constexpr int kT2 = NA * Q * Q * N;             // after the y contraction
  static constexpr int kPts = NA * 4 * NQ;               // values + 3 gradients
  // R, J v and J^T w take their face terms from the face kernel's buffer:
  // the six sides' lifted coefficients [6][2][NF][FN]
  static constexpr bool kFB = MODE == kResidual || MODE == kJvp || MODE == kVjp;
  static constexpr int kFaceLoop = NA * NNP              // neighbour data
                               + 2 * NA * 2 * FNP         // layer values + normal derivatives
                               + 2 * NA * 2 * Q * N       // after the first face contraction
                               + 2 * NA * 2 * FQ          // traces at face points
                               + 2 * NF * FQ              // face coefficients
                               + 2 * NF * Q * N           // transposed, first stage
                               + 2 * NF * FNP;            // transposed, at face nodes
  static constexpr int kFace = kFB ? 6 * 2 * NF * FN : kFaceLoop;
  // T1 is dead once T2 is formed, so it shares space with the point arrays
  static constexpr int kVol = kT2 + (kPts > kT1 ? kPts : kT1);
  static constexpr int kWork = kVol > kFace ? kVol : kFace;
  static constexpr int raw = kX + kOut + kWork;
  // stride between element regions: congruent to the element's thread count
  // modulo the bank count (32 words), so that a warp spanning two elements
  // keeps consecutive threads on consecutive banks
  static constexpr int kBankWords = 32;
  static constexpr int total = raw + ((NT - raw % kBankWords) % kBankWords + kBankWords) % kBankWords;
  static constexpr int kPrefetch = (NA * NN + NT - 1) / NT;  // neighbour values per thread
};

// Largest thread block of the hexahedral kernel; the elements per block (EB,
// chosen at launch by the autotuner) satisfy EB * tpe3d <= this.
constexpr int kMaxThreads3D = 256;
// Resident blocks per SM the register allocation is sized for: the
// double-float kernels are issue-bound on the FP32 pipe and need more warps in
// flight than their natural register count allows.
template <class R> struct MinBlocks3D { static constexpr int value = 1; };
template <> struct MinBlocks3D<df> { static constexpr int value = ENP_DF_MIN_BLOCKS; };

template <int P, int NF, int MODE, class R>
__global__ void __launch_bounds__(kMaxThreads3D, MinBlocks3D<R>::value)
op3d_kernel(const OpParams prm, const io_t<R>* __restrict__ u, const io_t<R>* __restrict__ v,
            io_t<R>* __restrict__ out) {
  using S = Smem3<P, NF, MODE, tpe3d<P, R>()>;
  using TO = TabOff<P>;
  constexpr int N = S::N, Q = S::Q, NN = S::NN, NQ = S::NQ, FN = S::FN, FQ = S::FQ;
  constexpr int NX = S::NX, NNP = S::NNP, FNP = S::FNP;
  constexpr int NV = S::NV, NA = S::NA, NT = tpe3d<P, R>(), PF = S::kPrefetch;
  constexpr bool kBlk = MODE == kBlockCol;
  constexpr int MODEc = kBlk ? kJvp : MODE;
  const PhysT<R>& ph = phys<R>(prm);
  extern __shared__ __align__(16) unsigned char smem3_raw[];
  const int es = threadIdx.x / NT, tid = threadIdx.x % NT;
  R* base = reinterpret_cast<R*>(smem3_raw) + es * S::total;
  R* XA = base;                 // [NA][NNP] padded nodal arrays
  R* RO = XA + S::kX;           // [NF][NNP]
  R* WK = RO + S::kOut;
  const int EB = blockDim.x / NT;   // elements per block, chosen at launch
  const int e = blockIdx.x * EB + es;
  const bool valid = e < prm.E;
  const int ee = valid ? e : prm.E - 1;   // invalid slots shadow a valid element, write nothing
  constexpr bool kPar = MODE == kParam;
  const int col = kBlk ? (int)blockIdx.y : -1;
  const int bidx = kBlk ? 0 : (kPar ? (int)blockIdx.y / prm.n_theta : (int)blockIdx.y);
  const int theta_j = kPar ? (int)blockIdx.y % prm.n_theta : -1;
  const long long boff = kBlk ? 0 : (long long)bidx * prm.batch_stride;
  const long long ooff = kPar ? ((long long)theta_j * prm.batch + bidx) * prm.batch_stride : boff;
  const long long EN = (long long)prm.E * NN;

  int idx[3];
  idx[0] = ee % prm.ne[0];
  idx[1] = (ee / prm.ne[0]) % prm.ne[1];
  idx[2] = ee / (prm.ne[0] * prm.ne[1]);
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

  for (int t = tid; t < NF * NN; t += NT) {
    const int f = t / NN, i = t % NN;
    const long long gi = boff + f * EN + (long long)ee * NN + i;
    const int pi = f * NNP + padded_node<N>(i);
    stage_copy(XA + pi, u + gi);
    if (NV == 2) {
      if (kBlk) XA[NF * NNP + pi] = R(t == col ? 1 : 0);
      else stage_copy(XA + NF * NNP + pi, v + gi);
    }
  }
  stage_wait();
  if constexpr (std::is_same<R, df>::value) {
    for (int t = tid; t < NF * NN; t += NT) {
      const int pi = (t / NN) * NNP + padded_node<N>(t % NN);
      stage_finish(XA + pi);
      if (NV == 2 && !kBlk) stage_finish(XA + NF * NNP + pi);
    }
  }
  // neighbour data of a face, fetched into registers one face ahead so that the
  // global loads overlap the computation of the previous stage
  const int stride[3] = {1, prm.ne[0], prm.ne[0] * prm.ne[1]};
  R pf[PF];
  auto prefetch = [&](int s) {
    const int a = s >> 1, hi = s & 1;
    const bool bnd = hi ? (idx[a] == prm.ne[a] - 1) : (idx[a] == 0);
    if (bnd) return;
    const int en = ee + (hi ? stride[a] : -stride[a]);
#pragma unroll
    for (int k = 0; k < PF; ++k) {
      const int t = tid + k * NT;
      if (t < NA * NN) {
        const int vv = t / (NF * NN), r = t % (NF * NN), f = r / NN, i = r % NN;
        const long long gi = boff + f * EN + (long long)en * NN + i;
        pf[k] = vv == 0 ? R(u[gi]) : (kBlk ? R(0) : R(v[gi]));
      }
    }
  };
  if constexpr (!S::kFB) prefetch(0);
  if constexpr (S::kFB) {
    // the six sides' lifted face terms are read after the volume terms: start
    // moving them into L2 now (one 128-byte line per work item)
    constexpr int PER = 2 * NF * FN;
    constexpr int LINES = (PER * (int)sizeof(R) + 127) / 128 + 1;  // + 1: unaligned start
    for (int q = tid; q < 6 * LINES; q += NT) {
      const int s = q / LINES, l = q % LINES;
      const int a = s >> 1, hi = s & 1;
      const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
      // run-time axes: selections, not indexed arrays (which would go to local memory)
      const long long gid = pick3(prm.foff, a) + (pick3(idx, a) + hi) +
                            (long long)(pick3(prm.ne, a) + 1) *
                                (pick3(idx, b0) + (long long)pick3(prm.ne, b0) * pick3(idx, b1));
      const char* src = reinterpret_cast<const char*>(reinterpret_cast<const R*>(prm.fbuf) +
                                                      (long long)bidx * prm.fbuf_stride +
                                                      (gid * 2 + (hi ? 0 : 1)) * PER);
      const int off = l * 128 < PER * (int)sizeof(R) ? l * 128 : PER * (int)sizeof(R) - 1;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(src + off));
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- volume
  R* T2 = WK;                   // [NA][N][Q][Q]
  R* PT = T2 + S::kT2;          // [NA][4][NQ]
  R* T1 = PT;                   // [NA][N][N][Q], dead before PT is written
  pencil<P, N, N, N, 0, 0, false, false, NA, NNP, Q * N * N, R, NX>(XA, T1, tid, NT);
  __syncthreads();
  pencil<P, Q, N, N, 1, 0, false, false, NA, Q * N * N, Q * Q * N>(T1, T2, tid, NT);
  __syncthreads();
  pencil<P, Q, Q, N, 2, 0, false, false, NA, Q * Q * N, 4 * NQ>(T2, PT, tid, NT);
  __syncthreads();
  pencil_grad3<P, NA, 4 * NQ>(PT, tid, NT);
  __syncthreads();

  {
    // points pt = tid, tid + NT, ...: with NT = Q^2 one thread runs down the z
    // line of its (kx, ky), and the x-y weight and coordinates are hoisted
    constexpr bool kLine = NT == Q * Q;
    const int kx0 = tid % Q, ky0 = (tid / Q) % Q;
    const R wxy0 = ctab<P, R>(TO::W + kx0) * ctab<P, R>(TO::W + ky0) * detJ;
    const R xp00 = lo[0] + R(0.5) * (ctab<P, R>(TO::X + kx0) + R(1)) * h[0];
    const R xp01 = lo[1] + R(0.5) * (ctab<P, R>(TO::X + ky0) + R(1)) * h[1];
#pragma unroll 1
    for (int pt = tid; pt < NQ; pt += NT) {
      const int kx = kLine ? kx0 : pt % Q, ky = kLine ? ky0 : (pt / Q) % Q, kz = pt / (Q * Q);
      const R wxy = kLine ? wxy0 : ctab<P, R>(TO::W + kx) * ctab<P, R>(TO::W + ky) * detJ;
      R xp[3];
      xp[0] = kLine ? xp00 : lo[0] + R(0.5) * (ctab<P, R>(TO::X + kx) + R(1)) * h[0];
      xp[1] = kLine ? xp01 : lo[1] + R(0.5) * (ctab<P, R>(TO::X + ky) + R(1)) * h[1];
      xp[2] = lo[2] + R(0.5) * (ctab<P, R>(TO::X + kz) + R(1)) * h[2];
      R uv[3];
      velocity(ph, xp, uv);
      const R w = wxy * ctab<P, R>(TO::W + kz);
      R c0[NF], g0[NF][3];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const R* V = PT + f * 4 * NQ;
        c0[f] = V[pt];
#pragma unroll
        for (int a = 0; a < 3; ++a) g0[f][a] = V[(1 + a) * NQ + pt] * sc[a];
      }
      R oS[NF], oG[NF][3];
      if (MODEc == kParam) {
        const PhysT<Tan<R>> pt = seed_phys<R>(ph, NF, theta_j);
        Tan<R> ct[NF], gt[NF][3], Sf[NF], Gf[NF][3];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          ct[f] = Tan<R>(c0[f]);
#pragma unroll
          for (int a = 0; a < 3; ++a) gt[f][a] = Tan<R>(g0[f][a]);
        }
        volume_flux<NF, 3, Tan<R>, R, Tan<R>>(pt, ct, gt, uv, Sf, Gf);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          oS[f] = Sf[f].d;
#pragma unroll
          for (int a = 0; a < 3; ++a) oG[f][a] = Gf[f][a].d;
        }
      } else if (MODEc == kResidual) {
        volume_flux<NF, 3, R, R>(ph, c0, g0, uv, oS, oG);
#pragma unroll
        for (int f = 0; f < NF; ++f)
          oS[f] -= prm.src ? R(prm.src[((long long)f * prm.E + ee) * NQ + pt]) : R(0);
      } else {
        R c1[NF], g1[NF][3];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const R* V = PT + (NF + f) * 4 * NQ;
          c1[f] = V[pt];
#pragma unroll
          for (int a = 0; a < 3; ++a) g1[f][a] = V[(1 + a) * NQ + pt] * sc[a];
        }
        if (MODEc == kJvp) {
          Tan<R> ct[NF], gt[NF][3], Sf[NF], Gf[NF][3];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            ct[f] = Tan<R>(c0[f], c1[f]);
#pragma unroll
            for (int a = 0; a < 3; ++a) gt[f][a] = Tan<R>(g0[f][a], g1[f][a]);
          }
          volume_flux<NF, 3, Tan<R>, R>(ph, ct, gt, uv, Sf, Gf);
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            oS[f] = Sf[f].d;
#pragma unroll
            for (int a = 0; a < 3; ++a) oG[f][a] = Gf[f][a].d;
          }
        } else {
          volume_flux_adjoint<NF, 3, R>(ph, c0, g0, uv, g1, oS, oG);
        }
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        R* V = PT + ((NV - 1) * NF + f) * 4 * NQ;
        V[pt] = w * oS[f];
#pragma unroll
        for (int a = 0; a < 3; ++a) V[(1 + a) * NQ + pt] = w * sc[a] * oG[f][a];
      }
    }
  }
  __syncthreads();
  R* PO = PT + (NV - 1) * NF * 4 * NQ;   // the NF output point arrays
  pencil<P, Q, Q, Q, 0, 1, true, true, NF, 4 * NQ, 4 * NQ>(PO + NQ, PO, tid, NT);
  __syncthreads();
  pencil<P, Q, Q, Q, 1, 1, true, true, NF, 4 * NQ, 4 * NQ>(PO + 2 * NQ, PO, tid, NT);
  __syncthreads();
  pencil<P, Q, Q, Q, 2, 1, true, true, NF, 4 * NQ, 4 * NQ>(PO + 3 * NQ, PO, tid, NT);
  __syncthreads();
  pencil<P, Q, Q, Q, 2, 0, true, false, NF, 4 * NQ, Q * Q * N>(PO, T2, tid, NT);
  __syncthreads();
  R* T1b = PT;  // the point arrays are dead once T2 holds the z-transposed values
  pencil<P, Q, Q, N, 1, 0, true, false, NF, Q * Q * N, Q * N * N>(T2, T1b, tid, NT);
  __syncthreads();
  pencil<P, Q, N, N, 0, 0, true, false, NF, Q * N * N, NNP, R, Q, NX>(T1b, RO, tid, NT);
  __syncthreads();

  // ---------------------------------------------------------------- faces
  if constexpr (S::kFB) {
    // the lifted coefficients of the six sides, left by the face kernel: side
    // (a, hi) of this element is the lower element (0) of face plane
    // idx[a] + 1 when hi, the upper one (1) of plane idx[a] otherwise
    R* FS = WK;  // [6][2][NF][FN]
    const R* fb = reinterpret_cast<const R*>(prm.fbuf) + (long long)bidx * prm.fbuf_stride;
    constexpr int PER = 2 * NF * FN;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      const int a = s >> 1, hi = s & 1;
      const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
      const long long gid = prm.foff[a] + (idx[a] + hi) +
                            (long long)(prm.ne[a] + 1) * (idx[b0] + (long long)prm.ne[b0] * idx[b1]);
      const R* src = fb + (gid * 2 + (hi ? 0 : 1)) * PER;
      for (int r = tid; r < PER; r += NT) stage_copy(FS + s * PER + r, src + r);
    }
    stage_wait();
    __syncthreads();
    // each row gathers its six face terms in side order (no two threads write
    // one row)
    for (int t = tid; t < NF * NN; t += NT) {
      const int f = t / NN, i = t % NN;
      const int c3[3] = {i % N, (i / N) % N, i / (N * N)};
      R acc = RO[f * NNP + padded_node<N>(i)];
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const int a = s >> 1, hi = s & 1;
        const int k = c3[a];
        const int j = a == 0 ? c3[1] + N * c3[2] : (a == 1 ? c3[0] + N * c3[2] : c3[0] + N * c3[1]);
        const R sv = FS[((s * 2 + 0) * NF + f) * FN + j];
        const R tv = FS[((s * 2 + 1) * NF + f) * FN + j];
        R add = ctab<P, R>(TO::dL + hi * N + k) * tv;
        if (k == (hi ? N - 1 : 0)) add += sv;
        acc += add;
      }
      RO[f * NNP + padded_node<N>(i)] = acc;
    }
    __syncthreads();
  } else {
  R* XN = WK;                                  // [NA][NNP] neighbour data
  R* FL = XN + NA * NNP;                       // [2 sides][NA][2][FNP] layer values, derivatives
  R* F1 = FL + 2 * NA * 2 * FNP;               // [2][NA][2][Q][N]
  R* TR = F1 + 2 * NA * 2 * Q * N;             // [2][NA][2][FQ]
  R* FC = TR + 2 * NA * 2 * FQ;                // [2][NF][FQ]: S then T coefficients
  R* G1 = FC + 2 * NF * FQ;                    // [2][NF][N][Q]
  R* G2 = G1 + 2 * NF * Q * N;                 // [2][NF][FNP]
#pragma unroll 1
  for (int s = 0; s < 6; ++s) {
    const int a = s >> 1, hi = s & 1;
    const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    const R nrm = hi ? R(1) : R(-1);
    const bool boundary = hi ? (idx[a] == prm.ne[a] - 1) : (idx[a] == 0);
    int tag = kInterior, bface = -1;
    R hn = h[a], diagn = diag;
    if (boundary) {
      const int loc = idx[b0] + prm.ne[b0] * idx[b1];
      bface = prm.side_off[s] + loc;
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
#pragma unroll
      for (int k = 0; k < PF; ++k) {
        const int t = tid + k * NT;
        if (t < NA * NN) {
          const int arr = t / NN, i = t % NN;
          XN[arr * NNP + padded_node<N>(i)] = pf[k];
        }
      }
    }
    if (s < 5) prefetch(s + 1);
    const bool active = !(tag == kWall || (tag == kInlet && MODEc != kResidual && MODEc != kParam));
    __syncthreads();
    // layer values and reference normal derivatives at the face nodes
    const int lay = hi ? N - 1 : 0, layo = hi ? 0 : N - 1;
    const int nsides = boundary ? 1 : 2;
    for (int w = tid; w < nsides * NA * FN; w += NT) {
      const int side = w / (NA * FN), r = w % (NA * FN), arr = r / FN, j = r % FN;
      const int j1 = j % N, j2 = j / N;
      const R* X = (side == 0 ? XA : XN) + arr * NNP;
      const int L = side == 0 ? lay : layo;
      const int dsel = side == 0 ? hi : 1 - hi;
      R d = R(0);
#pragma unroll
      for (int k = 0; k < N; ++k)
        d = mad(ctab<P, R>(TO::dL + dsel * N + k), X[face_node_pad<N>(a, k, j1, j2)], d);
      R* o = FL + ((side * NA + arr) * 2) * FNP;
      const int jp = j1 + NX * j2;
      o[jp] = X[face_node_pad<N>(a, L, j1, j2)];
      o[FNP + jp] = d;
    }
    __syncthreads();
    // 2D interpolation to the face Gauss points: along b0, then b1. Both sides
    // are always processed so that every thread reaches every barrier; on a
    // boundary face the second side holds stale values that are never read.
    pencil<P, N, N, 1, 0, 0, false, false, 4 * NA, FNP, Q * N, R, NX>(FL, F1, tid, NT);
    __syncthreads();
    pencil<P, Q, N, 1, 1, 0, false, false, 4 * NA, Q * N, FQ>(F1, TR, tid, NT);
    __syncthreads();
    // pointwise face fluxes, one thread per face point
    {
      const R area = R(0.25) * h[b0] * h[b1];
      const R delta = ph.cip * R(P * P) / (boundary ? diag : R(0.5) * (diag + diagn));
      const R sca = sc[a] * nrm;
      const R scn = R(2) / hn * nrm;
      const R phiapp = (tag >= kElectrode0)
          ? (prm.phiapp_batch ? R(prm.phiapp_batch[bidx * 4 + (tag - kElectrode0)])
                              : ph.phiapp[tag - kElectrode0])
          : R(0);
#pragma unroll 1
      for (int pt = tid; pt < FQ; pt += NT) {
      const int k1 = pt % Q, k2 = pt / Q;
      R xp[3];
      xp[a] = hi ? lo[a] + h[a] : lo[a];
      xp[b0] = lo[b0] + R(0.5) * (ctab<P, R>(TO::X + k1) + R(1)) * h[b0];
      xp[b1] = lo[b1] + R(0.5) * (ctab<P, R>(TO::X + k2) + R(1)) * h[b1];
      R uv[3];
      velocity(ph, xp, uv);
      const R un = uv[a] * nrm;
      const R w = ctab<P, R>(TO::W + k1) * ctab<P, R>(TO::W + k2) * area;
      auto trv = [&](int side, int vv, int f, int comp) -> R {
        return TR[(((side * NA) + vv * NF + f) * 2 + comp) * FQ + pt];
      };
      R cm[NF], dm[NF], cp[NF], dp[NF], g[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        cm[f] = trv(0, 0, f, 0);
        dm[f] = trv(0, 0, f, 1) * sca;
        cp[f] = boundary ? R(0) : trv(1, 0, f, 0);
        dp[f] = boundary ? R(0) : trv(1, 0, f, 1) * scn;
        g[f] = (tag == kDirichlet && prm.dirv)
                   ? R(prm.dirv[((long long)f * prm.NBF + bface) * prm.Nfq + pt]) : R(0);
      }
      R oS[NF], oT[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) { oS[f] = R(0); oT[f] = R(0); }
      if (active) {
        if (MODEc == kParam) {
          const PhysT<Tan<R>> pt = seed_phys<R>(ph, NF, theta_j);
          const Tan<R> phit(phiapp, (tag >= kElectrode0 && theta_j == 2 * NF - 1 + tag - kElectrode0)
                                        ? R(1) : R(0));
          Tan<R> tm[NF], tdm[NF], tp[NF], tdp[NF], Sf[NF], Tf[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            tm[f] = Tan<R>(cm[f]); tdm[f] = Tan<R>(dm[f]);
            tp[f] = Tan<R>(cp[f]); tdp[f] = Tan<R>(dp[f]);
          }
          if (boundary)
            face_boundary_flux<NF, Tan<R>, R, Tan<R>>(pt, tag, tm, tdm, g, un, delta, xp, phit, Sf, Tf);
          else
            face_interior_flux<NF, Tan<R>, R, Tan<R>>(pt, tm, tdm, tp, tdp, un, delta, Sf, Tf);
#pragma unroll
          for (int f = 0; f < NF; ++f) { oS[f] = Sf[f].d; oT[f] = Tf[f].d; }
        } else if (MODEc == kResidual) {
          if (boundary) face_boundary_flux<NF, R, R>(ph, tag, cm, dm, g, un, delta, xp, phiapp, oS, oT);
          else face_interior_flux<NF, R, R>(ph, cm, dm, cp, dp, un, delta, oS, oT);
        } else {
          R cm1[NF], dm1[NF], cp1[NF], dp1[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            cm1[f] = trv(0, 1, f, 0);
            dm1[f] = trv(0, 1, f, 1) * sca;
            cp1[f] = boundary ? R(0) : trv(1, 1, f, 0);
            dp1[f] = boundary ? R(0) : trv(1, 1, f, 1) * scn;
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
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        FC[f * FQ + pt] = w * oS[f];
        FC[(NF + f) * FQ + pt] = w * sca * oT[f];
      }
      }
    }
    __syncthreads();
    // transposed 2D contraction back to the face nodes, then into the rows
    pencil<P, Q, Q, 1, 1, 0, true, false, 2 * NF, FQ, Q * N>(FC, G1, tid, NT);
    __syncthreads();
    pencil<P, Q, N, 1, 0, 0, true, false, 2 * NF, Q * N, FNP, R, Q, NX>(G1, G2, tid, NT);
    __syncthreads();
    for (int w = tid; w < NF * FN; w += NT) {
      const int f = w / FN, j = w % FN, j1 = j % N, j2 = j / N;
      R* Rf = RO + f * NNP;
      const int jp = j1 + NX * j2;
      const R sv = G2[f * FNP + jp], tv = G2[(NF + f) * FNP + jp];
      if (active) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
          R add = ctab<P, R>(TO::dL + hi * N + k) * tv;
          if (k == lay) add += sv;
          Rf[face_node_pad<N>(a, k, j1, j2)] += add;
        }
      }
    }
    __syncthreads();
  }
  }  // face loop of the block-column and parameter modes

  if (valid) {
    if (kBlk) {
      const long long nb = NF * NN;
      for (int t = tid; t < NF * NN; t += NT)
        out[((long long)e * nb + t) * nb + col] = to_io(RO[(t / NN) * NNP + padded_node<N>(t % NN)]);
    } else {
      for (int t = tid; t < NF * NN; t += NT) {
        const int f = t / NN, i = t % NN;
        out[ooff + f * EN + (long long)e * NN + i] = to_io(RO[f * NNP + padded_node<N>(i)]);
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Face kernel of R, J v and J^T w: each face of the mesh once, for both of its
// sides. Threads per face: Q x Q for FP64; for FP32 and double-float the
// fewest threads that cover the Q x Q face points in about one pass of the
// pointwise fluxes (16, 16, 32 and 48 at p = 1..4), so that the costliest
// stage keeps its lanes busy; faces per block make up the block.
template <int P, class R>
__host__ __device__ constexpr int tpf3d() {
  if constexpr (std::is_same<R, double>::value) return (P + 2) * (P + 2);
  else return P <= 2 ? 16 : (P == 3 ? 32 : 48);
}

template <int P, int NF, int MODE, int NT>
struct SmemF {
  static constexpr int N = P + 1, Q = P + 2;
  static constexpr int NX = Pad<N>::X;
  static constexpr int NN = N * N * N, FN = N * N, FQ = Q * Q;
  static constexpr int NNP = NX * N * N, FNP = NX * N;
  static constexpr int NV = MODE == kResidual ? 1 : 2;
  static constexpr int NA = NV * NF;
  // Two regions, reused stage by stage: A holds both elements' data X, then
  // (once FL is formed) the interpolation F1 and the traces TR, then (once the
  // fluxes are formed) the transposed contractions G1 and G2; B holds FL, then
  // (once F1 is formed) the face coefficients FC.
  static constexpr int kX = 2 * NA * NNP;              // both elements' data
  static constexpr int kF1 = 2 * NA * 2 * Q * N;       // after the first face contraction
  static constexpr int kTR = 2 * NA * 2 * FQ;          // traces at the face points
  static constexpr int kG1 = 2 * 2 * NF * Q * N;
  static constexpr int kG2 = 2 * 2 * NF * FNP;
  static constexpr int kA0 = kX > kF1 + kTR ? kX : kF1 + kTR;
  static constexpr int kA = kA0 > kG1 + kG2 ? kA0 : kG1 + kG2;
  static constexpr int kFL = 2 * NA * 2 * FNP;         // layer values + normal derivatives
  static constexpr int kFC = 2 * 2 * NF * FQ;          // [side][S, T][NF] at face points
  static constexpr int kB = kFL > kFC ? kFL : kFC;
  static constexpr int raw = kA + kB;
  static constexpr int total = raw + ((NT - raw % 32) % 32 + 32) % 32;
};

// The stages of one face after both elements' data are in XS (the first
// region of `base`): layer values and normal derivatives, the 2D interpolation
// to the face points, the pointwise fluxes, and the transposed 2D contraction
// back to the face nodes. On return (after a barrier) the lifted coefficients
// of both sides are at face3d_g2(base): [side][S, T][NF][FNP]. All threads of
// the block take part in every barrier.
template <int P, int NF, int MODE, class R, int NTS>
__device__ __forceinline__ R* face3d_g2(R* base) {
  using S = SmemF<P, NF, MODE, NTS>;
  return base + S::kG1;
}
template <int P, int NF, int MODE, class R, int NTS>
__device__ __forceinline__ void face3d_stages(const OpParams& prm, R* base, int tid, int NT, int a,
                                              int ia, int j0, int j1, int bidx) {
  using S = SmemF<P, NF, MODE, NTS>;
  using TO = TabOff<P>;
  constexpr int N = S::N, Q = S::Q, FN = S::FN, FQ = S::FQ;
  constexpr int NX = S::NX, NNP = S::NNP, FNP = S::FNP, NA = S::NA;
  const PhysT<R>& ph = phys<R>(prm);
  R* XS = base;                  // [2][NA][NNP]
  R* F1 = base;                  // [2][NA][2][Q][N] (over XS, once FL is formed)
  R* TR = F1 + S::kF1;           // [2][NA][2][FQ]
  R* G1 = base;                  // [2][2][NF][N][Q] (over F1 and TR, once FC is formed)
  R* G2 = G1 + S::kG1;           // [2][2][NF][FNP]
  R* FL = base + S::kA;          // [2][NA][2][FNP]
  R* FC = FL;                    // [2][2][NF][FQ] (over FL, once F1 is formed)
  const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
  const bool hasL = ia > 0, hasU = ia < prm.ne[a];
  const R lo0 = vertex<R>(prm, b0, j0), lo1 = vertex<R>(prm, b1, j1);
  const R h0 = vertex<R>(prm, b0, j0 + 1) - lo0, h1 = vertex<R>(prm, b1, j1 + 1) - lo1;
  const R xa = vertex<R>(prm, a, ia);
  const R hL = hasL ? xa - vertex<R>(prm, a, ia - 1) : R(1);
  const R hU = hasU ? vertex<R>(prm, a, ia + 1) - xa : R(1);
  const R diagL = sqrtv(hL * hL + h0 * h0 + h1 * h1), diagU = sqrtv(hU * hU + h0 * h0 + h1 * h1);
  // face-layer values and reference normal derivatives: the lower element at
  // its upper face (layer N-1, derivative at xi = +1), the upper element at its
  // lower face (layer 0, derivative at xi = -1)
  // node (k along a, face node (j1, j2)) of a padded element array sits at
  // fbase(j1, j2) + k * fstr
  const int fstr = a == 0 ? 1 : (a == 1 ? NX : NX * N);
  for (int w = tid; w < 2 * NA * FN; w += NT) {
    const int sa = w / FN, j = w % FN;          // sa = side * NA + arr
    const int side = sa >= NA ? 1 : 0, arr = sa - side * NA;
    const int jn1 = j % N, jn2 = j / N;
    const int fbase = a == 0 ? NX * (jn1 + N * jn2) : (a == 1 ? jn1 + NX * N * jn2 : jn1 + NX * jn2);
    const R* X = XS + (side * NA + arr) * NNP + fbase;
    const int lay = side == 0 ? N - 1 : 0, dsel = side == 0 ? 1 : 0;
    R d = R(0);
#pragma unroll
    for (int k = 0; k < N; ++k) d = mad(ctab<P, R>(TO::dL + dsel * N + k), X[k * fstr], d);
    R* o = FL + ((side * NA + arr) * 2) * FNP;
    const int jp = jn1 + NX * jn2;
    o[jp] = X[lay * fstr];
    o[FNP + jp] = d;
  }
  __syncthreads();
  pencil<P, N, N, 1, 0, 0, false, false, 4 * NA, FNP, Q * N, R, NX>(FL, F1, tid, NT);
  __syncthreads();
  pencil<P, Q, N, 1, 1, 0, false, false, 4 * NA, Q * N, FQ>(F1, TR, tid, NT);
  __syncthreads();

  {
    const R area = R(0.25) * h0 * h1;
    const R scL = R(2) / hL, scU = R(2) / hU;
    const bool interior = hasL && hasU;
    // boundary face: the one element's own side and outward normal
    const int bside = hasL ? 0 : 1;
    const R nrm = bside == 0 ? R(1) : R(-1);
    const R sca = (bside == 0 ? scL : scU) * nrm;
    int tag = kInterior, bface = -1;
    if (!interior) {
      bface = prm.side_off[2 * a + (bside == 0 ? 1 : 0)] + j0 + prm.ne[b0] * j1;
      tag = prm.btag[bface];
    }
    const bool active = interior || !(tag == kWall || (tag == kInlet && MODE != kResidual));
    const R delta = ph.cip * R(P * P) /
                    (interior ? R(0.5) * (diagL + diagU) : (bside == 0 ? diagL : diagU));
    const R phiapp = (tag >= kElectrode0)
        ? (prm.phiapp_batch ? R(prm.phiapp_batch[bidx * 4 + (tag - kElectrode0)])
                            : ph.phiapp[tag - kElectrode0])
        : R(0);
#pragma unroll 1
    for (int pt = tid; pt < FQ; pt += NT) {
      const int k1 = pt % Q, k2 = pt / Q;
      const R xb0 = lo0 + R(0.5) * (ctab<P, R>(TO::X + k1) + R(1)) * h0;
      const R xb1 = lo1 + R(0.5) * (ctab<P, R>(TO::X + k2) + R(1)) * h1;
      // (x, y, z) of the point by selection (a, b0, b1 are run-time axes)
      R xp[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) xp[c] = c == a ? xa : (c == b0 ? xb0 : xb1);
      R uv[3];
      velocity(ph, xp, uv);
      const R ua = pick3(uv, a);
      const R w = ctab<P, R>(TO::W + k1) * ctab<P, R>(TO::W + k2) * area;
      const R* T0p = TR + pt;
      auto tr = [&](int side, int vv, int f, int comp) -> R {
        return T0p[(((side * NA) + vv * NF + f) * 2 + comp) * FQ];
      };
      R oSL[NF], oTL[NF], oSU[NF], oTU[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) { oSL[f] = oTL[f] = oSU[f] = oTU[f] = R(0); }
      if (interior) {
        // the lower element's view: outward normal +e_a, derivatives along it
        const R un = ua;
        R cm[NF], dm[NF], cp[NF], dp[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          cm[f] = tr(0, 0, f, 0); dm[f] = tr(0, 0, f, 1) * scL;
          cp[f] = tr(1, 0, f, 0); dp[f] = tr(1, 0, f, 1) * scU;
        }
        if (MODE == kResidual) {
          face_interior_flux2<NF, R, R>(ph, cm, dm, cp, dp, un, delta, oSL, oTL, oTU);
#pragma unroll
          for (int f = 0; f < NF; ++f) oSU[f] = -oSL[f];
        } else {
          R cm1[NF], dm1[NF], cp1[NF], dp1[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            cm1[f] = tr(0, 1, f, 0); dm1[f] = tr(0, 1, f, 1) * scL;
            cp1[f] = tr(1, 1, f, 0); dp1[f] = tr(1, 1, f, 1) * scU;
          }
          if (MODE == kJvp) {
            Tan<R> tm[NF], tdm[NF], tp[NF], tdp[NF], Sf[NF], Tf[NF], TfP[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              tm[f] = Tan<R>(cm[f], cm1[f]); tdm[f] = Tan<R>(dm[f], dm1[f]);
              tp[f] = Tan<R>(cp[f], cp1[f]); tdp[f] = Tan<R>(dp[f], dp1[f]);
            }
            face_interior_flux2<NF, Tan<R>, R>(ph, tm, tdm, tp, tdp, un, delta, Sf, Tf, TfP);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              oSL[f] = Sf[f].d; oTL[f] = Tf[f].d; oSU[f] = -Sf[f].d; oTU[f] = TfP[f].d;
            }
          } else {
            // J^T w: the rows of each side, differentiated with respect to both
            // sides' states; the upper side's rows seen from the upper element
            // (normal and normal derivatives flip)
            R acm[NF], adm[NF], acp[NF], adp[NF], bcm[NF], bdm[NF], bcp[NF], bdp[NF];
            R ncm[NF], ndm[NF], ncp[NF], ndp[NF], Sh[NF], Th[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              acm[f] = adm[f] = acp[f] = adp[f] = bcm[f] = bdm[f] = bcp[f] = bdp[f] = R(0);
              Sh[f] = cm1[f]; Th[f] = dm1[f];
            }
            face_interior_adjoint<NF, R>(ph, cm, dm, cp, dp, un, delta, Sh, Th, acm, adm, acp, adp);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              ncm[f] = cp[f]; ndm[f] = -dp[f]; ncp[f] = cm[f]; ndp[f] = -dm[f];
              Sh[f] = cp1[f]; Th[f] = -dp1[f];
            }
            face_interior_adjoint<NF, R>(ph, ncm, ndm, ncp, ndp, -un, delta, Sh, Th, bcm, bdm, bcp, bdp);
#pragma unroll
            for (int f = 0; f < NF; ++f) {
              oSL[f] = acm[f] + bcp[f]; oTL[f] = adm[f] - bdp[f];
              oSU[f] = bcm[f] + acp[f]; oTU[f] = bdm[f] - adp[f];
            }
          }
        }
      } else if (active) {
        const R un = ua * nrm;
        R cm[NF], dm[NF], g[NF], oS[NF], oT[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          cm[f] = tr(bside, 0, f, 0);
          dm[f] = tr(bside, 0, f, 1) * sca;
          g[f] = (tag == kDirichlet && prm.dirv)
                     ? R(prm.dirv[((long long)f * prm.NBF + bface) * prm.Nfq + pt]) : R(0);
          oS[f] = R(0); oT[f] = R(0);
        }
        if (MODE == kResidual) {
          face_boundary_flux<NF, R, R>(ph, tag, cm, dm, g, un, delta, xp, phiapp, oS, oT);
        } else {
          R cm1[NF], dm1[NF];
#pragma unroll
          for (int f = 0; f < NF; ++f) { cm1[f] = tr(bside, 1, f, 0); dm1[f] = tr(bside, 1, f, 1) * sca; }
          if (MODE == kJvp) {
            Tan<R> tm[NF], tdm[NF], Sf[NF], Tf[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) { tm[f] = Tan<R>(cm[f], cm1[f]); tdm[f] = Tan<R>(dm[f], dm1[f]); }
            face_boundary_flux<NF, Tan<R>, R>(ph, tag, tm, tdm, g, un, delta, xp, phiapp, Sf, Tf);
#pragma unroll
            for (int f = 0; f < NF; ++f) { oS[f] = Sf[f].d; oT[f] = Tf[f].d; }
          } else {
            R acm[NF], adm[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) acm[f] = adm[f] = R(0);
            face_boundary_adjoint<NF, R>(ph, tag, cm, dm, g, un, delta, xp, phiapp, cm1, dm1, acm, adm);
#pragma unroll
            for (int f = 0; f < NF; ++f) { oS[f] = acm[f]; oT[f] = adm[f]; }
          }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (bside == 0) { oSL[f] = oS[f]; oTL[f] = oT[f]; }
          else { oSU[f] = oS[f]; oTU[f] = oT[f]; }
        }
      }
      // weights, and the normal derivative of each side's test functions along
      // its own outward normal (+e_a for the lower side, -e_a for the upper)
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        FC[((0 * 2 + 0) * NF + f) * FQ + pt] = w * oSL[f];
        FC[((0 * 2 + 1) * NF + f) * FQ + pt] = w * scL * oTL[f];
        FC[((1 * 2 + 0) * NF + f) * FQ + pt] = w * oSU[f];
        FC[((1 * 2 + 1) * NF + f) * FQ + pt] = -(w * scU * oTU[f]);
      }
    }
  }
  __syncthreads();
  // transposed 2D contraction back to the face nodes, both sides
  pencil<P, Q, Q, 1, 1, 0, true, false, 4 * NF, FQ, Q * N>(FC, G1, tid, NT);
  __syncthreads();
  pencil<P, Q, N, 1, 0, 0, true, false, 4 * NF, Q * N, FNP, R, Q, NX>(G1, G2, tid, NT);
  __syncthreads();
}

template <int P, int NF, int MODE, class R>
__global__ void __launch_bounds__(kMaxThreads3D, MinBlocks3D<R>::value)
face3d_kernel(const OpParams prm, const io_t<R>* __restrict__ u, const io_t<R>* __restrict__ v) {
  constexpr int NT = tpf3d<P, R>();
  using S = SmemF<P, NF, MODE, NT>;
  constexpr int N = S::N, NN = S::NN, FN = S::FN;
  constexpr int NX = S::NX, NNP = S::NNP, FNP = S::FNP, NA = S::NA;
  extern __shared__ __align__(16) unsigned char smemf_raw[];
  const int fs = threadIdx.x / NT, tid = threadIdx.x % NT;
  R* base = reinterpret_cast<R*>(smemf_raw) + fs * S::total;
  R* XS = base;                  // [2][NA][NNP]
  const int FPB = blockDim.x / NT;
  const long long nf = prm.foff[3];
  const long long graw = (long long)blockIdx.x * FPB + fs;
  const bool valid = graw < nf;
  const long long g = valid ? graw : nf - 1;     // idle slots shadow a face, write nothing
  const int bidx = blockIdx.y;
  const long long boff = (long long)bidx * prm.batch_stride;
  const long long EN = (long long)prm.E * NN;

  const int a = (g >= prm.foff[1]) + (g >= prm.foff[2]);
  const long long fi = g - prm.foff[a];
  const int na0 = prm.ne[a] + 1;
  const int ia = (int)(fi % na0);
  const long long rr = fi / na0;
  const int nb0 = prm.ne[a == 0 ? 1 : 0];
  const int j0 = (int)(rr % nb0), j1 = (int)(rr / nb0);
  const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
  const long long gid = prm.foff[a] + ia + (long long)(prm.ne[a] + 1) * (j0 + (long long)prm.ne[b0] * j1);
  const bool hasL = ia > 0, hasU = ia < prm.ne[a];
  const int stride[3] = {1, prm.ne[0], prm.ne[0] * prm.ne[1]};
  const int sa = pick3(stride, a);
  const int eU = ia * sa + j0 * pick3(stride, b0) + j1 * pick3(stride, b1);  // valid when hasU
  const int eL = eU - sa;                                                   // valid when hasL

  // both elements' data (a missing side is zero and never read); node-outer, so
  // the padded offset is formed once per node
  {
    const long long gL = boff + (long long)(hasL ? eL : 0) * NN;
    const long long gU = boff + (long long)(hasU ? eU : 0) * NN;
    for (int i = tid; i < NN; i += NT) {
      const int pi = padded_node<N>(i);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long o = f * EN + i;
        if (hasL) stage_copy(XS + f * NNP + pi, u + gL + o);
        else XS[f * NNP + pi] = R(0);
        if (hasU) stage_copy(XS + (NA + f) * NNP + pi, u + gU + o);
        else XS[(NA + f) * NNP + pi] = R(0);
        if (NA > NF) {
          if (hasL) stage_copy(XS + (NF + f) * NNP + pi, v + gL + o);
          else XS[(NF + f) * NNP + pi] = R(0);
          if (hasU) stage_copy(XS + (NA + NF + f) * NNP + pi, v + gU + o);
          else XS[(NA + NF + f) * NNP + pi] = R(0);
        }
      }
    }
    stage_wait();
    if constexpr (std::is_same<R, df>::value) {
      for (int i = tid; i < NN; i += NT) {
        const int pi = padded_node<N>(i);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (hasL) stage_finish(XS + f * NNP + pi);
          if (hasU) stage_finish(XS + (NA + f) * NNP + pi);
          if (NA > NF) {
            if (hasL) stage_finish(XS + (NF + f) * NNP + pi);
            if (hasU) stage_finish(XS + (NA + NF + f) * NNP + pi);
          }
        }
      }
    }
  }
  __syncthreads();
  face3d_stages<P, NF, MODE, R, NT>(prm, base, tid, NT, a, ia, j0, j1, bidx);
  const R* G2 = face3d_g2<P, NF, MODE, R, NT>(base);
  if (valid) {
    R* fb = reinterpret_cast<R*>(prm.fbuf) + (long long)bidx * prm.fbuf_stride +
            gid * 2 * 2 * NF * FN;
    for (int w = tid; w < 2 * 2 * NF * FN; w += NT) {
      const int c = w / FN, j = w % FN;   // c = (side * 2 + S/T) * NF + f
      fb[w] = G2[c * FNP + (j % N) + NX * (j / N)];
    }
  }
}

}  // namespace enp
