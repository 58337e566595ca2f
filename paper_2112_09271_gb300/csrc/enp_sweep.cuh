// One element plane of the downwind block Gauss-Seidel sweep, in one launch.
//
// The sweep solves (D + L) z = x with D the element-diagonal blocks of J and L
// each element's coupling to its upstream neighbour along the flow axis a
// (Sec. 4: the block preconditioner of the Newton-Krylov solve, ordered along
// the advection of Eq. NPDG). Planes of elements are solved in flow order;
// within a plane every element is independent. One thread block takes one
// element e of the plane for one operating point b:
//   1. the face between e and its upstream neighbour: both elements' states,
//      the upstream element's tangent z_up and a zero tangent on e's side, run
//      through the face stages of the J v face kernel (the same arithmetic);
//   2. t = x_e minus e's side of the lifted face terms (its S and T
//      coefficients lifted onto e's nodes as the element kernel gathers them);
//   3. z_e = Binv_e t, with the inverse stored transposed (BT[c][r]).
// The first plane (no upstream plane) skips 1 and 2. This replaces a face-plane
// launch plus a block-apply launch per plane, and the face terms never leave
// shared memory.
#pragma once
#include <cuda_bf16.h>

#include "enp_operator3d.cuh"

namespace enp {

// Threads of the fused sweep block: at least the face kernel's and one row of
// the block per thread up to 256 rows.
template <int P, int NF, class TV>
__host__ __device__ constexpr int sweep_threads() {
  constexpr int nb = NF * (P + 1) * (P + 1) * (P + 1);
  constexpr int rows = ((nb < 256 ? nb : 256) + 31) / 32 * 32;
  constexpr int tf = tpf3d<P, TV>();
  return tf > rows ? tf : rows;
}

template <int P, int NF, class TV>
struct SweepSmem {
  static constexpr int NT = sweep_threads<P, NF, TV>();
  using F = SmemF<P, NF, kJvp, NT>;
  static constexpr int nb = NF * (P + 1) * (P + 1) * (P + 1);
  static constexpr size_t face_bytes = (size_t)F::total * sizeof(TV);
  static constexpr size_t t_off = (face_bytes + 15) / 16 * 16;   // t, in the accumulation type
  static constexpr size_t bytes = t_off + (size_t)nb * sizeof(double);
};

template <class TS, class TA, class TV, int NT>
__device__ __forceinline__ void sweep_gemv(const TS* __restrict__ B, const TA* ts, TV* zb, int n,
                                           int NN, long long EN, long long e) {
  for (int r = threadIdx.x; r < n; r += NT) {
    // sixteen independent partial sums keep sixteen loads per thread in flight:
    // a plane has few blocks per SM, and each streams its whole block inverse
    constexpr int K = 16;
    TA acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = TA(0);
    int c = 0;
    for (; c + K <= n; c += K) {
      TS bv[K];
#pragma unroll
      for (int q = 0; q < K; ++q) bv[q] = B[(long long)(c + q) * n + r];
#pragma unroll
      for (int q = 0; q < K; ++q) acc[q] += (TA)bv[q] * ts[c + q];
    }
    for (; c < n; ++c) acc[0] += (TA)B[(long long)c * n + r] * ts[c];
#pragma unroll
    for (int h = K / 2; h > 0; h /= 2)
#pragma unroll
      for (int q = 0; q < h; ++q) acc[q] += acc[q + h];
    const TA sum = acc[0];
    const int f = r / NN, i = r % NN;
    zb[f * EN + e * NN + i] = (TV)sum;
  }
}

// storage: 0 = FP64 inverses (accumulated in FP64), 1 = FP32, 2 = BF16 (both
// accumulated in FP32). z holds zeros on the planes not yet solved; upc is the
// linearisation point. dir = +1: flow along +e_a (planes 0, 1, ...), -1: along
// -e_a.
template <int P, int NF, class TV>
__global__ void __launch_bounds__(sweep_threads<P, NF, TV>())
sweep_fused_kernel(const OpParams prm, const void* __restrict__ binv, int storage,
                   const TV* __restrict__ x, TV* z, const TV* __restrict__ upc, int a, int k,
                   int dir, int upstream, int shared_blocks) {
  using SS = SweepSmem<P, NF, TV>;
  constexpr int NT = SS::NT;
  using S = typename SS::F;
  using TO = TabOff<P>;
  constexpr int N = S::N, NN = S::NN, NNP = S::NNP, NX = S::NX, FNP = S::FNP, NA = S::NA;
  constexpr int nb = SS::nb;
  extern __shared__ __align__(16) unsigned char sweep_raw[];
  TV* base = reinterpret_cast<TV*>(sweep_raw);
  const int tid = threadIdx.x;
  const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
  const int nb0 = prm.ne[b0];
  const int j0 = (int)(blockIdx.x % nb0), j1 = (int)(blockIdx.x / nb0);
  const int stride[3] = {1, prm.ne[0], prm.ne[0] * prm.ne[1]};
  const int sa = pick3(stride, a);
  const long long e = (long long)k * sa + (long long)j0 * pick3(stride, b0) +
                      (long long)j1 * pick3(stride, b1);
  const int b = blockIdx.y;
  const long long EN = (long long)prm.E * NN;
  const long long boff = (long long)b * prm.batch_stride;
  const long long blk = ((long long)(shared_blocks ? 0 : b) * prm.E + e) * (long long)nb * nb;
  {
    // the block inverse does not depend on the face terms: start moving it into
    // L2 now, so that the product below does not wait on HBM (blocks up to 64 KB:
    // a plane of larger ones exceeds L2, and their products stream from HBM)
    const size_t tsz = storage == 0 ? 8 : (storage == 1 ? 4 : 2);
    const char* p0 = reinterpret_cast<const char*>(binv) + blk * tsz;
    const size_t bytes = (size_t)nb * nb * tsz;
    if (bytes <= 65536) {
      for (size_t off = (size_t)tid * 128; off < bytes; off += (size_t)NT * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + off));
      if (tid == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(p0 + bytes - 1));
    }
  }
  // the face between e and its upstream neighbour: plane ia of direction a;
  // e is its upper element (side 1) when the flow runs along +e_a
  const int side = dir > 0 ? 1 : 0;
  const int ia = dir > 0 ? k : k + 1;
  if (upstream) {
    const long long eup = e - (long long)dir * sa;
    const long long eL = side == 1 ? eup : e, eU = side == 1 ? e : eup;
    const TV* vL = side == 1 ? z : nullptr;   // e's own tangent is zero
    const TV* vU = side == 1 ? nullptr : z;
    for (int i = tid; i < NN; i += NT) {
      const int pi = padded_node<N>(i);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const long long oL = boff + f * EN + eL * NN + i, oU = boff + f * EN + eU * NN + i;
        base[f * NNP + pi] = upc[oL];
        base[(NA + f) * NNP + pi] = upc[oU];
        base[(NF + f) * NNP + pi] = vL ? vL[oL] : TV(0);
        base[(NA + NF + f) * NNP + pi] = vU ? vU[oU] : TV(0);
      }
    }
    __syncthreads();
    face3d_stages<P, NF, kJvp, TV, NT>(prm, base, tid, NT, a, ia, j0, j1, b);
  }
  const TV* G2 = face3d_g2<P, NF, kJvp, TV, NT>(base);
  const int lay = side == 1 ? 0 : N - 1;
  const int dlo = TO::dL + (side == 1 ? 0 : N);
  auto fill_t = [&](auto* ts) {
    using TA = typename std::remove_pointer<decltype(ts)>::type;
    for (int c = tid; c < nb; c += NT) {
      const int f = c / NN, i = c % NN;
      TA t = (TA)x[boff + f * EN + e * NN + i];
      if (upstream) {
        const int c3[3] = {i % N, (i / N) % N, i / (N * N)};
        const int ka = pick3(c3, a);
        const int jb0 = pick3(c3, b0), jb1 = pick3(c3, b1);
        const int jp = jb0 + NX * jb1;
        const TA sv = (TA)G2[((side * 2 + 0) * NF + f) * FNP + jp];
        const TA tv = (TA)G2[((side * 2 + 1) * NF + f) * FNP + jp];
        TA add = (TA)ctab<P, TV>(dlo + ka) * tv;
        if (ka == lay) add += sv;
        t -= add;
      }
      ts[c] = t;
    }
  };
  TV* zb = z + boff;
  if (storage == 0) {
    double* ts = reinterpret_cast<double*>(sweep_raw + SS::t_off);
    fill_t(ts);
    __syncthreads();
    sweep_gemv<double, double, TV, NT>(reinterpret_cast<const double*>(binv) + blk, ts, zb, nb, NN,
                                       EN, e);
  } else {
    float* ts = reinterpret_cast<float*>(sweep_raw + SS::t_off);
    fill_t(ts);
    __syncthreads();
    if (storage == 1)
      sweep_gemv<float, float, TV, NT>(reinterpret_cast<const float*>(binv) + blk, ts, zb, nb, NN,
                                       EN, e);
    else
      sweep_gemv<__nv_bfloat16, float, TV, NT>(reinterpret_cast<const __nv_bfloat16*>(binv) + blk,
                                               ts, zb, nb, NN, EN, e);
  }
}

}  // namespace enp
