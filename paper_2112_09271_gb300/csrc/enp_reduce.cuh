// Device reductions shared by the solver and the allocation-free inner
// product: fixed-order dot products (a grid-stride loop per thread, a shuffle
// tree per warp, one partial per thread block, then one block per result), so
// that a result depends on the vector length only, not on timing or batch.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace enp {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 608;  // 4 blocks per SM on 152 SMs; partials per dot product

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// W consecutive values of a vector as one 16-byte load (W = 16 / sizeof(T)),
// or one value (W = 1).
template <class T, int W>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&a)[W]) {
  if constexpr (W == 1) {
    a[0] = p[0];
  } else if constexpr (sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    a[0] = t.x; a[1] = t.y;
  }
}

template <class T, int W>
__device__ __forceinline__ void store_vec(T* __restrict__ p, const T (&a)[W]) {
  if constexpr (W == 1) {
    p[0] = a[0];
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(a[0], a[1]);
  }
}

// Transposed butterfly: from v[0..7] on every lane, lane l ends with the sum
// over the warp's 32 lanes of v[l & 7] (9 shuffles instead of 8 x 5), in a
// fixed order.
template <class T>
__device__ __forceinline__ T warp_reduce8(T (&v)[8], int lane) {
  constexpr unsigned kAll = 0xffffffffu;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 4;
    const T send = up ? v[i] : v[i + 4];
    const T keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(kAll, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 2;
    const T send = up ? v[i] : v[i + 2];
    const T keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(kAll, send, 2);
  }
  {
    const bool up = lane & 1;
    const T send = up ? v[0] : v[1];
    const T keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(kAll, send, 1);
  }
  T r = v[0];
  r += __shfl_xor_sync(kAll, r, 8);
  r += __shfl_xor_sync(kAll, r, 16);
  return r;
}

// Partial sums of nd dot products <V_i, w> (i < nd) over each batch item:
// part[b][i][block]. V_i = V + i * vstride. The vectors are taken in groups of
// kDotGroup with one accumulator each per thread (few registers), W
// consecutive entries per 16-byte load; each thread runs over its units by
// grid stride, accumulating in the vector's own precision (FP32 vectors: FP32,
// no conversions on the FP64 pipe); the warp tree runs in that precision, the
// block and grid sums in FP64. Fixed reduction order for a given grid.
constexpr int kDotGroup = 8;

template <class T, int W>
__global__ void __launch_bounds__(kRedThreads)
multidot_partial(const T* __restrict__ V, long long vstride, int nd, const T* __restrict__ w,
                 long long n, long long bstride, double* __restrict__ part) {
  __shared__ double red[kRedThreads / 32][kDotGroup];
  const int b = blockIdx.y;
  const T* wb = w + b * bstride;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nu = n / W;
  for (int i0 = 0; i0 < nd; i0 += kDotGroup) {
    const int ni = min(kDotGroup, nd - i0);
    const T* V0 = V + i0 * vstride + b * bstride;
    T acc[kDotGroup];
#pragma unroll
    for (int i = 0; i < kDotGroup; ++i) acc[i] = T(0);
    for (long long u = blockIdx.x * (long long)kRedThreads + threadIdx.x; u < nu;
         u += (long long)gridDim.x * kRedThreads) {
      T wv[W];
      load_vec<T, W>(wb + u * W, wv);
#pragma unroll
      for (int i = 0; i < kDotGroup; ++i)
        if (i < ni) {
          T vv[W];
          load_vec<T, W>(V0 + i * vstride + u * W, vv);
#pragma unroll
          for (int c = 0; c < W; ++c) acc[i] += vv[c] * wv[c];
        }
    }
    const T r = warp_reduce8<T>(acc, lane);
    if (lane < kDotGroup) red[warp][lane] = (double)r;
    __syncthreads();
    if (threadIdx.x < ni) {
      double s = 0.0;
      for (int wv = 0; wv < kRedThreads / 32; ++wv) s += red[wv][threadIdx.x];
      part[((long long)b * nd + i0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// out[b][i] = sum over blocks of part[b][i][:], in block order.
static __global__ void finish_partials(const double* __restrict__ part, int nparts, int count,
                                double* __restrict__ out) {
  const int i = blockIdx.x;  // one block per (b, i)
  if (i >= count) return;
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += 32) s += part[(long long)i * nparts + k];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[i] = s;
}

}  // namespace enp

// Entries per 16-byte load usable on these vectors: every vector start (base
// pointers and the strides between vectors and operating points) 16-byte aligned.
template <class T>
inline int vec_width(long long n, long long vstride, const void* a, const void* b) {
  constexpr int W = 16 / sizeof(T);
  const bool ok = n % W == 0 && vstride % W == 0 &&
                  reinterpret_cast<uintptr_t>(a) % 16 == 0 && reinterpret_cast<uintptr_t>(b) % 16 == 0;
  return ok ? W : 1;
}

// Blocks of a reduction over n entries in units of W: about two units per
// thread, at most kRedBlocks. Depends on n only (not on the batch), so a point
// of a batch is reduced exactly as it is alone.
inline int red_blocks(long long n, int W) {
  const long long nu = n / W;
  const long long g = (nu + 2LL * enp::kRedThreads - 1) / (2LL * enp::kRedThreads);
  return (int)std::max(1LL, std::min<long long>(g, enp::kRedBlocks));
}
