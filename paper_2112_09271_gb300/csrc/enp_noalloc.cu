// Inner products without any device allocation.
//
// enp_inner_product keeps its per-block partial sums in scratch memory that
// the handle allocates with cudaMalloc. Some callers cannot allocate: a host
// application that owns all device memory through its own pool and forbids
// other allocations, or a latency-critical loop that cannot afford cudaMalloc's
// cost and implicit device synchronisation. For them, enp_inner_product_noalloc
// computes the same reduction with the partial sums in the fixed array below,
// which lives in the library's static device memory: every GPU that loads the
// library holds it (ENP_NOALLOC_MAX_BATCH x 608 doubles) until the process exits.
//
// Host code must not pass `g_noalloc_partials` itself to a kernel: in host code
// that name is a host-side stand-in, not a device address. The device address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current) and passed to the kernel.
#include <mutex>

#include "../../include/enp_dg.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 608;  // 4 blocks per SM on 152 SMs: partials per operating point
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[ENP_NOALLOC_MAX_BATCH * kBlocks];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One partial sum of <x_b, y_b> per thread block, in a fixed order: a
// grid-stride loop per thread, a shuffle tree per warp, then the warps in order.
// Every slot read later by the finishing kernel is written here first, so the
// array needs no clearing between calls.
__global__ void __launch_bounds__(kThreads)
dot_partial_noalloc(const double* __restrict__ x, const double* __restrict__ y, long long n,
                    double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  const int b = blockIdx.y;
  const double* xb = x + (long long)b * n;
  const double* yb = y + (long long)b * n;
  double acc = 0.0;
  for (long long k = blockIdx.x * (long long)kThreads + threadIdx.x; k < n;
       k += (long long)gridDim.x * kThreads)
    acc += xb[k] * yb[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    part[(long long)b * gridDim.x + blockIdx.x] = s;
  }
}

// out[b] = sum of the partials of operating point b, in block order.
__global__ void dot_finish_noalloc(const double* __restrict__ part, int nparts,
                                   double* __restrict__ out) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += 32) s += part[(long long)b * nparts + k];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[b] = s;
}

std::mutex g_mutex;
double* g_ptr[kMaxDevices] = {nullptr};

// Device address of the partials array on the current device, looked up on
// the first call on that device and cached.
enp_status scratch_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return ENP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return ENP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return ENP_ERR_CUDA;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return ENP_OK;
}

}  // namespace

extern "C" enp_status enp_inner_product_noalloc(const double* x, const double* y, long long n,
                                                int batch, double* out, void* stream) {
  if (!x || !y || !out || n < 0 || batch < 1) return ENP_ERR_INVALID_ARG;
  if (batch > ENP_NOALLOC_MAX_BATCH) return ENP_ERR_INVALID_ARG;  // more than the array holds
  double* part = nullptr;
  enp_status st = scratch_on_current_device(&part);
  if (st != ENP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dot_partial_noalloc<<<dim3(kBlocks, batch), kThreads, 0, s>>>(x, y, n, part);
  dot_finish_noalloc<<<batch, 32, 0, s>>>(part, kBlocks, out);
  return cudaGetLastError() == cudaSuccess ? ENP_OK : ENP_ERR_CUDA;
}
