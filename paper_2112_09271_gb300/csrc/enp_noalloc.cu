// Inner products without any device allocation.
//
// enp_inner_product keeps its per-block partial sums in scratch memory that
// the handle allocates with cudaMalloc. Some callers cannot allocate: a host
// application that owns all device memory through its own pool and forbids
// other allocations, or a latency-critical loop that cannot afford cudaMalloc's
// cost and implicit device synchronisation. For them, enp_inner_product_noalloc
// computes the same reduction (same kernels, grid and summation order, hence
// the same bits) with the partial sums in the fixed array below, which lives in
// the library's static device memory: every GPU that loads the library holds
// it (ENP_NOALLOC_MAX_BATCH x 608 doubles) until the process exits.
//
// Host code must not pass `g_noalloc_partials` itself to a kernel: in host code
// that name is a host-side stand-in, not a device address. The device address
// is looked up once per device with cudaGetSymbolAddress (with that device
// current) and passed to the kernel.
#include <mutex>

#include "../../include/enp_dg.h"
#include "enp_reduce.cuh"

namespace {

constexpr int kMaxDevices = 64;

// One partial per reduction block and operating point: the same reduction
// (kernels, grid and order) as enp_inner_product, whose partials live in
// handle-owned scratch.
static __device__ __align__(256) double g_noalloc_partials[ENP_NOALLOC_MAX_BATCH * enp::kRedBlocks];

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
  // every partial slot the finishing kernel reads is written first by the
  // partial kernel of the same call: the array needs no clearing
  const int W = vec_width<double>(n, 0, x, y);
  const int nb = red_blocks(n, W);
  const dim3 g(nb, batch);
  if (W == 1)
    enp::multidot_partial<double, 1><<<g, enp::kRedThreads, 0, s>>>(x, 0, 1, y, n, n, part);
  else
    enp::multidot_partial<double, 2><<<g, enp::kRedThreads, 0, s>>>(x, 0, 1, y, n, n, part);
  enp::finish_partials<<<batch, 32, 0, s>>>(part, nb, batch, out);
  return cudaGetLastError() == cudaSuccess ? ENP_OK : ENP_ERR_CUDA;
}
