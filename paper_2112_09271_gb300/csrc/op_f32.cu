// FP32 instantiations of the operator kernel (inner Krylov operator of the
// mixed-precision solve).
#include "enp_op_dispatch.cuh"
template cudaError_t enp::launch_op<float>(int, const OpParams&, const Tables*, const float*,
                                           const float*, float*, int, cudaStream_t);
template cudaError_t enp::prepare_tables<float>(int, const Tables&);
template int enp::eb3d_max<float>(int, int, int);
template void enp::eb3d_set<float>(int, int, int, int);
template int enp::eb3d_get<float>(int, int, int);
template int enp::fpb3d_max<float>(int, int, int);
template void enp::fpb3d_set<float>(int, int, int, int);
template int enp::fpb3d_get<float>(int, int, int);
template cudaError_t enp::launch_sweep_plane<float>(const OpParams&, const void*, int, const float*,
                                                  float*, const float*, int, cudaStream_t, int, int,
                                                  int, int, int);
