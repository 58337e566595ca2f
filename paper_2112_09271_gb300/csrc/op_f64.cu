// FP64 instantiations of the operator kernel: R(u), J(u)v and J(u)^T w.
#include "enp_op_dispatch.cuh"
template cudaError_t enp::launch_op<double>(int, const OpParams&, const Tables*, const double*,
                                            const double*, double*, int, cudaStream_t);
template cudaError_t enp::prepare_tables<double>(int, const Tables&);
template int enp::eb3d_max<double>(int, int, int);
template void enp::eb3d_set<double>(int, int, int, int);
template int enp::eb3d_get<double>(int, int, int);
template int enp::fpb3d_max<double>(int, int, int);
template void enp::fpb3d_set<double>(int, int, int, int);
template int enp::fpb3d_get<double>(int, int, int);
template cudaError_t enp::launch_sweep_plane<double>(const OpParams&, const void*, int, const double*,
                                                  double*, const double*, int, cudaStream_t, int, int,
                                                  int, int, int);
