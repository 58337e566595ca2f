// Entry of the double-float hexahedral operator: R(u), J(u)v, J(u)^T w and block columns with
// FP64 vectors in and out and double-float arithmetic on the FP32 pipe (the
// FP64-accurate operator). The kernels of each degree live in op_df_p<p>.cu.
#include "enp_op_dispatch.cuh"

cudaError_t enp::launch_op_df(int mode, const OpParams& prm, const double* u, const double* v,
                              double* out, int batch, cudaStream_t stream) {
  switch (prm.p) {
    case 1: return launch_df_p1(mode, prm, u, v, out, batch, stream);
    case 2: return launch_df_p2(mode, prm, u, v, out, batch, stream);
    case 3: return launch_df_p3(mode, prm, u, v, out, batch, stream);
    case 4: return launch_df_p4(mode, prm, u, v, out, batch, stream);
  }
  return cudaErrorInvalidConfiguration;
}

cudaError_t enp::prepare_tables_df(int p, const Tables& t) {
  switch (p) {
    case 1: return upload_tables_df_p1(t);
    case 2: return upload_tables_df_p2(t);
    case 3: return upload_tables_df_p3(t);
    case 4: return upload_tables_df_p4(t);
  }
  return cudaErrorInvalidConfiguration;
}

// Launch-shape hooks of the autotuner (shape arithmetic only, no kernels here).
template int enp::eb3d_max<enp::df>(int, int, int);
template void enp::eb3d_set<enp::df>(int, int, int, int);
template int enp::eb3d_get<enp::df>(int, int, int);
template int enp::fpb3d_max<enp::df>(int, int, int);
template void enp::fpb3d_set<enp::df>(int, int, int, int);
template int enp::fpb3d_get<enp::df>(int, int, int);
