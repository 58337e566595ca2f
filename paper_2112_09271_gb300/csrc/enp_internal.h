// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include "enp_common.cuh"

namespace enp {

// Launch the operator kernel for (dim, p, NF) chosen at run time.
// mode: 0 residual, 1 J v, 2 J^T w. Returns cudaErrorInvalidConfiguration if the
// shape is not compiled.
// R = double, float or df (double-float arithmetic on FP64 vectors: io_t<df> =
// double). With prm.arith == kArithDF, launch_op<double> on hexahedra runs the
// double-float kernels.
template <class R>
cudaError_t launch_op(int mode, const OpParams& prm, const Tables* tabs, const io_t<R>* u,
                      const io_t<R>* v, io_t<R>* out, int batch, cudaStream_t stream);

// The double-float hexahedral operator: R, J v, J^T w and block columns of
// degree prm.p (op_df.cu), compiled one degree per translation unit
// (op_df_p1.cu .. op_df_p4.cu), each with its own constant tables.
cudaError_t launch_op_df(int mode, const OpParams& prm, const double* u, const double* v,
                         double* out, int batch, cudaStream_t stream);
cudaError_t prepare_tables_df(int p, const Tables& t);
#define ENP_DF_DECL(PP)                                                                      \
  cudaError_t launch_df_p##PP(int mode, const OpParams& prm, const double* u, const double* v, \
                              double* out, int batch, cudaStream_t s);                        \
  cudaError_t upload_tables_df_p##PP(const Tables& t);
ENP_DF_DECL(1)
ENP_DF_DECL(2)
ENP_DF_DECL(3)
ENP_DF_DECL(4)
#undef ENP_DF_DECL

bool shape_supported(int dim, int p, int nf);

// Elements per block of the hexahedral kernel (autotuner hooks).
template <class R> int eb3d_max(int p, int nf, int mode);
template <class R> void eb3d_set(int p, int nf, int mode, int eb);
template <class R> int eb3d_get(int p, int nf, int mode);
// Faces per block of the hexahedral face kernel (modes 0..2).
template <class R> int fpb3d_max(int p, int nf, int mode);
template <class R> void fpb3d_set(int p, int nf, int mode, int fpb);
template <class R> int fpb3d_get(int p, int nf, int mode);

// Upload the degree-p basis tables to the constant memory the kernels of type R
// read (current device).
template <class R>
cudaError_t prepare_tables(int p, const Tables& t);

// One element plane k (along axis a, flow direction dir = +-1) of the downwind
// block Gauss-Seidel sweep for every operating point: z_e = Binv_e (x_e -
// J_(e,up) z_up), the upstream face term evaluated in the same launch
// (upstream = 0 for the first plane). binv: the transposed block inverses in
// `storage` (0 FP64, 1 FP32, 2 BF16), one set per point or one shared set;
// upc: the linearisation point (hexahedra).
template <class TV>
cudaError_t launch_sweep_plane(const OpParams& prm, const void* binv, int storage, const TV* x,
                               TV* z, const TV* upc, int batch, cudaStream_t s, int a, int k,
                               int dir, int upstream, int shared_blocks);

}  // namespace enp

struct enp_solver_ext;
void enp_solver_free(struct enp_dg* h);

struct enp_dg {
  enp::OpParams prm{};
  enp::Tables htab{};
  enp::Tables* d_tab = nullptr;
  double* d_xv[3] = {nullptr, nullptr, nullptr};
  float* d_xvf[3] = {nullptr, nullptr, nullptr};
  float2* d_xvdf[3] = {nullptr, nullptr, nullptr};
  uint8_t* d_btag = nullptr;
  double* d_src = nullptr;
  double* d_dir = nullptr;
  double* d_phiapp = nullptr;
  void* d_fbuf = nullptr;        // face coefficients of the hexahedral operator
  int batch = 1;
  long long n_dof = 0;           // per operating point
  cudaStream_t stream = nullptr;
  std::string err;
  enp_solver_ext* solver = nullptr;   // block-Jacobi, Krylov and reduction workspace
};
