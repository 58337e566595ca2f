// Run-time dispatch from (dim, p, fields, mode) to a compiled operator kernel.
// For kBlockCol, `batch` is the number of block columns (NF * Np): grid.y runs
// over the columns.
#pragma once
#include <mutex>

#include "enp_internal.h"
#include "enp_operator.cuh"
#include "enp_operator3d.cuh"
#include "enp_blockcols.cuh"
#include "enp_sweep.cuh"

namespace enp {

// The dynamic shared-memory limit of a kernel is a per-device attribute: each
// launch site keeps, per device, whether it has raised the limit (thread-safe).
struct SmemAttr {
  std::mutex mu;
  bool done[64] = {};
};
template <class K>
static cudaError_t raise_smem_limit(SmemAttr& st, K kern, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  std::lock_guard<std::mutex> g(st.mu);
  if (st.done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  // shared memory, not L1, bounds the resident blocks of these kernels
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) st.done[dev] = true;
  return e;
}

// Elements per block of the hexahedral kernel, per (p, fields, mode) and
// arithmetic type; 0 = the default (shared memory near 96 KB). One table per
// type for the whole library (the double-float kernels span several
// translation units).
template <class R>
inline int (&eb3d_table())[kMaxP + 1][4][5] {
  static int t[kMaxP + 1][4][5] = {};
  return t;
}
// Faces per block of the face kernel (modes R, J v, J^T w), the same way.
template <class R>
inline int (&fpb3d_table())[kMaxP + 1][4][3] {
  static int t[kMaxP + 1][4][3] = {};
  return t;
}

template <int P, int NF, int MODE, class R>
static constexpr size_t face_bytes() {
  return (size_t)SmemF<P, NF, MODE, tpf3d<P, R>()>::total * sizeof(R);
}
// The default faces per block (shared memory near 96 KB) and the largest
// feasible value (threads <= kMaxThreads3D, shared memory <= 200 KB).
template <int P, int NF, int MODE, class R>
static int default_fpb() {
  constexpr int TF = tpf3d<P, R>();
  int f = (int)((96 * 1024) / face_bytes<P, NF, MODE, R>());
  f = f < 1 ? 1 : f;
  if (f * TF > kMaxThreads3D) f = kMaxThreads3D / TF;
  return f < 1 ? 1 : f;
}
template <int P, int NF, int MODE, class R>
static int max_fpb() {
  constexpr int TF = tpf3d<P, R>();
  int f = kMaxThreads3D / TF;
  while (f > 1 && (size_t)f * face_bytes<P, NF, MODE, R>() > 200 * 1024) --f;
  return f < 1 ? 1 : f;
}

template <int P, int NF, int MODE, class R>
static int default_eb() {
  constexpr int NT = tpe3d<P, R>();
  constexpr size_t per_el = (size_t)Smem3<P, NF, MODE, NT>::total * sizeof(R);
  int eb = (int)((96 * 1024) / per_el);
  eb = eb < 1 ? 1 : eb;
  while (eb > 1 && eb * NT > kMaxThreads3D) --eb;
  return eb;
}

template <int P, int NF, int MODE, class R>
static int max_eb() {
  constexpr int NT = tpe3d<P, R>();
  constexpr size_t per_el = (size_t)Smem3<P, NF, MODE, NT>::total * sizeof(R);
  int eb = kMaxThreads3D / NT;
  while (eb > 1 && (size_t)eb * per_el > 200 * 1024) --eb;
  return eb < 1 ? 1 : eb;
}

// Columns of the element-diagonal blocks per (element, chunk of kBlockChunk
// columns), the state's point values and face traces formed once per chunk.
constexpr int kBlockChunk = 16;
template <int P, int NF, class R>
static cudaError_t launch_blockcols(const OpParams& prm, const io_t<R>* u, io_t<R>* out,
                                    cudaStream_t stream) {
  constexpr int NT = tpe3d<P, R>();
  constexpr size_t smem = (size_t)SmemB<P, NF, NT, kBlockChunk>::total * sizeof(R);
  static_assert(smem <= 200 * 1024, "block-column kernel shared memory");
  auto k = blockcol3d_kernel<P, NF, kBlockChunk, R>;
  static SmemAttr attr;
  cudaError_t e = raise_smem_limit(attr, k, smem);
  if (e != cudaSuccess) return e;
  constexpr int nb = NF * (P + 1) * (P + 1) * (P + 1);
  const dim3 grid((unsigned)prm.E, (nb + kBlockChunk - 1) / kBlockChunk);
  k<<<grid, NT, smem, stream>>>(prm, u, out);
  return cudaGetLastError();
}

template <int P, int NF, int MODE, class R>
static cudaError_t launch_3d_op(const OpParams& prm, const io_t<R>* u, const io_t<R>* v,
                                io_t<R>* out, int batch, cudaStream_t stream);

// Hexahedra: the thread-per-pencil kernel with EB elements per block (the FP32
// block columns: blockcol3d_kernel).
template <int P, int NF, int MODE, class R>
static cudaError_t launch_3d(const OpParams& prm, const io_t<R>* u, const io_t<R>* v, io_t<R>* out,
                             int batch, cudaStream_t stream) {
  if constexpr (MODE == kBlockCol) {
    (void)v;
    (void)batch;  // the nb columns
    return launch_blockcols<P, NF, R>(prm, u, out, stream);
  } else {
    return launch_3d_op<P, NF, MODE, R>(prm, u, v, out, batch, stream);
  }
}

template <int P, int NF, int MODE, class R>
static cudaError_t launch_3d_op(const OpParams& prm, const io_t<R>* u, const io_t<R>* v,
                                io_t<R>* out, int batch, cudaStream_t stream) {
  constexpr int NT = tpe3d<P, R>();
  using S3 = Smem3<P, NF, MODE, NT>;
  constexpr size_t per_el = (size_t)S3::total * sizeof(R);
  int eb = eb3d_table<R>()[P][NF][MODE];
  if (eb <= 0) eb = default_eb<P, NF, MODE, R>();
  const size_t smem = (size_t)eb * per_el;
  auto kern = op3d_kernel<P, NF, MODE, R>;
  static SmemAttr attr;
  cudaError_t ea = raise_smem_limit(attr, kern, (size_t)max_eb<P, NF, MODE, R>() * per_el);
  if (ea != cudaSuccess) return ea;
  if constexpr (S3::kFB) {
    // the faces first: each face once, both sides' terms into the face buffer
    constexpr int TF = tpf3d<P, R>();
    constexpr size_t per_face = face_bytes<P, NF, MODE, R>();
    int fpb = fpb3d_table<R>()[P][NF][MODE];
    if (fpb <= 0) fpb = default_fpb<P, NF, MODE, R>();
    auto fk = face3d_kernel<P, NF, MODE, R>;
    static SmemAttr fattr;
    cudaError_t ef = raise_smem_limit(fattr, fk, (size_t)max_fpb<P, NF, MODE, R>() * per_face);
    if (ef != cudaSuccess) return ef;
    const long long nf = prm.foff[3];
    dim3 fgrid((unsigned)((nf + fpb - 1) / fpb), batch);
    fk<<<fgrid, fpb * TF, fpb * per_face, stream>>>(prm, u, v);
  }
  dim3 grid((prm.E + eb - 1) / eb, batch);
  kern<<<grid, eb * NT, smem, stream>>>(prm, u, v, out);
  return cudaGetLastError();
}

template <int DIM, int P, int NF, int MODE, class R>
static cudaError_t launch_one(const OpParams& prm, const Tables* tabs, const io_t<R>* u,
                              const io_t<R>* v, io_t<R>* out, int batch, cudaStream_t stream) {
  if constexpr (DIM == 3) {
    (void)tabs;
    return launch_3d<P, NF, MODE, R>(prm, u, v, out, batch, stream);
  } else {
  using M = WarpSmem<DIM, P, NF, MODE>;
  constexpr size_t per_warp = (size_t)M::total * sizeof(R);
  constexpr int WPB = per_warp * 4 <= 96 * 1024 ? 4 : (per_warp * 2 <= 110 * 1024 ? 2 : 1);
  const size_t smem = ((size_t)TabSmem<P>::total + (size_t)WPB * M::total) * sizeof(R);
  auto kern = op_kernel<DIM, P, NF, MODE, WPB, R>;
  static SmemAttr attr;
  cudaError_t ea = raise_smem_limit(attr, kern, smem);
  if (ea != cudaSuccess) return ea;
  dim3 grid((prm.E + WPB - 1) / WPB, batch);
  kern<<<grid, WPB * 32, smem, stream>>>(prm, tabs, u, v, out);
  return cudaGetLastError();
  }
}

template <int DIM, int P, int NF, class R>
static cudaError_t launch_mode(int mode, const OpParams& prm, const Tables* t, const io_t<R>* u,
                               const io_t<R>* v, io_t<R>* out, int batch, cudaStream_t s) {
  if constexpr (std::is_same<R, df>::value) {
    // double-float: the residual, J v, J^T w and block columns (dR/dtheta
    // stays with the FP64 kernels)
    switch (mode) {
      case kResidual: return launch_one<DIM, P, NF, kResidual, R>(prm, t, u, v, out, batch, s);
      case kJvp: return launch_one<DIM, P, NF, kJvp, R>(prm, t, u, v, out, batch, s);
      case kVjp: return launch_one<DIM, P, NF, kVjp, R>(prm, t, u, v, out, batch, s);
      case kBlockCol: return launch_one<DIM, P, NF, kBlockCol, R>(prm, t, u, v, out, batch, s);
    }
    return cudaErrorNotSupported;
  } else {
    switch (mode) {
      case kResidual: return launch_one<DIM, P, NF, kResidual, R>(prm, t, u, v, out, batch, s);
      case kJvp: return launch_one<DIM, P, NF, kJvp, R>(prm, t, u, v, out, batch, s);
      case kVjp: return launch_one<DIM, P, NF, kVjp, R>(prm, t, u, v, out, batch, s);
      case kBlockCol: return launch_one<DIM, P, NF, kBlockCol, R>(prm, t, u, v, out, batch, s);
      case kParam:
        if constexpr (DIM == 3) return launch_one<DIM, P, NF, kParam, R>(prm, t, u, v, out, batch, s);
        return cudaErrorNotSupported;
    }
    return cudaErrorInvalidValue;
  }
}

template <int DIM, int P, class R>
static cudaError_t launch_nf(int mode, const OpParams& prm, const Tables* t, const io_t<R>* u,
                             const io_t<R>* v, io_t<R>* out, int batch, cudaStream_t s) {
  if (prm.NF == 2) return launch_mode<DIM, P, 2, R>(mode, prm, t, u, v, out, batch, s);
  if (prm.NF == 3) return launch_mode<DIM, P, 3, R>(mode, prm, t, u, v, out, batch, s);
  return cudaErrorInvalidConfiguration;
}

// One plane of the downwind block Gauss-Seidel sweep (sweep_fused_kernel).
template <int P, int NF, class TV>
static cudaError_t launch_sweep_pn(const OpParams& prm, const void* binv, int storage, const TV* x,
                                   TV* z, const TV* upc, int batch, cudaStream_t stream, int a,
                                   int k, int dir, int upstream, int shared_blocks) {
  using SS = SweepSmem<P, NF, TV>;
  auto kern = sweep_fused_kernel<P, NF, TV>;
  static SmemAttr attr;
  cudaError_t e = raise_smem_limit(attr, kern, SS::bytes);
  if (e != cudaSuccess) return e;
  const int nplane = prm.ne[a == 0 ? 1 : 0] * prm.ne[a == 2 ? 1 : 2];
  const dim3 grid((unsigned)nplane, (unsigned)batch);
  kern<<<grid, SS::NT, SS::bytes, stream>>>(prm, binv, storage, x, z, upc, a, k, dir, upstream,
                                            shared_blocks);
  return cudaGetLastError();
}

template <class TV>
cudaError_t launch_sweep_plane(const OpParams& prm, const void* binv, int storage, const TV* x,
                               TV* z, const TV* upc, int batch, cudaStream_t s, int a, int k,
                               int dir, int upstream, int shared_blocks) {
  if (prm.dim != 3 || storage < 0 || storage > 2 || (dir != 1 && dir != -1))
    return cudaErrorInvalidConfiguration;
#define ENP_SW(PP)                                                                              \
  case PP:                                                                                      \
    if (prm.NF == 2)                                                                            \
      return launch_sweep_pn<PP, 2, TV>(prm, binv, storage, x, z, upc, batch, s, a, k, dir,     \
                                        upstream, shared_blocks);                               \
    if (prm.NF == 3)                                                                            \
      return launch_sweep_pn<PP, 3, TV>(prm, binv, storage, x, z, upc, batch, s, a, k, dir,     \
                                        upstream, shared_blocks);                               \
    return cudaErrorInvalidConfiguration;
  switch (prm.p) { ENP_SW(1) ENP_SW(2) ENP_SW(3) ENP_SW(4) }
#undef ENP_SW
  return cudaErrorInvalidConfiguration;
}

// Elements-per-block of the hexahedral kernel: the largest feasible value for
// (p, fields, mode), and setting the value launches use (0 = default).
template <class R>
int eb3d_max(int p, int nf, int mode) {
#define ENP_EBM(PP, NFF, MM) \
  if (p == PP && nf == NFF && mode == MM && (MM != kParam || !std::is_same<R, df>::value)) return max_eb<PP, NFF, MM, R>();
#define ENP_EBM_P(PP) ENP_EBM(PP, 2, 0) ENP_EBM(PP, 2, 1) ENP_EBM(PP, 2, 2) ENP_EBM(PP, 2, 3) ENP_EBM(PP, 2, 4) \
  ENP_EBM(PP, 3, 0) ENP_EBM(PP, 3, 1) ENP_EBM(PP, 3, 2) ENP_EBM(PP, 3, 3) ENP_EBM(PP, 3, 4)
  ENP_EBM_P(1) ENP_EBM_P(2) ENP_EBM_P(3) ENP_EBM_P(4)
#undef ENP_EBM_P
#undef ENP_EBM
  return 1;
}

// Faces per block of the face kernel (modes 0..2), as above.
template <class R>
int fpb3d_max(int p, int nf, int mode) {
#define ENP_FBM(PP, NFF, MM) if (p == PP && nf == NFF && mode == MM) return max_fpb<PP, NFF, MM, R>();
#define ENP_FBM_P(PP) ENP_FBM(PP, 2, 0) ENP_FBM(PP, 2, 1) ENP_FBM(PP, 2, 2) \
  ENP_FBM(PP, 3, 0) ENP_FBM(PP, 3, 1) ENP_FBM(PP, 3, 2)
  ENP_FBM_P(1) ENP_FBM_P(2) ENP_FBM_P(3) ENP_FBM_P(4)
#undef ENP_FBM_P
#undef ENP_FBM
  return 1;
}

template <class R>
void fpb3d_set(int p, int nf, int mode, int fpb) {
  if (p >= 1 && p <= kMaxP && nf >= 2 && nf <= 3 && mode >= 0 && mode <= 2) fpb3d_table<R>()[p][nf][mode] = fpb;
}

template <class R>
int fpb3d_get(int p, int nf, int mode) {
  if (p >= 1 && p <= kMaxP && nf >= 2 && nf <= 3 && mode >= 0 && mode <= 2) return fpb3d_table<R>()[p][nf][mode];
  return 0;
}

template <class R>
void eb3d_set(int p, int nf, int mode, int eb) {
  if (p >= 1 && p <= kMaxP && nf >= 2 && nf <= 3 && mode >= 0 && mode <= 4) eb3d_table<R>()[p][nf][mode] = eb;
}

template <class R>
int eb3d_get(int p, int nf, int mode) {
  if (p >= 1 && p <= kMaxP && nf >= 2 && nf <= 3 && mode >= 0 && mode <= 4) return eb3d_table<R>()[p][nf][mode];
  return 0;
}

// Upload the degree-p tables to this translation unit's constant memory on
// the current device (idempotent: the tables depend on p only).
template <class R>
cudaError_t prepare_tables(int p, const Tables& t) {
  return upload_const_tables(p, t);
}

template <class R>
cudaError_t launch_op(int mode, const OpParams& prm, const Tables* t, const io_t<R>* u,
                      const io_t<R>* v, io_t<R>* out, int batch, cudaStream_t s) {
  if constexpr (std::is_same<R, double>::value) {
    // R, J v, J^T w and block columns in double-float arithmetic on hexahedra
    if (prm.arith == kArithDF && prm.dim == 3 && mode != kParam)
      return launch_op_df(mode, prm, u, v, out, batch, s);
  }
  if (prm.dim == 3) {
    switch (prm.p) {
      case 1: return launch_nf<3, 1, R>(mode, prm, t, u, v, out, batch, s);
      case 2: return launch_nf<3, 2, R>(mode, prm, t, u, v, out, batch, s);
      case 3: return launch_nf<3, 3, R>(mode, prm, t, u, v, out, batch, s);
      case 4: return launch_nf<3, 4, R>(mode, prm, t, u, v, out, batch, s);
    }
  }
  if (prm.dim == 2) {
    switch (prm.p) {
      case 1: return launch_nf<2, 1, R>(mode, prm, t, u, v, out, batch, s);
      case 2: return launch_nf<2, 2, R>(mode, prm, t, u, v, out, batch, s);
      case 3: return launch_nf<2, 3, R>(mode, prm, t, u, v, out, batch, s);
    }
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace enp

// The double-float hexahedral kernels of one degree PP (op_df_pPP.cu): the
// launcher and the upload of that translation unit's constant tables.
#define ENP_DF_DEGREE(PP)                                                                    \
  cudaError_t enp::launch_df_p##PP(int mode, const OpParams& prm, const double* u,             \
                                   const double* v, double* out, int batch, cudaStream_t s) { \
    if (prm.dim != 3) return cudaErrorInvalidConfiguration;                                   \
    return launch_nf<3, PP, df>(mode, prm, nullptr, u, v, out, batch, s);                     \
  }                                                                                           \
  cudaError_t enp::upload_tables_df_p##PP(const Tables& t) { return upload_const_tables(PP, t); }
