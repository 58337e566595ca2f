// Element block-Jacobi preconditioner, Krylov and Newton solvers, c_m recovery.
//
//  * block setup: the element-diagonal blocks of J(u) (volume terms plus this
//    element's own-side face terms, all fields coupled), one column per grid.y
//    of the J v kernel, then batched Gauss-Jordan inversion with partial
//    pivoting; the inverse is stored transposed in FP64, FP32 or BF16.
//  * block apply: y_e = B_e^{-1} x_e, one thread block per element, threads over
//    rows, reading the stored inverse once (an HBM-bound batched GEMV).
//  * FGMRES(m) with right preconditioning (flexible: the preconditioner may
//    change between iterations), classical Gram-Schmidt applied twice, dot
//    products reduced on the device in a fixed order (warp shuffles, then one
//    partial per block, then one block), so results do not depend on timing.
//  * Newton's method with backtracking line search on ||R|| (Sec. 4).
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <type_traits>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/enp_dg.h"
#include "enp_internal.h"
#include "enp_reduce.cuh"

namespace enp {

// ------------------------------------------------------------------ c_m
// Eq. substitution: c_m = -(1/z_m) sum_{k<m} z_k c_k, node by node.
__global__ void recover_cm_kernel(const double* __restrict__ u, double* __restrict__ cm, int NF,
                                  long long EN, double zk0, double zk1, double zk2, double inv_zm,
                                  long long batch_stride, int batch) {
  const double zk[3] = {zk0, zk1, zk2};
  long long total = EN * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long b = t / EN, i = t % EN;
    double s = 0.0;
    for (int k = 0; k < NF - 1; ++k) s += zk[k] * u[b * batch_stride + (k + 1) * EN + i];
    cm[t] = -inv_zm * s;
  }
}


// w[b] -= sum_i V_i[b] h[b][i]  (h on the device, [batch][nd], nd <= 256),
// in the vector's precision with the coefficients staged once per block, W
// entries per 16-byte load. With NORM, also the partial sums of ||w_new||^2
// per block, part[b][block] (thread sums in the vector's precision, then FP64).
template <class T, int W, bool NORM>
__global__ void __launch_bounds__(kRedThreads)
multi_axpy(const T* __restrict__ V, long long vstride, int nd, const double* __restrict__ h,
           T* __restrict__ w, long long n, long long bstride, double* __restrict__ part) {
  __shared__ T hs[256];
  __shared__ double red[kRedThreads / 32];
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) hs[i] = (T)h[b * nd + i];
  __syncthreads();
  const long long nu = n / W;
  T nrm = T(0);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < nu;
       u += (long long)gridDim.x * blockDim.x) {
    T acc[W];
    load_vec<T, W>(w + b * bstride + u * W, acc);
    const T* Vu = V + b * bstride + u * W;
#pragma unroll 4
    for (int i = 0; i < nd; ++i) {
      T vv[W];
      load_vec<T, W>(Vu + i * vstride, vv);
      const T hi = hs[i];
#pragma unroll
      for (int c = 0; c < W; ++c) acc[c] -= hi * vv[c];
    }
    store_vec<T, W>(w + b * bstride + u * W, acc);
    if (NORM) {
#pragma unroll
      for (int c = 0; c < W; ++c) nrm += acc[c] * acc[c];
    }
  }
  if (NORM) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double s = warp_sum((double)nrm);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int wv = 0; wv < kRedThreads / 32; ++wv) t += red[wv];
      part[(long long)b * gridDim.x + blockIdx.x] = t;
    }
  }
}

// y[b] = sum_{i<nd} V_i[b] c[b * cstride + i] (+ y[b] if accumulate), nd <= 256
template <class T, class TY>
__global__ void combine(const T* __restrict__ V, long long vstride, int nd,
                        const double* __restrict__ c, int cstride, TY* __restrict__ y,
                        long long n, long long bstride, int accumulate) {
  __shared__ T cs_[256];
  const int b = blockIdx.y;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) cs_[i] = (T)c[b * cstride + i];
  __syncthreads();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    T acc = accumulate ? (T)y[b * bstride + k] : T(0);
    for (int i = 0; i < nd; ++i) acc += cs_[i] * V[i * vstride + b * bstride + k];
    y[b * bstride + k] = (TY)acc;
  }
}

// y[b] = a[b] * x[b] (+ beta * y) with per-batch scalars on the device, in the
// precision of TY
template <class TX, class TY>
__global__ void scale_copy(const TX* __restrict__ x, const double* __restrict__ a, double beta,
                           TY* __restrict__ y, long long n, long long bstride) {
  const int b = blockIdx.y;
  const TY ab = (TY)a[b], bb = (TY)beta;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    TY v = ab * (TY)x[b * bstride + k];
    if (beta != 0.0) v += bb * y[b * bstride + k];
    y[b * bstride + k] = v;
  }
}

// z[b] = x[b] + lam[b] y[b] (per operating point step lengths)
__global__ void axpy_batched(const double* __restrict__ x, const double* __restrict__ lam,
                             const double* __restrict__ y, double* __restrict__ z, long long n,
                             int B) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n * B;
       k += (long long)gridDim.x * blockDim.x)
    z[k] = x[k] + lam[k / n] * y[k];
}

// y[b] = s[b] x[b] (per operating point scale, e.g. 0 to freeze a converged point)
__global__ void scale_batched(const double* __restrict__ x, const double* __restrict__ sc,
                              double* __restrict__ y, long long n, int B) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n * B;
       k += (long long)gridDim.x * blockDim.x)
    y[k] = sc[k / n] * x[k];
}

// Potential-only operator (the initial guess of Sec. 4.3): the species rows of
// J v are the identity, y_species = v_species.
template <class T>
__global__ void species_rows_copy(const T* __restrict__ v, T* __restrict__ y, long long EN,
                                  int NF, long long bstride, int B) {
  const long long per = (long long)(NF - 1) * EN;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * B;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, i = EN + t % per;
    y[b * bstride + i] = v[b * bstride + i];
  }
}

// ... and the species rows of the residual are c_k - c_k^in.
__global__ void species_rows_offset(const double* __restrict__ u, double* __restrict__ r,
                                    long long EN, int NF, long long bstride, int B, double c0,
                                    double c1, double c2) {
  const double cin[3] = {c0, c1, c2};
  const long long per = (long long)(NF - 1) * EN;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * B;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, i = EN + t % per;
    r[b * bstride + i] = u[b * bstride + i] - cin[(t % per) / EN];
  }
}

// ... and the species rows of every element-diagonal block are unit rows
// (blocks [nblk][nb][nb] row-major, rows f * Np + i).
template <class T>
__global__ void block_species_identity(T* __restrict__ blk, long long nblk, int nb, int Np) {
  const long long per = (long long)(nb - Np) * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * nblk;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k = t / per, rc = t % per;
    const int row = Np + (int)(rc / nb), col = (int)(rc % nb);
    blk[k * nb * nb + (long long)row * nb + col] = row == col ? T(1) : T(0);
  }
}

// c_k = c_k^in at every node of every operating point.
__global__ void species_fill(double* __restrict__ u, long long EN, int NF, long long bstride, int B,
                             double c0, double c1, double c2) {
  const double cin[3] = {c0, c1, c2};
  const long long per = (long long)(NF - 1) * EN;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * B;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, i = EN + t % per;
    u[b * bstride + i] = cin[(t % per) / EN];
  }
}

template <class TX, class TY>
__global__ void convert_kernel(const TX* __restrict__ x, TY* __restrict__ y, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    y[k] = (TY)x[k];
}

// ------------------------------------------------------------------ FGMRES state
// Per operating point b, on the device: H [m+1][m] (column j built in
// iteration j), g [m+1], cs, sn [m], hcol [m+1], scalars. One thread per b.
struct KrylovDev {
  double *H, *g, *cs, *sn, *hcol, *dh, *hn2, *inv, *beta, *bn2, *tol, *resn, *coef;
  int* jconv;   // -2 done before the cycle, -1 running, j converged at iteration j
};

__global__ void krylov_tolerance(KrylovDev K, int B, double rtol, double atol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  K.tol[b] = fmax(rtol * sqrt(K.bn2[b]), atol);
}

// Start of a cycle: beta = ||r0||, g = beta e1, scale factor 1/beta, done flags.
__global__ void krylov_cycle_init(KrylovDev K, int B, int m, int* any_running, int* nonfinite) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double beta = sqrt(K.dh[b]);
  K.beta[b] = beta;
  K.resn[b] = beta;
  if (!isfinite(beta)) atomicOr(nonfinite, 1);
  for (int i = 0; i <= m; ++i) K.g[(long long)b * (m + 1) + i] = 0.0;
  K.g[(long long)b * (m + 1)] = beta;
  const bool done = !(beta > K.tol[b]);
  K.jconv[b] = done ? -2 : -1;
  K.inv[b] = done ? 0.0 : 1.0 / beta;
  if (!done) atomicOr(any_running, 1);
}

// One warp per (b, i): dh[b][i] = the partials of <V_i, w>_b summed in block
// order (as finish_partials), added into the Hessenberg column (first pass:
// stored).
__global__ void krylov_hcol_finish(KrylovDev K, const double* __restrict__ part, int nparts,
                                   int B, int m, int nd, int first) {
  const int t = blockIdx.x;
  if (t >= B * nd) return;
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += 32) s += part[(long long)t * nparts + k];
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    const int b = t / nd, i = t % nd;
    K.dh[t] = s;
    K.hcol[(long long)b * (m + 1) + i] = first ? s : K.hcol[(long long)b * (m + 1) + i] + s;
  }
}

// Iteration j of Arnoldi with Givens rotations, one warp per running point:
// ||w||^2 summed from its partials in block order; the new Hessenberg column
// and the earlier rotations staged in shared memory by the warp, then rotated
// by lane 0 with the running entry in a register.
__global__ void krylov_norm_givens(KrylovDev K, const double* __restrict__ part, int nparts, int B,
                                   int m, int j, int* nonfinite) {
  __shared__ double s_h[256], s_cs[256], s_sn[256];  // m <= 255
  const int b = blockIdx.x;
  if (b >= B) return;
  const int lane = threadIdx.x;
  double s = 0.0;
  for (int k = lane; k < nparts; k += 32) s += part[(long long)b * nparts + k];
  s = warp_sum(s);
  const double* hc = K.hcol + (long long)b * (m + 1);
  double* cs = K.cs + (long long)b * m;
  double* sn = K.sn + (long long)b * m;
  for (int r = lane; r <= j; r += 32) s_h[r] = hc[r];
  for (int r = lane; r < j; r += 32) { s_cs[r] = cs[r]; s_sn[r] = sn[r]; }
  __syncwarp();
  if (lane != 0) return;
  K.hn2[b] = s;
  const double hn = sqrt(s);
  if (K.jconv[b] != -1) { K.inv[b] = 0.0; return; }
  double* H = K.H + (long long)b * (m + 1) * m;
  double* g = K.g + (long long)b * (m + 1);
  double a = s_h[0];  // entry r of the column, already rotated by rotations < r
  for (int r = 0; r < j; ++r) {
    const double c = s_h[r + 1], cr = s_cs[r], sr = s_sn[r];
    H[(long long)r * m + j] = cr * a + sr * c;
    a = -sr * a + cr * c;
  }
  const double c = hn;
  const double rr = hypot(a, c);
  const double cj = rr > 0 ? a / rr : 1.0, sj = rr > 0 ? c / rr : 0.0;
  cs[j] = cj;
  sn[j] = sj;
  H[(long long)j * m + j] = rr;
  H[(long long)(j + 1) * m + j] = 0.0;
  const double gj = g[j];
  g[j + 1] = -sj * gj;
  g[j] = cj * gj;
  const double res = fabs(g[j + 1]);
  K.resn[b] = res;
  if (!isfinite(res)) atomicOr(nonfinite, 1);
  if (res <= K.tol[b] || hn == 0.0) K.jconv[b] = j;
  K.inv[b] = (hn > 0 && K.jconv[b] == -1) ? 1.0 / hn : 0.0;
}

// Back substitution for the update coefficients of every point (columns beyond
// its convergence iteration are zero).
__global__ void krylov_solve_upper(KrylovDev K, int B, int m, int jm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int jc = K.jconv[b];
  const int ji = jc == -2 ? 0 : (jc >= 0 ? jc + 1 : jm);
  const double* H = K.H + (long long)b * (m + 1) * m;
  const double* g = K.g + (long long)b * (m + 1);
  double* y = K.coef + (long long)b * m;
  for (int r = m - 1; r >= ji; --r) y[r] = 0.0;
  for (int r = ji - 1; r >= 0; --r) {
    double s = g[r];
    for (int c = r + 1; c < ji; ++c) s -= H[(long long)r * m + c] * y[c];
    const double d = H[(long long)r * m + r];
    y[r] = d != 0.0 ? s / d : 0.0;
  }
}

// r = b - r (batched, elementwise)
template <class T>
__global__ void b_minus(const T* __restrict__ b, T* __restrict__ r, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    r[k] = b[k] - r[k];
}

// ------------------------------------------------------------------ two-level
// Coarse space: one potential value per element (the element mean mode,
// P = constant on the element's Phi nodes). A0 = P^T J_PhiPhi P is a 7-point
// stencil on the element grid, stored [batch][cell][7] with entries
// (self, -x, +x, -y, +y, -z, +z). Coarser levels aggregate 2 x 2 x 2 cells
// (Galerkin: the stencil stays 7-point), smoothed by red-black Gauss-Seidel.

// Element colour (ix + 2 iy + 3 iz) mod 7: the seven cells of a 7-point
// stencil have offsets 0, +-1, +-2, +-3 (mod 7), all distinct, so every cell's
// stencil holds exactly one cell of each colour and seven probes recover A0.
__device__ __forceinline__ int cell_colour(int ix, int iy, int iz) {
  return (ix + 2 * iy + 3 * iz) % 7;
}

// v = indicator of the Phi field on the elements of colour c (other fields 0).
template <class T>
__global__ void coarse_colour_vector(T* __restrict__ v, int nx, int ny, int nz, int Np,
                                     long long bstride, int E, int colour) {
  const int b = blockIdx.y;
  const long long n = (long long)E * Np;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / Np);
    const int ix = e % nx, iy = (e / nx) % ny, iz = e / (nx * ny);
    v[b * bstride + t] = (cell_colour(ix, iy, iz) == colour) ? T(1) : T(0);
  }
}

// Sum of the Phi rows of element K of J v, filed under the direction of the
// colour-c element in K's stencil (if that element exists).
template <class T>
__global__ void coarse_gather(const T* __restrict__ jv, double* __restrict__ A, int nx, int ny,
                              int nz, int Np, long long bstride, int colour) {
  const int b = blockIdx.y;
  const int E = nx * ny * nz;
  for (int K = blockIdx.x * blockDim.x + threadIdx.x; K < E; K += gridDim.x * blockDim.x) {
    const int ix = K % nx, iy = (K / nx) % ny, iz = K / (nx * ny);
    // offset of the colour-c cell relative to K, as a colour difference
    const int d = ((colour - cell_colour(ix, iy, iz)) % 7 + 7) % 7;
    int dir = -1;
    switch (d) {
      case 0: dir = 0; break;
      case 6: dir = ix > 0 ? 1 : -1; break;
      case 1: dir = ix < nx - 1 ? 2 : -1; break;
      case 5: dir = iy > 0 ? 3 : -1; break;
      case 2: dir = iy < ny - 1 ? 4 : -1; break;
      case 4: dir = iz > 0 ? 5 : -1; break;
      case 3: dir = iz < nz - 1 ? 6 : -1; break;
    }
    if (dir < 0) continue;
    const T* row = jv + b * bstride + (long long)K * Np;  // field 0 block starts at 0
    double s = 0.0;
    for (int i = 0; i < Np; ++i) s += (double)row[i];
    A[((long long)b * E + K) * 7 + dir] = s;
  }
}

// Galerkin aggregation of a 7-point level onto 2 x 2 x 2 blocks of cells.
__global__ void coarse_aggregate(const double* __restrict__ Af, int fx, int fy, int fz,
                                 double* __restrict__ Ac, int cx, int cy, int cz) {
  const int b = blockIdx.y;
  const int Nc = cx * cy * cz, Nf = fx * fy * fz;
  for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < Nc; C += gridDim.x * blockDim.x) {
    const int jx = C % cx, jy = (C / cx) % cy, jz = C / (cx * cy);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int ix = 2 * jx + dx, iy = 2 * jy + dy, iz = 2 * jz + dz;
          if (ix >= fx || iy >= fy || iz >= fz) continue;
          const double* a = Af + ((long long)b * Nf + ix + fx * (iy + fy * iz)) * 7;
          acc[0] += a[0];
          // x neighbours: inside the aggregate -> self, outside -> the coarse neighbour
          acc[dx == 0 ? 1 : 0] += a[1];
          acc[dx == 1 ? 2 : 0] += a[2];
          acc[dy == 0 ? 3 : 0] += a[3];
          acc[dy == 1 ? 4 : 0] += a[4];
          acc[dz == 0 ? 5 : 0] += a[5];
          acc[dz == 1 ? 6 : 0] += a[6];
        }
    double* o = Ac + ((long long)b * Nc + C) * 7;
    for (int d = 0; d < 7; ++d) o[d] = acc[d];
  }
}

// The V-cycle runs in FP32 (it only preconditions: FGMRES is flexible, and the
// outer residual stays in the caller's precision). Each level's stencil is kept
// packed per cell as 8 floats: the 7 entries and the inverse diagonal (0 where
// the diagonal is 0: such a cell is left unchanged by smoothing).
constexpr int kPack = 8;

// (a0..a6 as float, 1 / a0) per cell, from the FP64 stencil
__global__ void coarse_pack32(const double* __restrict__ A, float* __restrict__ A32,
                              long long ncells) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncells;
       c += (long long)gridDim.x * blockDim.x) {
    const double* a = A + c * 7;
    float* o = A32 + c * kPack;
    for (int d = 0; d < 7; ++d) o[d] = (float)a[d];
    o[7] = a[0] != 0.0 ? (float)(1.0 / a[0]) : 0.0f;
  }
}

__device__ __forceinline__ float stencil_off(const float* __restrict__ a, const float* __restrict__ x,
                                             int i, int nx, int ny, int nz, int ix, int iy, int iz) {
  float s = 0.0f;
  if (ix > 0) s += a[1] * x[i - 1];
  if (ix < nx - 1) s += a[2] * x[i + 1];
  if (iy > 0) s += a[3] * x[i - nx];
  if (iy < ny - 1) s += a[4] * x[i + nx];
  if (iz > 0) s += a[5] * x[i - nx * ny];
  if (iz < nz - 1) s += a[6] * x[i + nx * ny];
  return s;
}

// The per-cell steps of the V-cycle, shared by the grid-wide kernels (large
// levels) and the one-block kernel (small levels), so both give the same bits.
// Ab, xb, bb: one operating point's packed stencil, iterate and right-hand side.

// Gauss-Seidel update of cell i if it has parity `colour` (red-black).
__device__ __forceinline__ void gs_cell(const float* __restrict__ Ab, float* __restrict__ xb,
                                        const float* __restrict__ bb, int nx, int ny, int nz,
                                        int colour, int i) {
  const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
  if (((ix + iy + iz) & 1) != colour) return;
  const float* a = Ab + (long long)i * kPack;
  if (a[7] == 0.0f) return;
  xb[i] = (bb[i] - stencil_off(a, xb, i, nx, ny, nz, ix, iy, iz)) * a[7];
}

__device__ __forceinline__ float residual_cell(const float* __restrict__ Ab,
                                               const float* __restrict__ xb,
                                               const float* __restrict__ bb, int nx, int ny,
                                               int nz, int i) {
  const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
  const float* a = Ab + (long long)i * kPack;
  return bb[i] - a[0] * xb[i] - stencil_off(a, xb, i, nx, ny, nz, ix, iy, iz);
}

// sum of the fine values over the 2 x 2 x 2 aggregate of coarse cell C
__device__ __forceinline__ float restrict_cell(const float* __restrict__ rf, int fx, int fy,
                                               int fz, int cx, int cy, int C) {
  const int jx = C % cx, jy = (C / cx) % cy, jz = C / (cx * cy);
  float s = 0.0f;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int ix = 2 * jx + dx, iy = 2 * jy + dy, iz = 2 * jz + dz;
        if (ix < fx && iy < fy && iz < fz) s += rf[ix + fx * (iy + fy * iz)];
      }
  return s;
}

// the coarse value of the aggregate that holds fine cell i
__device__ __forceinline__ float prolong_cell(const float* __restrict__ xc, int cx, int cy,
                                              int fx, int fy, int i) {
  const int ix = i % fx, iy = (i / fx) % fy, iz = i / (fx * fy);
  return xc[ix / 2 + cx * (iy / 2 + cy * (iz / 2))];
}

// One half-sweep of red-black Gauss-Seidel on cells of parity `colour`.
__global__ void coarse_gs(const float* __restrict__ A, float* __restrict__ x,
                          const float* __restrict__ bvec, int nx, int ny, int nz, int colour) {
  const int b = blockIdx.y;
  const int N = nx * ny * nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    gs_cell(A + (long long)b * N * kPack, x + (long long)b * N, bvec + (long long)b * N, nx, ny,
            nz, colour, i);
}

// r = b - A x
__global__ void coarse_residual(const float* __restrict__ A, const float* __restrict__ x,
                                const float* __restrict__ bvec, float* __restrict__ r, int nx,
                                int ny, int nz) {
  const int b = blockIdx.y;
  const int N = nx * ny * nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    r[(long long)b * N + i] = residual_cell(A + (long long)b * N * kPack, x + (long long)b * N,
                                            bvec + (long long)b * N, nx, ny, nz, i);
}

// b_c = sum of the fine residual over each 2 x 2 x 2 aggregate
__global__ void coarse_restrict(const float* __restrict__ rf, int fx, int fy, int fz,
                                float* __restrict__ bc, int cx, int cy, int cz) {
  const int b = blockIdx.y;
  const int Nc = cx * cy * cz, Nf = fx * fy * fz;
  for (int C = blockIdx.x * blockDim.x + threadIdx.x; C < Nc; C += gridDim.x * blockDim.x)
    bc[(long long)b * Nc + C] = restrict_cell(rf + (long long)b * Nf, fx, fy, fz, cx, cy, C);
}

// x_f += omega x_c on every fine cell of the aggregate
__global__ void coarse_prolong(const float* __restrict__ xc, int cx, int cy, int cz,
                               float* __restrict__ xf, int fx, int fy, int fz, float omega) {
  const int b = blockIdx.y;
  const int Nc = cx * cy * cz, Nf = fx * fy * fz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Nf; i += gridDim.x * blockDim.x)
    xf[(long long)b * Nf + i] += omega * prolong_cell(xc + (long long)b * Nc, cx, cy, fx, fy, i);
}

// The coarsest level (at most kCoarsestCells cells) is solved with its dense
// inverse, computed in FP64 at setup by the block Gauss-Jordan kernel below and
// stored in FP32. If that matrix is singular to working accuracy (a potential
// fixed by no boundary condition), it is smoothed instead: x = 0, then
// `sweeps` red-black Gauss-Seidel sweeps inside one thread block per operating
// point, with the stencil, x and b held in shared memory.
constexpr int kCoarsestCells = 128;

// dense[b][i][j] = the FP64 stencil rows of a level as a dense n x n matrix
// (one block per operating point)
__global__ void coarse_dense(const double* __restrict__ A, int nx, int ny, int nz,
                             double* __restrict__ dense) {
  const int b = blockIdx.x;
  const int N = nx * ny * nz;
  double* D = dense + (long long)b * N * N;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) D[t] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const double* a = A + ((long long)b * N + i) * 7;
    double* row = D + (long long)i * N;
    row[i] = a[0];
    if (ix > 0) row[i - 1] = a[1];
    if (ix < nx - 1) row[i + 1] = a[2];
    if (iy > 0) row[i - nx] = a[3];
    if (iy < ny - 1) row[i + nx] = a[4];
    if (iz > 0) row[i - nx * ny] = a[5];
    if (iz < nz - 1) row[i + nx * ny] = a[6];
  }
}

// Row r of inv * b with the inverse stored transposed (M[c][r]).
__device__ __forceinline__ float dense_row(const float* __restrict__ M,
                                           const float* __restrict__ bb, int N, int r) {
  float s = 0.0f;
  for (int c = 0; c < N; ++c) s += M[(long long)c * N + r] * bb[c];
  return s;
}

// x_b = inv_b r_b, one block per operating point.
__global__ void __launch_bounds__(kCoarsestCells)
coarse_dense_apply(const float* __restrict__ invT, const float* __restrict__ rhs, int N,
                   float* __restrict__ x) {
  const int b = blockIdx.x;
  for (int r = threadIdx.x; r < N; r += blockDim.x)
    x[(long long)b * N + r] = dense_row(invT + (long long)b * N * N, rhs + (long long)b * N, N, r);
}

__global__ void __launch_bounds__(kCoarsestCells)
coarse_solve_small(const float* __restrict__ A, float* __restrict__ x,
                   const float* __restrict__ bvec, int nx, int ny, int nz, int sweeps) {
  __shared__ float sA[kCoarsestCells * kPack];
  __shared__ float sx[kCoarsestCells];
  __shared__ float sb[kCoarsestCells];
  const int b = blockIdx.x;
  const int N = nx * ny * nz;  // <= kCoarsestCells, checked by the host
  const float* Ab = A + (long long)b * N * kPack;
  for (int i = threadIdx.x; i < kPack * N; i += blockDim.x) sA[i] = Ab[i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sx[i] = 0.0f;
    sb[i] = bvec[(long long)b * N + i];
  }
  __syncthreads();
  for (int sw = 0; sw < sweeps; ++sw)
    for (int colour = 0; colour < 2; ++colour) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) gs_cell(sA, sx, sb, nx, ny, nz, colour, i);
      __syncthreads();
    }
  for (int i = threadIdx.x; i < N; i += blockDim.x) x[(long long)b * N + i] = sx[i];
}

// The small levels of the V-cycle (at most kTailCells cells) run in one
// thread block per operating point, with a barrier between steps, instead of
// one launch per half-sweep: levels l0 .. nl-2 are smoothed, their residuals
// restricted, the coarsest solved (its inverse, or smoothing), and the
// corrections prolonged and post-smoothed, as in the grid-wide kernels.
constexpr int kTailCells = 8192;
constexpr int kTailThreads = 1024;
constexpr int kMaxLevels = 16;

struct LevelDev {
  int nx, ny, nz, n;
  const float* A;
  float *x, *b, *r;
};

struct VcycleTail {
  int l0, nl;
  LevelDev L[kMaxLevels];
  const float* inv;  // coarsest inverse, transposed, [B][n][n]; null: smoothing
  int smooth, coarsest_sweeps;
  float omega;       // over-correction of the prolongated coarse values
};

__global__ void __launch_bounds__(kTailThreads) coarse_vcycle_tail(const VcycleTail T) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int l = T.l0; l < T.nl - 1; ++l) {
    const LevelDev L = T.L[l], C = T.L[l + 1];
    const int N = L.n;
    const float* Ab = L.A + (long long)b * N * kPack;
    float* xb = L.x + (long long)b * N;
    const float* bb = L.b + (long long)b * N;
    float* rb = L.r + (long long)b * N;
    for (int i = tid; i < N; i += nt) xb[i] = 0.0f;
    __syncthreads();
    for (int sw = 0; sw < T.smooth; ++sw)
      for (int colour = 0; colour < 2; ++colour) {
        for (int i = tid; i < N; i += nt) gs_cell(Ab, xb, bb, L.nx, L.ny, L.nz, colour, i);
        __syncthreads();
      }
    for (int i = tid; i < N; i += nt) rb[i] = residual_cell(Ab, xb, bb, L.nx, L.ny, L.nz, i);
    __syncthreads();
    for (int c = tid; c < C.n; c += nt)
      C.b[(long long)b * C.n + c] = restrict_cell(rb, L.nx, L.ny, L.nz, C.nx, C.ny, c);
    __syncthreads();
  }
  {
    const LevelDev L = T.L[T.nl - 1];
    const int N = L.n;
    float* xb = L.x + (long long)b * N;
    const float* bb = L.b + (long long)b * N;
    if (T.inv) {
      for (int r = tid; r < N; r += nt) xb[r] = dense_row(T.inv + (long long)b * N * N, bb, N, r);
    } else {
      const float* Ab = L.A + (long long)b * N * kPack;
      for (int i = tid; i < N; i += nt) xb[i] = 0.0f;
      __syncthreads();
      for (int sw = 0; sw < T.coarsest_sweeps; ++sw)
        for (int colour = 0; colour < 2; ++colour) {
          for (int i = tid; i < N; i += nt) gs_cell(Ab, xb, bb, L.nx, L.ny, L.nz, colour, i);
          __syncthreads();
        }
    }
    __syncthreads();
  }
  for (int l = T.nl - 2; l >= T.l0; --l) {
    const LevelDev L = T.L[l], C = T.L[l + 1];
    const int N = L.n;
    const float* Ab = L.A + (long long)b * N * kPack;
    float* xb = L.x + (long long)b * N;
    const float* bb = L.b + (long long)b * N;
    for (int i = tid; i < N; i += nt)
      xb[i] += T.omega * prolong_cell(C.x + (long long)b * C.n, C.nx, C.ny, L.nx, L.ny, i);
    __syncthreads();
    for (int sw = 0; sw < T.smooth; ++sw)
      for (int colour = 1; colour >= 0; --colour) {
        for (int i = tid; i < N; i += nt) gs_cell(Ab, xb, bb, L.nx, L.ny, L.nz, colour, i);
        __syncthreads();
      }
  }
}

// b0[K] = sum over the Phi nodes of element K of r (P^T r), summed in FP64;
// one warp per element
template <class TV>
__global__ void coarse_from_fine(const TV* __restrict__ r, float* __restrict__ b0, int E, int Np,
                                 long long bstride) {
  const int b = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int K = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; K < E; K += nw) {
    const TV* row = r + b * bstride + (long long)K * Np;
    double s = 0.0;
    for (int i = lane; i < Np; i += 32) s += (double)row[i];
    s = warp_sum(s);
    if (lane == 0) b0[(long long)b * E + K] = (float)s;
  }
}

// acc += x
__global__ void axpy_f32(const float* __restrict__ x, float* __restrict__ acc, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    acc[t] += x[t];
}

// z[Phi nodes of K] += x0[K] (P x0)
template <class TV>
__global__ void coarse_to_fine(const float* __restrict__ x0, TV* __restrict__ z, int E, int Np,
                               long long bstride) {
  const int b = blockIdx.y;
  const long long n = (long long)E * Np;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    z[b * bstride + t] += (TV)x0[(long long)b * E + t / Np];
}

// ------------------------------------------------------------------ block inverse
// In-place Gauss-Jordan inversion with partial (row) pivoting of one n x n
// block per thread block. The matrix lives in shared memory when it fits
// (SMEM = true), else in global memory, with the odd leading dimension n + 1
// (no shared-memory bank conflicts down a column). Lane l of every warp owns
// the rows i = l (mod 32), warp w the columns j = w (mod nwarps). Step k:
//   (1) stage the pivot row (old row p) and the pivot column (rows k and p
//       exchanged), and move row k to row p;
//   (2) rank-1 update of every entry, A_ij -= A_ik A_kj / A_kk, the column
//       entries of the thread's rows held in registers;
//   (3) overwrite row k (scaled pivot row) and column k (-A_ik / A_kk), while
//       warp 0 finds the next pivot in column k+1 (in the matrix's type).
// A non-finite pivot, or one not above piv_rtol times the largest |A_ij| (an
// exact zero when piv_rtol = 0), sets *singular. Row swaps are undone at the end
// as column swaps in reverse order. The inverse is written transposed
// (out[e][c][r] = inv[r][c]) in type TS.
constexpr int kGjRows = 8;  // rows per lane held in registers: n <= 256

template <class T>
__device__ __forceinline__ void gj_pivot(const T* A, int ld, int n, int col, int lane, int* s_p,
                                         int* s_bad, T thr) {
  T best = T(-1);
  int bi = col;
  for (int i = col + lane; i < n; i += 32) {
    const T a = fabs(A[(long long)i * ld + col]);
    if (a > best) { best = a; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { *s_p = bi; *s_bad = (!(best > thr) || !isfinite(best)) ? 1 : 0; }
}

template <class T, class TS, bool SMEM, class TB>
__global__ void gj_invert(const TB* __restrict__ blocks, T* __restrict__ work, TS* __restrict__ out,
                          int n, int* __restrict__ singular, T piv_rtol) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const long long e = blockIdx.x;
  const int ld = n + 1;
  const long long na = (long long)n * ld;
  T* A = SMEM ? reinterpret_cast<T*>(gsm) : work + e * na;
  T* prow = SMEM ? A + na : reinterpret_cast<T*>(gsm);   // [n] pivot row (old row p)
  T* pcol = prow + n;                                     // [n] pivot column after the swap
  int* piv = reinterpret_cast<int*>(pcol + n);            // [n] row chosen at each step
  __shared__ int s_p;
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const TB* src = blocks + e * (long long)n * n;
  __shared__ T s_thr;
  __shared__ T s_wmax[32];
  T amax = T(0);
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) {
      const T a = (T)src[(long long)i * n + j];
      A[(long long)i * ld + j] = a;
      amax = fmax(amax, fabs(a));
    }
  // pivots at or below piv_rtol * max |A_ij| count as singular (0: exact zero only)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_down_sync(0xffffffffu, amax, o));
  if (lane == 0) s_wmax[warp] = amax;
  __syncthreads();
  if (tid == 0) {
    T mx = T(0);
    for (int w = 0; w < nw; ++w) mx = fmax(mx, s_wmax[w]);
    s_thr = piv_rtol > T(0) ? piv_rtol * mx : T(0);
  }
  __syncthreads();
  if (warp == 0) gj_pivot<T>(A, ld, n, 0, lane, &s_p, &s_bad, s_thr);
  __syncthreads();
  const bool regs = n <= 32 * kGjRows;
  for (int k = 0; k < n; ++k) {
    if (s_bad) break;
    const int p = s_p;
    // (1)
    for (int j = tid; j < n; j += nt) {
      const T vp = A[(long long)p * ld + j], vk = A[(long long)k * ld + j];
      prow[j] = vp;
      if (p != k) A[(long long)p * ld + j] = vk;
    }
    for (int i = tid; i < n; i += nt) {
      const int si = (i == k) ? p : ((i == p) ? k : i);
      pcol[i] = A[(long long)si * ld + k];
    }
    if (tid == 0) piv[k] = p;
    __syncthreads();
    // (2)
    const T pinv = T(1) / prow[k];
    if (regs) {
      T pc[kGjRows];
#pragma unroll
      for (int r = 0; r < kGjRows; ++r) {
        const int i = lane + 32 * r;
        pc[r] = i < n ? pcol[i] : T(0);
      }
      for (int j = warp; j < n; j += nw) {
        const T rj = prow[j] * pinv;
        T* colj = A + j;
#pragma unroll
        for (int r = 0; r < kGjRows; ++r) {
          const int i = lane + 32 * r;
          if (i < n) colj[(long long)i * ld] -= pc[r] * rj;
        }
      }
    } else {
      for (int j = warp; j < n; j += nw) {
        const T rj = prow[j] * pinv;
        for (int i = lane; i < n; i += 32) A[(long long)i * ld + j] -= pcol[i] * rj;
      }
    }
    __syncthreads();
    // (3)
    for (int j = tid; j < n; j += nt) A[(long long)k * ld + j] = (j == k) ? pinv : prow[j] * pinv;
    for (int i = tid; i < n; i += nt)
      if (i != k) A[(long long)i * ld + k] = -pcol[i] * pinv;
    if (warp == 0 && k + 1 < n) gj_pivot<T>(A, ld, n, k + 1, lane, &s_p, &s_bad, s_thr);
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) atomicOr(singular, 1);
    return;
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < n; i += nt) {
        T tmp = A[(long long)i * ld + k];
        A[(long long)i * ld + k] = A[(long long)i * ld + p];
        A[(long long)i * ld + p] = tmp;
      }
    __syncthreads();
  }
  TS* o = out + e * (long long)n * n;
  for (int c = warp; c < n; c += nw)
    for (int r = lane; r < n; r += 32) o[(long long)c * n + r] = (TS)A[(long long)r * ld + c];
}

// Gauss-Jordan inversion of one n x n block per thread block with the whole
// matrix in registers (FP32 arithmetic): warp w owns the rows i = w + NW r
// (r < RPW), lane l the columns j = l + 32 c (c < CPL); entries beyond n are
// identity padding that no step changes. Partial pivoting without row
// exchanges: step k pivots in place on (p, k), p the row not yet used with the
// largest |M_pk| (the exchange step of Gauss-Jordan elimination):
//   M_pj <- M_pj / M_pk (j != k),  M_pk <- 1 / M_pk,
//   M_ik <- -M_ik / M_pk (i != p), M_ij <- M_ij - M_ik M_pj / M_pk otherwise;
// after n steps with rows p_0..p_{n-1}, M_{p_k, j} = inv(A)_{k, p_j}. Two
// barriers per step: the lanes owning column k publish it (double-buffered,
// with |M_ik| or -1 for used rows), every warp finds the pivot from it in the
// same order (so all agree), the warp owning row p publishes that row. The
// inverse is staged in shared memory and written transposed, out[e][c][r] =
// inv[r][c], in type TS. A pivot not above piv_rtol max|A_ij| (exactly zero
// when piv_rtol = 0), or not finite, sets *singular.
template <class TB, class TS, int NW, int RPW, int CPL>
__global__ void __launch_bounds__(NW * 32, 1)
gj_invert_regs(const TB* __restrict__ blocks, TS* __restrict__ out, int n,
               int* __restrict__ singular, float piv_rtol) {
  constexpr int NR = NW * RPW;   // padded rows
  constexpr int NC = 32 * CPL;   // padded columns
  extern __shared__ __align__(16) unsigned char gsm[];
  float* stage = reinterpret_cast<float*>(gsm);        // [n][n + 1] transposed inverse
  __shared__ float colv[2][NR];                        // the pivot column, double-buffered
  __shared__ float candv[2][32];                       // per warp: largest |M_ik| over its unused rows
  __shared__ int candi[2][32];                         //           and that row
  __shared__ float rowv[NC];
  __shared__ int piv[NC], stepof[NR];
  __shared__ float s_wmax[NW];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long e = blockIdx.x;
  const TB* src = blocks + e * (long long)n * n;
  float M[RPW][CPL];
  float amax = 0.f;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int i = w + NW * r;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = lane + 32 * c;
      const float a = (i < n && j < n) ? (float)src[(long long)i * n + j] : (i == j ? 1.f : 0.f);
      M[r][c] = a;
      if (i < n && j < n) amax = fmaxf(amax, fabsf(a));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, o));
  if (lane == 0) s_wmax[w] = amax;
  unsigned used = 0u;  // bit r: row w + NW r already a pivot row (same in every lane)
  // publish column kc (from lane kc % 32 of every warp): its values for the
  // update, and the warp's pivot candidate among its unused rows
  auto publish = [&](int kc, int buf) {
    if (lane == (kc & 31)) {
      const int cc = kc >> 5;
      float best = -1.f;
      int bi = 0;
#pragma unroll
      for (int c = 0; c < CPL; ++c)
        if (c == cc) {
#pragma unroll
          for (int r = 0; r < RPW; ++r) {
            const int i = w + NW * r;
            const float v = M[r][c];
            colv[buf][i] = v;
            const float av = (i < n && !((used >> r) & 1u)) ? fabsf(v) : -1.f;
            if (av > best) { best = av; bi = i; }   // rows ascend with r: ties keep the lower
          }
        }
      candv[buf][w] = best;
      candi[buf][w] = bi;
    }
  };
  publish(0, 0);
  __syncthreads();
  float thr = 0.f;
  if (piv_rtol > 0.f) {
    float mx = 0.f;
    for (int t = 0; t < NW; ++t) mx = fmaxf(mx, s_wmax[t]);
    thr = piv_rtol * mx;
  }
  bool bad = false;
  for (int k = 0; k < n; ++k) {
    const int buf = k & 1;
    // the pivot row: the best of the warps' candidates, ties to the lower row
    float best = lane < NW ? candv[buf][lane] : -1.f;
    int bi = lane < NW ? candi[buf][lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > thr) || !isfinite(best)) { bad = true; break; }  // the same in every thread
    const int p = bi;
    const float pinv = __frcp_rn(colv[buf][p]);
    const int wp = p % NW, rp = p / NW;
    // the pivot row, from the warp that owns it
    if (w == wp) {
      used |= 1u << rp;
#pragma unroll
      for (int r = 0; r < RPW; ++r)
        if (r == rp) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) rowv[lane + 32 * c] = M[r][c];
        }
    }
    if (tid == 0) { piv[k] = p; stepof[p] = k; }
    __syncthreads();
    float rj[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = lane + 32 * c;
      rj[c] = (j == k ? 1.f : rowv[j]) * pinv;
    }
    // column k becomes -M_ik / M_pk: cleared here, the update below fills it
    if (lane == (k & 31)) {
      const int ck = k >> 5;
#pragma unroll
      for (int c = 0; c < CPL; ++c)
        if (c == ck) {
#pragma unroll
          for (int r = 0; r < RPW; ++r) M[r][c] = 0.f;
        }
    }
    // M_ij -= M_ik M_pj / M_pk off the pivot row
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int i = w + NW * r;
      const float ci = i == p ? 0.f : colv[buf][i];
#pragma unroll
      for (int c = 0; c < CPL; ++c) M[r][c] = fmaf(-ci, rj[c], M[r][c]);
    }
    // the pivot row becomes M_pj / M_pk, and 1 / M_pk at k
    if (w == wp) {
#pragma unroll
      for (int r = 0; r < RPW; ++r)
        if (r == rp) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) M[r][c] = rj[c];
        }
    }
    if (k + 1 < n) publish(k + 1, buf ^ 1);
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicOr(singular, 1);
    return;
  }
  // inv[step(i)][p_j] = M_ij; out[c][r] = inv[r][c]: stage[p_j][step(i)], rows
  // padded to n + 1 so that a warp's scattered rows p_j fall in different banks
  const int ld = n + 1;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int i = w + NW * r;
    if (i >= n) continue;
    const int si = stepof[i];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = lane + 32 * c;
      if (j < n) stage[piv[j] * ld + si] = M[r][c];
    }
  }
  __syncthreads();
  TS* o = out + e * (long long)n * n;
  for (int row = w; row < n; row += NW)
    for (int col = lane; col < n; col += 32) o[(long long)row * n + col] = (TS)stage[row * ld + col];
}

// The same register-resident Gauss-Jordan for blocks of up to 256 x 256, whose
// 65,536 entries exceed one SM's registers: each block is spread over a
// cluster of two CTAs on two SMs. Global row i lives in CTA i % 2 as local row
// i / 2 (warp w: local rows w + 16 r, r < 8; lane l: columns l + 32 c, c < 8).
// Each CTA publishes its rows' part of the pivot column in its own shared
// memory, with each warp's best unused row and that row's values; after a
// cluster barrier every warp of both CTAs reads both halves (the other through
// distributed shared memory), finds the same pivot and reads the pivot row
// from the owning CTA: one cluster barrier per step. The inverse is staged in
// the shared memory of the CTA that owns each output row (out[c][.] in CTA
// c % 2) and written out coalesced. Singular pivots and the output order are
// as in gj_invert_regs.
constexpr int kGjcNW = 16, kGjcRPW = 8, kGjcCPL = 8;
constexpr int kGjcRows = kGjcNW * kGjcRPW;  // local rows per CTA (128)
constexpr int kGjcCols = 32 * kGjcCPL;      // columns (256)

template <class TS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGjcNW * 32, 1)
gj_invert_cluster(const float* __restrict__ blocks, TS* __restrict__ out, int n,
                  int* __restrict__ singular) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), peer = rank ^ 1;
  extern __shared__ __align__(16) unsigned char gcs[];
  float* stage = reinterpret_cast<float*>(gcs);   // [(n + 1) / 2][n]: out rows c with c % 2 == rank
  __shared__ float colv[2][kGjcRows];
  __shared__ float candv[2][kGjcNW];   // per warp: largest |M_ik| over its unused rows
  __shared__ int candi[2][kGjcNW];     //           and that (global) row
  __shared__ float rowc[2][kGjcNW][kGjcCols];   //      and that row's values
  __shared__ int piv[kGjcCols], stepof[2 * kGjcRows];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long e = blockIdx.x / 2;
  const float* src = blocks + e * (long long)n * n;
  // the peer's copies ([2][...] arrays, row-major as here)
  const float* colv_p = cluster.map_shared_rank(&colv[0][0], peer);
  const float* candv_p = cluster.map_shared_rank(&candv[0][0], peer);
  const int* candi_p = cluster.map_shared_rank(&candi[0][0], peer);
  const float* rowc_p = cluster.map_shared_rank(&rowc[0][0][0], peer);
  float* stage_p = cluster.map_shared_rank(stage, peer);
  float M[kGjcRPW][kGjcCPL];
  // global row of local row li in this CTA: 2 li + rank
#pragma unroll
  for (int r = 0; r < kGjcRPW; ++r) {
    const int i = 2 * (w + kGjcNW * r) + rank;
#pragma unroll
    for (int c = 0; c < kGjcCPL; ++c) {
      const int j = lane + 32 * c;
      M[r][c] = (i < n && j < n) ? src[(long long)i * n + j] : (i == j ? 1.f : 0.f);
    }
  }
  unsigned used = 0u;
  // publish column kc (from lane kc % 32 of every warp): its values, the
  // warp's pivot candidate among its unused rows and that row's values, so
  // that the step that picks it needs one cluster barrier, not two
  auto publish = [&](int kc, int buf) {
    const int src_lane = kc & 31;
    int br = -1;  // the candidate's local row slot r
    if (lane == src_lane) {
      const int cc = kc >> 5;
      float best = -1.f;
#pragma unroll
      for (int c = 0; c < kGjcCPL; ++c)
        if (c == cc) {
#pragma unroll
          for (int r = 0; r < kGjcRPW; ++r) {
            const int li = w + kGjcNW * r, i = 2 * li + rank;
            const float v = M[r][c];
            colv[buf][li] = v;
            const float av = (i < n && !((used >> r) & 1u)) ? fabsf(v) : -1.f;
            if (av > best) { best = av; br = r; }   // rows ascend with r: ties keep the lower
          }
        }
      candv[buf][w] = best;
      candi[buf][w] = 2 * (w + kGjcNW * (br < 0 ? 0 : br)) + rank;
    }
    br = __shfl_sync(0xffffffffu, br, src_lane);
    if (br >= 0) {
#pragma unroll
      for (int r = 0; r < kGjcRPW; ++r)
        if (r == br) {
#pragma unroll
          for (int c = 0; c < kGjcCPL; ++c) rowc[buf][w][lane + 32 * c] = M[r][c];
        }
    }
  };
  publish(0, 0);
  cluster.sync();
  bool bad = false;
  for (int k = 0; k < n; ++k) {
    const int buf = k & 1;
    // pivot: the best of both CTAs' warp candidates, ties to the lower row
    const int q = lane & (kGjcNW - 1);
    const bool mine = (lane < kGjcNW) == (rank == 0);   // lanes < 16: CTA 0's warps
    float best = mine ? candv[buf][q] : candv_p[buf * kGjcNW + q];
    int bi = mine ? candi[buf][q] : candi_p[buf * kGjcNW + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (!(best > 0.f) || !isfinite(best)) { bad = true; break; }  // the same in both CTAs
    const int p = bi, owner = p & 1, lp = p >> 1;
    const float pivv = owner == rank ? colv[buf][lp] : colv_p[buf * kGjcRows + lp];
    const float pinv = __frcp_rn(pivv);
    const int wp = lp % kGjcNW;
    const bool own = owner == rank && w == wp;
    const int rp = lp / kGjcNW;
    if (own) used |= 1u << rp;
    if (tid == 0) { piv[k] = p; stepof[p] = k; }
    // the pivot row: its warp's published candidate row, in the owning CTA
    const float* rsrc = (owner == rank ? &rowc[0][0][0] : rowc_p) +
                        ((size_t)buf * kGjcNW + wp) * kGjcCols;
    float rj[kGjcCPL];
#pragma unroll
    for (int c = 0; c < kGjcCPL; ++c) {
      const int j = lane + 32 * c;
      rj[c] = (j == k ? 1.f : rsrc[j]) * pinv;
    }
    // column k becomes -M_ik / M_pk: cleared here, the update below fills it
    if (lane == (k & 31)) {
      const int ck = k >> 5;
#pragma unroll
      for (int c = 0; c < kGjcCPL; ++c)
        if (c == ck) {
#pragma unroll
          for (int r = 0; r < kGjcRPW; ++r) M[r][c] = 0.f;
        }
    }
    // M_ij -= M_ik M_pj / M_pk off the pivot row
#pragma unroll
    for (int r = 0; r < kGjcRPW; ++r) {
      const int li = w + kGjcNW * r, i = 2 * li + rank;
      const float ci = i == p ? 0.f : colv[buf][li];
#pragma unroll
      for (int c = 0; c < kGjcCPL; ++c) M[r][c] = fmaf(-ci, rj[c], M[r][c]);
    }
    // the pivot row becomes M_pj / M_pk, and 1 / M_pk at k
    if (own) {
#pragma unroll
      for (int r = 0; r < kGjcRPW; ++r)
        if (r == rp) {
#pragma unroll
          for (int c = 0; c < kGjcCPL; ++c) M[r][c] = rj[c];
        }
    }
    if (k + 1 < n) publish(k + 1, buf ^ 1);
    cluster.sync();
  }
  if (bad) {
    if (tid == 0 && rank == 0) atomicOr(singular, 1);
    cluster.sync();  // no CTA leaves while the other may still read its shared memory
    return;
  }
  // inv[step(i)][p_j] = M_ij -> out[p_j][step(i)], staged in CTA p_j % 2
#pragma unroll
  for (int r = 0; r < kGjcRPW; ++r) {
    const int i = 2 * (w + kGjcNW * r) + rank;
    if (i >= n) continue;
    const int si = stepof[i];
#pragma unroll
    for (int c = 0; c < kGjcCPL; ++c) {
      const int j = lane + 32 * c;
      if (j < n) {
        const int oc = piv[j];
        float* dst = (oc & 1) == rank ? stage : stage_p;
        dst[(oc >> 1) * n + si] = M[r][c];
      }
    }
  }
  cluster.sync();
  TS* o = out + e * (long long)n * n;
  const int nrow = (n - rank + 1) / 2;  // output rows c = 2 q + rank < n
  for (int t = tid; t < nrow * n; t += kGjcNW * 32) {
    const int q = t / n, r = t % n;
    o[(long long)(2 * q + rank) * n + r] = (TS)stage[q * n + r];
  }
}

// y_e = Binv_e x_e with the inverse stored transposed (BT[c][r]); accumulation in TA.
template <class TS, class TA, class TV>
__global__ void bj_apply_kernel(const TS* __restrict__ BT, const TV* __restrict__ x,
                                TV* __restrict__ y, int n, int NF, int Np, long long EN,
                                long long bstride, int shared_blocks) {
  extern __shared__ __align__(16) unsigned char xsm_raw[];
  TA* xs = reinterpret_cast<TA*>(xsm_raw);
  const long long e = blockIdx.x;
  const int b = blockIdx.y;
  const long long E = EN / Np;
  const TV* xb = x + b * bstride;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const int f = c / Np, i = c % Np;
    xs[c] = (TA)xb[f * EN + e * Np + i];
  }
  __syncthreads();
  const TS* B = BT + ((long long)(shared_blocks ? 0 : b) * E + e) * (long long)n * n;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    // eight independent partial sums keep eight loads per thread in flight
    TA acc[8] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
    int c = 0;
    for (; c + 8 <= n; c += 8) {
      TS bv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) bv[k] = B[(long long)(c + k) * n + r];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += (TA)bv[k] * xs[c + k];
    }
    for (; c < n; ++c) acc[0] += (TA)B[(long long)c * n + r] * xs[c];
    const TA s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    const int f = r / Np, i = r % Np;
    y[b * bstride + f * EN + e * Np + i] = (TV)s;
  }
}

// ------------------------------------------------- graph-driven Newton iteration
// Device-side control of a Newton solve whose iterations run as one CUDA graph
// launch with conditional WHILE nodes (the FGMRES restart cycles, the
// backtracking line search, and the Newton steps between preconditioner
// setups): the host takes part once per setup.
struct NewtonCtl {
  int it;          // Newton iterations of the solve
  int since;       // Newton iterations since the last preconditioner setup
  int kry_total;   // FGMRES iterations of the solve
  int kry_solve;   // FGMRES iterations of the current inner solve
  int bt;          // backtracking steps of the current line search
  int nonfinite;   // a non-finite residual or Krylov value
  int kfail;       // an inner solve stopped at its iteration limit
  int pad;
  double hist[64]; // largest ||R|| after each Newton iteration
};

struct NewtonDev {
  double *rn, *tol, *lam, *rnew2, *negmask;  // [B]
  int *mask, *acc;                           // [B]
  NewtonCtl* c;
};

__global__ void ng_arm(cudaGraphConditionalHandle h) { cudaGraphSetConditional(h, 1u); }

// Start of a Newton iteration: the running points (||R|| above tolerance), the
// right-hand-side scale -1 / 0, full steps for the line search.
__global__ void ng_begin(NewtonDev A, int B) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int run = A.rn[b] > A.tol[b] ? 1 : 0;
    A.mask[b] = run;
    A.negmask[b] = run ? -1.0 : 0.0;
    A.lam[b] = run ? 1.0 : 0.0;
    A.acc[b] = run ? 0 : 1;
  }
  if (threadIdx.x == 0) { A.c->kry_solve = 0; A.c->bt = 0; }
}

// After an FGMRES restart cycle: count its iterations (up to each point's
// convergence when the cycle finished every point), and continue while a point
// runs, the inner limit is not reached and nothing is non-finite.
__global__ void ng_krylov_count(KrylovDev K, NewtonDev A, const int* __restrict__ dflag, int B,
                                int m, int max_it, cudaGraphConditionalHandle h) {
  __shared__ int s_used;
  if (threadIdx.x == 0) s_used = 0;
  __syncthreads();
  int running = 0, used = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const int j = K.jconv[b];
    if (j == -1) running = 1;
    if (j >= 0) used = max(used, j + 1);
  }
  atomicMax(&s_used, used);
  running = __syncthreads_or(running);
  if (threadIdx.x == 0) {
    const int its = A.c->kry_solve + (running ? m : s_used);
    A.c->kry_solve = its;
    const int nonf = dflag[1];
    if (nonf) A.c->nonfinite = 1;
    if (running && its >= max_it) A.c->kfail = 1;
    cudaGraphSetConditional(h, (running && its < max_it && !nonf) ? 1u : 0u);
  }
}

// Armijo test of every point still searching: accept, or halve its step.
__global__ void ng_ls_accept(NewtonDev A, int B, double c_armijo, int max_bt,
                             cudaGraphConditionalHandle h) {
  const int bt = A.c->bt;
  int any = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (A.acc[b]) continue;
    const double rnew = sqrt(A.rnew2[b]);
    if (rnew <= (1.0 - c_armijo * A.lam[b]) * A.rn[b] || bt >= max_bt) {
      A.acc[b] = 1;
    } else {
      A.lam[b] *= 0.5;
      any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    A.c->bt = bt + 1;
    cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

// End of a Newton iteration: the new norms, the history, and whether to go on
// (a point above tolerance, under the iteration limit, and the preconditioner
// still within its lag).
__global__ void ng_end(NewtonDev A, int B, int max_it, int per_setup,
                       cudaGraphConditionalHandle h) {
  __shared__ unsigned long long s_max;
  if (threadIdx.x == 0) s_max = 0ull;
  __syncthreads();
  int any = 0, nonf = 0;
  double mx = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const double r = sqrt(A.rnew2[b]);
    A.rn[b] = r;
    if (!isfinite(r)) nonf = 1;
    if (r > A.tol[b]) any = 1;
    mx = fmax(mx, isnan(r) ? INFINITY : r);
  }
  atomicMax(&s_max, (unsigned long long)__double_as_longlong(mx));  // non-negative: bits ordered
  any = __syncthreads_or(any);
  nonf = __syncthreads_or(nonf);
  if (threadIdx.x == 0) {
    NewtonCtl* c = A.c;
    c->kry_total += c->kry_solve;
    c->it += 1;
    c->since += 1;
    if (c->it < 64) c->hist[c->it] = __longlong_as_double((long long)s_max);
    if (nonf) c->nonfinite = 1;
    const bool go = any && c->it < max_it && c->since < per_setup && !c->nonfinite && !c->kfail;
    cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

}  // namespace enp

// ====================================================================== host
using enp::OpParams;

namespace {

int grid_for(long long n, int threads = 256) {
  long long g = (n + threads - 1) / threads;
  return (int)std::max(1LL, std::min(g, 152LL * 8));
}

struct SolverState {
  // block-Jacobi
  int nb = 0;
  int storage = -1;               // 0 f64, 1 f32, 2 bf16
  double* blocks = nullptr;       // [E][nb][nb] assembled blocks of one point (FP64 setup)
  size_t blocks_count = 0;
  float* blocks32 = nullptr;      // [E][nb][nb] assembled blocks of one point (FP32 setup)
  float* u32 = nullptr;           // the linearisation point in FP32
  size_t blocks32_count = 0, u32_count = 0;
  void* binv = nullptr;           // [sets][E][nb][nb] inverse, transposed, in `storage`
  int binv_sets = 0;              // batch, or 1 when one set is shared
  void* gj_work = nullptr;        // global work for blocks too large for shared memory
  size_t gj_work_bytes = 0;
  int* d_flag = nullptr;
  // reductions
  double* part = nullptr;
  size_t part_count = 0;
  double* dsmall = nullptr;       // device small vectors
  size_t dsmall_count = 0;
  // Krylov workspace
  void* V = nullptr;
  void* Z = nullptr;
  size_t krylov_bytes = 0;
  double* dRdtheta = nullptr;     // parameter Jacobian workspace [n_theta][batch][n]
  size_t dRdtheta_count = 0;
  // CUDA graph of one FGMRES restart cycle, on handle-owned copies of the inputs
  cudaStream_t gstream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  void* gbuf = nullptr;           // [3][B][n] of the Krylov type: u_lin, b, x
  size_t gbuf_bytes = 0;
  const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};
  int gkey_i[4] = {0, 0, 0, 0};
  // graph-driven Newton iteration (enp_newton_opts.device_loop): the graph, the
  // streams its nested bodies were captured on, handle-owned copies of the
  // Newton vectors, the device control block, and the key it was captured for
  cudaStream_t nstream[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t nexec = nullptr;
  void* nbuf = nullptr;           // u, r, du, ut, rt (FP64) [+ u, b, x in FP32]
  size_t nbuf_bytes = 0;
  void* nsmall = nullptr;         // NewtonCtl + per-point arrays
  size_t nsmall_bytes = 0;
  std::vector<char> nkey;
  // preconditioner generation: bumped whenever its configuration changes or a
  // buffer it reads is reallocated, so that a captured FGMRES cycle is replayed
  // only with the preconditioner it was captured with
  unsigned long long pc_gen = 1, gkey_gen = 0;
  // two-level preconditioner: element-mean potential correction
  int sweep_mode = 2;             // downwind block Gauss-Seidel: 0 off, 1 on, 2 automatic
  bool potential_only = false;    // the potential rows alone (enp_initial_guess)
  int pc_shared = -1;             // >= 0: one set of block inverses, of this operating
                                  // point, for the whole batch (enp_set_shared_blocks)
  int pc_shared_built = 0;        // the stored inverses are one shared set
  bool sweep_ready = false;
  int sweep_axis = 0, sweep_dir = 1;
  double* upc64 = nullptr;        // the linearisation point of the last setup
  float* upc32 = nullptr;
  size_t upc64_count = 0, upc32_count = 0;
  bool coarse = false;            // enabled by enp_set_preconditioner
  int coarse_cycles = 1;          // V-cycles per application (enp_set_coarse_options)
  int coarse_smooth = 2;          // Gauss-Seidel sweeps before and after the coarse step
  float coarse_omega = 1.8f;      // prolongation over-correction
  float* cx_acc = nullptr;        // [B][n0] accumulated level-0 solution (cycles > 1)
  float* cb_keep = nullptr;       // [B][n0] level-0 right-hand side (cycles > 1)
  size_t cx_acc_count = 0, cb_keep_count = 0;
  bool coarse_ready = false;
  struct Level { int nx, ny, nz, n; double* A; float *A32, *x, *b, *r; };  // A: FP64 stencil
  std::vector<Level> levels;      // level 0: the element grid
  bool coarse_direct = false;     // coarsest level solved by its dense inverse
  double* cdense = nullptr;       // [B][n][n] coarsest matrix
  float* cinv = nullptr;          // [B][n][n] its inverse, transposed, in FP32
  size_t cdense_count = 0, cinv_count = 0;
  double* cwork = nullptr;        // Jv scratch for the coarse setup [B][n]
  size_t cwork_count = 0;
};

}  // namespace

struct enp_solver_ext {
  SolverState s;
};

namespace {

SolverState& state_of(enp_handle h) {
  if (!h->solver) h->solver = new enp_solver_ext();
  return h->solver->s;
}

enp_status cuda_err(enp_handle h, cudaError_t e, const char* what) {
  h->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? ENP_ERR_OOM : ENP_ERR_CUDA;
}

template <class P>
cudaError_t ensure(P** p, size_t& have, size_t want_count) {
  if (*p && have >= want_count) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  have = 0;
  cudaError_t e = cudaMalloc((void**)p, want_count * sizeof(P));
  if (e == cudaSuccess) have = want_count;
  return e;
}

// J(u) v as the solvers apply it; in potential-only mode (the initial guess)
// the species rows are the identity.
template <class TV>
cudaError_t apply_jv(enp_handle h, const OpParams& P, const TV* ulin, const TV* v, TV* out, int B) {
  cudaError_t e = enp::launch_op<TV>(enp::kJvp, P, h->d_tab, ulin, v, out, B, h->stream);
  if (e == cudaSuccess && state_of(h).potential_only) {
    const long long EN = (long long)P.E * P.Np;
    enp::species_rows_copy<TV><<<grid_for((P.NF - 1) * EN * B), 256, 0, h->stream>>>(
        v, out, EN, P.NF, P.batch_stride, B);
    e = cudaGetLastError();
  }
  return e;
}

// R(u) as the Newton solver evaluates it; in potential-only mode the species
// rows are c_k - c_k^in.
cudaError_t apply_residual(enp_handle h, const double* u, double* r, int B) {
  const OpParams& P = h->prm;
  cudaError_t e = enp::launch_op<double>(enp::kResidual, P, h->d_tab, u, nullptr, r, B, h->stream);
  if (e == cudaSuccess && state_of(h).potential_only) {
    const long long EN = (long long)P.E * P.Np;
    enp::species_rows_offset<<<grid_for((P.NF - 1) * EN * B), 256, 0, h->stream>>>(
        u, r, EN, P.NF, P.batch_stride, B, P.cin[0], P.cin[1], P.cin[2]);
    e = cudaGetLastError();
  }
  return e;
}

// Partials of <V_i, w>_b (i < nd) into S.part; *nparts = the partials per dot.
template <class T>
cudaError_t dot_partials(enp_handle h, const T* V, long long vstride, int nd, const T* w,
                         int* nparts) {
  SolverState& S = state_of(h);
  const long long n = h->n_dof;
  const int B = h->batch;
  cudaError_t e = ensure(&S.part, S.part_count, (size_t)B * std::max(nd, 1) * enp::kRedBlocks);
  if (e != cudaSuccess) return e;
  const int W = vec_width<T>(n, vstride, V, w);
  const int nb = red_blocks(n, W);
  const dim3 g(nb, B);
  if (W == 1)
    enp::multidot_partial<T, 1><<<g, enp::kRedThreads, 0, h->stream>>>(V, vstride, nd, w, n, n, S.part);
  else
    enp::multidot_partial<T, 16 / sizeof(T)><<<g, enp::kRedThreads, 0, h->stream>>>(V, vstride, nd,
                                                                                   w, n, n, S.part);
  *nparts = nb;
  return cudaGetLastError();
}

// w -= sum_i V_i h_i (h: device [B][nd]); with part, also the partials of
// ||w_new||^2 into part (their count per point in *nparts).
template <class T>
cudaError_t axpy_many(enp_handle h, const T* V, long long vstride, int nd, const double* hc, T* w,
                      double* part, int* nparts) {
  const long long n = h->n_dof;
  const int B = h->batch;
  const int W = vec_width<T>(n, vstride, V, w);
  const int nb = red_blocks(n, W);
  const dim3 g(nb, B);
  constexpr int WV = 16 / sizeof(T);
  if (part) {
    if (W == 1)
      enp::multi_axpy<T, 1, true><<<g, enp::kRedThreads, 0, h->stream>>>(V, vstride, nd, hc, w, n, n, part);
    else
      enp::multi_axpy<T, WV, true><<<g, enp::kRedThreads, 0, h->stream>>>(V, vstride, nd, hc, w, n, n, part);
    *nparts = nb;
  } else {
    if (W == 1)
      enp::multi_axpy<T, 1, false><<<g, enp::kRedThreads, 0, h->stream>>>(V, vstride, nd, hc, w, n, n, nullptr);
    else
      enp::multi_axpy<T, WV, false><<<g, enp::kRedThreads, 0, h->stream>>>(V, vstride, nd, hc, w, n, n, nullptr);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t multidot(enp_handle h, const T* V, long long vstride, int nd, const T* w,
                     double* out) {
  int np = 0;
  cudaError_t e = dot_partials<T>(h, V, vstride, nd, w, &np);
  if (e != cudaSuccess) return e;
  enp::finish_partials<<<h->batch * nd, 32, 0, h->stream>>>(state_of(h).part, np, h->batch * nd, out);
  return cudaGetLastError();
}

// Gram-Schmidt of w against V_0..V_j, twice (classical, CGS2), then ||w||^2
// and the Givens update of Arnoldi iteration j: seven launches, the partial
// sums finished inside the kernels that consume them.
template <class TV>
cudaError_t arnoldi_orthogonalise(enp_handle h, const enp::KrylovDev& K, TV* V, long long vs,
                                  int j, TV* w, int m, int* nonfinite) {
  SolverState& S = state_of(h);
  const int B = h->batch;
  const int nd = j + 1;
  cudaError_t e = cudaSuccess;
  int np = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if ((e = dot_partials<TV>(h, V, vs, nd, w, &np)) != cudaSuccess) return e;
    enp::krylov_hcol_finish<<<B * nd, 32, 0, h->stream>>>(K, S.part, np, B, m, nd, pass == 0);
    if ((e = axpy_many<TV>(h, V, vs, nd, K.dh, w, pass == 1 ? S.part : nullptr, &np)) !=
        cudaSuccess)
      return e;
  }
  enp::krylov_norm_givens<<<B, 32, 0, h->stream>>>(K, S.part, np, B, m, j, nonfinite);
  return cudaGetLastError();
}

cudaError_t small(enp_handle h, size_t count) {
  SolverState& S = state_of(h);
  return ensure(&S.dsmall, S.dsmall_count, count);
}

}  // namespace


namespace {

constexpr int kCoarsestSweeps = 100;

cudaError_t coarse_levels(enp_handle h) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  if (!S.levels.empty()) return cudaSuccess;
  int nx = P.ne[0], ny = P.ne[1], nz = P.ne[2];
  const int B = h->batch;
  while (true) {
    SolverState::Level L{nx, ny, nz, nx * ny * nz, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaError_t e = cudaMalloc(&L.A, sizeof(double) * 7 * (size_t)L.n * B);
    if (e == cudaSuccess) e = cudaMalloc(&L.A32, sizeof(float) * enp::kPack * (size_t)L.n * B);
    if (e == cudaSuccess) e = cudaMalloc(&L.x, sizeof(float) * (size_t)L.n * B);
    if (e == cudaSuccess) e = cudaMalloc(&L.b, sizeof(float) * (size_t)L.n * B);
    if (e == cudaSuccess) e = cudaMalloc(&L.r, sizeof(float) * (size_t)L.n * B);
    S.levels.push_back(L);
    if (e != cudaSuccess) return e;
    if (L.n <= enp::kCoarsestCells) break;
    nx = (nx + 1) / 2; ny = (ny + 1) / 2; nz = (nz + 1) / 2;
  }
  return cudaSuccess;
}

// A0 = P^T J_PhiPhi P from 7 coloured J v passes at u, then the hierarchy.
cudaError_t coarse_setup(enp_handle h, const double* u) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  const int B = h->batch;
  cudaError_t e = coarse_levels(h);
  if (e != cudaSuccess) return e;
  const long long ntot = h->n_dof * B;
  if ((e = ensure(&S.cwork, S.cwork_count, (size_t)2 * ntot)) != cudaSuccess) return e;
  SolverState::Level& L0 = S.levels[0];
  cudaMemsetAsync(L0.A, 0, sizeof(double) * 7 * (size_t)L0.n * B, h->stream);
  // seven J v products with the FP64 operator, or with the FP32 one when the
  // block inverses are stored in single or half precision (mixed solves)
  auto probe = [&](auto* uu, auto* v, auto* jv) -> cudaError_t {
    using T = std::remove_pointer_t<decltype(v)>;
    cudaMemsetAsync(v, 0, sizeof(T) * ntot, h->stream);
    const int gx = grid_for((long long)P.E * P.Np);
    for (int c = 0; c < 7; ++c) {
      enp::coarse_colour_vector<T><<<dim3(gx, B), 256, 0, h->stream>>>(v, P.ne[0], P.ne[1], P.ne[2],
                                                                        P.Np, P.batch_stride, P.E, c);
      cudaError_t er = enp::launch_op<T>(enp::kJvp, P, h->d_tab, uu, v, jv, B, h->stream);
      if (er != cudaSuccess) return er;
      enp::coarse_gather<T><<<dim3(grid_for(P.E), B), 256, 0, h->stream>>>(
          jv, L0.A, P.ne[0], P.ne[1], P.ne[2], P.Np, P.batch_stride, c);
    }
    return cudaGetLastError();
  };
  if (S.storage == 0) {
    e = probe(u, S.cwork, S.cwork + ntot);
  } else {
    float* w32 = reinterpret_cast<float*>(S.cwork);  // 2 ntot doubles hold 2 ntot floats
    e = probe(static_cast<const float*>(S.u32), w32, w32 + ntot);
  }
  if (e != cudaSuccess) return e;
  for (size_t l = 0; l + 1 < S.levels.size(); ++l) {
    const auto& F = S.levels[l];
    const auto& C = S.levels[l + 1];
    enp::coarse_aggregate<<<dim3(grid_for(C.n), B), 256, 0, h->stream>>>(F.A, F.nx, F.ny, F.nz, C.A,
                                                                         C.nx, C.ny, C.nz);
  }
  for (const auto& L : S.levels)
    enp::coarse_pack32<<<grid_for((long long)L.n * B), 256, 0, h->stream>>>(L.A, L.A32,
                                                                         (long long)L.n * B);
  // the coarsest level: dense inverse by Gauss-Jordan in FP64 (n <=
  // kCoarsestCells, in shared memory), stored in FP32, or Gauss-Seidel
  // smoothing if it is singular
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const auto& Lc = S.levels.back();
  const size_t nn = (size_t)Lc.n * Lc.n * B;
  if ((e = ensure(&S.cdense, S.cdense_count, nn)) != cudaSuccess) return e;
  if ((e = ensure(&S.cinv, S.cinv_count, nn)) != cudaSuccess) return e;
  enp::coarse_dense<<<B, 256, 0, h->stream>>>(Lc.A, Lc.nx, Lc.ny, Lc.nz, S.cdense);
  const int nc = Lc.n;
  const size_t smem = sizeof(double) * ((size_t)nc * (nc + 1) + 2 * nc) + sizeof(int) * nc;
  auto k = enp::gj_invert<double, float, true, double>;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return e;
  cudaMemsetAsync(S.d_flag, 0, sizeof(int), h->stream);
  // a pivot below 1e-10 of the largest entry: singular to working accuracy
  k<<<B, 512, smem, h->stream>>>(S.cdense, nullptr, S.cinv, nc, S.d_flag, 1e-10);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int flag = 0;
  if ((e = cudaMemcpyAsync(&flag, S.d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
    return e;
  S.coarse_direct = flag == 0;
  {
    const size_t n0 = (size_t)S.levels[0].n * B;
    if ((e = ensure(&S.cx_acc, S.cx_acc_count, n0)) != cudaSuccess ||
        (e = ensure(&S.cb_keep, S.cb_keep_count, n0)) != cudaSuccess)
      return e;
  }
  S.coarse_ready = true;
  return cudaSuccess;
}

void vcycle(enp_handle h, size_t l) {
  SolverState& S = state_of(h);
  const int B = h->batch;
  auto& L = S.levels[l];
  if (L.n <= enp::kTailCells && S.levels.size() <= (size_t)enp::kMaxLevels) {
    // this level and all below it in one launch
    enp::VcycleTail T{};
    T.l0 = (int)l;
    T.nl = (int)S.levels.size();
    for (size_t k = 0; k < S.levels.size(); ++k) {
      const auto& Q = S.levels[k];
      T.L[k] = enp::LevelDev{Q.nx, Q.ny, Q.nz, Q.n, Q.A32, Q.x, Q.b, Q.r};
    }
    T.inv = S.coarse_direct ? S.cinv : nullptr;
    T.smooth = S.coarse_smooth;
    T.omega = S.coarse_omega;
    T.coarsest_sweeps = kCoarsestSweeps;
    enp::coarse_vcycle_tail<<<B, enp::kTailThreads, 0, h->stream>>>(T);
    return;
  }
  if (l + 1 == S.levels.size()) {
    if (S.coarse_direct)
      enp::coarse_dense_apply<<<B, enp::kCoarsestCells, 0, h->stream>>>(S.cinv, L.b, L.n, L.x);
    else
      enp::coarse_solve_small<<<B, enp::kCoarsestCells, 0, h->stream>>>(L.A32, L.x, L.b, L.nx,
                                                                      L.ny, L.nz, kCoarsestSweeps);
    return;
  }
  const dim3 g(grid_for(L.n), B);
  cudaMemsetAsync(L.x, 0, sizeof(float) * (size_t)L.n * B, h->stream);
  for (int sw = 0; sw < S.coarse_smooth; ++sw) {
    enp::coarse_gs<<<g, 256, 0, h->stream>>>(L.A32, L.x, L.b, L.nx, L.ny, L.nz, 0);
    enp::coarse_gs<<<g, 256, 0, h->stream>>>(L.A32, L.x, L.b, L.nx, L.ny, L.nz, 1);
  }
  auto& C = S.levels[l + 1];
  enp::coarse_residual<<<g, 256, 0, h->stream>>>(L.A32, L.x, L.b, L.r, L.nx, L.ny, L.nz);
  enp::coarse_restrict<<<dim3(grid_for(C.n), B), 256, 0, h->stream>>>(L.r, L.nx, L.ny, L.nz, C.b,
                                                                      C.nx, C.ny, C.nz);
  vcycle(h, l + 1);
  enp::coarse_prolong<<<g, 256, 0, h->stream>>>(C.x, C.nx, C.ny, C.nz, L.x, L.nx, L.ny, L.nz,
                                                S.coarse_omega);
  for (int sw = 0; sw < S.coarse_smooth; ++sw) {
    enp::coarse_gs<<<g, 256, 0, h->stream>>>(L.A32, L.x, L.b, L.nx, L.ny, L.nz, 1);
    enp::coarse_gs<<<g, 256, 0, h->stream>>>(L.A32, L.x, L.b, L.nx, L.ny, L.nz, 0);
  }
}

// z += P V(P^T r): the coarse correction of the two-level preconditioner.
template <class TV>
cudaError_t coarse_apply(enp_handle h, const TV* r, TV* z) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  const int B = h->batch;
  auto& L0 = S.levels[0];
  enp::coarse_from_fine<TV><<<dim3(grid_for(32LL * P.E), B), 256, 0, h->stream>>>(r, L0.b, P.E, P.Np,
                                                                               P.batch_stride);
  vcycle(h, 0);
  if (S.coarse_cycles > 1) {
    // further cycles on the level-0 residual: x += V(b - A0 x); the buffers
    // were allocated by the setup (no allocation here: this may be captured)
    const size_t n0 = (size_t)L0.n * B;
    if (!S.cx_acc || !S.cb_keep || S.cx_acc_count < n0 || S.cb_keep_count < n0)
      return cudaErrorInvalidValue;
    cudaMemcpyAsync(S.cb_keep, L0.b, sizeof(float) * n0, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(S.cx_acc, L0.x, sizeof(float) * n0, cudaMemcpyDeviceToDevice, h->stream);
    const dim3 g0(grid_for(L0.n), B);
    for (int c = 1; c < S.coarse_cycles; ++c) {
      enp::coarse_residual<<<g0, 256, 0, h->stream>>>(L0.A32, S.cx_acc, S.cb_keep, L0.b, L0.nx,
                                                      L0.ny, L0.nz);
      vcycle(h, 0);
      enp::axpy_f32<<<grid_for((long long)n0), 256, 0, h->stream>>>(L0.x, S.cx_acc, (long long)n0);
    }
    cudaMemcpyAsync(L0.x, S.cx_acc, sizeof(float) * n0, cudaMemcpyDeviceToDevice, h->stream);
  }
  enp::coarse_to_fine<TV><<<dim3(grid_for((long long)P.E * P.Np), B), 256, 0, h->stream>>>(
      L0.x, z, P.E, P.Np, P.batch_stride);
  return cudaGetLastError();
}

}  // namespace

void enp_solver_free(enp_handle h) {
  if (!h || !h->solver) return;
  SolverState& S = h->solver->s;
  if (S.nexec) cudaGraphExecDestroy(S.nexec);
  for (auto& st : S.nstream)
    if (st) cudaStreamDestroy(st);
  cudaFree(S.nbuf); cudaFree(S.nsmall);
  cudaFree(S.blocks); cudaFree(S.binv); cudaFree(S.gj_work); cudaFree(S.d_flag);
  cudaFree(S.blocks32); cudaFree(S.u32);
  cudaFree(S.part); cudaFree(S.dsmall); cudaFree(S.V); cudaFree(S.dRdtheta);
  for (auto& L : S.levels) {
    cudaFree(L.A); cudaFree(L.A32); cudaFree(L.x); cudaFree(L.b); cudaFree(L.r);
  }
  cudaFree(S.cwork); cudaFree(S.cdense); cudaFree(S.cinv);
  cudaFree(S.cx_acc); cudaFree(S.cb_keep);
  cudaFree(S.upc64); cudaFree(S.upc32);
  if (S.gexec) cudaGraphExecDestroy(S.gexec);
  if (S.gstream) cudaStreamDestroy(S.gstream);
  cudaFree(S.gbuf);
  delete h->solver;
  h->solver = nullptr;
}

// Elements along the flow axis from which the automatic mode uses the sweep:
// on the plate reactor (Pe = 1e4) block-Jacobi is faster at 96 elements along
// the flow and the sweep 1.5x faster at 192 (one FP32 linear solve).
constexpr int kSweepAutoElements = 128;

// Whether the next setup builds the sweep, and along which axis and direction:
// the plate-flow axis in the sign of its mean speed, or the largest component
// of a constant velocity.
static bool sweep_wanted(enp_handle h) {
  SolverState& S = state_of(h);
  const auto& pd = h->prm.pd;
  double speed;
  if (pd.vel_kind == 1) {
    S.sweep_axis = pd.velA;
    S.sweep_dir = pd.vp[4] < 0.0 ? -1 : 1;
    speed = std::fabs(pd.vp[4]);
  } else {
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (std::fabs(pd.vp[d]) > std::fabs(pd.vp[ax])) ax = d;
    S.sweep_axis = ax;
    S.sweep_dir = pd.vp[ax] < 0.0 ? -1 : 1;
    speed = std::fabs(pd.vp[ax]);
  }
  if (h->prm.dim != 3 || S.sweep_mode == 0) return false;
  if (S.sweep_mode == 1) return true;
  return speed > 0.0 && h->prm.ne[S.sweep_axis] >= kSweepAutoElements;
}

extern "C" {

enp_status enp_recover_cm(enp_handle h, const double* u, double* cm) {
  if (!h || !u || !cm) return ENP_ERR_INVALID_ARG;
  const OpParams& P = h->prm;
  const long long EN = (long long)P.E * P.Np;
  double zk[3] = {0, 0, 0};
  for (int k = 0; k < P.NF - 1 && k < 3; ++k) zk[k] = P.z[k];
  enp::recover_cm_kernel<<<grid_for(EN * h->batch), 256, 0, h->stream>>>(
      u, cm, P.NF, EN, zk[0], zk[1], zk[2], 1.0 / P.z[P.NF - 1], P.batch_stride, h->batch);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "recover_cm");
}

enp_status enp_inner_product(enp_handle h, const double* x, const double* y, double* out) {
  if (!h || !x || !y || !out) return ENP_ERR_INVALID_ARG;
  cudaError_t e = small(h, (size_t)h->batch);
  if (e == cudaSuccess) e = multidot<double>(h, x, 0, 1, y, state_of(h).dsmall);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, state_of(h).dsmall, sizeof(double) * h->batch, cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "inner_product");
}

enp_status enp_block_diagonal(enp_handle h, const double* u, double* blocks) {
  if (!h || !u || !blocks) return ENP_ERR_INVALID_ARG;
  const OpParams& P = h->prm;
  const int nb = P.NF * P.Np;
  const long long bsz = (long long)P.E * nb * nb;
  for (int b = 0; b < h->batch; ++b) {
    OpParams Pb = P;
    if (P.phiapp_batch) Pb.phiapp_batch = P.phiapp_batch + 4 * b;
    cudaError_t e = enp::launch_op<double>(enp::kBlockCol, Pb, h->d_tab, u + b * P.batch_stride,
                                           nullptr, blocks + b * bsz, nb, h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "block columns");
  }
  return ENP_OK;
}

enp_status enp_block_jacobi_setup(enp_handle h, const double* u, int storage) {
  // buffers the preconditioner's apply reads; a reallocation invalidates any
  // captured FGMRES cycle
  auto pc_ptrs = [](const SolverState& Q) {
    return std::vector<const void*>{Q.binv, Q.cinv, Q.upc64, Q.upc32, Q.cx_acc, Q.cb_keep,
                                    Q.levels.empty() ? nullptr : (const void*)Q.levels[0].A32};
  };
  if (!h || !u || storage < 0 || storage > 2) return ENP_ERR_INVALID_ARG;
  SolverState& S = state_of(h);
  const std::vector<const void*> pc_before = pc_ptrs(S);
  const OpParams& P = h->prm;
  const int nb = P.NF * P.Np;
  const size_t nn = (size_t)nb * nb;
  const bool f64 = storage == 0;  // FP64 storage: FP64 assembly and inversion; else FP32
  // one set of inverses per operating point, or (pc_shared >= 0) one set, of
  // that point, for the whole batch; either way the blocks are assembled and
  // inverted one operating point at a time, so the assembly staging holds one
  // point's blocks
  const int shared = S.pc_shared >= 0 && S.pc_shared < h->batch ? 1 : 0;
  const int nsets = shared ? 1 : h->batch;
  const long long nblk = (long long)P.E;  // blocks per set
  cudaError_t e;
  const size_t esz = storage == 0 ? 8 : (storage == 1 ? 4 : 2);
  if (!S.binv || S.nb != nb || S.storage != storage || S.binv_sets != nsets) {
    cudaFree(S.binv);
    S.binv = nullptr;
    S.binv_sets = 0;
    e = cudaMalloc(&S.binv, esz * nn * nblk * nsets);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc block inverses");
    S.binv_sets = nsets;
  }
  if (!S.d_flag) {
    e = cudaMalloc(&S.d_flag, sizeof(int));
    if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc flag");
  }
  if (f64) {
    if (!S.blocks || S.nb != nb || S.blocks_count < nn * nblk) {
      cudaFree(S.blocks);
      S.blocks = nullptr;
      S.blocks_count = 0;
      e = cudaMalloc(&S.blocks, sizeof(double) * nn * nblk);
      if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc blocks");
      S.blocks_count = nn * nblk;
    }
  } else {
    const long long ntot = h->n_dof * h->batch;
    if ((e = ensure(&S.blocks32, S.blocks32_count, nn * nblk)) != cudaSuccess ||
        (e = ensure(&S.u32, S.u32_count, (size_t)ntot)) != cudaSuccess)
      return cuda_err(h, e, "cudaMalloc FP32 blocks");
    enp::convert_kernel<double, float><<<grid_for(ntot), 256, 0, h->stream>>>(u, S.u32, ntot);
  }
  S.nb = nb;
  S.storage = storage;
  S.pc_shared_built = shared;
  cudaMemsetAsync(S.d_flag, 0, sizeof(int), h->stream);
  const size_t telt = f64 ? 8 : 4;
  const size_t smem_full = telt * ((size_t)nb * (nb + 1) + 2 * nb) + sizeof(int) * nb;
  const bool in_smem = smem_full <= 200 * 1024;
  const int threads = 512;
  // the global-memory work copy serves only the generic kernel on blocks too
  // large for shared memory (FP64 beyond 160, FP32 beyond 256 unknowns)
  const bool generic = f64 || nb > enp::kGjcCols;
  if (generic && !in_smem) {
    e = ensure((char**)&S.gj_work, S.gj_work_bytes, telt * (size_t)nb * (nb + 1) * nblk);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc inversion work");
  }
  const size_t smem = in_smem ? smem_full : telt * 2 * nb + sizeof(int) * nb;
  for (int set = 0; set < nsets; ++set) {
    const int b = shared ? S.pc_shared : set;
    OpParams Pb = P;
    if (P.phiapp_batch) Pb.phiapp_batch = P.phiapp_batch + 4 * b;
    // assemble operating point b's blocks: column j of every block per grid.y
    if (f64) {
      e = enp::launch_op<double>(enp::kBlockCol, Pb, h->d_tab, u + b * P.batch_stride, nullptr,
                                 S.blocks, nb, h->stream);
      if (e != cudaSuccess) return cuda_err(h, e, "block columns");
      if (S.potential_only)
        enp::block_species_identity<double><<<grid_for((long long)(nb - P.Np) * nb * nblk), 256, 0,
                                              h->stream>>>(S.blocks, nblk, nb, P.Np);
    } else {
      e = enp::launch_op<float>(enp::kBlockCol, Pb, h->d_tab, S.u32 + b * P.batch_stride, nullptr,
                                S.blocks32, nb, h->stream);
      if (e != cudaSuccess) return cuda_err(h, e, "FP32 block columns");
      if (S.potential_only)
        enp::block_species_identity<float><<<grid_for((long long)(nb - P.Np) * nb * nblk), 256, 0,
                                             h->stream>>>(S.blocks32, nblk, nb, P.Np);
    }
    void* out = (char*)S.binv + esz * nn * nblk * set;
#define ENP_GJ(T, TS, SM, TB, SRC)                                                              \
  {                                                                                             \
    auto k = enp::gj_invert<T, TS, SM, TB>;                                                     \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
    if (e == cudaSuccess) {                                                                     \
      k<<<(unsigned)nblk, threads, smem, h->stream>>>(SRC, (T*)S.gj_work, (TS*)out, nb,         \
                                                      S.d_flag, T(0));                          \
      e = cudaGetLastError();                                                                   \
    }                                                                                           \
  }
  // FP32 inversion of blocks up to 192 x 192: the register-resident kernel
#define ENP_GJR(TS, NW, RPW, CPL)                                                                 \
  {                                                                                               \
    auto k = enp::gj_invert_regs<float, TS, NW, RPW, CPL>;                                        \
    const size_t sm = sizeof(float) * (size_t)nb * (nb + 1);                                      \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);            \
    if (e == cudaSuccess) {                                                                       \
      k<<<(unsigned)nblk, NW * 32, sm, h->stream>>>(S.blocks32, (TS*)out, nb, S.d_flag, 0.f);     \
      e = cudaGetLastError();                                                                     \
    }                                                                                             \
  }
// FP32 inversion of blocks up to 256 x 256: a two-CTA cluster per block
#define ENP_GJC(TS)                                                                               \
  {                                                                                               \
    auto k = enp::gj_invert_cluster<TS>;                                                          \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);            \
    if (e == cudaSuccess) {                                                                       \
      k<<<(unsigned)(2 * nblk), enp::kGjcNW * 32, sm, h->stream>>>(S.blocks32, (TS*)out, nb,      \
                                                                  S.d_flag);                      \
      e = cudaGetLastError();                                                                     \
    }                                                                                             \
  }
#define ENP_GJR_ANY(TS)                                          \
  if (nb <= 32) ENP_GJR(TS, 4, 8, 1)                             \
  else if (nb <= 64) ENP_GJR(TS, 8, 8, 2)                        \
  else if (nb <= 96) ENP_GJR(TS, 8, 12, 3)                       \
  else if (nb <= 128) ENP_GJR(TS, 16, 8, 4)                      \
  else ENP_GJR(TS, 16, 12, 6)
    const bool regs = !f64 && nb <= 192;
    const bool clus = !f64 && !regs && nb <= enp::kGjcCols;
    if (regs) {
      if (storage == 1) ENP_GJR_ANY(float)
      else ENP_GJR_ANY(__nv_bfloat16)
    } else if (clus) {
      const size_t sm = sizeof(float) * (size_t)((nb + 1) / 2) * nb;
      if (storage == 1) ENP_GJC(float) else ENP_GJC(__nv_bfloat16)
    } else if (storage == 0) {
      if (in_smem) ENP_GJ(double, double, true, double, S.blocks) else ENP_GJ(double, double, false, double, S.blocks)
    } else if (storage == 1) {
      if (in_smem) ENP_GJ(float, float, true, float, S.blocks32) else ENP_GJ(float, float, false, float, S.blocks32)
    } else {
      if (in_smem) ENP_GJ(float, __nv_bfloat16, true, float, S.blocks32)
      else ENP_GJ(float, __nv_bfloat16, false, float, S.blocks32)
    }
#undef ENP_GJ
#undef ENP_GJC
#undef ENP_GJR_ANY
#undef ENP_GJR
    if (e != cudaSuccess) break;
  }
  if (e != cudaSuccess) return cuda_err(h, e, "block inversion");
  int flag = 0;
  e = cudaMemcpyAsync(&flag, S.d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_err(h, e, "block inversion sync");
  if (flag) {
    h->err = "singular or non-finite element block";
    return ENP_ERR_NONFINITE;
  }
  if (S.coarse) {
    if ((e = coarse_setup(h, u)) != cudaSuccess) return cuda_err(h, e, "coarse setup");
  }
  S.sweep_ready = false;
  if (sweep_wanted(h)) {
    // the sweep's upstream couplings are J v face terms at this u: keep a copy
    const long long ntot = h->n_dof * h->batch;
    if ((e = ensure(&S.upc64, S.upc64_count, (size_t)ntot)) != cudaSuccess ||
        (e = ensure(&S.upc32, S.upc32_count, (size_t)ntot)) != cudaSuccess)
      return cuda_err(h, e, "cudaMalloc sweep state");
    cudaMemcpyAsync(S.upc64, u, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, h->stream);
    enp::convert_kernel<double, float><<<grid_for(ntot), 256, 0, h->stream>>>(u, S.upc32, ntot);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(h, e, "sweep setup");
    S.sweep_ready = true;
  }
  if (pc_ptrs(S) != pc_before) ++S.pc_gen;
  return ENP_OK;
}

}  // extern "C"

// Apply the stored block inverse to a vector of type TV (double or float).
template <class TV>
static cudaError_t bj_apply_plain(enp_handle h, const TV* x, TV* y);

// The preconditioner: block-Jacobi, plus the coarse potential correction when
// the two-level preconditioner is enabled and set up.
template <class TV>
static cudaError_t sweep_apply(enp_handle h, const TV* x, TV* z);

template <class TV>
static cudaError_t bj_apply_any(enp_handle h, const TV* x, TV* y) {
  SolverState& S = state_of(h);
  cudaError_t e = S.sweep_ready ? sweep_apply<TV>(h, x, y) : bj_apply_plain<TV>(h, x, y);
  if (e == cudaSuccess && S.coarse && S.coarse_ready) e = coarse_apply<TV>(h, x, y);
  return e;
}

template <class TV>
static cudaError_t bj_apply_plain(enp_handle h, const TV* x, TV* y) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  const int nb = S.nb;
  const long long EN = (long long)P.E * P.Np;
  dim3 g(P.E, h->batch);
  int threads = std::min(256, ((nb + 31) / 32) * 32);
  if (S.storage == 0) {
    size_t sm = sizeof(double) * nb;
    enp::bj_apply_kernel<double, double, TV><<<g, threads, sm, h->stream>>>(
        (const double*)S.binv, x, y, nb, P.NF, P.Np, EN, P.batch_stride, S.pc_shared_built);
  } else if (S.storage == 1) {
    size_t sm = sizeof(float) * nb;
    enp::bj_apply_kernel<float, float, TV><<<g, threads, sm, h->stream>>>(
        (const float*)S.binv, x, y, nb, P.NF, P.Np, EN, P.batch_stride, S.pc_shared_built);
  } else {
    size_t sm = sizeof(float) * nb;
    enp::bj_apply_kernel<__nv_bfloat16, float, TV><<<g, threads, sm, h->stream>>>(
        (const __nv_bfloat16*)S.binv, x, y, nb, P.NF, P.Np, EN, P.batch_stride, S.pc_shared_built);
  }
  return cudaGetLastError();
}

// Downwind block Gauss-Seidel: z = (D + L)^-1 x with D the element blocks and L
// the couplings of each element to its upstream neighbour along the flow axis;
// the element planes are solved in flow order, one launch per plane, each
// element evaluating its upstream face term from the plane solved before.
template <class TV>
static cudaError_t sweep_apply(enp_handle h, const TV* x, TV* z) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  const int B = h->batch;
  const long long ntot = h->n_dof * B;
  cudaError_t e = cudaMemsetAsync(z, 0, sizeof(TV) * ntot, h->stream);
  if (e != cudaSuccess) return e;
  const int a = S.sweep_axis, dir = S.sweep_dir;
  const int nk = P.ne[a];
  const TV* upc = std::is_same<TV, double>::value ? reinterpret_cast<const TV*>(S.upc64)
                                                  : reinterpret_cast<const TV*>(S.upc32);
  for (int step = 0; step < nk; ++step) {
    const int k = dir > 0 ? step : nk - 1 - step;
    if ((e = enp::launch_sweep_plane<TV>(P, S.binv, S.storage, x, z, upc, B, h->stream, a, k, dir,
                                         step > 0 ? 1 : 0, S.pc_shared_built)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

extern "C" enp_status enp_set_shared_blocks(enp_handle h, int point) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (point < -1 || point >= h->batch) {
    h->err = "point must be -1 or an operating point of the batch";
    return ENP_ERR_INVALID_ARG;
  }
  SolverState& S = state_of(h);
  if (S.pc_shared != point) {
    S.pc_shared = point;
    ++S.pc_gen;
  }
  return ENP_OK;
}

extern "C" enp_status enp_set_preconditioner(enp_handle h, int two_level) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (two_level < 0 || two_level > 1) {
    h->err = "two_level must be 0 or 1";
    return ENP_ERR_INVALID_ARG;
  }
  if (two_level == 1 && h->prm.dim != 3) {
    h->err = "the two-level preconditioner needs a hexahedral mesh";
    return ENP_ERR_UNSUPPORTED;
  }
  SolverState& S = state_of(h);
  S.coarse = two_level == 1;
  S.coarse_ready = false;
  ++S.pc_gen;
  return ENP_OK;
}

extern "C" enp_status enp_set_sweep(enp_handle h, int on) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (on < 0 || on > 2) {
    h->err = "on must be 0, 1 or 2";
    return ENP_ERR_INVALID_ARG;
  }
  if (on == 1 && h->prm.dim != 3) {
    h->err = "the sweep needs a hexahedral mesh";
    return ENP_ERR_UNSUPPORTED;
  }
  SolverState& S = state_of(h);
  S.sweep_mode = on;
  S.sweep_ready = false;
  ++S.pc_gen;
  return ENP_OK;
}

extern "C" enp_status enp_set_coarse_options(enp_handle h, int cycles, int smooth, double omega) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (cycles < 1 || cycles > 8 || smooth < 1 || smooth > 8 || !(omega > 0.0) || !(omega <= 3.0)) {
    h->err = "coarse options out of range";
    return ENP_ERR_INVALID_ARG;
  }
  SolverState& S = state_of(h);
  S.coarse_cycles = cycles;
  S.coarse_smooth = smooth;
  S.coarse_omega = (float)omega;
  ++S.pc_gen;
  return ENP_OK;
}

extern "C" enp_status enp_coarse_operator(enp_handle h, double* a0) {
  if (!h || !a0) return ENP_ERR_INVALID_ARG;
  SolverState& S = state_of(h);
  if (!S.coarse || !S.coarse_ready || S.levels.empty()) {
    h->err = "the two-level preconditioner has not been set up";
    return ENP_ERR_INVALID_ARG;
  }
  const auto& L = S.levels[0];
  cudaError_t e = cudaMemcpyAsync(a0, L.A, sizeof(double) * 7 * (size_t)L.n * h->batch,
                                  cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "coarse operator copy");
}

extern "C" enp_status enp_block_jacobi_apply(enp_handle h, const double* x, double* y) {
  if (!h || !x || !y) return ENP_ERR_INVALID_ARG;
  if (!h->solver || state_of(h).storage < 0) {
    h->err = "enp_block_jacobi_setup has not been called";
    return ENP_ERR_INVALID_ARG;
  }
  cudaError_t e = bj_apply_any<double>(h, x, y);
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "block apply");
}

extern "C" enp_status enp_block_jacobi_apply_f32(enp_handle h, const float* x, float* y) {
  if (!h || !x || !y) return ENP_ERR_INVALID_ARG;
  if (!h->solver || state_of(h).storage < 0) {
    h->err = "enp_block_jacobi_setup has not been called";
    return ENP_ERR_INVALID_ARG;
  }
  cudaError_t e = bj_apply_any<float>(h, x, y);
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "block apply (FP32)");
}

// ---------------------------------------------------------------- FGMRES
// Solves J(u_lin) x = b (right-preconditioned by the block-Jacobi inverse set
// up last; identity if none) for every operating point of the batch. TV is the
// Krylov vector type: double (FP64 operator) or float (FP32 operator, inner
// solve of the mixed-precision Newton method). The Hessenberg matrix, the
// Givens rotations and the scale factors stay on the device; the host reads the
// convergence flags every kCheckEvery iterations and once per cycle.
constexpr int kCheckEvery = 8;

template <class TV>
static enp_status fgmres_any(enp_handle h, const TV* ulin, const TV* b, TV* x,
                             const enp_krylov_opts* o, enp_krylov_stats* st) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  const long long n = h->n_dof;
  const int B = h->batch;
  const int m = std::max(1, std::min(o->restart, 255));  // coefficient staging holds 256
  const long long ntot = n * B;
  const bool precond = S.storage >= 0;
  cudaError_t e;
  const size_t vbytes = sizeof(TV) * ntot;
  const size_t need = vbytes * (size_t)(m + 1) + vbytes * (size_t)m;
  if (S.krylov_bytes < need) {
    cudaFree(S.V); S.V = nullptr; S.krylov_bytes = 0;
    e = cudaMalloc(&S.V, need);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc Krylov basis");
    S.krylov_bytes = need;
  }
  TV* V = (TV*)S.V;                                  // [m+1][B][n]
  TV* Z = (TV*)((char*)S.V + vbytes * (m + 1));      // [m][B][n]
  const long long vs = ntot;
  // device small arrays
  const size_t nH = (size_t)B * (m + 1) * m, nG = (size_t)B * (m + 1), nM = (size_t)B * m;
  const size_t nsmall = nH + 2 * nG + 2 * nM + nM + (size_t)B * (m + 1) + 7 * (size_t)B + 4;
  e = small(h, nsmall);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc small");
  double* q = S.dsmall;
  enp::KrylovDev K;
  K.H = q; q += nH;
  K.g = q; q += nG;
  K.hcol = q; q += nG;
  K.cs = q; q += nM;
  K.sn = q; q += nM;
  K.coef = q; q += nM;
  K.dh = q; q += (size_t)B * (m + 1);
  K.hn2 = q; q += B;
  K.inv = q; q += B;
  K.beta = q; q += B;
  K.bn2 = q; q += B;
  K.tol = q; q += B;
  K.resn = q; q += B;
  int* flags = reinterpret_cast<int*>(q); q += B;   // jconv
  int* dflag = reinterpret_cast<int*>(q);           // [0] any running, [1] non-finite
  K.jconv = flags;
  const int gx = grid_for(n);
  dim3 gv(gx, B);
  const int tb = std::min(B, 256), gbk = (B + tb - 1) / tb;
  auto apply_A = [&](const TV* in, TV* outv) -> cudaError_t {
    return apply_jv<TV>(h, P, ulin, in, outv, B);
  };
  std::vector<int> hj(B);
  std::vector<double> hres(B), hb(B);
  int hflag[2] = {0, 0};
  // ||b|| and the tolerances
  if ((e = multidot<TV>(h, b, 0, 1, b, K.bn2)) != cudaSuccess) return cuda_err(h, e, "fgmres norm");
  enp::krylov_tolerance<<<gbk, tb, 0, h->stream>>>(K, B, o->rtol, o->atol);
  int total_it = 0;
  double first_norm = -1.0;
  bool all_done = false, nonfinite = false;
  while (!all_done && total_it < o->max_it) {
    // r0 = b - A x -> V0
    if ((e = apply_A(x, V)) != cudaSuccess) return cuda_err(h, e, "fgmres A x");
    enp::b_minus<TV><<<grid_for(ntot), 256, 0, h->stream>>>(b, V, ntot);
    if ((e = multidot<TV>(h, V, 0, 1, V, K.dh)) != cudaSuccess) return cuda_err(h, e, "fgmres r0");
    cudaMemsetAsync(dflag, 0, 2 * sizeof(int), h->stream);
    enp::krylov_cycle_init<<<gbk, tb, 0, h->stream>>>(K, B, m, dflag, dflag + 1);
    cudaMemcpyAsync(hflag, dflag, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(hres.data(), K.resn, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_err(h, e, "fgmres sync");
    if (hflag[1]) { nonfinite = true; break; }
    if (first_norm < 0) {
      first_norm = 0;
      for (int i = 0; i < B; ++i) first_norm = std::max(first_norm, hres[i]);
    }
    if (!hflag[0]) { all_done = true; break; }
    enp::scale_copy<TV, TV><<<gv, 256, 0, h->stream>>>(V, K.inv, 0.0, V, n, n);
    int j = 0;
    bool cycle_done = false;
    const int cycle_start = total_it;
    for (; j < m && total_it < o->max_it; ++j) {
      TV* vj = V + j * vs;
      TV* zj = Z + j * vs;
      TV* w = V + (j + 1) * vs;
      if (precond) e = bj_apply_any<TV>(h, vj, zj);
      else e = cudaMemcpyAsync(zj, vj, vbytes, cudaMemcpyDeviceToDevice, h->stream);
      if (e != cudaSuccess) return cuda_err(h, e, "fgmres precondition");
      if ((e = apply_A(zj, w)) != cudaSuccess) return cuda_err(h, e, "fgmres A z");
      if ((e = arnoldi_orthogonalise<TV>(h, K, V, vs, j, w, m, dflag + 1)) != cudaSuccess)
        return cuda_err(h, e, "fgmres orthogonalisation");
      enp::scale_copy<TV, TV><<<gv, 256, 0, h->stream>>>(w, K.inv, 0.0, w, n, n);
      ++total_it;
      if ((j + 1) % kCheckEvery == 0 || j + 1 == m || total_it >= o->max_it) {
        cudaMemcpyAsync(hj.data(), K.jconv, B * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        cudaMemcpyAsync(hflag + 1, dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
        if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_err(h, e, "fgmres sync");
        if (hflag[1]) { nonfinite = true; break; }
        cycle_done = true;
        for (int i = 0; i < B; ++i) cycle_done = cycle_done && hj[i] != -1;
        if (cycle_done) {
          // count iterations up to each point's convergence, not up to this check
          int used = 0;
          for (int i = 0; i < B; ++i) if (hj[i] >= 0) used = std::max(used, hj[i] + 1);
          total_it = cycle_start + used;
          ++j;
          break;
        }
      }
    }
    if (nonfinite) break;
    const int jm = j;
    enp::krylov_solve_upper<<<gbk, tb, 0, h->stream>>>(K, B, m, jm);
    enp::combine<TV, TV><<<gv, 256, 0, h->stream>>>(Z, vs, jm, K.coef, m, x, n, n, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(h, e, "fgmres update");
    all_done = cycle_done;
  }
  if (nonfinite) { h->err = "non-finite value in FGMRES"; return ENP_ERR_NONFINITE; }
  // true residual of the final iterate
  if ((e = apply_A(x, V)) != cudaSuccess) return cuda_err(h, e, "fgmres final A x");
  enp::b_minus<TV><<<grid_for(ntot), 256, 0, h->stream>>>(b, V, ntot);
  if ((e = multidot<TV>(h, V, 0, 1, V, K.dh)) != cudaSuccess) return cuda_err(h, e, "fgmres final r");
  std::vector<double> hr2(B), htol(B), hbn(B);
  cudaMemcpyAsync(hr2.data(), K.dh, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(htol.data(), K.tol, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(hbn.data(), K.bn2, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_err(h, e, "fgmres sync");
  double worst_rel = 0.0, worst = 0.0;
  bool conv = all_done;
  for (int i = 0; i < B; ++i) {
    const double r = std::sqrt(hr2[i]), bn = std::sqrt(hbn[i]);
    if (!(r <= htol[i] * 1.0001)) conv = false;  // the true residual, not the estimate
    worst = std::max(worst, r);
    worst_rel = std::max(worst_rel, bn > 0 ? r / bn : r);
  }
  if (st) {
    st->iterations = total_it;
    st->residual_norm = worst;
    st->relative_residual = worst_rel;
    st->initial_norm = first_norm < 0 ? 0.0 : first_norm;
    st->converged = conv ? 1 : 0;
  }
  if (!conv) { h->err = "FGMRES reached max_it"; return ENP_ERR_NOT_CONVERGED; }
  return ENP_OK;
}

// FGMRES with each restart cycle (r0, m Arnoldi iterations, update) captured
// once in a CUDA graph and replayed: one launch and one host read per cycle.
// The inputs are copied into handle-owned buffers so that the graph's pointers
// stay fixed across calls. Iterations are counted up to each point's
// convergence; the graph itself always runs whole cycles (a converged point is
// frozen, so the extra iterations do not change x).
template <class TV>
static enp_status fgmres_graph(enp_handle h, const TV* ulin, const TV* b, TV* x,
                               const enp_krylov_opts* o, enp_krylov_stats* st) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  const long long n = h->n_dof;
  const int B = h->batch;
  const int m = std::max(1, std::min(o->restart, 255));  // coefficient staging holds 256
  const long long ntot = n * B;
  const bool precond = S.storage >= 0;
  cudaError_t e;
  const size_t vbytes = sizeof(TV) * ntot;
  const size_t need = vbytes * (size_t)(m + 1) + vbytes * (size_t)m;
  cudaStream_t user = h->stream;
  auto fail_cuda = [&](cudaError_t er, const char* what) { h->stream = user; return cuda_err(h, er, what); };
  if (!S.gstream && (e = cudaStreamCreateWithFlags(&S.gstream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_err(h, e, "create graph stream");
  if (S.krylov_bytes < need) {
    if (S.gexec) { cudaGraphExecDestroy(S.gexec); S.gexec = nullptr; }
    cudaFree(S.V); S.V = nullptr; S.krylov_bytes = 0;
    if ((e = cudaMalloc(&S.V, need)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc Krylov basis");
    S.krylov_bytes = need;
  }
  if (S.gbuf_bytes < 3 * vbytes) {
    if (S.gexec) { cudaGraphExecDestroy(S.gexec); S.gexec = nullptr; }
    cudaFree(S.gbuf); S.gbuf = nullptr; S.gbuf_bytes = 0;
    if ((e = cudaMalloc(&S.gbuf, 3 * vbytes)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc graph inputs");
    S.gbuf_bytes = 3 * vbytes;
  }
  TV* ug = (TV*)S.gbuf;
  TV* bg = ug + ntot;
  TV* xg = bg + ntot;
  TV* V = (TV*)S.V;
  TV* Z = (TV*)((char*)S.V + vbytes * (m + 1));
  const long long vs = ntot;
  const size_t nH = (size_t)B * (m + 1) * m, nG = (size_t)B * (m + 1), nM = (size_t)B * m;
  const size_t nsmall = nH + 2 * nG + 2 * nM + nM + (size_t)B * (m + 1) + 7 * (size_t)B + 4;
  if ((e = small(h, nsmall)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc small");
  if ((e = ensure(&S.part, S.part_count, (size_t)B * (m + 1) * enp::kRedBlocks)) != cudaSuccess)
    return cuda_err(h, e, "cudaMalloc partials");
  double* q = S.dsmall;
  enp::KrylovDev K;
  K.H = q; q += nH;
  K.g = q; q += nG;
  K.hcol = q; q += nG;
  K.cs = q; q += nM;
  K.sn = q; q += nM;
  K.coef = q; q += nM;
  K.dh = q; q += (size_t)B * (m + 1);
  K.hn2 = q; q += B;
  K.inv = q; q += B;
  K.beta = q; q += B;
  K.bn2 = q; q += B;
  K.tol = q; q += B;
  K.resn = q; q += B;
  int* flags = reinterpret_cast<int*>(q); q += B;
  int* dflag = reinterpret_cast<int*>(q);
  K.jconv = flags;
  const int gx = grid_for(n);
  dim3 gv(gx, B);
  const int tb = std::min(B, 256), gbk = (B + tb - 1) / tb;
  // inputs into the graph's buffers, ordered after the caller's stream
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(S.gstream, ev, 0);
  h->stream = S.gstream;
  cudaMemcpyAsync(ug, ulin, vbytes, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(bg, b, vbytes, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(xg, x, vbytes, cudaMemcpyDeviceToDevice, h->stream);
  if ((e = multidot<TV>(h, bg, 0, 1, bg, K.bn2)) != cudaSuccess) { cudaEventDestroy(ev); return fail_cuda(e, "fgmres norm"); }
  enp::krylov_tolerance<<<gbk, tb, 0, h->stream>>>(K, B, o->rtol, o->atol);
  auto apply_A = [&](const TV* in, TV* outv) -> cudaError_t {
    return apply_jv<TV>(h, P, ug, in, outv, B);
  };
  const bool same = S.gexec && S.gkey[0] == (const void*)S.V && S.gkey[1] == S.binv &&
                    S.gkey[2] == (const void*)S.gbuf && S.gkey[3] == (const void*)S.dsmall &&
                    S.gkey_i[0] == m && S.gkey_i[1] == S.storage && S.gkey_i[2] == (int)sizeof(TV) &&
                    S.gkey_i[3] == B && S.gkey_gen == S.pc_gen;
  if (!same) {
    if (S.gexec) { cudaGraphExecDestroy(S.gexec); S.gexec = nullptr; }
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
      cudaEventDestroy(ev); return fail_cuda(e, "begin capture");
    }
    apply_A(xg, V);
    enp::b_minus<TV><<<grid_for(ntot), 256, 0, h->stream>>>(bg, V, ntot);
    multidot<TV>(h, V, 0, 1, V, K.dh);
    cudaMemsetAsync(dflag, 0, 2 * sizeof(int), h->stream);
    enp::krylov_cycle_init<<<gbk, tb, 0, h->stream>>>(K, B, m, dflag, dflag + 1);
    enp::scale_copy<TV, TV><<<gv, 256, 0, h->stream>>>(V, K.inv, 0.0, V, n, n);
    for (int j = 0; j < m; ++j) {
      TV* vj = V + j * vs;
      TV* zj = Z + j * vs;
      TV* w = V + (j + 1) * vs;
      if (precond) bj_apply_any<TV>(h, vj, zj);
      else cudaMemcpyAsync(zj, vj, vbytes, cudaMemcpyDeviceToDevice, h->stream);
      apply_A(zj, w);
      arnoldi_orthogonalise<TV>(h, K, V, vs, j, w, m, dflag + 1);
      enp::scale_copy<TV, TV><<<gv, 256, 0, h->stream>>>(w, K.inv, 0.0, w, n, n);
    }
    enp::krylov_solve_upper<<<gbk, tb, 0, h->stream>>>(K, B, m, m);
    enp::combine<TV, TV><<<gv, 256, 0, h->stream>>>(Z, vs, m, K.coef, m, xg, n, n, 1);
    e = cudaStreamEndCapture(h->stream, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S.gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) { S.gexec = nullptr; cudaEventDestroy(ev); return fail_cuda(e, "capture FGMRES cycle"); }
    S.gkey[0] = S.V; S.gkey[1] = S.binv; S.gkey[2] = S.gbuf; S.gkey[3] = S.dsmall;
    S.gkey_i[0] = m; S.gkey_i[1] = S.storage; S.gkey_i[2] = (int)sizeof(TV); S.gkey_i[3] = B;
    S.gkey_gen = S.pc_gen;
  }
  std::vector<int> hj(B);
  int hflag[2] = {0, 0};
  std::vector<double> hres(B);
  int total_it = 0;
  double first_norm = -1.0;
  bool all_done = false, nonfinite = false;
  for (int cycle = 0; !all_done && total_it < o->max_it; ++cycle) {
    if ((e = cudaGraphLaunch(S.gexec, h->stream)) != cudaSuccess) { cudaEventDestroy(ev); return fail_cuda(e, "graph launch"); }
    cudaMemcpyAsync(hj.data(), K.jconv, B * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(hflag, dflag, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(hres.data(), K.beta, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) { cudaEventDestroy(ev); return fail_cuda(e, "graph sync"); }
    if (first_norm < 0) {
      first_norm = 0;
      for (int i = 0; i < B; ++i) first_norm = std::max(first_norm, hres[i]);
    }
    if (hflag[1]) { nonfinite = true; break; }
    all_done = true;
    int used = 0;
    for (int i = 0; i < B; ++i) {
      if (hj[i] == -1) all_done = false;
      if (hj[i] >= 0) used = std::max(used, hj[i] + 1);
    }
    total_it += all_done ? used : m;
  }
  enp_status ret = ENP_OK;
  if (nonfinite) { h->err = "non-finite value in FGMRES"; ret = ENP_ERR_NONFINITE; }
  // true residual of the final iterate
  std::vector<double> hr2(B), htol(B), hbn(B);
  if (ret == ENP_OK) {
    apply_A(xg, V);
    enp::b_minus<TV><<<grid_for(ntot), 256, 0, h->stream>>>(bg, V, ntot);
    multidot<TV>(h, V, 0, 1, V, K.dh);
    cudaMemcpyAsync(hr2.data(), K.dh, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(htol.data(), K.tol, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(hbn.data(), K.bn2, B * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  cudaMemcpyAsync(x, xg, vbytes, cudaMemcpyDeviceToDevice, h->stream);
  cudaEventRecord(ev, h->stream);
  cudaStreamWaitEvent(user, ev, 0);
  e = cudaStreamSynchronize(h->stream);
  cudaEventDestroy(ev);
  h->stream = user;
  if (e != cudaSuccess) return cuda_err(h, e, "graph final sync");
  if (ret != ENP_OK) return ret;
  double worst_rel = 0.0, worst = 0.0;
  bool conv = all_done;
  for (int i = 0; i < B; ++i) {
    const double r = std::sqrt(hr2[i]), bn = std::sqrt(hbn[i]);
    if (!(r <= htol[i] * 1.0001)) conv = false;
    worst = std::max(worst, r);
    worst_rel = std::max(worst_rel, bn > 0 ? r / bn : r);
  }
  if (st) {
    st->iterations = total_it;
    st->residual_norm = worst;
    st->relative_residual = worst_rel;
    st->initial_norm = first_norm < 0 ? 0.0 : first_norm;
    st->converged = conv ? 1 : 0;
  }
  if (!conv) { h->err = "FGMRES reached max_it"; return ENP_ERR_NOT_CONVERGED; }
  return ENP_OK;
}

extern "C" enp_status enp_fgmres_solve(enp_handle h, const double* u_lin, const double* b, double* x,
                                       const enp_krylov_opts* o, enp_krylov_stats* st) {
  if (!h || !u_lin || !b || !x || !o || o->restart < 1 || o->max_it < 1) return ENP_ERR_INVALID_ARG;
  if (o->graph) return fgmres_graph<double>(h, u_lin, b, x, o, st);
  return fgmres_any<double>(h, u_lin, b, x, o, st);
}

extern "C" enp_status enp_fgmres_solve_f32(enp_handle h, const float* u_lin, const float* b, float* x,
                                           const enp_krylov_opts* o, enp_krylov_stats* st) {
  if (!h || !u_lin || !b || !x || !o || o->restart < 1 || o->max_it < 1) return ENP_ERR_INVALID_ARG;
  if (o->graph) return fgmres_graph<float>(h, u_lin, b, x, o, st);
  return fgmres_any<float>(h, u_lin, b, x, o, st);
}

// ---------------------------------------------------------------- Newton
// Newton's method with backtracking line search (Sec. 4), independently for
// every operating point of the batch: solve J du = -R with FGMRES (FP64, or
// with the FP32 operator when opts->mixed), then halve each point's step until
// ||R_b(u_b + lam_b du_b)|| <= (1 - c lam_b) ||R_b(u_b)||. A point that has met
// its tolerance gets a zero right-hand side (FGMRES leaves it at du = 0). The
// block-Jacobi preconditioner is rebuilt at every Newton iterate. Norms in the
// statistics are the largest over the operating points.
// ---------------------------------------------------------------------------
// Graph-driven Newton iteration. One CUDA graph holds a WHILE node over Newton
// steps; its body forms -R on the running points, solves J du = -R by FGMRES
// (a WHILE node over restart cycles, each cycle the sequence of fgmres_graph),
// runs the backtracking line search (a WHILE node over trial steps) and
// updates u and R. Device kernels count iterations and set the loop
// conditions, so one launch carries the solve from one preconditioner setup to
// the next (opts->pc_lag Newton steps), to convergence, to max_it, or to an
// inner solve that stopped at its limit; the host sets up the preconditioner
// between launches. The Newton vectors live in handle-owned buffers (u is
// copied in and out) so that the captured graph is reused across calls.

// The graph being captured on stream s, and a conditional handle in it.
static cudaError_t capture_handle(cudaStream_t s, cudaGraphConditionalHandle* hnd) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive || !g) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(hnd, g, 1, cudaGraphCondAssignDefault);
}

// Append a WHILE node on handle hnd at the capture point of stream s and start
// capturing its body on stream sb.
static cudaError_t begin_while(cudaStream_t s, cudaStream_t sb, cudaGraphConditionalHandle hnd) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
      cudaSuccess)
    return e;
  return cudaStreamBeginCaptureToGraph(sb, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeRelaxed);
}

static cudaError_t end_while(cudaStream_t sb) {
  cudaGraph_t g = nullptr;
  return cudaStreamEndCapture(sb, &g);
}

template <class TV>
static enp_status newton_device(enp_handle h, double* u_user, const enp_newton_opts* o,
                                enp_newton_stats* st) {
  SolverState& S = state_of(h);
  const OpParams& P = h->prm;
  constexpr bool mixed = std::is_same<TV, float>::value;
  const long long n = h->n_dof;
  const int B = h->batch;
  const long long ntot = n * B;
  const int m = std::max(1, std::min(o->krylov.restart, 255));
  const int per_setup = std::max(o->pc_lag, 1);
  cudaStream_t user = h->stream;
  cudaError_t e;
  using clk = std::chrono::steady_clock;
  auto seconds_since = [](clk::time_point t0) {
    return std::chrono::duration<double>(clk::now() - t0).count();
  };
  auto fail = [&](cudaError_t er, const char* what) { h->stream = user; return cuda_err(h, er, what); };
  // handle-owned Newton vectors
  const size_t vb64 = sizeof(double) * ntot, vb32 = sizeof(float) * ntot;
  const size_t nbuf_need = 5 * vb64 + (mixed ? 3 * vb32 : 0);
  if (S.nbuf_bytes < nbuf_need) {
    if (S.nexec) { cudaGraphExecDestroy(S.nexec); S.nexec = nullptr; }
    cudaFree(S.nbuf); S.nbuf = nullptr; S.nbuf_bytes = 0;
    if ((e = cudaMalloc(&S.nbuf, nbuf_need)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc newton vectors");
    S.nbuf_bytes = nbuf_need;
  }
  double* u = (double*)S.nbuf;
  double *r = u + ntot, *du = r + ntot, *ut = du + ntot, *rt = ut + ntot;
  float* u32 = mixed ? (float*)(rt + ntot) : nullptr;
  float* b32 = mixed ? u32 + ntot : nullptr;
  float* x32 = mixed ? b32 + ntot : nullptr;
  const size_t nsm_need = sizeof(enp::NewtonCtl) + (size_t)B * (5 * sizeof(double) + 2 * sizeof(int));
  if (S.nsmall_bytes < nsm_need) {
    if (S.nexec) { cudaGraphExecDestroy(S.nexec); S.nexec = nullptr; }
    cudaFree(S.nsmall); S.nsmall = nullptr; S.nsmall_bytes = 0;
    if ((e = cudaMalloc(&S.nsmall, nsm_need)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc newton state");
    S.nsmall_bytes = nsm_need;
  }
  enp::NewtonDev A;
  A.c = (enp::NewtonCtl*)S.nsmall;
  A.rn = (double*)(A.c + 1);
  A.tol = A.rn + B; A.lam = A.tol + B; A.rnew2 = A.lam + B; A.negmask = A.rnew2 + B;
  A.mask = (int*)(A.negmask + B); A.acc = A.mask + B;
  for (auto& sx : S.nstream)
    if (!sx && (e = cudaStreamCreateWithFlags(&sx, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_err(h, e, "create graph streams");
  // u in, the initial residual and tolerances (eager, on the caller's stream)
  cudaMemcpyAsync(u, u_user, vb64, cudaMemcpyDeviceToDevice, user);
  if ((e = apply_residual(h, u, r, B)) != cudaSuccess ||
      (e = multidot<double>(h, r, 0, 1, r, A.rnew2)) != cudaSuccess)
    return cuda_err(h, e, "newton residual");
  std::vector<double> r0(B), tol(B), rnh(B);
  cudaMemcpyAsync(r0.data(), A.rnew2, sizeof(double) * B, cudaMemcpyDeviceToHost, user);
  if ((e = cudaStreamSynchronize(user)) != cudaSuccess) return cuda_err(h, e, "newton sync");
  double r0max = 0.0;
  for (int b = 0; b < B; ++b) {
    r0[b] = std::sqrt(r0[b]);
    if (!std::isfinite(r0[b])) { h->err = "non-finite initial residual"; return ENP_ERR_NONFINITE; }
    tol[b] = std::max(o->rtol * r0[b], o->atol);
    r0max = std::max(r0max, r0[b]);
  }
  cudaMemcpyAsync(A.rn, r0.data(), sizeof(double) * B, cudaMemcpyHostToDevice, user);
  cudaMemcpyAsync(A.tol, tol.data(), sizeof(double) * B, cudaMemcpyHostToDevice, user);
  cudaMemsetAsync(A.c, 0, sizeof(enp::NewtonCtl), user);
  // Krylov workspace (as fgmres_graph)
  const size_t vbytes = sizeof(TV) * ntot;
  const size_t kneed = vbytes * (size_t)(2 * m + 1);
  if (S.krylov_bytes < kneed) {
    if (S.gexec) { cudaGraphExecDestroy(S.gexec); S.gexec = nullptr; }
    cudaFree(S.V); S.V = nullptr; S.krylov_bytes = 0;
    if ((e = cudaMalloc(&S.V, kneed)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc Krylov basis");
    S.krylov_bytes = kneed;
  }
  const size_t nH = (size_t)B * (m + 1) * m, nG = (size_t)B * (m + 1), nM = (size_t)B * m;
  const size_t nsmallk = nH + 2 * nG + 2 * nM + nM + (size_t)B * (m + 1) + 7 * (size_t)B + 4;
  enp_newton_stats acc{};
  acc.initial_norm = r0max;
  acc.history[0] = r0max;
  int setups = 0;
  double t_setup = 0.0, t_graph = 0.0;
  enp_status status = ENP_OK;
  enp::NewtonCtl ch{};
  while (true) {
    cudaMemcpyAsync(&ch, A.c, sizeof(ch), cudaMemcpyDeviceToHost, user);
    cudaMemcpyAsync(rnh.data(), A.rn, sizeof(double) * B, cudaMemcpyDeviceToHost, user);
    if ((e = cudaStreamSynchronize(user)) != cudaSuccess) return cuda_err(h, e, "newton sync");
    if (ch.nonfinite) { status = ENP_ERR_NONFINITE; h->err = "non-finite residual"; break; }
    bool conv = true;
    for (int b = 0; b < B; ++b) conv = conv && rnh[b] <= tol[b];
    if (conv) break;
    if (ch.it >= o->max_it) { status = ENP_ERR_NOT_CONVERGED; h->err = "Newton reached max_it"; break; }
    // preconditioner at the current u, then up to per_setup Newton steps on the device
    const auto t0 = clk::now();
    enp_status s2 = enp_block_jacobi_setup(h, u, o->bj_storage);  // synchronises
    t_setup += seconds_since(t0);
    ++setups;
    if (s2 != ENP_OK) { status = s2; break; }
    cudaMemsetAsync(&A.c->since, 0, sizeof(int), user);
    cudaMemsetAsync(&A.c->kfail, 0, sizeof(int), user);
    if ((e = small(h, nsmallk)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc small");
    if ((e = ensure(&S.part, S.part_count, (size_t)B * (m + 1) * enp::kRedBlocks)) != cudaSuccess)
      return cuda_err(h, e, "cudaMalloc partials");
    // the capture key: every pointer and setting the captured sequence bakes in,
    // including the operator parameters the kernels receive by value
    const double kv[] = {
        (double)(uintptr_t)S.V, (double)(uintptr_t)S.binv, (double)(uintptr_t)S.dsmall,
        (double)(uintptr_t)S.part, (double)(uintptr_t)S.nbuf, (double)(uintptr_t)S.nsmall,
        (double)m, (double)S.storage, (double)sizeof(TV), (double)B, (double)S.pc_gen,
        (double)S.potential_only, o->krylov.rtol, o->krylov.atol, (double)o->krylov.max_it,
        (double)o->max_it, o->armijo_c, (double)o->max_backtracks, (double)per_setup};
    std::vector<char> key(sizeof(kv) + sizeof(OpParams));
    std::memcpy(key.data(), kv, sizeof(kv));
    std::memcpy(key.data() + sizeof(kv), &P, sizeof(OpParams));
    if (!S.nexec || S.nkey != key) {
      if (S.nexec) { cudaGraphExecDestroy(S.nexec); S.nexec = nullptr; }
      double* q = S.dsmall;
      enp::KrylovDev K;
      K.H = q; q += nH;
      K.g = q; q += nG;
      K.hcol = q; q += nG;
      K.cs = q; q += nM;
      K.sn = q; q += nM;
      K.coef = q; q += nM;
      K.dh = q; q += (size_t)B * (m + 1);
      K.hn2 = q; q += B;
      K.inv = q; q += B;
      K.beta = q; q += B;
      K.bn2 = q; q += B;
      K.tol = q; q += B;
      K.resn = q; q += B;
      int* dflag = reinterpret_cast<int*>(q + B);
      K.jconv = reinterpret_cast<int*>(q);
      TV* V = (TV*)S.V;
      TV* Z = (TV*)((char*)S.V + vbytes * (m + 1));
      const long long vs = ntot;
      TV* xk = mixed ? (TV*)x32 : (TV*)du;
      const TV* bk = mixed ? (const TV*)b32 : (const TV*)rt;
      const TV* uk = mixed ? (const TV*)u32 : (const TV*)u;
      const bool precond = S.storage >= 0;
      const int gx = grid_for(n), gt = grid_for(ntot);
      const dim3 gv(gx, B);
      const int tb = std::min(B, 256), gbk = (B + tb - 1) / tb;
      // one eager J v launch so that every kernel's attributes are set outside capture
      if (mixed) enp::convert_kernel<double, float><<<gt, 256, 0, user>>>(u, u32, ntot);
      cudaMemsetAsync(xk, 0, vbytes, user);
      if ((e = apply_jv<TV>(h, P, uk, xk, (TV*)V, B)) != cudaSuccess) return fail(e, "newton warm-up");
      if ((e = cudaStreamSynchronize(user)) != cudaSuccess) return fail(e, "newton warm-up");
      cudaStream_t s0 = S.nstream[0], s1 = S.nstream[1], s2s = S.nstream[2];
      cudaGraph_t graph = nullptr;
      cudaGraphConditionalHandle hN, hK, hL;
      auto capture = [&]() -> cudaError_t {
        cudaError_t er;
        h->stream = s0;
        if ((er = cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed)) != cudaSuccess) return er;
        if ((er = capture_handle(s0, &hN)) != cudaSuccess) return er;
        if ((er = begin_while(s0, s1, hN)) != cudaSuccess) return er;
        h->stream = s1;
        enp::ng_begin<<<1, 256, 0, s1>>>(A, B);
        enp::scale_batched<<<gt, 256, 0, s1>>>(r, A.negmask, rt, n, B);
        if (mixed) {
          enp::convert_kernel<double, float><<<gt, 256, 0, s1>>>(u, u32, ntot);
          enp::convert_kernel<double, float><<<gt, 256, 0, s1>>>(rt, b32, ntot);
        }
        cudaMemsetAsync(xk, 0, vbytes, s1);
        multidot<TV>(h, bk, 0, 1, bk, K.bn2);
        enp::krylov_tolerance<<<gbk, tb, 0, s1>>>(K, B, o->krylov.rtol, o->krylov.atol);
        // FGMRES restart cycles
        if ((er = capture_handle(s1, &hK)) != cudaSuccess) return er;
        enp::ng_arm<<<1, 1, 0, s1>>>(hK);
        if ((er = begin_while(s1, s2s, hK)) != cudaSuccess) return er;
        h->stream = s2s;
        apply_jv<TV>(h, P, uk, xk, V, B);
        enp::b_minus<TV><<<gt, 256, 0, s2s>>>(bk, V, ntot);
        multidot<TV>(h, V, 0, 1, V, K.dh);
        cudaMemsetAsync(dflag, 0, 2 * sizeof(int), s2s);
        enp::krylov_cycle_init<<<gbk, tb, 0, s2s>>>(K, B, m, dflag, dflag + 1);
        enp::scale_copy<TV, TV><<<gv, 256, 0, s2s>>>(V, K.inv, 0.0, V, n, n);
        for (int j = 0; j < m; ++j) {
          TV* vj = V + j * vs;
          TV* zj = Z + j * vs;
          TV* w = V + (j + 1) * vs;
          if (precond) bj_apply_any<TV>(h, vj, zj);
          else cudaMemcpyAsync(zj, vj, vbytes, cudaMemcpyDeviceToDevice, s2s);
          apply_jv<TV>(h, P, uk, zj, w, B);
          arnoldi_orthogonalise<TV>(h, K, V, vs, j, w, m, dflag + 1);
          enp::scale_copy<TV, TV><<<gv, 256, 0, s2s>>>(w, K.inv, 0.0, w, n, n);
        }
        enp::krylov_solve_upper<<<gbk, tb, 0, s2s>>>(K, B, m, m);
        enp::combine<TV, TV><<<gv, 256, 0, s2s>>>(Z, vs, m, K.coef, m, xk, n, n, 1);
        enp::ng_krylov_count<<<1, 256, 0, s2s>>>(K, A, dflag, B, m, o->krylov.max_it, hK);
        if ((er = end_while(s2s)) != cudaSuccess) return er;
        h->stream = s1;
        if (mixed) enp::convert_kernel<float, double><<<gt, 256, 0, s1>>>(x32, du, ntot);
        // backtracking line search
        if ((er = capture_handle(s1, &hL)) != cudaSuccess) return er;
        enp::ng_arm<<<1, 1, 0, s1>>>(hL);
        if ((er = begin_while(s1, s2s, hL)) != cudaSuccess) return er;
        h->stream = s2s;
        enp::axpy_batched<<<gt, 256, 0, s2s>>>(u, A.lam, du, ut, n, B);
        apply_residual(h, ut, rt, B);
        multidot<double>(h, rt, 0, 1, rt, A.rnew2);
        enp::ng_ls_accept<<<1, 256, 0, s2s>>>(A, B, o->armijo_c, o->max_backtracks, hL);
        if ((er = end_while(s2s)) != cudaSuccess) return er;
        h->stream = s1;
        cudaMemcpyAsync(u, ut, vb64, cudaMemcpyDeviceToDevice, s1);
        cudaMemcpyAsync(r, rt, vb64, cudaMemcpyDeviceToDevice, s1);
        enp::ng_end<<<1, 256, 0, s1>>>(A, B, o->max_it, per_setup, hN);
        if ((er = end_while(s1)) != cudaSuccess) return er;
        h->stream = s0;
        return cudaStreamEndCapture(s0, &graph);
      };
      e = capture();
      h->stream = user;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&S.nexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        // leave no stream in capture mode
        for (auto sx : S.nstream) {
          cudaStreamCaptureStatus cs;
          if (cudaStreamIsCapturing(sx, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g2 = nullptr;
            cudaStreamEndCapture(sx, &g2);
            if (g2) cudaGraphDestroy(g2);
          }
        }
        cudaGetLastError();
        S.nexec = nullptr;
        return cuda_err(h, e, "capture Newton graph");
      }
      S.nkey = key;
    }
    const auto tg = clk::now();
    if ((e = cudaGraphLaunch(S.nexec, user)) != cudaSuccess) return cuda_err(h, e, "Newton graph launch");
    if ((e = cudaStreamSynchronize(user)) != cudaSuccess) return cuda_err(h, e, "Newton graph");
    t_graph += seconds_since(tg);
  }
  cudaMemcpyAsync(u_user, u, vb64, cudaMemcpyDeviceToDevice, user);
  cudaStreamSynchronize(user);
  if (st) {
    *st = acc;
    st->iterations = ch.it;
    st->krylov_iterations = ch.kry_total;
    st->setups = setups;
    st->setup_seconds = t_setup;
    st->krylov_seconds = t_graph;
    double mx = 0.0;
    for (double x : rnh) mx = std::max(mx, std::isnan(x) ? INFINITY : x);
    st->residual_norm = mx;
    for (int i = 1; i < 64 && i <= ch.it; ++i) st->history[i] = ch.hist[i];
    st->converged = status == ENP_OK ? 1 : 0;
  }
  return status;
}

extern "C" enp_status enp_newton_solve(enp_handle h, double* u, const enp_newton_opts* o,
                                       enp_newton_stats* st) {
  if (!h || !u || !o || o->max_it < 0) return ENP_ERR_INVALID_ARG;
  if (o->device_loop) return o->mixed ? newton_device<float>(h, u, o, st) : newton_device<double>(h, u, o, st);
  SolverState& S = state_of(h);
  const long long n = h->n_dof;
  const long long ntot = n * h->batch;
  const int B = h->batch;
  cudaError_t e;
  double *r = nullptr, *du = nullptr, *ut = nullptr, *rt = nullptr, *dvec = nullptr;
  float *u32 = nullptr, *b32 = nullptr, *x32 = nullptr;
  auto cleanup = [&]() {
    cudaFree(r); cudaFree(du); cudaFree(ut); cudaFree(rt); cudaFree(dvec);
    cudaFree(u32); cudaFree(b32); cudaFree(x32);
  };
  e = cudaMalloc(&r, sizeof(double) * ntot);
  if (e == cudaSuccess) e = cudaMalloc(&du, sizeof(double) * ntot);
  if (e == cudaSuccess) e = cudaMalloc(&ut, sizeof(double) * ntot);
  if (e == cudaSuccess) e = cudaMalloc(&rt, sizeof(double) * ntot);
  if (e == cudaSuccess) e = cudaMalloc(&dvec, sizeof(double) * 2 * B);
  if (e == cudaSuccess && o->mixed) {
    e = cudaMalloc(&u32, sizeof(float) * ntot);
    if (e == cudaSuccess) e = cudaMalloc(&b32, sizeof(float) * ntot);
    if (e == cudaSuccess) e = cudaMalloc(&x32, sizeof(float) * ntot);
  }
  if (e != cudaSuccess) { cleanup(); return cuda_err(h, e, "cudaMalloc newton work"); }
  double* dlam = dvec;       // [B] step lengths
  auto norms = [&](const double* v, std::vector<double>& out) -> cudaError_t {
    cudaError_t er = small(h, (size_t)B * 4);
    if (er != cudaSuccess) return er;
    er = multidot<double>(h, v, 0, 1, v, S.dsmall);
    if (er != cudaSuccess) return er;
    out.assign(B, 0.0);
    er = cudaMemcpyAsync(out.data(), S.dsmall, sizeof(double) * B, cudaMemcpyDeviceToHost, h->stream);
    if (er != cudaSuccess) return er;
    er = cudaStreamSynchronize(h->stream);
    for (auto& x : out) x = std::sqrt(x);
    return er;
  };
  auto maxof = [](const std::vector<double>& v) {
    double m = 0;
    for (double x : v) m = std::max(m, std::isnan(x) ? INFINITY : x);
    return m;
  };
  const int gx = grid_for(ntot);
  enp_status status = ENP_OK;
  std::vector<double> rn, r0, tol(B), lam(B), mask(B), rnew;
  if ((e = apply_residual(h, u, r, B)) != cudaSuccess ||
      (e = norms(r, rn)) != cudaSuccess) { cleanup(); return cuda_err(h, e, "newton residual"); }
  r0 = rn;
  for (int b = 0; b < B; ++b) {
    if (!std::isfinite(rn[b])) { cleanup(); h->err = "non-finite initial residual"; return ENP_ERR_NONFINITE; }
    tol[b] = std::max(o->rtol * r0[b], o->atol);
  }
  int it = 0, kry_total = 0, setups = 0, since_setup = 0;
  bool rebuild = true;
  double t_setup = 0.0, t_krylov = 0.0;
  using clk = std::chrono::steady_clock;
  auto seconds_since = [](clk::time_point t0) {
    return std::chrono::duration<double>(clk::now() - t0).count();
  };
  if (st) { std::memset(st, 0, sizeof(*st)); st->initial_norm = maxof(r0); st->history[0] = maxof(rn); }
  while (true) {
    bool all_conv = true;
    for (int b = 0; b < B; ++b) {
      mask[b] = rn[b] <= tol[b] ? 0.0 : 1.0;
      all_conv = all_conv && mask[b] == 0.0;
    }
    if (all_conv) break;
    if (it >= o->max_it) { status = ENP_ERR_NOT_CONVERGED; h->err = "Newton reached max_it"; break; }
    enp_status s2 = ENP_OK;
    if (rebuild || since_setup >= std::max(o->pc_lag, 1)) {
      const auto t0 = clk::now();
      s2 = enp_block_jacobi_setup(h, u, o->bj_storage);  // synchronises
      t_setup += seconds_since(t0);
      ++setups;
      since_setup = 0;
      rebuild = false;
    }
    if (s2 != ENP_OK) { status = s2; break; }
    ++since_setup;
    enp_krylov_stats ks{};
    const auto tk = clk::now();
    enp_krylov_opts ko = o->krylov;
    // right-hand side -R on the running points, 0 on the converged ones
    for (int b = 0; b < B; ++b) lam[b] = -mask[b];
    cudaMemcpyAsync(dlam, lam.data(), sizeof(double) * B, cudaMemcpyHostToDevice, h->stream);
    enp::scale_batched<<<gx, 256, 0, h->stream>>>(r, dlam, rt, n, B);
    cudaMemsetAsync(du, 0, sizeof(double) * ntot, h->stream);
    if (o->mixed) {
      enp::convert_kernel<double, float><<<gx, 256, 0, h->stream>>>(u, u32, ntot);
      enp::convert_kernel<double, float><<<gx, 256, 0, h->stream>>>(rt, b32, ntot);
      cudaMemsetAsync(x32, 0, sizeof(float) * ntot, h->stream);
      s2 = ko.graph ? fgmres_graph<float>(h, u32, b32, x32, &ko, &ks)
                    : fgmres_any<float>(h, u32, b32, x32, &ko, &ks);
      enp::convert_kernel<float, double><<<gx, 256, 0, h->stream>>>(x32, du, ntot);
    } else {
      s2 = ko.graph ? fgmres_graph<double>(h, u, rt, du, &ko, &ks)
                    : fgmres_any<double>(h, u, rt, du, &ko, &ks);
    }
    cudaStreamSynchronize(h->stream);
    t_krylov += seconds_since(tk);
    kry_total += ks.iterations;
    if (s2 != ENP_OK && s2 != ENP_ERR_NOT_CONVERGED) { status = s2; break; }
    if (s2 == ENP_ERR_NOT_CONVERGED) rebuild = true;  // a stale preconditioner may be the cause
    // backtracking line search, one step length per operating point
    std::vector<int> accepted(B, 0);
    for (int b = 0; b < B; ++b) { lam[b] = mask[b] > 0 ? 1.0 : 0.0; accepted[b] = mask[b] == 0.0; }
    for (int bt = 0;; ++bt) {
      cudaMemcpyAsync(dlam, lam.data(), sizeof(double) * B, cudaMemcpyHostToDevice, h->stream);
      enp::axpy_batched<<<gx, 256, 0, h->stream>>>(u, dlam, du, ut, n, B);
      if ((e = apply_residual(h, ut, rt, B)) != cudaSuccess ||
          (e = norms(rt, rnew)) != cudaSuccess) { cleanup(); return cuda_err(h, e, "newton line search"); }
      bool all_acc = true;
      for (int b = 0; b < B; ++b) {
        if (accepted[b]) continue;
        if (rnew[b] <= (1.0 - o->armijo_c * lam[b]) * rn[b] || bt >= o->max_backtracks) accepted[b] = 1;
        else lam[b] *= 0.5;
        all_acc = all_acc && accepted[b];
      }
      if (all_acc) break;
    }
    cudaMemcpyAsync(u, ut, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(r, rt, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, h->stream);
    rn = rnew;
    ++it;
    if (st && it < 64) st->history[it] = maxof(rn);
    if (!std::isfinite(maxof(rn))) { status = ENP_ERR_NONFINITE; h->err = "non-finite residual"; break; }
  }
  cudaStreamSynchronize(h->stream);
  if (st) {
    st->iterations = it;
    st->krylov_iterations = kry_total;
    st->setups = setups;
    st->setup_seconds = t_setup;
    st->krylov_seconds = t_krylov;
    st->residual_norm = maxof(rn);
    st->converged = (status == ENP_OK) ? 1 : 0;
  }
  cleanup();
  return status;
}

extern "C" enp_status enp_initial_guess(enp_handle h, double* u, const enp_newton_opts* o,
                                        enp_newton_stats* st) {
  if (!h || !u || !o) return ENP_ERR_INVALID_ARG;
  const OpParams& P = h->prm;
  SolverState& S = state_of(h);
  const int B = h->batch;
  const long long EN = (long long)P.E * P.Np;
  enp::species_fill<<<grid_for((P.NF - 1) * EN * B), 256, 0, h->stream>>>(
      u, EN, P.NF, P.batch_stride, B, P.cin[0], P.cin[1], P.cin[2]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(h, e, "initial concentrations");
  // Newton on the potential rows with the concentrations held: the species rows
  // of the system are c - c^in (zero here) with unit Jacobian rows, so every
  // Newton step leaves c = c^in; the sweep (which couples species across
  // elements) is off meanwhile
  const int sweep_mode = S.sweep_mode;
  S.sweep_mode = 0;
  S.potential_only = true;
  ++S.pc_gen;
  enp_status s = enp_newton_solve(h, u, o, st);
  S.potential_only = false;
  S.sweep_mode = sweep_mode;
  S.sweep_ready = false;
  ++S.pc_gen;
  return s;
}

extern "C" enp_status enp_newton_continuation(enp_handle h, double* u, const double* phi_app,
                                              const enp_continuation_opts* c,
                                              const enp_newton_opts* o,
                                              enp_continuation_stats* st) {
  if (!h || !u || !phi_app || !c || !o) return ENP_ERR_INVALID_ARG;
  if (!(c->step_min > 0.0) || !(c->step0 >= c->step_min) || !(c->step_max >= c->step0) ||
      !(c->step_max <= 1.0) || !(c->grow >= 1.0) || c->stage_max_it < 1) {
    h->err = "continuation options out of range";
    return ENP_ERR_INVALID_ARG;
  }
  const int B = h->batch;
  const long long ntot = h->n_dof * B;
  double* ut = nullptr;
  cudaError_t e = cudaMalloc(&ut, sizeof(double) * ntot);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc continuation iterate");
  std::vector<double> phi(4 * (size_t)B);
  enp_continuation_stats cs{};
  double lam = 0.0, dl = c->step0;
  enp_status status = ENP_OK;
  // ENP_CONTINUATION_LOG set: progress lines per stage on stderr (long runs)
  const bool log = std::getenv("ENP_CONTINUATION_LOG") != nullptr;
  const auto t_start = std::chrono::steady_clock::now();
  while (true) {
    const double nl = std::min(1.0, lam + dl);
    const bool last = nl >= 1.0;
    for (size_t i = 0; i < phi.size(); ++i) phi[i] = (last ? 1.0 : nl) * phi_app[i];
    enp_status s2 = enp_set_phi_app(h, phi.data());
    if (s2 != ENP_OK) { status = s2; break; }
    e = cudaMemcpyAsync(ut, u, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) { status = cuda_err(h, e, "continuation copy"); break; }
    enp_newton_opts so = *o;
    if (!last) { so.rtol = c->stage_rtol; so.max_it = c->stage_max_it; }
    enp_newton_stats ns{};
    s2 = enp_newton_solve(h, ut, &so, &ns);
    ++cs.stages;
    cs.newton_iterations += ns.iterations;
    cs.krylov_iterations += ns.krylov_iterations;
    cs.last = ns;
    if (log) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      std::fprintf(stderr,
                   "continuation stage %d: lambda %.4f status %d newton %d krylov %d ||R||/||R0|| %.3e "
                   "elapsed %.1f s\n",
                   cs.stages, last ? 1.0 : nl, (int)s2, ns.iterations, ns.krylov_iterations,
                   ns.initial_norm > 0 ? ns.residual_norm / ns.initial_norm : 0.0, el);
      // the Newton history of the stage: ||R|| / ||R_0|| after each iteration
      std::fprintf(stderr, "  history");
      for (int i = 0; i <= ns.iterations && i < 64; ++i)
        std::fprintf(stderr, " %.2e", ns.initial_norm > 0 ? ns.history[i] / ns.initial_norm : 0.0);
      std::fprintf(stderr, "\n");
      std::fflush(stderr);
    }
    if (s2 == ENP_OK) {
      e = cudaMemcpyAsync(u, ut, sizeof(double) * ntot, cudaMemcpyDeviceToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) { status = cuda_err(h, e, "continuation copy"); break; }
      lam = last ? 1.0 : nl;
      if (last) break;
      dl = std::min(dl * c->grow, c->step_max);
    } else if (s2 == ENP_ERR_NOT_CONVERGED || s2 == ENP_ERR_NONFINITE) {
      ++cs.failed_stages;  // discard the stage's iterate, retry with half the increment
      dl *= 0.5;
      if (dl < c->step_min) {
        status = ENP_ERR_NOT_CONVERGED;
        h->err = "continuation increment fell below step_min";
        break;
      }
    } else {
      status = s2;
      break;
    }
  }
  enp_set_phi_app(h, phi_app);
  cs.lambda = lam;
  if (st) *st = cs;
  cudaFree(ut);
  return status;
}

// dtheta[b][j] = <w_b, dR_b/dtheta_j> for theta = (D_1..D_m, c_in_1..c_in_{m-1},
// phi_app_0..phi_app_3): the parameter part of the adjoint.
namespace enp {
// out[j] = sum over operating points b (in order) of v[b][j].
__global__ void sum_over_batch_kernel(const double* __restrict__ v, int B, int nt,
                                      double* __restrict__ out) {
  for (int j = threadIdx.x; j < nt; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += v[(long long)b * nt + j];
    out[j] = s;
  }
}
}  // namespace enp

// <w_b, dR_b/dtheta_j> for every operating point into S.dsmall[b][j] (device).
static enp_status param_dots(enp_handle h, const double* u, const double* w, size_t extra) {
  SolverState& S = state_of(h);
  const int nt = h->prm.n_theta, B = h->batch;
  const long long n = h->n_dof;
  cudaError_t e = ensure(&S.dRdtheta, S.dRdtheta_count, (size_t)nt * B * n);
  if (e != cudaSuccess) return cuda_err(h, e, "cudaMalloc parameter Jacobian");
  enp_status st = enp_param_jacobian(h, u, S.dRdtheta);
  if (st != ENP_OK) return st;
  if ((e = small(h, (size_t)B * nt + extra)) != cudaSuccess) return cuda_err(h, e, "cudaMalloc small");
  if ((e = multidot<double>(h, S.dRdtheta, (long long)B * n, nt, w, S.dsmall)) != cudaSuccess)
    return cuda_err(h, e, "parameter dots");
  return ENP_OK;
}

extern "C" enp_status enp_param_vjp_total(enp_handle h, const double* u, const double* w,
                                          double* dtheta) {
  if (!h || !u || !w || !dtheta) return ENP_ERR_INVALID_ARG;
  const int nt = h->prm.n_theta, B = h->batch;
  enp_status st = param_dots(h, u, w, (size_t)nt);
  if (st != ENP_OK) return st;
  SolverState& S = state_of(h);
  double* tot = S.dsmall + (size_t)B * nt;
  enp::sum_over_batch_kernel<<<1, 32, 0, h->stream>>>(S.dsmall, B, nt, tot);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dtheta, tot, sizeof(double) * nt, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "parameter vjp (total)");
}

extern "C" enp_status enp_param_vjp(enp_handle h, const double* u, const double* w,
                                    double* dtheta) {
  if (!h || !u || !w || !dtheta) return ENP_ERR_INVALID_ARG;
  const int nt = h->prm.n_theta, B = h->batch;
  enp_status st = param_dots(h, u, w, 0);
  if (st != ENP_OK) return st;
  SolverState& S = state_of(h);
  cudaError_t e = cudaMemcpyAsync(dtheta, S.dsmall, sizeof(double) * B * nt, cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? ENP_OK : cuda_err(h, e, "parameter vjp");
}
