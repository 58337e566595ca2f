// Host side of the C ABI declared in include/enp_dg.h: handle creation (mesh
// upload, basis tables), problem data, and the operator entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/enp_dg.h"
#include "enp_internal.h"

using enp::OpParams;
using enp::Tables;

namespace {

// The physical coefficients of P in arithmetic type T (see PhysT).
template <class T>
void fill_phys(const OpParams& P, enp::PhysT<T>& o) {
  std::memset(&o, 0, sizeof(o));
  const int m = P.m;
  for (int k = 0; k < enp::kMaxSpecies; ++k) {
    o.D[k] = (T)P.D[k]; o.cin[k] = (T)P.cin[k]; o.mig[k] = (T)P.mig[k];
    o.acoef[k] = (T)P.acoef[k]; o.kcoef[k] = (T)P.kcoef[k]; o.z[k] = (T)P.z[k];
    o.zratio[k] = (T)(-P.z[k] / P.z[m - 1]);
  }
  o.neg_inv_zm = (T)(-1.0 / P.z[m - 1]);
  for (int i = 0; i < 8; ++i) o.vp[i] = (T)P.vp[i];
  o.vel_coef = (T)P.vel_coef;
  o.vel_kind = P.vel_kind;
  o.velA = (int)P.vp[0];
  o.velN = (int)P.vp[1];
  o.J0 = (T)P.J0; o.e1 = (T)P.e1; o.e2 = (T)P.e2;
  o.gam = (T)P.gam; o.gam1 = (T)(P.gam - 1.0); o.inv_cref = (T)P.inv_cref;
  o.ox_species_scale = (T)P.ox_species_scale; o.ox_charge_scale = (T)P.ox_charge_scale;
  for (int j = 0; j < 4; ++j) o.phiapp[j] = (T)P.phiapp[j];
  o.J0axis = P.J0axis;
  o.J0lo = (T)P.J0lo;
  o.J0half = (T)(0.5 * (P.J0hi - P.J0lo));
  o.J0inv_half = P.J0hi > P.J0lo ? (T)(1.0 / (0.5 * (P.J0hi - P.J0lo))) : (T)0;
  o.cip = (T)P.cip;
  o.bv_ox = P.bv_ox;
  const double zm = P.z[m - 1];
  for (int k = 0; k < enp::kMaxSpecies; ++k) {
    o.dmig[k] = (T)(P.z[k] * P.F / P.RT);
    o.da[k] = (T)(P.F * P.z[k]);
    o.dkc_own[k] = (T)(P.z[k] * P.z[k] * P.F * P.F / P.RT);
    o.dkc_m[k] = (T)(-P.z[k] * zm * P.F * P.F / P.RT);
  }
}

enp_status fail(enp_handle h, enp_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

enp_status cuda_fail(enp_handle h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (h) h->err = m;
  return e == cudaErrorMemoryAllocation ? ENP_ERR_OOM : ENP_ERR_CUDA;
}

// ---------------------------------------------------------------- 1D rules
// Legendre P_n(x) by the three-term recurrence.
double legendre_p(int n, double x) {
  if (n == 0) return 1.0;
  double a = 1.0, b = x;
  for (int k = 1; k < n; ++k) {
    double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
    a = b; b = c;
  }
  return b;
}

// Gauss-Legendre rule by Golub-Welsch: eigenvalues of the symmetric tridiagonal
// Jacobi matrix (off-diagonal k / sqrt(4k^2 - 1)) are the points; the weights are
// 2 times the squared first components of the normalised eigenvectors. The small
// dense eigenproblem is solved with cyclic Jacobi rotations.
void gauss_rule(int q, double* x, double* w) {
  std::vector<double> A(q * q, 0.0), V(q * q, 0.0);
  for (int k = 1; k < q; ++k) {
    double b = k / std::sqrt(4.0 * k * k - 1.0);
    A[k * q + k - 1] = A[(k - 1) * q + k] = b;
  }
  for (int i = 0; i < q; ++i) V[i * q + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < q; ++i)
      for (int j = i + 1; j < q; ++j) off += A[i * q + j] * A[i * q + j];
    if (off < 1e-34) break;
    for (int pp = 0; pp < q; ++pp)
      for (int r = pp + 1; r < q; ++r) {
        double apr = A[pp * q + r];
        if (std::fabs(apr) < 1e-300) continue;
        double theta = (A[r * q + r] - A[pp * q + pp]) / (2.0 * apr);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < q; ++k) {  // A <- A G (columns pp, r)
          double akp = A[k * q + pp], akr = A[k * q + r];
          A[k * q + pp] = c * akp - s * akr;
          A[k * q + r] = s * akp + c * akr;
        }
        for (int k = 0; k < q; ++k) {  // A <- G^T A (rows pp, r)
          double apk = A[pp * q + k], ark = A[r * q + k];
          A[pp * q + k] = c * apk - s * ark;
          A[r * q + k] = s * apk + c * ark;
        }
        for (int k = 0; k < q; ++k) {
          double vkp = V[k * q + pp], vkr = V[k * q + r];
          V[k * q + pp] = c * vkp - s * vkr;
          V[k * q + r] = s * vkp + c * vkr;
        }
      }
  }
  std::vector<int> ord(q);
  for (int i = 0; i < q; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[a * q + a] < A[b * q + b]; });
  for (int i = 0; i < q; ++i) {
    int j = ord[i];
    x[i] = A[j * q + j];
    w[i] = 2.0 * V[0 * q + j] * V[0 * q + j];
  }
  // symmetric rule: symmetrise to remove the last rounding
  for (int i = 0; i < q / 2; ++i) {
    double xs = 0.5 * (x[q - 1 - i] - x[i]), ws = 0.5 * (w[i] + w[q - 1 - i]);
    x[i] = -xs; x[q - 1 - i] = xs; w[i] = w[q - 1 - i] = ws;
  }
  if (q % 2) x[q / 2] = 0.0;
}

// Gauss-Lobatto nodes: the zeros of P_{p+1} - P_{p-1} (which is proportional to
// (1 - x^2) P_p'(x)), found by Newton with derivative (2p + 1) P_p.
void lobatto_nodes(int p, double* x) {
  x[0] = -1.0; x[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double t = -std::cos(M_PI * j / p);
    for (int it = 0; it < 60; ++it) {
      double f = legendre_p(p + 1, t) - legendre_p(p - 1, t);
      double df = (2.0 * p + 1.0) * legendre_p(p, t);
      double dt = f / df;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[j] = t;
  }
  for (int j = 0; j < (p + 1) / 2; ++j) {  // symmetrise
    double s = 0.5 * (x[p - j] - x[j]);
    x[j] = -s; x[p - j] = s;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
}

void barycentric_weights(int n, const double* x, double* lam) {
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0 / prod;
  }
}

// Differentiation matrix D[i][j] = l_j'(x_i) of the Lagrange basis on nodes x.
void diff_matrix(int n, const double* x, double* D) {
  std::vector<double> lam(n);
  barycentric_weights(n, x, lam.data());
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * n + j] = d;
      diag -= d;
    }
    D[i * n + i] = diag;
  }
}

void build_tables(int p, Tables& t) {
  const int n = p + 1, q = p + 2;
  std::memset(&t, 0, sizeof(t));
  double xl[enp::kMaxN], lam[enp::kMaxN];
  gauss_rule(q, t.xq, t.wq);
  lobatto_nodes(p, xl);
  barycentric_weights(n, xl, lam);
  for (int a = 0; a < q; ++a) {
    double x = t.xq[a];
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (x == xl[j]) hit = j;
    double den = 0.0;
    if (hit < 0)
      for (int j = 0; j < n; ++j) den += lam[j] / (x - xl[j]);
    for (int j = 0; j < n; ++j)
      t.B[a * n + j] = hit >= 0 ? (j == hit ? 1.0 : 0.0) : (lam[j] / (x - xl[j])) / den;
  }
  diff_matrix(q, t.xq, t.Dq);
  std::vector<double> DL(n * n);
  diff_matrix(n, xl, DL.data());
  for (int j = 0; j < n; ++j) {
    t.dL[j] = DL[0 * n + j];          // at x = -1
    t.dL[n + j] = DL[(n - 1) * n + j];  // at x = +1
  }
}

}  // namespace

bool enp::shape_supported(int dim, int p, int nf) {
  if (nf < 2 || nf > 3) return false;
  if (dim == 3) return p >= 1 && p <= 4;
  if (dim == 2) return p >= 1 && p <= 3;
  return false;
}

extern "C" {

enp_status enp_dg_create(enp_handle* out, const enp_mesh_desc* mesh, const enp_physics_desc* ph,
                         const enp_disc_desc* disc, void* stream) {
  if (!out) return ENP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !ph || !disc) return ENP_ERR_INVALID_ARG;
  const int dim = mesh->dim;
  if (dim != 2 && dim != 3) return ENP_ERR_INVALID_ARG;
  if (ph->m < 2 || ph->m > ENP_MAX_SPECIES || ph->z[ph->m - 1] == 0.0) return ENP_ERR_INVALID_ARG;
  if (!(ph->F > 0) || !(ph->RT > 0)) return ENP_ERR_INVALID_ARG;
  if (ph->bv_oxidant < -1 || ph->bv_oxidant >= ph->m) return ENP_ERR_INVALID_ARG;
  if (ph->velocity_kind != ENP_VEL_CONSTANT && ph->velocity_kind != ENP_VEL_PLATE)
    return ENP_ERR_INVALID_ARG;
  if (ph->velocity_kind == ENP_VEL_PLATE) {
    int A = (int)ph->vel_params[0], N = (int)ph->vel_params[1];
    if (A < 0 || A >= dim || N < 0 || N >= dim || !(ph->vel_params[3] > 0)) return ENP_ERR_INVALID_ARG;
  }
  if (ph->bv_J0_axis >= dim || (ph->bv_J0_axis >= 0 && !(ph->bv_J0_hi > ph->bv_J0_lo)))
    return ENP_ERR_INVALID_ARG;
  if (disc->batch < 1 || disc->batch > 65535 || disc->p < 1) return ENP_ERR_INVALID_ARG;
  if (disc->q != disc->p + 2) return ENP_ERR_UNSUPPORTED;
  if (!enp::shape_supported(dim, disc->p, ph->m)) return ENP_ERR_UNSUPPORTED;
  long long E = 1;
  for (int a = 0; a < dim; ++a) {
    if (mesh->n_el[a] < 1 || !mesh->coords[a]) return ENP_ERR_INVALID_ARG;
    for (int i = 0; i < mesh->n_el[a]; ++i)
      if (!(mesh->coords[a][i + 1] > mesh->coords[a][i])) return ENP_ERR_INVALID_ARG;
    E *= mesh->n_el[a];
  }
  if (E > (1LL << 30)) return ENP_ERR_INVALID_ARG;

  enp_handle h = new enp_dg();
  OpParams& P = h->prm;
  P.dim = dim;
  for (int a = 0; a < 3; ++a) P.ne[a] = a < dim ? mesh->n_el[a] : 1;
  P.E = (int)E;
  P.m = ph->m; P.NF = ph->m;
  P.p = disc->p; P.n = disc->p + 1; P.q = disc->q;
  P.Np = 1; P.Nq = 1; P.Nfq = 1;
  for (int a = 0; a < dim; ++a) { P.Np *= P.n; P.Nq *= P.q; }
  for (int a = 0; a < dim - 1; ++a) P.Nfq *= P.q;
  // boundary faces, side-major
  std::vector<uint8_t> tags;
  P.NBF = 0;
  for (int s = 0; s < 2 * dim; ++s) {
    int a = s / 2, nf = 1;
    for (int b = 0; b < dim; ++b)
      if (b != a) nf *= P.ne[b];
    P.side_off[s] = P.NBF;
    if (!mesh->face_tag[s]) { delete h; return ENP_ERR_INVALID_ARG; }
    for (int i = 0; i < nf; ++i) {
      uint8_t t = mesh->face_tag[s][i];
      if (t < ENP_FACE_WALL || t > ENP_FACE_ELECTRODE0 + 3) { delete h; return ENP_ERR_INVALID_ARG; }
      tags.push_back(t);
    }
    P.NBF += nf;
  }
  P.side_off[2 * dim] = P.NBF;
  const int m = ph->m;
  for (int k = 0; k < ENP_MAX_SPECIES; ++k) {
    P.z[k] = k < m ? ph->z[k] : 0.0;
    P.D[k] = k < m ? ph->D[k] : 0.0;
    P.cin[k] = k < m ? ph->c_in[k] : 0.0;
    P.mig[k] = P.acoef[k] = P.kcoef[k] = 0.0;
  }
  const double zm = ph->z[m - 1], mum = ph->D[m - 1] / ph->RT;
  for (int k = 0; k < m - 1; ++k) {
    const double muk = ph->D[k] / ph->RT;
    P.mig[k] = ph->z[k] * muk * ph->F;                              // z_k mu_k F
    P.acoef[k] = ph->F * ph->z[k] * (ph->D[k] - ph->D[m - 1]);      // a_km
    P.kcoef[k] = ph->z[k] * (ph->z[k] * muk - zm * mum) * ph->F * ph->F;  // kappa coefficient
  }
  P.F = ph->F;
  P.RT = ph->RT;
  P.vel_kind = ph->velocity_kind;
  for (int i = 0; i < 8; ++i) P.vp[i] = ph->vel_params[i];
  P.vel_coef = ph->velocity_kind == ENP_VEL_PLATE
                   ? 6.0 * ph->vel_params[4] / (ph->vel_params[3] * ph->vel_params[3]) : 0.0;
  P.bv_ox = ph->bv_oxidant;
  P.J0 = ph->bv_J0;
  P.e1 = ph->bv_alpha1 * ph->bv_n * ph->F / ph->RT;
  P.e2 = ph->bv_alpha2 * ph->bv_n * ph->F / ph->RT;
  P.gam = ph->bv_gamma;
  P.inv_cref = 1.0 / ph->bv_c_ref;
  P.ox_species_scale = -1.0 / (ph->bv_n * ph->F);
  P.ox_charge_scale = ph->bv_oxidant >= 0 ? -ph->z[ph->bv_oxidant] / ph->bv_n : 0.0;
  for (int j = 0; j < 4; ++j) P.phiapp[j] = ph->bv_phi_app[j];
  P.J0axis = ph->bv_J0_axis; P.J0lo = ph->bv_J0_lo; P.J0hi = ph->bv_J0_hi;
  P.cip = disc->C_IP;
  P.src = nullptr; P.dirv = nullptr; P.phiapp_batch = nullptr;
  P.batch_stride = (long long)P.NF * P.E * P.Np;
  fill_phys<double>(P, P.pd);
  fill_phys<float>(P, P.pf);
  fill_phys<enp::df>(P, P.pdf);
  P.arith = enp::kArithF64;
  P.batch = disc->batch;
  P.n_theta = 2 * P.m + 3;
  h->batch = disc->batch;
  h->n_dof = P.batch_stride;
  h->stream = (cudaStream_t)stream;
  build_tables(P.p, h->htab);

  cudaError_t e;
  for (int a = 0; a < dim; ++a) {
    e = cudaMalloc(&h->d_xv[a], sizeof(double) * (P.ne[a] + 1));
    if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "cudaMalloc coords"); enp_dg_destroy(h); return s; }
    e = cudaMemcpy(h->d_xv[a], mesh->coords[a], sizeof(double) * (P.ne[a] + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "upload coords"); enp_dg_destroy(h); return s; }
    P.xv[a] = h->d_xv[a];
    std::vector<float> cf(mesh->coords[a], mesh->coords[a] + P.ne[a] + 1);
    e = cudaMalloc(&h->d_xvf[a], sizeof(float) * (P.ne[a] + 1));
    if (e == cudaSuccess)
      e = cudaMemcpy(h->d_xvf[a], cf.data(), sizeof(float) * (P.ne[a] + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "upload coords (FP32)"); enp_dg_destroy(h); return s; }
    P.xvf[a] = h->d_xvf[a];
    std::vector<float2> cd(P.ne[a] + 1);
    for (int i = 0; i <= P.ne[a]; ++i) {
      const enp::df x(mesh->coords[a][i]);
      cd[i] = make_float2(x.hi, x.lo);
    }
    e = cudaMalloc(&h->d_xvdf[a], sizeof(float2) * (P.ne[a] + 1));
    if (e == cudaSuccess)
      e = cudaMemcpy(h->d_xvdf[a], cd.data(), sizeof(float2) * (P.ne[a] + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "upload coords (double-float)"); enp_dg_destroy(h); return s; }
    P.xvdf[a] = h->d_xvdf[a];
  }
  for (int a = dim; a < 3; ++a) { P.xv[a] = nullptr; P.xvf[a] = nullptr; P.xvdf[a] = nullptr; }
  e = cudaMalloc(&h->d_btag, tags.size());
  if (e == cudaSuccess) e = cudaMemcpy(h->d_btag, tags.data(), tags.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_tab, sizeof(Tables));
  if (e == cudaSuccess) e = cudaMemcpy(h->d_tab, &h->htab, sizeof(Tables), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "upload tables"); enp_dg_destroy(h); return s; }
  P.btag = h->d_btag;
  P.fbuf = nullptr;
  P.fbuf_stride = 0;
  for (int a = 0; a < 4; ++a) P.foff[a] = 0;
  if (dim == 3) {
    long long off = 0;
    for (int a = 0; a < 3; ++a) {
      const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
      P.foff[a] = off;
      off += (long long)(P.ne[a] + 1) * P.ne[b0] * P.ne[b1];
    }
    P.foff[3] = off;
    P.fbuf_stride = off * 2 * 2 * P.NF * (long long)P.n * P.n;
    e = cudaMalloc(&h->d_fbuf, sizeof(double) * P.fbuf_stride * P.batch);
    if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "cudaMalloc face buffer"); enp_dg_destroy(h); return s; }
    P.fbuf = h->d_fbuf;
  }
  e = enp::prepare_tables<double>(P.p, h->htab);
  if (e == cudaSuccess) e = enp::prepare_tables<float>(P.p, h->htab);
  if (e == cudaSuccess && dim == 3) e = enp::prepare_tables_df(P.p, h->htab);
  if (e != cudaSuccess) { enp_status s = cuda_fail(h, e, "upload constant tables"); enp_dg_destroy(h); return s; }
  *out = h;
  return ENP_OK;
}

enp_status enp_dg_destroy(enp_handle h) {
  if (!h) return ENP_ERR_INVALID_ARG;
  enp_solver_free(h);
  for (int a = 0; a < 3; ++a) { cudaFree(h->d_xv[a]); cudaFree(h->d_xvf[a]); cudaFree(h->d_xvdf[a]); }
  cudaFree(h->d_btag);
  cudaFree(h->d_tab);
  cudaFree(h->d_src);
  cudaFree(h->d_dir);
  cudaFree(h->d_phiapp);
  cudaFree(h->d_fbuf);
  delete h;
  return ENP_OK;
}

enp_status enp_dg_sizes(enp_handle h, long long* n_dof, int* n_fields, int* n_nodes,
                        int* n_qpoints, int* n_bfaces) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (n_dof) *n_dof = h->n_dof;
  if (n_fields) *n_fields = h->prm.NF;
  if (n_nodes) *n_nodes = h->prm.Np;
  if (n_qpoints) *n_qpoints = h->prm.Nq;
  if (n_bfaces) *n_bfaces = h->prm.NBF;
  return ENP_OK;
}

enp_status enp_set_stream(enp_handle h, void* stream) {
  if (!h) return ENP_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return ENP_OK;
}

enp_status enp_set_sources(enp_handle h, const double* src, const double* dir) {
  if (!h) return ENP_ERR_INVALID_ARG;
  const OpParams& P = h->prm;
  size_t ns = (size_t)P.NF * P.E * P.Nq, nd = (size_t)P.NF * P.NBF * P.Nfq;
  cudaError_t e;
  if (src) {
    if (!h->d_src) {
      e = cudaMalloc(&h->d_src, ns * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc sources");
    }
    e = cudaMemcpyAsync(h->d_src, src, ns * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy sources");
  }
  if (dir) {
    if (!h->d_dir) {
      e = cudaMalloc(&h->d_dir, nd * sizeof(double));
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc dirichlet");
    }
    e = cudaMemcpyAsync(h->d_dir, dir, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy dirichlet");
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_sources");
  h->prm.src = src ? h->d_src : nullptr;
  h->prm.dirv = dir ? h->d_dir : nullptr;
  return ENP_OK;
}

enp_status enp_set_phi_app(enp_handle h, const double* phi_app) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (!phi_app) { h->prm.phiapp_batch = nullptr; return ENP_OK; }
  cudaError_t e;
  if (!h->d_phiapp) {
    e = cudaMalloc(&h->d_phiapp, sizeof(double) * 4 * h->batch);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc phi_app");
  }
  e = cudaMemcpy(h->d_phiapp, phi_app, sizeof(double) * 4 * h->batch, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy phi_app");
  h->prm.phiapp_batch = h->d_phiapp;
  return ENP_OK;
}

enp_status enp_quadrature_points(enp_handle h, double* xq, double* xbq) {
  if (!h) return ENP_ERR_INVALID_ARG;
  const OpParams& P = h->prm;
  const Tables& T = h->htab;
  std::vector<double> xv[3];
  for (int a = 0; a < P.dim; ++a) {
    xv[a].resize(P.ne[a] + 1);
    cudaError_t e = cudaMemcpy(xv[a].data(), P.xv[a], sizeof(double) * (P.ne[a] + 1),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "read coords");
  }
  const int q = P.q;
  if (xq) {
    std::vector<double> hq((size_t)P.E * P.Nq * 3, 0.0);
    for (int e = 0; e < P.E; ++e) {
      int idx[3] = {e % P.ne[0], (e / P.ne[0]) % P.ne[1], e / (P.ne[0] * P.ne[1])};
      for (int pt = 0; pt < P.Nq; ++pt) {
        int k[3] = {pt % q, (pt / q) % q, pt / (q * q)};
        for (int a = 0; a < P.dim; ++a) {
          double lo = xv[a][idx[a]], hh = xv[a][idx[a] + 1] - lo;
          hq[((size_t)e * P.Nq + pt) * 3 + a] = lo + 0.5 * (T.xq[k[a]] + 1.0) * hh;
        }
      }
    }
    cudaError_t e = cudaMemcpy(xq, hq.data(), hq.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "write xq");
  }
  if (xbq) {
    std::vector<double> hb((size_t)P.NBF * P.Nfq * 3, 0.0);
    for (int s = 0; s < 2 * P.dim; ++s) {
      int a = s / 2, hi = s & 1, b[2] = {0, 0}, nb = 0;
      for (int c = 0; c < P.dim; ++c)
        if (c != a) b[nb++] = c;
      int n0 = P.ne[b[0]], n1 = P.dim == 3 ? P.ne[b[1]] : 1;
      for (int j1 = 0; j1 < n1; ++j1)
        for (int j0 = 0; j0 < n0; ++j0) {
          int bf = P.side_off[s] + j0 + n0 * j1;
          for (int pt = 0; pt < P.Nfq; ++pt) {
            double* o = &hb[((size_t)bf * P.Nfq + pt) * 3];
            o[a] = hi ? xv[a][P.ne[a]] : xv[a][0];
            double l0 = xv[b[0]][j0], h0 = xv[b[0]][j0 + 1] - l0;
            o[b[0]] = l0 + 0.5 * (T.xq[pt % q] + 1.0) * h0;
            if (P.dim == 3) {
              double l1 = xv[b[1]][j1], h1 = xv[b[1]][j1 + 1] - l1;
              o[b[1]] = l1 + 0.5 * (T.xq[pt / q] + 1.0) * h1;
            }
          }
        }
    }
    cudaError_t e = cudaMemcpy(xbq, hb.data(), hb.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(h, e, "write xbq");
  }
  return ENP_OK;
}

static enp_status run_op_f64(enp_handle h, int mode, const double* u, const double* v, double* out) {
  if (!h || !u || !out || (mode != 0 && !v)) return fail(h, ENP_ERR_INVALID_ARG, "null argument");
  cudaError_t e = enp::launch_op<double>(mode, h->prm, h->d_tab, u, v, out, h->batch, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "operator launch");
  return ENP_OK;
}

enp_status enp_residual(enp_handle h, const double* u, double* r) { return run_op_f64(h, 0, u, nullptr, r); }
enp_status enp_jvp(enp_handle h, const double* u, const double* v, double* jv) { return run_op_f64(h, 1, u, v, jv); }
enp_status enp_vjp(enp_handle h, const double* u, const double* w, double* jtw) { return run_op_f64(h, 2, u, w, jtw); }

enp_status enp_jvp_f32(enp_handle h, const float* u, const float* v, float* jv) {
  if (!h || !u || !v || !jv) return fail(h, ENP_ERR_INVALID_ARG, "null argument");
  cudaError_t e = enp::launch_op<float>(1, h->prm, h->d_tab, u, v, jv, h->batch, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "operator launch (f32)");
  return ENP_OK;
}

enp_status enp_param_count(enp_handle h, int* n_theta) {
  if (!h || !n_theta) return ENP_ERR_INVALID_ARG;
  *n_theta = h->prm.n_theta;
  return ENP_OK;
}

enp_status enp_param_jacobian(enp_handle h, const double* u, double* dRdtheta) {
  if (!h || !u || !dRdtheta) return fail(h, ENP_ERR_INVALID_ARG, "null argument");
  if (h->prm.dim != 3) return fail(h, ENP_ERR_UNSUPPORTED, "dR/dtheta is built for hexahedra");
  cudaError_t e = enp::launch_op<double>(enp::kParam, h->prm, h->d_tab, u, nullptr, dRdtheta,
                                         h->batch * h->prm.n_theta, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "parameter Jacobian launch");
  return ENP_OK;
}

}  // extern "C"

// Time every feasible elements-per-block value of the hexahedral kernel for
// each operator mode on this handle's mesh (three launches each, CUDA events)
// and keep the fastest. The block-column pass follows the J v choice.
template <class R>
static cudaError_t tune_launch(int mode, const OpParams& P, const Tables* t, enp::io_t<R>* u,
                               enp::io_t<R>* v, enp::io_t<R>* out, cudaStream_t s) {
  if constexpr (std::is_same<R, enp::df>::value) return enp::launch_op_df(mode, P, u, v, out, 1, s);
  else return enp::launch_op<R>(mode, P, t, u, v, out, 1, s);
}

// The tile shapes of one operator mode: faces per block of the face kernel
// (modes R, J v, J^T w), then elements per block of the element kernel, each
// timed over its feasible range (three launches of the whole operator, CUDA
// events) with the other at its current value; the fastest is kept.
template <class R>
static cudaError_t tune_mode(enp_handle h, int mode, enp::io_t<R>* u, enp::io_t<R>* v,
                             enp::io_t<R>* out, int* chosen, int* chosen_fpb) {
  OpParams P = h->prm;
  P.arith = enp::kArithF64;  // launch_op<double> then runs the FP64 kernels themselves
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t err = cudaSuccess;
  auto time_it = [&](float* ms) -> cudaError_t {
    cudaError_t er = tune_launch<R>(mode, P, h->d_tab, u, v, out, h->stream);
    if (er != cudaSuccess) return er;
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < 3; ++r) tune_launch<R>(mode, P, h->d_tab, u, v, out, h->stream);
    cudaEventRecord(e1, h->stream);
    er = cudaEventSynchronize(e1);
    *ms = 0.f;
    cudaEventElapsedTime(ms, e0, e1);
    return er;
  };
  int best_fpb = 0;
  if (mode <= enp::kVjp) {
    const int fx = enp::fpb3d_max<R>(P.p, P.NF, mode);
    float best = 1e30f;
    for (int f = 1; f <= fx && err == cudaSuccess; ++f) {
      enp::fpb3d_set<R>(P.p, P.NF, mode, f);
      float ms = 0.f;
      err = time_it(&ms);
      if (err == cudaSuccess && ms < best) { best = ms; best_fpb = f; }
    }
    enp::fpb3d_set<R>(P.p, P.NF, mode, best_fpb);
  }
  const int mx = enp::eb3d_max<R>(P.p, P.NF, mode);
  float best = 1e30f;
  int best_eb = 0;
  for (int eb = 1; eb <= mx && err == cudaSuccess; ++eb) {
    enp::eb3d_set<R>(P.p, P.NF, mode, eb);
    float ms = 0.f;
    err = time_it(&ms);
    if (err == cudaSuccess && ms < best) { best = ms; best_eb = eb; }
  }
  enp::eb3d_set<R>(P.p, P.NF, mode, best_eb);
  if (mode == enp::kJvp) enp::eb3d_set<R>(P.p, P.NF, enp::kBlockCol, best_eb);
  if (chosen) *chosen = best_eb;
  if (chosen_fpb) *chosen_fpb = best_fpb;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

extern "C" {

enp_status enp_autotune(enp_handle h, int* chosen) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (h->prm.dim != 3) return ENP_OK;  // the quad kernel has a fixed shape
  const size_t n = (size_t)h->n_dof;
  double *u = nullptr, *v = nullptr, *o = nullptr;
  cudaError_t e = cudaMalloc(&u, 3 * n * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc autotune");
  v = u + n;
  o = v + n;
  cudaMemsetAsync(u, 0, 3 * n * sizeof(double), h->stream);
  int c[5] = {0, 0, 0, 0, 0}, f[5] = {0, 0, 0, 0, 0};
  if (h->prm.arith == enp::kArithDF) {  // the FP64-accurate operator runs in double-float
    e = tune_mode<enp::df>(h, enp::kResidual, u, v, o, &c[0], &f[0]);
    if (e == cudaSuccess) e = tune_mode<enp::df>(h, enp::kJvp, u, v, o, &c[1], &f[1]);
    if (e == cudaSuccess) e = tune_mode<enp::df>(h, enp::kVjp, u, v, o, &c[2], &f[2]);
  } else {
    e = tune_mode<double>(h, enp::kResidual, u, v, o, &c[0], &f[0]);
    if (e == cudaSuccess) e = tune_mode<double>(h, enp::kJvp, u, v, o, &c[1], &f[1]);
    if (e == cudaSuccess) e = tune_mode<double>(h, enp::kVjp, u, v, o, &c[2], &f[2]);
  }
  if (e == cudaSuccess)
    e = tune_mode<float>(h, enp::kJvp, (float*)u, (float*)v, (float*)o, &c[3], &f[3]);
  if (e == cudaSuccess)
    e = tune_mode<float>(h, enp::kResidual, (float*)u, (float*)v, (float*)o, &c[4], &f[4]);
  cudaFree(u);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  if (chosen)
    for (int i = 0; i < 5; ++i) chosen[i] = c[i];
  return ENP_OK;
}

enp_status enp_set_arithmetic(enp_handle h, int arith) {
  if (!h) return ENP_ERR_INVALID_ARG;
  if (arith != ENP_ARITH_F64 && arith != ENP_ARITH_DF32)
    return fail(h, ENP_ERR_INVALID_ARG, "arith must be ENP_ARITH_F64 or ENP_ARITH_DF32");
  h->prm.arith = (arith == ENP_ARITH_DF32 && h->prm.dim == 3) ? enp::kArithDF : enp::kArithF64;
  return ENP_OK;
}

enp_status enp_get_arithmetic(enp_handle h, int* arith) {
  if (!h || !arith) return ENP_ERR_INVALID_ARG;
  *arith = h->prm.arith == enp::kArithDF ? ENP_ARITH_DF32 : ENP_ARITH_F64;
  return ENP_OK;
}

enp_status enp_launch_shapes(enp_handle h, int* eb, int* fpb) {
  if (!h) return ENP_ERR_INVALID_ARG;
  const OpParams& P = h->prm;
  if (P.dim != 3) {
    for (int i = 0; i < 5; ++i) { if (eb) eb[i] = 0; if (fpb) fpb[i] = 0; }
    return ENP_OK;
  }
  const bool dfa = P.arith == enp::kArithDF;
  const int modes[5] = {enp::kResidual, enp::kJvp, enp::kVjp, enp::kJvp, enp::kResidual};
  for (int i = 0; i < 5; ++i) {
    const int md = modes[i];
    if (i < 3) {
      if (eb) eb[i] = dfa ? enp::eb3d_get<enp::df>(P.p, P.NF, md) : enp::eb3d_get<double>(P.p, P.NF, md);
      if (fpb) fpb[i] = dfa ? enp::fpb3d_get<enp::df>(P.p, P.NF, md) : enp::fpb3d_get<double>(P.p, P.NF, md);
    } else {
      if (eb) eb[i] = enp::eb3d_get<float>(P.p, P.NF, md);
      if (fpb) fpb[i] = enp::fpb3d_get<float>(P.p, P.NF, md);
    }
  }
  return ENP_OK;
}

const char* enp_last_error(enp_handle h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
