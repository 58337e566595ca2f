"""Test infrastructure: the CPU FP64 oracle for the CNP discontinuous Galerkin operator.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import
this package. It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``enp_oracle.cpp`` (full-quadrature, element-by-element
assembly of Eq. NPDG and Eq. chargeDG of Sec. 3.3, forward dual numbers for
J(u)v). This module builds it with the host compiler, binds it through ctypes,
and adds a Newton solver with a sparse direct linear solve (scipy SuperLU) for
the manufactured-solution pins on small meshes (Sec. 4 "Newton's method with
backtracking line search", Sec. 5.1).

Pin status of each function (what fixes it other than itself) is listed in the
tests: tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enp_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, OpenMP). Returns its path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        lib.oracle_create.restype = P
        lib.oracle_create.argtypes = [I, P, P, P, I, P, P, P, D, D, I, P, I, P, I, I, D]
        lib.oracle_destroy.argtypes = [P]
        lib.oracle_num_threads.restype = I
        lib.oracle_set_threads.argtypes = [I]
        lib.oracle_rules.argtypes = [I, I, P, P, P]
        lib.oracle_quad_points.argtypes = [P, P, P]
        lib.oracle_node_points.argtypes = [P, P]
        lib.oracle_eval_quad.argtypes = [P, P, P, P]
        lib.oracle_residual.argtypes = [P, P, P, P, P, I, P]
        lib.oracle_jvp.argtypes = [P, P, P, P, P, P, I, P]
        lib.oracle_vjp_entries.argtypes = [P, P, P, P, P, P, I, P]
        lib.oracle_param_jacobian.argtypes = [P, P, P, P, I, P]
        lib.oracle_jacobian_coo.restype = LL
        lib.oracle_jacobian_coo.argtypes = [P, P, P, P, P, P, P, LL]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def rules(p: int, q: int):
    """(Gauss-Legendre points, weights) with q points and the p+1 Gauss-Lobatto nodes."""
    lib = _load()
    xg, wg, xn = np.zeros(q), np.zeros(q), np.zeros(p + 1)
    lib.oracle_rules(p, q, _ptr(xg), _ptr(wg), _ptr(xn))
    return xg, wg, xn


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


class Oracle:
    """The oracle for one problem (a ``workloads.Problem``).

    Vectors are flat float64 arrays in the layout [field][element][node],
    field 0 = Phi, field k = c_k; elements lexicographic (x fastest); nodes the
    tensor Gauss-Lobatto nodes, lexicographic (x fastest).
    """

    def __init__(self, prob, src=None, dirichlet=None):
        lib = _load()
        self.prob = prob
        self._lib = lib
        ne = np.array(list(prob.n_el[: prob.dim]) + [1] * (3 - prob.dim), dtype=np.int32)
        coords = np.concatenate([np.asarray(prob.coords[a], dtype=np.float64)
                                 for a in range(prob.dim)])
        tags = np.concatenate([np.asarray(t, dtype=np.uint8) for t in prob.tags])
        z = np.zeros(4); D = np.zeros(4); cin = np.zeros(4)
        z[: prob.m] = prob.z; D[: prob.m] = prob.D; cin[: prob.m] = prob.c_in
        vp = np.zeros(8); vp[: len(prob.vel_params)] = prob.vel_params
        bvp = prob.bv_params()
        self._keep = (ne, coords, tags, z, D, cin, vp, bvp)
        self.h = lib.oracle_create(prob.dim, _ptr(ne), _ptr(coords), _ptr(tags), prob.m,
                                   _ptr(z), _ptr(D), _ptr(cin), prob.F, prob.RT,
                                   prob.vel_kind, _ptr(vp), prob.bv_oxidant, _ptr(bvp),
                                   prob.p, prob.q, prob.C_IP)
        if not self.h:
            raise ValueError("oracle_create rejected the problem")
        self.src = _f64(src)
        self.dirichlet = _f64(dirichlet)
        self.N = prob.n_dof

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.oracle_destroy(h)
            self.h = None

    def _elems(self, elems):
        if elems is None:
            return None, 0
        e = np.ascontiguousarray(elems, dtype=np.int32)
        return e, len(e)

    def residual(self, u, elems=None, out=None):
        """R(u) (Eq. NPDG, Eq. chargeDG); with ``elems`` only those elements' rows."""
        u = _f64(u)
        r = np.zeros(self.N) if out is None else out
        e, n = self._elems(elems)
        self._lib.oracle_residual(self.h, _ptr(u), _ptr(self.src), _ptr(self.dirichlet),
                                  _ptr(e), n, _ptr(r))
        return r

    def jvp(self, u, v, elems=None):
        """J(u) v by forward dual numbers."""
        u, v = _f64(u), _f64(v)
        r = np.zeros(self.N)
        e, n = self._elems(elems)
        self._lib.oracle_jvp(self.h, _ptr(u), _ptr(v), _ptr(self.src), _ptr(self.dirichlet),
                             _ptr(e), n, _ptr(r))
        return r

    def vjp_entries(self, u, w, cols):
        """(J(u)^T w)[cols], one dual sweep per column."""
        u, w = _f64(u), _f64(w)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros(len(cols))
        self._lib.oracle_vjp_entries(self.h, _ptr(u), _ptr(w), _ptr(self.src),
                                     _ptr(self.dirichlet), _ptr(cols), len(cols), _ptr(out))
        return out

    def param_jacobian(self, u):
        """dR/dtheta [n_theta, N] for theta = (D_1..D_m, c_in_1..c_in_{m-1},
        phi_app_0..phi_app_3), one dual sweep per parameter."""
        nt = 2 * self.prob.m + 3
        out = np.zeros((nt, self.N))
        u = _f64(u)
        for j in range(nt):
            self._lib.oracle_param_jacobian(self.h, _ptr(u), _ptr(self.src), _ptr(self.dirichlet),
                                            j, _ptr(out[j]))
        return out

    def jacobian(self, u):
        """The assembled Jacobian J(u) as a scipy CSR matrix."""
        import scipy.sparse as sp
        P = self.prob
        nb = P.n_fields * P.Np
        cap = P.E * (2 * P.dim + 1) * nb * nb
        ri = np.zeros(cap, dtype=np.int64); ci = np.zeros(cap, dtype=np.int64)
        vals = np.zeros(cap)
        nnz = self._lib.oracle_jacobian_coo(self.h, _ptr(_f64(u)), _ptr(self.src),
                                            _ptr(self.dirichlet), _ptr(ri), _ptr(ci),
                                            _ptr(vals), cap)
        if nnz < 0:
            raise RuntimeError("jacobian capacity exceeded")
        return sp.csr_matrix((vals[:nnz], (ri[:nnz], ci[:nnz])), shape=(self.N, self.N))

    def quad_points(self):
        """(volume quadrature points [E, Nq, 3], boundary-face points [NBF, Nfq, 3])."""
        P = self.prob
        xq = np.zeros((P.E, P.Nq, 3)); xb = np.zeros((P.n_bfaces, P.Nfq, 3))
        self._lib.oracle_quad_points(self.h, _ptr(xq), _ptr(xb))
        return xq, xb

    def eval_quad(self, u):
        """(field values at volume quadrature points [NF, E, Nq], JxW [E, Nq])."""
        P = self.prob
        vals = np.zeros((P.n_fields, P.E, P.Nq)); jxw = np.zeros((P.E, P.Nq))
        self._lib.oracle_eval_quad(self.h, _ptr(_f64(u)), _ptr(vals), _ptr(jxw))
        return vals, jxw

    def node_points(self):
        """Physical coordinates of the nodes of one field, [E, Np, 3]."""
        P = self.prob
        xn = np.zeros((P.E, P.Np, 3))
        self._lib.oracle_node_points(self.h, _ptr(xn))
        return xn

    def block_diagonal(self, u):
        """The element-diagonal blocks of the assembled J(u): [E, nb, nb] with
        row/column index f * Np + i (the "element-wise Jacobi" of Sec. 4.2)."""
        P = self.prob
        J = self.jacobian(u).tocsr()
        nb = P.n_fields * P.Np
        out = np.zeros((P.E, nb, nb))
        loc = np.arange(nb)
        f, i = loc // P.Np, loc % P.Np
        for e in range(P.E):
            g = f * P.E * P.Np + e * P.Np + i
            out[e] = J[g][:, g].toarray()
        return out

    def block_jacobi_apply(self, blocks, x):
        """y_e = B_e^{-1} x_e for every element (dense LU solves)."""
        P = self.prob
        xe = x.reshape(P.n_fields, P.E, P.Np).transpose(1, 0, 2).reshape(P.E, -1)
        ye = np.linalg.solve(blocks, xe[..., None])[..., 0]
        return ye.reshape(P.E, P.n_fields, P.Np).transpose(1, 0, 2).reshape(-1)

    def linear_solve(self, u, b):
        """x with J(u) x = b, by a sparse direct solve (SuperLU)."""
        import scipy.sparse.linalg as spla
        return spla.spsolve(self.jacobian(u).tocsc(), np.asarray(b, dtype=np.float64))

    def newton_solve(self, u0, rtol=1e-10, max_it=30, c_armijo=1e-4):
        """Newton's method with a backtracking line search on ||R||, each linear
        system solved directly (sparse LU). Small meshes only."""
        import scipy.sparse.linalg as spla
        u = _f64(u0).copy()
        r = self.residual(u)
        r0 = np.linalg.norm(r)
        hist = [r0]
        for _ in range(max_it):
            if np.linalg.norm(r) <= rtol * max(r0, 1e-300):
                break
            J = self.jacobian(u).tocsc()
            du = spla.spsolve(J, -r)
            lam, nr = 1.0, np.linalg.norm(r)
            while True:
                ut = u + lam * du
                rt = self.residual(ut)
                if np.linalg.norm(rt) <= (1 - c_armijo * lam) * nr or lam < 1e-4:
                    break
                lam *= 0.5
            u, r = ut, rt
            hist.append(np.linalg.norm(r))
        return u, hist


def potential_initial_guess(orc, prob, phi0, rtol=1e-12, max_it=30, c_armijo=1e-4):
    """The initial guess of Sec. 4.3 ("Implementation"): every concentration at
    its inlet value c_k^in, and the potential from the charge-conservation
    equation at these constant concentrations, R_Phi(Phi; c^in) = 0 (the rows of
    Eq. chargeDG). With Butler-Volmer electrodes that equation is nonlinear in
    Phi, so it is solved by Newton's method with backtracking on ||R_Phi||, each
    step a direct solve with the Phi-Phi block of the assembled Jacobian (the
    paper hands the same equation to its potential-block solver). phi0: the
    starting potential [E * Np]. Returns (u [n_dof], history of ||R_Phi||)."""
    import scipy.sparse.linalg as spla
    n_phi = prob.E * prob.Np
    u = np.zeros(prob.n_dof)
    u[:n_phi] = _f64(phi0)
    for k in range(prob.m - 1):
        u[(k + 1) * n_phi:(k + 2) * n_phi] = prob.c_in[k]
    r = orc.residual(u)[:n_phi]
    r0 = np.linalg.norm(r)
    hist = [r0]
    for _ in range(max_it):
        if np.linalg.norm(r) <= rtol * max(r0, 1e-300):
            break
        A = orc.jacobian(u).tocsr()[:n_phi, :n_phi].tocsc()
        dphi = spla.spsolve(A, -r)
        lam, nr = 1.0, np.linalg.norm(r)
        while True:
            ut = u.copy()
            ut[:n_phi] += lam * dphi
            rt = orc.residual(ut)[:n_phi]
            if np.linalg.norm(rt) <= (1 - c_armijo * lam) * nr or lam < 1e-4:
                break
            lam *= 0.5
        u, r = ut, rt
        hist.append(np.linalg.norm(r))
    return u, hist


def recover_cm(prob, u):
    """The eliminated concentration c_m = -(1/z_m) sum_{k<m} z_k c_k
    (Eq. substitution), node by node: [E * Np]."""
    uu = np.asarray(u, dtype=np.float64).reshape(prob.n_fields, prob.E * prob.Np)
    s = np.zeros(prob.E * prob.Np)
    for k in range(prob.m - 1):
        s = s + prob.z[k] * uu[k + 1]
    return -s / prob.z[prob.m - 1]
