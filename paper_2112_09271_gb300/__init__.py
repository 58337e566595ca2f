"""Python binding of the GB300 CNP discontinuous Galerkin operator (libenp_dg.so).

Argument marshalling only: every step of the operator, the preconditioner and
the solvers runs in the library's CUDA kernels. PyTorch supplies device memory
and streams. There is no fallback: if the shared library is missing or cannot
be loaded, every entry point raises.

The C ABI is declared in include/enp_dg.h; each method here has the name of the
C function it calls, without the ``enp_`` prefix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libenp_dg.so")
SOURCES = ["enp_api.cu", "op_f64.cu", "op_f32.cu", "op_df.cu", "op_df_p1.cu", "op_df_p2.cu",
           "op_df_p3.cu", "op_df_p4.cu", "enp_solver.cu", "enp_noalloc.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", ARCH, "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr"]

ENP_OK, ENP_ERR_INVALID_ARG, ENP_ERR_CUDA, ENP_ERR_OOM, ENP_ERR_NONFINITE = 0, 1, 2, 3, 4
ENP_ERR_NOT_CONVERGED, ENP_ERR_TIMEOUT, ENP_ERR_UNSUPPORTED = 5, 6, 7
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NONFINITE", 5: "NOT_CONVERGED",
           6: "TIMEOUT", 7: "UNSUPPORTED"}


class EnpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (one object per source, in parallel)
    and link libenp_dg.so in-tree. Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)
                   if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(_ROOT, "include", "enp_dg.h"))
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(_BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ----------------------------------------------------------------- ctypes ABI
class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_el", ctypes.c_int * 3),
                ("coords", ctypes.c_void_p * 3), ("face_tag", ctypes.c_void_p * 6)]


class PhysicsDesc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("z", ctypes.c_double * 4), ("D", ctypes.c_double * 4),
                ("c_in", ctypes.c_double * 4), ("F", ctypes.c_double), ("RT", ctypes.c_double),
                ("velocity_kind", ctypes.c_int), ("vel_params", ctypes.c_double * 8),
                ("bv_oxidant", ctypes.c_int), ("bv_J0", ctypes.c_double),
                ("bv_alpha1", ctypes.c_double), ("bv_alpha2", ctypes.c_double),
                ("bv_n", ctypes.c_double), ("bv_gamma", ctypes.c_double),
                ("bv_c_ref", ctypes.c_double), ("bv_phi_app", ctypes.c_double * 4),
                ("bv_J0_axis", ctypes.c_int), ("bv_J0_lo", ctypes.c_double),
                ("bv_J0_hi", ctypes.c_double)]


class DiscDesc(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("q", ctypes.c_int), ("C_IP", ctypes.c_double),
                ("batch", ctypes.c_int)]


class KrylovOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_it", ctypes.c_int), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("graph", ctypes.c_int)]


class KrylovStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("initial_norm", ctypes.c_double), ("residual_norm", ctypes.c_double),
                ("relative_residual", ctypes.c_double)]


class NewtonOpts(ctypes.Structure):
    _fields_ = [("max_it", ctypes.c_int), ("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("armijo_c", ctypes.c_double), ("max_backtracks", ctypes.c_int),
                ("bj_storage", ctypes.c_int), ("mixed", ctypes.c_int), ("krylov", KrylovOpts),
                ("pc_lag", ctypes.c_int), ("device_loop", ctypes.c_int)]


class NewtonStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("krylov_iterations", ctypes.c_int),
                ("converged", ctypes.c_int), ("initial_norm", ctypes.c_double),
                ("residual_norm", ctypes.c_double), ("history", ctypes.c_double * 64),
                ("setups", ctypes.c_int), ("setup_seconds", ctypes.c_double),
                ("krylov_seconds", ctypes.c_double)]


class ContinuationOpts(ctypes.Structure):
    _fields_ = [("step0", ctypes.c_double), ("step_max", ctypes.c_double),
                ("step_min", ctypes.c_double), ("grow", ctypes.c_double),
                ("stage_rtol", ctypes.c_double), ("stage_max_it", ctypes.c_int)]


class ContinuationStats(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int), ("failed_stages", ctypes.c_int),
                ("newton_iterations", ctypes.c_int), ("krylov_iterations", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("last", NewtonStats)]


BJ_F64, BJ_F32, BJ_BF16 = 0, 1, 2
ARITH_F64, ARITH_DF32 = 0, 1

_lib = None

# (name, restype, argtypes) of every exported function declared in include/enp_dg.h
_V, _I, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
_PROTOS = [
    ("enp_dg_create", _I, [ctypes.POINTER(_V), ctypes.POINTER(MeshDesc),
                           ctypes.POINTER(PhysicsDesc), ctypes.POINTER(DiscDesc), _V]),
    ("enp_dg_destroy", _I, [_V]),
    ("enp_dg_sizes", _I, [_V, ctypes.POINTER(_LL), ctypes.POINTER(_I), ctypes.POINTER(_I),
                          ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("enp_set_stream", _I, [_V, _V]),
    ("enp_set_sources", _I, [_V, _V, _V]),
    ("enp_set_phi_app", _I, [_V, _V]),
    ("enp_quadrature_points", _I, [_V, _V, _V]),
    ("enp_residual", _I, [_V, _V, _V]),
    ("enp_jvp", _I, [_V, _V, _V, _V]),
    ("enp_jvp_f32", _I, [_V, _V, _V, _V]),
    ("enp_vjp", _I, [_V, _V, _V, _V]),
    ("enp_recover_cm", _I, [_V, _V, _V]),
    ("enp_inner_product", _I, [_V, _V, _V, _V]),
    ("enp_block_diagonal", _I, [_V, _V, _V]),
    ("enp_block_jacobi_setup", _I, [_V, _V, _I]),
    ("enp_block_jacobi_apply", _I, [_V, _V, _V]),
    ("enp_block_jacobi_apply_f32", _I, [_V, _V, _V]),
    ("enp_set_preconditioner", _I, [_V, _I]),
    ("enp_set_shared_blocks", _I, [_V, _I]),
    ("enp_set_coarse_options", _I, [_V, _I, _I, ctypes.c_double]),
    ("enp_set_sweep", _I, [_V, _I]),
    ("enp_coarse_operator", _I, [_V, _V]),
    ("enp_fgmres_solve", _I, [_V, _V, _V, _V, _V, _V]),
    ("enp_fgmres_solve_f32", _I, [_V, _V, _V, _V, _V, _V]),
    ("enp_newton_solve", _I, [_V, _V, _V, _V]),
    ("enp_newton_continuation", _I, [_V, _V, _V, _V, _V, _V]),
    ("enp_initial_guess", _I, [_V, _V, _V, _V]),
    ("enp_autotune", _I, [_V, _V]),
    ("enp_launch_shapes", _I, [_V, _V, _V]),
    ("enp_param_count", _I, [_V, ctypes.POINTER(_I)]),
    ("enp_param_jacobian", _I, [_V, _V, _V]),
    ("enp_param_vjp", _I, [_V, _V, _V, _V]),
    ("enp_param_vjp_total", _I, [_V, _V, _V, _V]),
    ("enp_inner_product_noalloc", _I, [_V, _V, _LL, _I, _V, _V]),
    ("enp_set_arithmetic", _I, [_V, _I]),
    ("enp_get_arithmetic", _I, [_V, ctypes.POINTER(_I)]),
    ("enp_last_error", ctypes.c_char_p, [_V]),
]

NOALLOC_MAX_BATCH = 32


def load(path: str | None = None):
    """Load libenp_dg.so (built in-tree by ``build()``) and declare its prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise EnpError(ENP_ERR_UNSUPPORTED,
                       f"{path} is missing: call paper_2112_09271_gb300.build() first")
    lib = ctypes.CDLL(path)
    for name, res, args in _PROTOS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return [p[0] for p in _PROTOS]


def _dptr(t, dtype):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


class Operator:
    """One CNP DG operator (a handle of the C library).

    ``prob`` is any object with the attributes of ``workloads.Problem`` (dim,
    n_el, coords, tags, m, z, D, c_in, F, RT, vel_kind, vel_params, bv_*, p, q,
    C_IP). Vectors are CUDA tensors [batch * m * E * Np] in the library layout.
    """

    def __init__(self, prob, batch: int = 1, stream=None):
        import torch
        lib = load()
        self.prob = prob
        self.batch = batch
        dim = prob.dim
        self._coords = [np.ascontiguousarray(prob.coords[a], dtype=np.float64) for a in range(dim)]
        self._tags = [np.ascontiguousarray(t, dtype=np.uint8) for t in prob.tags]
        mesh = MeshDesc()
        mesh.dim = dim
        for a in range(3):
            mesh.n_el[a] = int(prob.n_el[a]) if a < dim else 1
            mesh.coords[a] = self._coords[a].ctypes.data if a < dim else None
        for s in range(6):
            mesh.face_tag[s] = self._tags[s].ctypes.data if s < 2 * dim else None
        ph = PhysicsDesc()
        ph.m = prob.m
        for k in range(4):
            ph.z[k] = prob.z[k] if k < prob.m else 0.0
            ph.D[k] = prob.D[k] if k < prob.m else 0.0
            ph.c_in[k] = prob.c_in[k] if k < prob.m else 0.0
        ph.F, ph.RT = prob.F, prob.RT
        ph.velocity_kind = prob.vel_kind
        for i in range(8):
            ph.vel_params[i] = prob.vel_params[i] if i < len(prob.vel_params) else 0.0
        ph.bv_oxidant = prob.bv_oxidant
        ph.bv_J0, ph.bv_alpha1, ph.bv_alpha2 = prob.bv_J0, prob.bv_alpha1, prob.bv_alpha2
        ph.bv_n, ph.bv_gamma, ph.bv_c_ref = prob.bv_n, prob.bv_gamma, prob.bv_c_ref
        for j in range(4):
            ph.bv_phi_app[j] = prob.bv_phi_app[j]
        ph.bv_J0_axis, ph.bv_J0_lo, ph.bv_J0_hi = prob.bv_J0_axis, prob.bv_J0_lo, prob.bv_J0_hi
        disc = DiscDesc(prob.p, prob.q, prob.C_IP, batch)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib.enp_dg_create(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(ph),
                               ctypes.byref(disc), ctypes.c_void_p(stream.cuda_stream))
        if st != ENP_OK:
            raise EnpError(st, "enp_dg_create failed")
        self.h = h
        self._lib = lib
        n = ctypes.c_longlong(); nf = ctypes.c_int(); nn = ctypes.c_int(); nq = ctypes.c_int()
        nb = ctypes.c_int()
        self._check(lib.enp_dg_sizes(h, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nn),
                                     ctypes.byref(nq), ctypes.byref(nb)))
        self.n_dof, self.n_fields, self.n_nodes = n.value, nf.value, nn.value
        self.n_qpoints, self.n_bfaces = nq.value, nb.value
        self.n = self.n_dof * batch

    def _check(self, st):
        if st != ENP_OK:
            msg = self._lib.enp_last_error(self.h)
            raise EnpError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self._lib.enp_dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _new(self, like_dtype):
        import torch
        return torch.empty(self.n, dtype=like_dtype, device="cuda")

    def set_arithmetic(self, arith):
        """Arithmetic of the FP64 operator on hexahedra: ARITH_F64 (native FP64)
        or ARITH_DF32 (double-float on the FP32 pipe; R, J v and J^T w)."""
        self._check(self._lib.enp_set_arithmetic(self.h, int(arith)))

    @property
    def arithmetic(self):
        c = ctypes.c_int()
        self._check(self._lib.enp_get_arithmetic(self.h, ctypes.byref(c)))
        return c.value

    def set_sources(self, src=None, dirichlet=None):
        import torch
        s = _dptr(src, torch.float64) if src is not None else None
        d = _dptr(dirichlet, torch.float64) if dirichlet is not None else None
        self._check(self._lib.enp_set_sources(self.h, s, d))

    def set_phi_app(self, phi_app):
        a = None if phi_app is None else np.ascontiguousarray(phi_app, dtype=np.float64)
        if a is not None and a.size != 4 * self.batch:
            raise ValueError("phi_app must have batch x 4 entries")
        self._phi = a
        self._check(self._lib.enp_set_phi_app(self.h, None if a is None else a.ctypes.data))

    def quadrature_points(self):
        import torch
        P = self.prob
        xq = torch.empty((P.E, self.n_qpoints, 3), dtype=torch.float64, device="cuda")
        xb = torch.empty((self.n_bfaces, P.q ** (P.dim - 1), 3), dtype=torch.float64,
                         device="cuda")
        self._check(self._lib.enp_quadrature_points(self.h, ctypes.c_void_p(xq.data_ptr()),
                                                    ctypes.c_void_p(xb.data_ptr())))
        return xq, xb

    def residual(self, u, out=None):
        import torch
        out = self._new(torch.float64) if out is None else out
        self._check(self._lib.enp_residual(self.h, _dptr(u, torch.float64),
                                           _dptr(out, torch.float64)))
        return out

    def jvp(self, u, v, out=None):
        import torch
        out = self._new(torch.float64) if out is None else out
        self._check(self._lib.enp_jvp(self.h, _dptr(u, torch.float64), _dptr(v, torch.float64),
                                      _dptr(out, torch.float64)))
        return out

    def jvp_f32(self, u, v, out=None):
        import torch
        out = self._new(torch.float32) if out is None else out
        self._check(self._lib.enp_jvp_f32(self.h, _dptr(u, torch.float32),
                                          _dptr(v, torch.float32), _dptr(out, torch.float32)))
        return out

    def recover_cm(self, u, out=None):
        import torch
        P = self.prob
        out = torch.empty(self.batch * P.E * self.n_nodes, dtype=torch.float64,
                          device="cuda") if out is None else out
        self._check(self._lib.enp_recover_cm(self.h, _dptr(u, torch.float64),
                                             _dptr(out, torch.float64)))
        return out

    def inner_product(self, x, y):
        import torch
        out = np.zeros(self.batch)
        self._check(self._lib.enp_inner_product(self.h, _dptr(x, torch.float64),
                                                _dptr(y, torch.float64),
                                                ctypes.c_void_p(out.ctypes.data)))
        return out

    def block_diagonal(self, u, out=None):
        import torch
        nb = self.n_fields * self.n_nodes
        out = torch.empty(self.batch * self.prob.E * nb * nb, dtype=torch.float64,
                          device="cuda") if out is None else out
        self._check(self._lib.enp_block_diagonal(self.h, _dptr(u, torch.float64),
                                                 _dptr(out, torch.float64)))
        return out

    def block_jacobi_setup(self, u, storage=BJ_F64):
        import torch
        self._check(self._lib.enp_block_jacobi_setup(self.h, _dptr(u, torch.float64),
                                                     int(storage)))

    def block_jacobi_apply(self, x, out=None):
        import torch
        out = self._new(torch.float64) if out is None else out
        self._check(self._lib.enp_block_jacobi_apply(self.h, _dptr(x, torch.float64),
                                                     _dptr(out, torch.float64)))
        return out

    def block_jacobi_apply_f32(self, x, out=None):
        """The preconditioner on FP32 vectors (the mixed-precision inner solve's)."""
        import torch
        out = self._new(torch.float32) if out is None else out
        self._check(self._lib.enp_block_jacobi_apply_f32(self.h, _dptr(x, torch.float32),
                                                         _dptr(out, torch.float32)))
        return out

    def set_preconditioner(self, two_level):
        """0: block-Jacobi; 1: block-Jacobi plus the coarse potential correction
        (takes effect at the next block_jacobi_setup)."""
        self._check(self._lib.enp_set_preconditioner(self.h, int(two_level)))

    def set_shared_blocks(self, point):
        """-1: block inverses per operating point; b >= 0: the inverses of point
        b serve the whole batch (next setup)."""
        self._check(self._lib.enp_set_shared_blocks(self.h, int(point)))

    def set_sweep(self, on):
        """1: downwind block Gauss-Seidel instead of block-Jacobi; 0: block-Jacobi;
        2 (the default): the sweep on long channels (next setup)."""
        self._check(self._lib.enp_set_sweep(self.h, int(on)))

    def set_coarse_options(self, cycles=1, smooth=2, omega=1.0):
        """V-cycles per application, smoothing sweeps, prolongation over-correction."""
        self._check(self._lib.enp_set_coarse_options(self.h, int(cycles), int(smooth),
                                                     float(omega)))

    def coarse_operator(self):
        """The level-0 coarse operator [batch][E][7] of the last two-level setup."""
        import torch
        out = torch.empty(self.batch * self.prob.E * 7, dtype=torch.float64, device="cuda")
        self._check(self._lib.enp_coarse_operator(self.h, _dptr(out, torch.float64)))
        return out

    def fgmres_solve(self, u_lin, b, x, restart=30, max_it=300, rtol=1e-8, atol=0.0,
                     raise_on_fail=True, graph=False):
        """Solve J(u_lin) x = b in place on x; returns the stats as a dict."""
        import torch
        f32 = u_lin.dtype == torch.float32
        dt = torch.float32 if f32 else torch.float64
        o = KrylovOpts(restart, max_it, rtol, atol, int(graph))
        st = KrylovStats()
        fn = self._lib.enp_fgmres_solve_f32 if f32 else self._lib.enp_fgmres_solve
        rc = fn(self.h, _dptr(u_lin, dt), _dptr(b, dt), _dptr(x, dt), ctypes.byref(o),
                ctypes.byref(st))
        if rc != ENP_OK and (raise_on_fail or rc != ENP_ERR_NOT_CONVERGED):
            self._check(rc)
        return {k: getattr(st, k) for k, _ in KrylovStats._fields_} | {"status": rc}

    def newton_solve(self, u, max_it=20, rtol=1e-10, atol=0.0, armijo_c=1e-4,
                     max_backtracks=12, bj_storage=BJ_F64, mixed=False, krylov_restart=30,
                     krylov_max_it=500, krylov_rtol=1e-3, raise_on_fail=True, graph=False,
                     pc_lag=1, device_loop=False):
        """Newton with backtracking line search in place on u; returns the stats.
        device_loop: the Newton iterations between preconditioner setups as one
        graph launch with device-side loops."""
        import torch
        o = NewtonOpts(max_it, rtol, atol, armijo_c, max_backtracks, bj_storage, int(mixed),
                       KrylovOpts(krylov_restart, krylov_max_it, krylov_rtol, 0.0, int(graph)),
                       int(pc_lag), int(device_loop))
        st = NewtonStats()
        rc = self._lib.enp_newton_solve(self.h, _dptr(u, torch.float64), ctypes.byref(o),
                                        ctypes.byref(st))
        if rc != ENP_OK and raise_on_fail:
            self._check(rc)
        out = {k: getattr(st, k) for k, _ in NewtonStats._fields_ if k != "history"}
        out["history"] = list(st.history[: st.iterations + 1])
        out["status"] = rc
        return out

    def initial_guess(self, u, max_it=30, rtol=1e-8, atol=0.0, armijo_c=1e-4,
                      max_backtracks=12, bj_storage=BJ_F64, mixed=False, krylov_restart=50,
                      krylov_max_it=4000, krylov_rtol=1e-2, raise_on_fail=True, graph=False,
                      pc_lag=1, device_loop=False):
        """The initial guess of Sec. 4.3 in place on u: c = c_in everywhere and
        Phi from the charge-conservation equation at constant c, by Newton from
        the Phi in u (inner FGMRES to 1e-2, as the paper); returns the stats."""
        import torch
        o = NewtonOpts(max_it, rtol, atol, armijo_c, max_backtracks, bj_storage, int(mixed),
                       KrylovOpts(krylov_restart, krylov_max_it, krylov_rtol, 0.0, int(graph)),
                       int(pc_lag), int(device_loop))
        st = NewtonStats()
        rc = self._lib.enp_initial_guess(self.h, _dptr(u, torch.float64), ctypes.byref(o),
                                         ctypes.byref(st))
        if rc != ENP_OK and raise_on_fail:
            self._check(rc)
        out = {k: getattr(st, k) for k, _ in NewtonStats._fields_ if k != "history"}
        out["history"] = list(st.history[: st.iterations + 1])
        out["status"] = rc
        return out

    def newton_continuation(self, u, phi_app, step0=0.125, step_max=0.25, step_min=1.0 / 512,
                            grow=1.5, stage_rtol=1e-6, stage_max_it=10, max_it=30, rtol=1e-10,
                            atol=0.0, armijo_c=1e-4, max_backtracks=12, bj_storage=BJ_F64,
                            mixed=False, krylov_restart=50, krylov_max_it=4000,
                            krylov_rtol=1e-3, graph=False, pc_lag=1, raise_on_fail=True,
                            device_loop=False):
        """Continuation in the applied potential up to phi_app ([batch][4]), in
        place on u; returns the stats (the last stage's Newton stats under 'last')."""
        import numpy as np
        import torch
        ph = np.ascontiguousarray(np.asarray(phi_app, dtype=np.float64).reshape(self.batch, 4))
        c = ContinuationOpts(step0, step_max, step_min, grow, stage_rtol, stage_max_it)
        o = NewtonOpts(max_it, rtol, atol, armijo_c, max_backtracks, bj_storage, int(mixed),
                       KrylovOpts(krylov_restart, krylov_max_it, krylov_rtol, 0.0, int(graph)),
                       int(pc_lag), int(device_loop))
        st = ContinuationStats()
        rc = self._lib.enp_newton_continuation(
            self.h, _dptr(u, torch.float64), ph.ctypes.data_as(ctypes.c_void_p),
            ctypes.byref(c), ctypes.byref(o), ctypes.byref(st))
        if rc != ENP_OK and raise_on_fail:
            self._check(rc)
        out = {k: getattr(st, k) for k, _ in ContinuationStats._fields_ if k not in ("last", "lambda_")}
        out["lambda"] = st.lambda_
        last = {k: getattr(st.last, k) for k, _ in NewtonStats._fields_ if k != "history"}
        last["history"] = list(st.last.history[: st.last.iterations + 1])
        out["last"] = last
        out["status"] = rc
        return out

    def autotune(self):
        """Pick the tile shapes (faces per block of the face kernel, elements
        per block of the element kernel) for this shape; returns the elements
        per block for R, J v, J^T w (FP64-accurate), J v, R (FP32)."""
        c = (ctypes.c_int * 5)()
        self._check(self._lib.enp_autotune(self.h, c))
        return list(c)

    def launch_shapes(self):
        """(elements per block, faces per block) in use for R, J v, J^T w
        (FP64-accurate), J v, R (FP32); 0 = default."""
        eb, fpb = (ctypes.c_int * 5)(), (ctypes.c_int * 5)()
        self._check(self._lib.enp_launch_shapes(self.h, eb, fpb))
        return list(eb), list(fpb)

    @property
    def n_theta(self):
        c = ctypes.c_int()
        self._check(self._lib.enp_param_count(self.h, ctypes.byref(c)))
        return c.value

    def param_jacobian(self, u, out=None):
        """dR/dtheta for theta = (D_1..D_m, c_in_1..c_in_{m-1}, phi_app_0..3):
        a CUDA tensor [n_theta, batch * m * E * Np]."""
        import torch
        nt = self.n_theta
        out = torch.empty((nt, self.n), dtype=torch.float64, device="cuda") if out is None else out
        self._check(self._lib.enp_param_jacobian(self.h, _dptr(u, torch.float64),
                                                 _dptr(out, torch.float64)))
        return out

    def param_vjp(self, u, w):
        """<w, dR/dtheta_j> per operating point: numpy [batch, n_theta]."""
        import torch
        out = np.zeros((self.batch, self.n_theta))
        self._check(self._lib.enp_param_vjp(self.h, _dptr(u, torch.float64),
                                            _dptr(w, torch.float64),
                                            ctypes.c_void_p(out.ctypes.data)))
        return out

    def param_vjp_total(self, u, w):
        """sum_b <w_b, dR_b/dtheta_j>, summed over operating points on the
        device: numpy [n_theta]."""
        import torch
        out = np.zeros(self.n_theta)
        self._check(self._lib.enp_param_vjp_total(self.h, _dptr(u, torch.float64),
                                                  _dptr(w, torch.float64),
                                                  ctypes.c_void_p(out.ctypes.data)))
        return out

    def vjp(self, u, w, out=None):
        import torch
        out = self._new(torch.float64) if out is None else out
        self._check(self._lib.enp_vjp(self.h, _dptr(u, torch.float64), _dptr(w, torch.float64),
                                      _dptr(out, torch.float64)))
        return out


def residual_function(op):
    """A torch.autograd.Function for u -> R(u) with the operator ``op``: the
    forward pass runs enp_residual, the backward pass enp_vjp (J(u)^T g) and
    enp_param_vjp (the gradient with respect to theta, returned through the
    ``theta`` input, a tensor of n_theta entries whose value is not used: the
    parameters live in the handle). Element-local recomputation, no stored
    quadrature-point state."""
    import torch

    class _Residual(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u, theta):
            ctx.save_for_backward(u)
            return op.residual(u.detach().contiguous())

        @staticmethod
        def backward(ctx, g):
            (u,) = ctx.saved_tensors
            g = g.contiguous()
            gu = op.vjp(u.detach().contiguous(), g) if ctx.needs_input_grad[0] else None
            gt = None
            if ctx.needs_input_grad[1]:
                d = op.param_vjp_total(u.detach().contiguous(), g)
                gt = torch.tensor(d, dtype=torch.float64, device=u.device)
            return gu, gt

    return _Residual.apply
