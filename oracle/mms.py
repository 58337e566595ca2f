"""Test infrastructure: manufactured solutions for the CNP model (Sec. 5.1).

Given exact fields c_k(x) (k < m) and Phi(x), the volume sources are the strong
forms evaluated at the exact solution:
  species k (Eq. NP2):   R_k = -div(D_k grad c_k) + div(c_k q_k),
                         q_k = u - z_k mu_k F grad Phi, mu_k = D_k / RT (Eq. NE);
  charge    (Eq. charge2): f = -div(sum_k a_k grad c_k) - div(kappa grad Phi),
                         a_k = F z_k (D_k - D_m),
                         kappa = sum_{k<m} z_k (z_k mu_k - z_m mu_m) F^2 c_k.
These are derived symbolically (sympy) from the PDEs, not from the weak form,
so they check the discontinuous Galerkin terms rather than repeat them.
sympy is imported lazily: it is needed only by CPU tests.
"""
from __future__ import annotations

import numpy as np


def _velocity_expr(prob, X):
    import sympy as sp
    if prob.vel_kind == 0:
        return [sp.Float(prob.vel_params[a]) for a in range(3)]
    A, N = int(prob.vel_params[0]), int(prob.vel_params[1])
    y0, H, uavg = prob.vel_params[2], prob.vel_params[3], prob.vel_params[4]
    s = X[N] - y0
    u = [sp.Integer(0)] * 3
    u[A] = 6 * uavg * s * (H - s) / H ** 2
    return u


def build(prob, c_exprs, phi_expr):
    """Returns (exact(xyz) -> [NF, npts], sources(xyz) -> [NF, npts]) as numpy
    callables; c_exprs are sympy expressions in x, y, z for c_1..c_{m-1}."""
    import sympy as sp
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    dim = prob.dim
    grad = lambda e: [sp.diff(e, X[a]) for a in range(dim)]
    div = lambda v: sum(sp.diff(v[a], X[a]) for a in range(dim))
    u = _velocity_expr(prob, X)
    m, F, RT = prob.m, prob.F, prob.RT
    zs, Ds = prob.z, prob.D
    mu = [Ds[k] / RT for k in range(m)]
    gphi = grad(phi_expr)
    src = []
    # charge equation source f
    flux = [0] * dim
    kap = sum(zs[k] * (zs[k] * mu[k] - zs[m - 1] * mu[m - 1]) * F ** 2 * c_exprs[k]
              for k in range(m - 1))
    for k in range(m - 1):
        ak = F * zs[k] * (Ds[k] - Ds[m - 1])
        gc = grad(c_exprs[k])
        for a in range(dim):
            flux[a] += ak * gc[a]
    for a in range(dim):
        flux[a] += kap * gphi[a]
    src.append(-div(flux))
    for k in range(m - 1):
        qk = [u[a] - zs[k] * mu[k] * F * gphi[a] for a in range(dim)]
        gc = grad(c_exprs[k])
        src.append(-div([Ds[k] * gc[a] for a in range(dim)])
                   + div([c_exprs[k] * qk[a] for a in range(dim)]))
    exact = [phi_expr] + list(c_exprs)
    fe = [sp.lambdify((x, y, z), e, "numpy") for e in exact]
    fs = [sp.lambdify((x, y, z), sp.simplify(e), "numpy") for e in src]

    def ev(funcs, xyz):
        xyz = np.asarray(xyz).reshape(-1, 3)
        out = np.zeros((len(funcs), len(xyz)))
        for i, f in enumerate(funcs):
            out[i] = np.broadcast_to(f(xyz[:, 0], xyz[:, 1], xyz[:, 2]), (len(xyz),))
        return out

    return (lambda xyz: ev(fe, xyz)), (lambda xyz: ev(fs, xyz))


def problem_data(orc, exact, sources):
    """(nodal interpolant u* [NF*E*Np], sources [NF][E][Nq], Dirichlet data
    [NF][NBF][Nfq]) for an ``oracle.Oracle`` and the callables from ``build``."""
    P = orc.prob
    xn = orc.node_points()
    xq, xb = orc.quad_points()
    u = exact(xn.reshape(-1, 3)).reshape(P.n_fields, P.E, P.Np).reshape(-1)
    s = sources(xq.reshape(-1, 3)).reshape(P.n_fields, P.E, P.Nq).reshape(-1)
    d = exact(xb.reshape(-1, 3)).reshape(P.n_fields, P.n_bfaces, P.Nfq).reshape(-1)
    return u, s, d


def l2_errors(orc, u, exact):
    """Per-field L2 error of the discrete solution against the exact one."""
    vals, jxw = orc.eval_quad(u)
    xq, _ = orc.quad_points()
    ex = exact(xq.reshape(-1, 3)).reshape(vals.shape)
    return np.sqrt(((vals - ex) ** 2 * jxw[None]).sum(axis=(1, 2)))
