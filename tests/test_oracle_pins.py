"""Pins for the oracle's residual R(u), J(u)v and J(u)^T w against what the paper and
the mathematics fix, independently of the oracle's own code:

* polynomial consistency: the SIPG/upwind scheme is consistent, so the interpolant
  of an exact solution in Q^p (with its strong-form sources and Dirichlet data)
  has R = 0 to rounding (Sec. 3, Eq. NPDG/chargeDG; sources from the PDEs Eq. NP2
  and Eq. charge2, derived symbolically);
* global conservation: testing with v = 1 leaves only boundary and source terms,
  computed here from Gauss-Lobatto face sums and numpy's Gauss-Legendre weights
  (Eq. NPDG in conservation form; the inlet/outlet/electrode terms of Sec. 3.3);
* symmetry of the interior-penalty blocks (the "symmetric interior penalty" of
  Sec. 3.2), constants in the kernel of the potential block under natural
  boundary conditions, and positive definiteness with Dirichlet faces;
* p = 0 reduction to the textbook first-order upwind finite-volume scheme;
* J(u)v against central finite differences of R; the assembled J against Jv and
  J^T w (for the dual-number machinery).
The manufactured-solution convergence rates are in test_oracle_mms.py.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import mms


def _with(prob, **kw):
    import dataclasses
    return dataclasses.replace(prob, **kw)


def _all_tags(prob, tag):
    return [np.full_like(t, tag) for t in prob.tags]


# ------------------------------------------------------------ consistency
CONSISTENCY_CASES = [
    # (name, config, p, c-expressions, phi-expression, velocity override)
    ("2d_p1", "mms2d_n3", 1, ["2 + x + 0.5*y + 0.25*x*y"], "0.3 - x + 0.7*y + 0.1*x*y", None),
    ("2d_p2", "mms2d_n3", 2, ["2 + x + 0.5*y**2 - 0.3*x*y + 0.2*x**2*y"],
     "0.5 - x + y**2 + 0.2*x*y", None),
    ("2d_p3", "mms2d_n2", 3, ["3 + x**3 - 0.5*y**2 + 0.3*x*y**3"], "x**2*y - 0.4*y**3 + x",
     None),
    ("3d_p2_plate", "cube_n2_p2", 2, ["2 + 0.5*x + 0.3*y*z + 0.2*z**2 - 0.1*x**2*y"],
     "x - y + 0.5*x*z + 0.1*y**2", "plate"),
    ("3d_p1_3ions", "channel_n1", 1, ["1 + 0.2*x + 0.1*y*z", "2 - 0.1*x*y + 0.3*z"],
     "0.2*x - 0.1*y + 0.05*x*y*z", "plate"),
]


@pytest.mark.parametrize("case", CONSISTENCY_CASES, ids=[c[0] for c in CONSISTENCY_CASES])
def test_polynomial_consistency(case):
    sp = pytest.importorskip("sympy")
    _, cfg, p, cs, ph, vel = case
    P = W.config(cfg, p=p)
    P = _with(P, tags=_all_tags(P, W.DIRICHLET), bv_oxidant=-1)
    if P.dim == 2:
        P = _with(P, vel_kind=W.VEL_CONSTANT, vel_params=[1.0, 0.5, 0, 0, 0, 0, 0, 0])
    x, y, z = sp.symbols("x y z")
    loc = {"x": x, "y": y, "z": z}
    exact, sources = mms.build(P, [sp.sympify(c, locals=loc) for c in cs],
                               sp.sympify(ph, locals=loc))
    orc0 = oracle.Oracle(P)
    u, s, d = mms.problem_data(orc0, exact, sources)
    orc = oracle.Oracle(P, src=s, dirichlet=d)
    r = orc.residual(u)
    # scale: the size of the individual terms, seen through a perturbed state
    rng = np.random.default_rng(0)
    scale = np.abs(orc.residual(u + 1e-3 * rng.standard_normal(u.size))).max()
    assert scale > 1e-6
    assert np.abs(r).max() < 1e-11 * max(1.0, np.abs(u).max()), np.abs(r).max()
    # and a mistaken Dirichlet trace is seen: shift the exterior data
    bad = oracle.Oracle(P, src=s, dirichlet=d + 1e-3)
    assert np.abs(bad.residual(u)).max() > 1e-8


# ------------------------------------------------------------ conservation
def _gll_weights(p):
    _, _, xn = oracle.rules(p, p + 2)
    Pp = np.polynomial.legendre.Legendre.basis(p)
    return 2.0 / (p * (p + 1) * Pp(xn) ** 2)


@pytest.mark.parametrize("cfg,grad_phi", [("cube_n3_p2", None), ("channel_n1", None),
                                          ("mms2d_n3", None), ("cube_n3_p2", (0.4, -0.3, 0.2)),
                                          ("channel_n1", (-0.5, 0.25, 0.1)),
                                          ("mms2d_n3", (0.6, 0.3, 0.0))])
def test_global_conservation(cfg, grad_phi):
    """Sum over all rows of species k = outlet flux + inlet flux - electrode
    reaction - source; sum of the potential rows = -electrode current - source.
    With grad_phi the potential is the linear function grad_phi . x (exactly in
    Q^p), there are no electrodes, and the outlet flux carries the migration
    velocity q_k . n = u . n - z_k mu_k F dPhi/dn."""
    P = W.config(cfg)
    ubar = [0.7, 0.2, 0.1] if P.dim == 3 else [0.7, 0.2, 0.0]
    tags = [t.copy() for t in P.tags]
    tags[0][:] = W.INLET
    tags[1][:] = W.OUTLET
    for s in range(2, 2 * P.dim):
        keep = tags[s] >= W.ELECTRODE0
        tags[s][:] = W.OUTLET if s % 2 else W.INLET
        tags[s][keep] = W.ELECTRODE0 if s == 2 else W.ELECTRODE0 + 1
    if P.dim == 2:
        tags[2][3:5] = W.ELECTRODE0
    if P.bv_oxidant < 0:
        P = _with(P, bv_oxidant=0, bv_J0=0.3, bv_phi_app=[0.4, -0.2, 0, 0])
    P = _with(P, tags=tags, vel_kind=W.VEL_CONSTANT, vel_params=ubar + [0.0] * 5,
              bv_J0_axis=-1)
    src = W.random_sources(P, 11)
    phi0 = 0.05
    u = W.random_state(P, 12).reshape(P.n_fields, P.E, P.Np)
    gphi = np.zeros(3)
    if grad_phi is not None:
        tags = [np.where(t >= W.ELECTRODE0, W.WALL, t).astype(np.uint8) for t in tags]
        P = _with(P, tags=tags)
        gphi = np.asarray(grad_phi, dtype=float)
        xn = oracle.Oracle(P).node_points().reshape(P.E, P.Np, 3)
        u[0] = phi0 + xn @ gphi
    else:
        u[0] = phi0
    u = u.reshape(-1)
    orc = oracle.Oracle(P, src=src)
    r = orc.residual(u).reshape(P.n_fields, P.E, P.Np)
    tot = r.sum(axis=(1, 2))

    # independent boundary integrals: Gauss-Lobatto face sums of nodal values
    n = P.p + 1
    wl = _gll_weights(P.p)
    uu = u.reshape(P.n_fields, P.E, *([n] * P.dim)[::-1])  # [f][e][(z)][y][x]
    ne = P.n_el
    expect = np.zeros(P.n_fields)
    mu_fac = [P.z[k] * P.D[k] / P.RT * P.F for k in range(P.m)]

    def c_ox(vals):
        if P.bv_oxidant < P.m - 1:
            return vals[P.bv_oxidant + 1]
        return -sum(P.z[k] * vals[k + 1] for k in range(P.m - 1)) / P.z[P.m - 1]

    for s in range(2 * P.dim):
        a, hi = s // 2, s & 1
        others = [b for b in range(P.dim) if b != a]
        nrm = 1.0 if hi else -1.0
        un = ubar[a] * nrm
        shape = [ne[b] for b in others]
        for loc in range(int(np.prod(shape))):
            idx = [0, 0, 0]
            if P.dim == 3:
                idx[others[0]] = loc % shape[0]
                idx[others[1]] = loc // shape[0]
            else:
                idx[others[0]] = loc
            idx[a] = ne[a] - 1 if hi else 0
            e = idx[0] + ne[0] * (idx[1] + ne[1] * idx[2])
            hs = [P.coords[b][idx[b] + 1] - P.coords[b][idx[b]] for b in others]
            jac = np.prod([h / 2 for h in hs])
            # nodal values on the face, as an array over the other axes
            sl = [slice(None)] * P.dim
            sl[P.dim - 1 - a] = -1 if hi else 0
            face = uu[:, e][(slice(None),) + tuple(sl)]  # [f][...] axes reversed
            wt = wl if P.dim == 2 else np.outer(wl, wl)
            integ = lambda vals: jac * float(np.sum(wt * vals))
            tag = tags[s][loc]
            if tag == W.INLET:
                for k in range(P.m - 1):
                    expect[k + 1] += un * P.c_in[k] * jac * float(np.sum(wt))
            elif tag == W.OUTLET:
                for k in range(P.m - 1):
                    qn = un - mu_fac[k] * gphi[a] * nrm
                    expect[k + 1] += qn * integ(face[k + 1])
            elif tag >= W.ELECTRODE0:
                j = tag - W.ELECTRODE0
                fac = P.bv_n * P.F / P.RT
                eta = P.bv_phi_app[j] - phi0
                co = c_ox(face)
                Jn = P.bv_J0 * (math.exp(P.bv_alpha1 * fac * eta)
                                - (co / P.bv_c_ref) * math.exp(-P.bv_alpha2 * fac * eta))
                if P.bv_oxidant < P.m - 1:
                    expect[P.bv_oxidant + 1] -= integ(Jn) / (P.bv_n * P.F)
                expect[0] -= P.z[P.bv_oxidant] / P.bv_n * integ(Jn)
    # sources: numpy Gauss-Legendre weights times the element Jacobians
    xg, wg = np.polynomial.legendre.leggauss(P.q)
    wq = wg if P.dim == 2 else np.einsum("i,j,k->kji", wg, wg, wg).reshape(-1)
    if P.dim == 2:
        wq = np.outer(wg, wg).reshape(-1)
    srcr = src.reshape(P.n_fields, P.E, P.Nq)
    for e in range(P.E):
        idx = [e % ne[0], (e // ne[0]) % ne[1], e // (ne[0] * ne[1])]
        jac = np.prod([(P.coords[a][idx[a] + 1] - P.coords[a][idx[a]]) / 2 for a in range(P.dim)])
        expect -= jac * srcr[:, e] @ wq
    np.testing.assert_allclose(tot, expect, rtol=1e-11, atol=1e-11 * np.abs(expect).max())
    assert np.abs(r).max() > 1e3 * np.abs(tot - expect).max()  # the sum is not trivially 0


# ------------------------------------------------------------ SIPG structure
def _blocks(P, J):
    nf = P.n_fields
    n1 = P.E * P.Np
    return lambda f, g: J[f * n1:(f + 1) * n1, g * n1:(g + 1) * n1]


@pytest.mark.parametrize("cfg", ["cube_n2_p2", "mms2d_n3", "channel_n1"])
def test_potential_block_symmetric_any_state(cfg):
    P = W.config(cfg)
    u = W.random_state(P, 5, c_amp=0.3)
    J = oracle.Oracle(P, dirichlet=W.random_dirichlet(P, 6)).jacobian(u)
    A = _blocks(P, J)(0, 0).toarray()
    if P.bv_oxidant >= 0:  # the Butler-Volmer term adds a diagonal-type boundary mass
        pass
    asym = np.abs(A - A.T).max() / np.abs(A).max()
    assert asym < 1e-13, asym


def test_potential_block_kernel_and_definiteness():
    P = W.config("cube_n2_p2")
    u = W.random_state(P, 5, c_amp=0.3)
    walls = _with(P, tags=_all_tags(P, W.WALL), bv_oxidant=-1)
    A = _blocks(walls, oracle.Oracle(walls).jacobian(u))(0, 0).toarray()
    ones = np.ones(A.shape[0])
    assert np.abs(A @ ones).max() < 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-8 * ev[-1]  # one zero mode only
    dirich = _with(P, tags=_all_tags(P, W.DIRICHLET), bv_oxidant=-1)
    A = _blocks(dirich, oracle.Oracle(dirich).jacobian(u))(0, 0).toarray()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev[0] > 1e-8 * ev[-1]


def test_species_block_symmetric_without_transport():
    P = W.config("cube_n2_p2")
    P = _with(P, tags=_all_tags(P, W.DIRICHLET), bv_oxidant=-1, vel_kind=W.VEL_CONSTANT,
              vel_params=[0.0] * 8)
    u = W.random_state(P, 9).reshape(P.n_fields, P.E, P.Np)
    u[0] = 0.3  # constant potential: q_k = u = 0
    J = oracle.Oracle(P).jacobian(u.reshape(-1))
    A = _blocks(P, J)(1, 1).toarray()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    # coercive with the penalty C_IP = 10 (Sec. 3.2): positive definite; the
    # penalty-free form of the same block is indefinite on this mesh
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev[0] > 1e-8 * ev[-1]
    P0 = _with(P, C_IP=0.0)
    A0 = _blocks(P0, oracle.Oracle(P0).jacobian(u.reshape(-1)))(1, 1).toarray()
    assert np.linalg.eigvalsh(0.5 * (A0 + A0.T))[0] < 0
    # with flow the upwind term makes it non-symmetric
    P2 = _with(P, vel_params=[1.0, 0.3, 0.0, 0, 0, 0, 0, 0])
    A2 = _blocks(P2, oracle.Oracle(P2).jacobian(u.reshape(-1)))(1, 1).toarray()
    assert np.abs(A2 - A2.T).max() > 1e-3 * np.abs(A2).max()


# ------------------------------------------------------------ p = 0 upwind
@pytest.mark.parametrize("dim,dirichlet", [(2, False), (3, False), (2, True), (3, True)])
def test_p0_is_first_order_upwind_finite_volume(dim, dirichlet):
    """At p = 0 every gradient and the penalty (p^2 = 0) vanish, leaving the
    textbook upwind finite-volume scheme: flux u.n c_upwind through each face,
    with c_in on inlets, the cell value on outlets, and on Dirichlet faces the
    exterior state g as the upwind value where u.n < 0."""
    P = W.config("mms2d_n4" if dim == 2 else "cube_n3_p0", p=0)
    ubar = [1.0, -0.4, 0.25]
    tags = []
    for s in range(2 * dim):
        a, hi = s // 2, s & 1
        out = (ubar[a] > 0) == bool(hi)
        t = W.DIRICHLET if dirichlet else (W.OUTLET if out else W.INLET)
        tags.append(np.full_like(P.tags[s], t))
    P = _with(P, tags=tags, vel_kind=W.VEL_CONSTANT, vel_params=ubar + [0.0] * 5,
              bv_oxidant=-1)
    rng = np.random.default_rng(3)
    coords = [np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, P.n_el[a]))])
              for a in range(dim)]
    P = _with(P, coords=coords)
    src = W.random_sources(P, 4)
    gd = W.random_dirichlet(P, 6, amp=0.5).reshape(P.n_fields, P.n_bfaces, P.Nfq)
    u = W.random_state(P, 5, c_amp=0.5)
    r = oracle.Oracle(P, src=src, dirichlet=gd.reshape(-1)).residual(u).reshape(P.n_fields, P.E)
    side_off = np.concatenate([[0], np.cumsum([len(t) for t in P.tags])])
    xg1, wg1 = np.polynomial.legendre.leggauss(P.q)
    wface = wg1 if dim == 2 else np.outer(wg1, wg1).reshape(-1)  # point order irrelevant: sum
    c = u.reshape(P.n_fields, P.E)[1]
    ne = P.n_el
    fv = np.zeros(P.E)
    xg, wg = np.polynomial.legendre.leggauss(P.q)
    wsum = wg.sum() ** dim
    s1 = src.reshape(P.n_fields, P.E, P.Nq)
    for e in range(P.E):
        idx = [e % ne[0], (e // ne[0]) % ne[1], e // (ne[0] * ne[1])]
        h = [coords[a][idx[a] + 1] - coords[a][idx[a]] for a in range(dim)]
        vol = np.prod(h)
        wq = np.ones(P.Nq) * 0
        # source integral: sum of the quadrature values times the weights
        if dim == 2:
            wq = np.outer(wg, wg).reshape(-1)
        else:
            wq = np.einsum("i,j,k->ijk", wg, wg, wg).reshape(-1)
        fv[e] -= vol / 2 ** dim * s1[1, e] @ wq
        for a in range(dim):
            area = vol / h[a]
            for hi in (0, 1):
                n = 1.0 if hi else -1.0
                un = ubar[a] * n
                nb = list(idx)
                nb[a] += 1 if hi else -1
                if 0 <= nb[a] < ne[a]:
                    en = nb[0] + ne[0] * (nb[1] + ne[1] * nb[2])
                    cup = c[e] if un > 0 else c[en]
                    fv[e] += area * un * cup
                elif dirichlet:
                    others = [b for b in range(dim) if b != a]
                    loc = idx[others[0]] + (ne[others[0]] * idx[others[1]] if dim == 3 else 0)
                    bf = side_off[2 * a + hi] + loc
                    if un > 0:
                        fv[e] += area * un * c[e]
                    else:  # mean of the exterior state over the face
                        gmean = gd[1, bf] @ wface / wface.sum()
                        fv[e] += area * un * gmean
                elif un < 0:
                    fv[e] += area * un * P.c_in[0]
                else:
                    fv[e] += area * un * c[e]
    np.testing.assert_allclose(r[1], fv, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(r[0], -np.array([np.prod(
        [coords[a][([e % ne[0], (e // ne[0]) % ne[1], e // (ne[0] * ne[1])][a]) + 1]
         - coords[a][[e % ne[0], (e // ne[0]) % ne[1], e // (ne[0] * ne[1])][a]]
         for a in range(dim)]) / 2 ** dim * (s1[0, e] @ (np.outer(wg, wg).reshape(-1) if dim == 2
                                             else np.einsum("i,j,k->ijk", wg, wg, wg).reshape(-1)))
        for e in range(P.E)]), rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ derivatives
DERIV_CASES = ["mms2d_n3", "cube_n2_p3", "channel_n1", "reactor_n1_p2"]


@pytest.mark.parametrize("cfg", DERIV_CASES)
def test_jvp_matches_central_differences(cfg):
    P = W.config(cfg)
    orc = oracle.Oracle(P, src=W.random_sources(P, 1), dirichlet=W.random_dirichlet(P, 2))
    u = W.random_state(P, 3)
    v = W.random_vector(P, 4)
    jv = orc.jvp(u, v)
    h = 1e-6
    fd = (orc.residual(u + h * v) - orc.residual(u - h * v)) / (2 * h)
    assert np.linalg.norm(jv - fd) / np.linalg.norm(jv) < 1e-7


@pytest.mark.parametrize("cfg", ["mms2d_n3", "cube_n2_p2", "cube_n3_p1", "channel_n1"])
def test_assembled_jacobian_consistent(cfg):
    P = W.config(cfg)
    orc = oracle.Oracle(P, dirichlet=W.random_dirichlet(P, 2))
    u = W.random_state(P, 3)
    v, w = W.random_vector(P, 4), W.random_vector(P, 5)
    J = orc.jacobian(u)
    jv = orc.jvp(u, v)
    assert np.linalg.norm(J @ v - jv) <= 1e-13 * np.linalg.norm(jv)
    cols = np.arange(0, P.n_dof, 5)
    jtw = orc.vjp_entries(u, w, cols)
    ref = (J.T @ w)[cols]
    assert np.linalg.norm(jtw - ref) <= 1e-13 * np.linalg.norm(ref)
    # <w, J v> = <J^T w, v>
    full = orc.vjp_entries(u, w, np.arange(P.n_dof))
    assert abs(w @ jv - full @ v) <= 1e-12 * abs(w @ jv)


def test_element_subset_rows_match_full():
    P = W.config("cube_n3_p2")
    orc = oracle.Oracle(P)
    u = W.random_state(P, 3)
    full = orc.residual(u).reshape(P.n_fields, P.E, P.Np)
    el = np.array([0, 5, 13, 26])
    part = orc.residual(u, elems=el).reshape(P.n_fields, P.E, P.Np)
    np.testing.assert_array_equal(part[:, el], full[:, el])
    mask = np.ones(P.E, bool); mask[el] = False
    assert np.all(part[:, mask] == 0)


# ------------------------------------------------------------ c_m, blocks
@pytest.mark.parametrize("cfg", ["cube_n2_p2", "channel_n1"])
def test_recovered_cm_satisfies_electroneutrality(cfg):
    """Eq. electroneutrality: sum_{k=1}^{m} z_k c_k = 0 with c_m from Eq. substitution."""
    P = W.config(cfg)
    u = W.random_state(P, 3)
    cm = oracle.recover_cm(P, u)
    uu = u.reshape(P.n_fields, -1)
    total = sum(P.z[k] * uu[k + 1] for k in range(P.m - 1)) + P.z[P.m - 1] * cm
    assert np.abs(total).max() < 1e-14 * np.abs(uu[1:]).max()


def test_block_diagonal_and_block_solve_are_consistent():
    """The diagonal blocks equal the element-local Jacobian with the neighbours'
    unknowns frozen: J applied to a vector supported on one element, restricted
    to that element's rows, equals the block times the vector."""
    P = W.config("cube_n3_p2")
    orc = oracle.Oracle(P)
    u = W.random_state(P, 3)
    blocks = orc.block_diagonal(u)
    e = 13
    rng = np.random.default_rng(1)
    v = np.zeros(P.n_dof).reshape(P.n_fields, P.E, P.Np)
    v[:, e] = rng.standard_normal((P.n_fields, P.Np))
    jv = orc.jvp(u, v.reshape(-1)).reshape(P.n_fields, P.E, P.Np)
    np.testing.assert_allclose(jv[:, e].reshape(-1), blocks[e] @ v[:, e].reshape(-1),
                               rtol=1e-12, atol=1e-14)
    x = rng.standard_normal(P.n_dof)
    y = orc.block_jacobi_apply(blocks, x).reshape(P.n_fields, P.E, P.Np)
    np.testing.assert_allclose(blocks[e] @ y[:, e].reshape(-1),
                               x.reshape(P.n_fields, P.E, P.Np)[:, e].reshape(-1), rtol=1e-10)


# ------------------------------------------------------------ dR/dtheta
def _perturb(P, j, h):
    """The problem with parameter j of theta = (D_1..D_m, c_in_1..c_in_{m-1},
    phi_app_0..3) shifted by h."""
    m = P.m
    D, cin, phi = list(P.D), list(P.c_in), list(P.bv_phi_app)
    if j < m:
        D[j] += h
    elif j < 2 * m - 1:
        cin[j - m] += h
    else:
        phi[j - (2 * m - 1)] += h
    return _with(P, D=D, c_in=cin, bv_phi_app=phi)


@pytest.mark.parametrize("cfg", ["cube_n2_p2", "channel_n1"])
def test_param_jacobian_matches_central_differences(cfg):
    """The dual sweep seeded on each parameter (D_k through mu_k, a_km and kappa
    of Eq. NE / Eq. charge2; c_in through the inlet term; phi_app through
    Eq. bv) against central differences of R in that parameter."""
    P = W.config(cfg)
    tags = [t.copy() for t in P.tags]
    tags[0][:] = W.INLET  # inlet, outlet and both electrodes present
    P = _with(P, tags=tags)
    u = W.random_state(P, 3)
    dR = oracle.Oracle(P).param_jacobian(u)
    assert dR.shape[0] == 2 * P.m + 3
    for j in range(dR.shape[0]):
        base = ([P.D[k] for k in range(P.m)] + list(P.c_in[: P.m - 1]) + list(P.bv_phi_app))[j]
        h = 1e-6 * max(abs(base), 1e-3)
        fd = (oracle.Oracle(_perturb(P, j, h)).residual(u)
              - oracle.Oracle(_perturb(P, j, -h)).residual(u)) / (2 * h)
        scale = max(np.abs(dR[j]).max(), 1e-300)
        if np.abs(fd).max() < 1e-12 and np.abs(dR[j]).max() < 1e-12:
            continue  # electrodes 2, 3 absent: both derivatives vanish
        assert np.abs(dR[j] - fd).max() <= 1e-6 * scale, (j, np.abs(dR[j] - fd).max(), scale)
