"""Parity of the CUDA operator (through the C ABI) with the FP64 CPU oracle.

R(u), J(u)v and J(u)^T w are compared element by element on the same seeded
inputs, as a norm-wise relative error ||x_gpu - x_oracle|| / ||x_oracle|| taken
per field (the potential rows and each species' rows separately, so that an
error confined to one field is not hidden by the others' larger norms): the
FP64-accurate operator must agree to 1e-12 (the exact result up to rounding
order: the oracle uses full quadrature, the GPU sum factorisation), in both of
its arithmetics: native FP64, and double-float on the FP32 pipe (about 48
significant bits, relative rounding 2^-48). Small meshes are checked in full;
the full-size workloads on sampled elements, which the oracle computes row
block by row block. J(u)^T w is checked against the oracle's assembled
transpose (dual-number columns).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
ARITHS = ["f64", "df32"]
_ORACLE_CACHE = {}


def _enp():
    import paper_2112_09271_gb300 as enp
    enp.build()
    return enp


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _relf(a, b, nf):
    """Largest per-field relative error of one operating point: a and b hold
    nf equal field blocks in field order (the library layout [field][element]
    [node], or sampled rows grouped by field)."""
    a, b = np.asarray(a).reshape(nf, -1), np.asarray(b).reshape(nf, -1)
    return max(_rel(a[f], b[f]) for f in range(nf))


def _set_arith(op, arith):
    enp = _enp()
    op.set_arithmetic(enp.ARITH_DF32 if arith == "df32" else enp.ARITH_F64)


def _setup(cfg, seed=0, sources=True, arith="f64"):
    import torch
    enp = _enp()
    P = W.config(cfg) if isinstance(cfg, str) else cfg
    src = W.random_sources(P, 100 + seed) if sources else None
    dirv = W.random_dirichlet(P, 200 + seed) if sources else None
    orc = oracle.Oracle(P, src=src, dirichlet=dirv)
    op = enp.Operator(P)
    _set_arith(op, arith)
    if sources:
        op.set_sources(torch.tensor(src, device="cuda"), torch.tensor(dirv, device="cuda"))
    return P, orc, op


def _cached(key, fn):
    """The oracle's result for key, computed once per test session (the two
    arithmetics are checked against the same reference)."""
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = fn()
    return _ORACLE_CACHE[key]


SMALL = ["mms2d_n3", "mms2d_n4", "cube_n3_p1", "cube_n3_p2", "cube_n3_p3", "cube_n2_p4",
         "channel_n1", "channel_n2", "reactor_n1_p2", "cube_graded", "cube_dirichlet_graded"]

# graded vertex coordinates: neighbouring elements differ in size along every axis,
# so the two sides of a face have different lengths, normal scalings and diagonals
GRADED = [np.array([0.0, 0.22, 0.61, 1.0]), np.array([0.0, 0.45, 0.7, 1.0]),
          np.array([0.0, 0.3, 0.52, 1.0])]


def _small(cfg):
    import dataclasses
    if cfg == "mms2d_n4":
        return W.config("mms2d_n4", p=3)
    if cfg == "channel_n1":
        return W.config("channel_n1", p=2)
    if cfg == "cube_graded":
        return dataclasses.replace(W.config("cube_n3_p2"), coords=[c.copy() for c in GRADED])
    if cfg == "cube_dirichlet_graded":
        P = W.config("cube_n3_p3")
        return dataclasses.replace(P, coords=[c.copy() for c in GRADED],
                                   tags=[np.full_like(t, W.DIRICHLET) for t in P.tags])
    return W.config(cfg)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("cfg", SMALL)
def test_residual_matches_oracle(cfg, arith):
    import torch
    P, orc, op = _setup(_small(cfg), sources=True, arith=arith)
    u = W.random_state(P, 1)
    r = op.residual(torch.tensor(u, device="cuda")).cpu().numpy()
    ref = _cached((cfg, "res"), lambda: orc.residual(u))
    e = _relf(r, ref, P.n_fields)
    assert e < TOL64, e


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("cfg", SMALL)
def test_jvp_matches_oracle(cfg, arith):
    import torch
    P, orc, op = _setup(_small(cfg), sources=True, arith=arith)
    u, v = W.random_state(P, 1), W.random_vector(P, 2)
    jv = op.jvp(torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")).cpu().numpy()
    ref = _cached((cfg, "jvp"), lambda: orc.jvp(u, v))
    e = _relf(jv, ref, P.n_fields)
    assert e < TOL64, e


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("cfg", SMALL)
def test_vjp_matches_oracle_transpose(cfg, arith):
    import torch
    P, orc, op = _setup(_small(cfg), sources=True, arith=arith)
    u, w = W.random_state(P, 1), W.random_vector(P, 3)
    jtw = op.vjp(torch.tensor(u, device="cuda"), torch.tensor(w, device="cuda")).cpu().numpy()
    ref = _cached((cfg, "vjp"), lambda: orc.vjp_entries(u, w, np.arange(P.n_dof)))
    e = _relf(jtw, ref, P.n_fields)
    assert e < TOL64, e


@pytest.mark.parametrize("arith", ARITHS)
def test_vjp_is_the_adjoint_of_jvp_on_gpu(arith):
    import torch
    P, orc, op = _setup("cube_n4_p3", sources=False, arith=arith)
    u = torch.tensor(W.random_state(P, 1), device="cuda")
    v = torch.tensor(W.random_vector(P, 2), device="cuda")
    w = torch.tensor(W.random_vector(P, 3), device="cuda")
    lhs = torch.dot(w, op.jvp(u, v)).item()
    rhs = torch.dot(op.vjp(u, w), v).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


FULL = [("cube16_p3", 48), ("channel64_p3", 24), ("cube24_p2", 24), ("reactor192_p2", 24)]


def _sample_elements(P, nsample):
    rng = np.random.default_rng(5)
    return np.unique(np.concatenate([rng.choice(P.E, nsample, replace=False),
                                     [0, P.E - 1, P.n_el[0] * P.n_el[1] // 2]]))


@pytest.mark.parametrize("cfg,nsample", FULL)
def test_full_size_sampled_rows(cfg, nsample):
    """At the benchmark sizes, in the launch configuration the bench uses: the
    GPU computes every row, the oracle the rows of sampled elements (including
    boundary and electrode elements); both arithmetics of the FP64 operator,
    after autotuning as in the bench."""
    import torch
    P = W.config(cfg)
    enp = _enp()
    op = enp.Operator(P)
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    v = W.random_vector(P, 3)
    w = W.random_vector(P, 4)
    el = _sample_elements(P, nsample)
    rr = orc.residual(u, elems=el).reshape(P.n_fields, P.E, P.Np)[:, el]
    jr = orc.jvp(u, v, elems=el).reshape(P.n_fields, P.E, P.Np)[:, el]
    # J^T w on the columns of a few sampled elements, field by field
    cols = np.concatenate([f * P.E * P.Np + e * P.Np + np.arange(P.Np)
                           for f in range(P.n_fields) for e in el[:6]])
    tr = orc.vjp_entries(u, w, cols)
    ud, vd, wd = (torch.tensor(x, device="cuda") for x in (u, v, w))
    for arith in ARITHS:
        _set_arith(op, arith)
        op.autotune()
        r = op.residual(ud).cpu().numpy().reshape(P.n_fields, P.E, P.Np)[:, el]
        jv = op.jvp(ud, vd).cpu().numpy().reshape(P.n_fields, P.E, P.Np)[:, el]
        jtw = op.vjp(ud, wd).cpu().numpy()[cols]
        errs = (_relf(r, rr, P.n_fields), _relf(jv, jr, P.n_fields),
                _relf(jtw, tr, P.n_fields))
        assert max(errs) < TOL64, (arith, errs)


@pytest.mark.parametrize("cfg", ["cube16_p3", "channel64_p3", "reactor192_p2"])
def test_double_float_operator_agrees_with_fp64_on_every_row(cfg):
    """At full size, every row: the double-float operator against the native
    FP64 one (both are checked against the oracle on sampled rows above; here
    no row of the full mesh escapes). The two differ by rounding only: 2^-48
    per double-float operation against 2^-53."""
    import torch
    P = W.config(cfg)
    enp = _enp()
    op = enp.Operator(P)
    ud = torch.tensor(W.random_state(P, 2), device="cuda")
    vd = torch.tensor(W.random_vector(P, 3), device="cuda")
    out = {}
    for arith in ARITHS:
        _set_arith(op, arith)
        out[arith] = [op.residual(ud).cpu().numpy(), op.jvp(ud, vd).cpu().numpy(),
                      op.vjp(ud, vd).cpu().numpy()]
    errs = [_relf(a, b, P.n_fields) for a, b in zip(out["df32"], out["f64"])]
    assert max(errs) < TOL64, errs


@pytest.mark.parametrize("cfg,nsample", [("channel64_p3", 16), ("reactor192_p2", 16)])
def test_full_size_jvp_f32_sampled_rows(cfg, nsample):
    """The FP32 inner operator of the mixed-precision solves, at the benchmark
    sizes (including the plate reactor's Butler-Volmer electrode): sampled rows
    against the oracle, to single precision."""
    import torch
    P = W.config(cfg)
    enp = _enp()
    op = enp.Operator(P)
    op.autotune()
    orc = oracle.Oracle(P)
    u, v = W.random_state(P, 2), W.random_vector(P, 3)
    el = _sample_elements(P, nsample)
    jr = orc.jvp(u, v, elems=el).reshape(P.n_fields, P.E, P.Np)[:, el]
    jv = op.jvp_f32(torch.tensor(u, device="cuda", dtype=torch.float32),
                    torch.tensor(v, device="cuda", dtype=torch.float32)).cpu().numpy()
    jv = jv.reshape(P.n_fields, P.E, P.Np)[:, el].astype(np.float64)
    assert _rel(jv, jr) < 2e-5, _rel(jv, jr)


@pytest.mark.parametrize("cfg", ["cube_n3_p3", "channel_n2", "reactor_n1_p2"])
def test_jvp_f32_matches_oracle_to_single_precision(cfg):
    import torch
    P, orc, op = _setup(cfg, sources=False)
    u, v = W.random_state(P, 1), W.random_vector(P, 2)
    jv = op.jvp_f32(torch.tensor(u, device="cuda", dtype=torch.float32),
                    torch.tensor(v, device="cuda", dtype=torch.float32)).cpu().numpy()
    ref = orc.jvp(u, v)
    assert _rel(jv.astype(np.float64), ref) < 2e-5


@pytest.mark.parametrize("arith", ARITHS)
def test_batched_operating_points_match_single_runs(arith):
    import torch
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 3
    phis = np.array([[0.1 * 38.92 * (b + 1), 0.0, 0.0, 0.0] for b in range(B)])
    opb = enp.Operator(P, batch=B)
    _set_arith(opb, arith)
    opb.set_phi_app(phis)
    u = np.concatenate([W.random_state(P, 10 + b) for b in range(B)])
    v = np.concatenate([W.random_vector(P, 20 + b) for b in range(B)])
    ud, vd = torch.tensor(u, device="cuda"), torch.tensor(v, device="cuda")
    rb = opb.residual(ud).cpu().numpy().reshape(B, -1)
    jb = opb.jvp(ud, vd).cpu().numpy().reshape(B, -1)
    import dataclasses
    for b in range(B):
        Pb = dataclasses.replace(P, bv_phi_app=list(phis[b]))
        orc = oracle.Oracle(Pb)
        ub, vb = u.reshape(B, -1)[b], v.reshape(B, -1)[b]
        assert _relf(rb[b], orc.residual(ub), P.n_fields) < TOL64
        assert _relf(jb[b], orc.jvp(ub, vb), P.n_fields) < TOL64


def test_unsupported_and_invalid_inputs_raise():
    import dataclasses
    enp = _enp()
    P = W.config("cube_n2_p3")
    with pytest.raises(enp.EnpError) as ei:
        enp.Operator(dataclasses.replace(P, q=P.p + 1))
    assert ei.value.status == enp.ENP_ERR_UNSUPPORTED
    bad = [c.copy() for c in P.coords]
    bad[0][1] = bad[0][0]
    with pytest.raises(enp.EnpError) as ei:
        enp.Operator(dataclasses.replace(P, coords=bad))
    assert ei.value.status == enp.ENP_ERR_INVALID_ARG
