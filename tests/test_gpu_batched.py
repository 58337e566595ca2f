"""Batched operating points and graph-captured Krylov cycles.

* FGMRES replaying one CUDA-graph-captured restart cycle gives bit for bit the
  iterate of the eager loop (same kernels, same order; a converged point is
  frozen in both).
* Newton over a batch of applied potentials (the Phi_app sweep of the reactor
  workload, Sec. 5.2) solves every operating point independently: each one's
  solution is bit for bit its single-point solution, and matches the oracle's
  direct-solve Newton solution for that potential.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _enp():
    import paper_2112_09271_gb300 as enp
    enp.build()
    return enp


def _cuda(x):
    import torch
    return torch.tensor(np.asarray(x), device="cuda")


def _initial(P, batch=1):
    u = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u[k] = P.c_in[k - 1]
    return np.tile(u.reshape(-1), batch)


@pytest.mark.parametrize("f32", [False, True])
def test_graph_fgmres_equals_eager(f32):
    import torch
    enp = _enp()
    P = W.config("cube_n3_p2")
    op = enp.Operator(P)
    u = _cuda(W.random_state(P, 2))
    b = _cuda(W.random_vector(P, 6))
    op.block_jacobi_setup(u, enp.BJ_F32)
    if f32:
        u, b = u.float(), b.float()
    res = []
    for graph in (False, True):
        x = torch.zeros_like(b)
        # FP32 vectors: the true residual cannot go much below 1e-6 relative
        st = op.fgmres_solve(u, b, x, restart=10, max_it=400, rtol=1e-4 if f32 else 1e-6,
                             graph=graph)
        assert st["converged"] == 1
        res.append((x.cpu().numpy(), st["iterations"]))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


@pytest.mark.parametrize("mixed,graph", [(False, False), (True, True)])
def test_batched_newton_equals_single_solves(mixed, graph):
    enp = _enp()
    P = W.config("cube_n3_p2")
    phis = [0.5, 1.17, 2.0]
    B = len(phis)
    kw = dict(max_it=30, rtol=1e-10, krylov_rtol=1e-3, bj_storage=enp.BJ_F32 if mixed else enp.BJ_F64,
              mixed=mixed, graph=graph, krylov_restart=30, krylov_max_it=2000)
    singles = []
    for ph in phis:
        Pb = dataclasses.replace(P, bv_phi_app=[ph, 0.0, 0.0, 0.0])
        op1 = enp.Operator(Pb)
        u1 = _cuda(_initial(P))
        st1 = op1.newton_solve(u1, **kw)
        assert st1["converged"] == 1, st1
        singles.append(u1.cpu().numpy())
    op = enp.Operator(P, batch=B)
    op.set_phi_app(np.array([[ph, 0.0, 0.0, 0.0] for ph in phis]))
    ub = _cuda(_initial(P, B))
    st = op.newton_solve(ub, **kw)
    assert st["converged"] == 1, st
    got = ub.cpu().numpy().reshape(B, -1)
    for i, ph in enumerate(phis):
        np.testing.assert_array_equal(got[i], singles[i])
        orc = oracle.Oracle(dataclasses.replace(P, bv_phi_app=[ph, 0.0, 0.0, 0.0]))
        ref, _ = orc.newton_solve(_initial(P), rtol=1e-12)
        assert np.linalg.norm(got[i] - ref) <= 1e-8 * np.linalg.norm(ref)


def test_autotune_keeps_results():
    """The tile shapes chosen by the autotuner (faces per block, elements per
    block) change the block decomposition, not the arithmetic: results are
    unchanged bit for bit, in FP64 and double-float."""
    import torch
    enp = _enp()
    P = W.config("channel_n2")
    op = enp.Operator(P)
    u, v = _cuda(W.random_state(P, 1)), _cuda(W.random_vector(P, 2))
    before = (op.residual(u).cpu().numpy(), op.jvp(u, v).cpu().numpy())
    chosen = op.autotune()
    assert len(chosen) == 5 and all(c >= 1 for c in chosen)
    eb, fpb = op.launch_shapes()
    assert eb == chosen and all(f >= 1 for f in fpb)
    after = (op.residual(u).cpu().numpy(), op.jvp(u, v).cpu().numpy())
    np.testing.assert_array_equal(before[0], after[0])
    np.testing.assert_array_equal(before[1], after[1])
    # every face tile shape gives the same bits (each face is computed by one
    # group of threads whatever the number of faces per block)
    op.set_arithmetic(enp.ARITH_DF32)
    op.autotune()
    d_after = op.jvp(u, v).cpu().numpy()
    op2 = enp.Operator(P)
    op2.set_arithmetic(enp.ARITH_DF32)
    np.testing.assert_array_equal(op2.jvp(u, v).cpu().numpy(), d_after)


@pytest.mark.parametrize("mixed", [False, True])
def test_continuation_reaches_strongly_driven_electrodes(mixed):
    """Applied potentials 0.1 to 0.8 V on the plate reactor (Butler-Volmer
    exponents up to e^31, Sec. 5.2): Newton from c = c_in, Phi = Phi_app / 2
    fails at the top of the range, continuation in Phi_app reaches it. At the
    end every operating point satisfies the oracle's residual equations at its
    target potential to the tolerance, and the applied potentials of the
    handle are the target ones."""
    enp = _enp()
    P = W.config("reactor_n1_p2")
    volts = np.array([0.1, 0.35, 0.6, 0.8])
    phis = 38.92 * volts
    B = len(phis)
    target = np.array([[ph, 0.0, 0.0, 0.0] for ph in phis])
    op = enp.Operator(P, batch=B)
    op.set_preconditioner(1)
    kw = dict(bj_storage=enp.BJ_F32 if mixed else enp.BJ_F64, mixed=mixed, graph=mixed)
    u = _cuda(W.reactor_initial_state(P, phis * 0.125))
    st = op.newton_continuation(u, target, **kw)
    assert st["status"] == enp.ENP_OK and st["lambda"] == 1.0, st
    assert st["last"]["residual_norm"] <= 1e-10 * st["last"]["initial_norm"]
    got = u.cpu().numpy().reshape(B, -1)
    for i in range(B):
        orc = oracle.Oracle(dataclasses.replace(P, bv_phi_app=list(target[i])))
        r = np.linalg.norm(orc.residual(got[i]))
        assert r <= 2e-10 * st["last"]["initial_norm"], (i, r)
    # the handle is left at the target potentials: its residual there is small
    import torch
    r = torch.empty_like(u)
    op.residual(u, out=r)
    assert float(r.norm()) <= 2e-10 * st["last"]["initial_norm"] * np.sqrt(B)


def test_continuation_rejects_bad_options():
    enp = _enp()
    P = W.config("reactor_n1_p2")
    op = enp.Operator(P)
    u = _cuda(W.reactor_initial_state(P, [1.0]))
    with pytest.raises(enp.EnpError) as ei:
        op.newton_continuation(u, [[1.0, 0, 0, 0]], step0=0.5, step_max=0.25)
    assert ei.value.status == enp.ENP_ERR_INVALID_ARG
