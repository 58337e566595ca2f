"""The graph-driven Newton iteration (enp_newton_opts.device_loop = 1): the
Newton steps between preconditioner setups as one CUDA graph launch with
conditional WHILE nodes over the FGMRES restart cycles, the line-search trial
steps and the Newton steps (device-side counts and stopping tests).

* It takes the same iterates as the host-driven loop with graph-captured
  restart cycles, bit for bit: batched operating points, FP64 and mixed
  precision, block-Jacobi and two-level preconditioners, every setup or every
  third (pc_lag = 3).
* Its solution satisfies the oracle's residual equations to the Newton
  tolerance and lies within tolerance times conditioning of the oracle's
  direct-solve Newton solution; a second solve replays the graph and gives the
  same bits.
* The continuation in the applied potential (0.1-0.8 V on the plate reactor)
  reaches the same states with it.
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


def _initial(P, B=1):
    u = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u[k] = P.c_in[k - 1]
    return np.tile(u.reshape(-1), B)


@pytest.mark.parametrize("mixed,two_level,pc_lag", [(False, 0, 1), (True, 1, 1), (True, 1, 3),
                                                    (False, 1, 3)])
def test_device_loop_takes_the_host_loops_iterates(mixed, two_level, pc_lag):
    enp = _enp()
    P = W.config("cube_n3_p2")
    phis = [0.5, 1.17, 2.0]
    B = len(phis)
    kw = dict(max_it=30, rtol=1e-10, krylov_rtol=1e-3, mixed=mixed,
              bj_storage=enp.BJ_F32 if mixed else enp.BJ_F64, graph=True, krylov_restart=30,
              krylov_max_it=2000, pc_lag=pc_lag)
    out = []
    for device_loop in (False, True):
        op = enp.Operator(P, batch=B)
        op.set_phi_app(np.array([[ph, 0.0, 0.0, 0.0] for ph in phis]))
        op.set_preconditioner(two_level)
        u = _cuda(_initial(P, B))
        st = op.newton_solve(u, device_loop=device_loop, **kw)
        assert st["converged"] == 1, st
        out.append((u.cpu().numpy(), st))
    (ue, se), (ud, sd) = out
    assert sd["iterations"] == se["iterations"]
    assert sd["krylov_iterations"] == se["krylov_iterations"]
    assert sd["setups"] == se["setups"]
    np.testing.assert_array_equal(ud, ue)
    np.testing.assert_allclose(sd["history"], se["history"], rtol=0, atol=0)


def test_device_loop_matches_oracle_newton_and_reuses_its_graph():
    enp = _enp()
    P = W.config("reactor_n1_p2")
    ph = 0.3 * 38.92
    Pb = dataclasses.replace(P, bv_phi_app=[ph, 0.0, 0.0, 0.0])
    op = enp.Operator(Pb)
    op.set_preconditioner(1)
    u0 = W.reactor_initial_state(P, [ph])
    orc = oracle.Oracle(Pb)
    ref, _ = orc.newton_solve(u0, rtol=1e-12, max_it=40)
    r0 = np.linalg.norm(orc.residual(u0))
    sols = []
    for _ in range(2):  # the second solve replays the captured graph
        u = _cuda(u0)
        st = op.newton_solve(u, max_it=40, rtol=1e-10, krylov_rtol=1e-3, mixed=True,
                             bj_storage=enp.BJ_F32, krylov_restart=50, krylov_max_it=4000,
                             device_loop=True)
        assert st["converged"] == 1, st
        got = u.cpu().numpy()
        # the oracle's residual at the GPU solution meets the tolerance; the
        # solution error is that tolerance times the conditioning (the
        # Butler-Volmer electrode at 0.3 V)
        assert np.linalg.norm(orc.residual(got)) <= 2e-10 * r0
        assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
        sols.append(got)
    np.testing.assert_array_equal(sols[0], sols[1])


def test_device_loop_continuation_reaches_the_same_states():
    enp = _enp()
    P = W.config("reactor_n1_p2")
    phis = 38.92 * np.array([0.1, 0.45, 0.8])
    B = len(phis)
    target = np.array([[ph, 0.0, 0.0, 0.0] for ph in phis])
    res = []
    for device_loop in (False, True):
        op = enp.Operator(P, batch=B)
        op.set_preconditioner(1)
        u = _cuda(W.reactor_initial_state(P, phis * 0.125))
        st = op.newton_continuation(u, target, bj_storage=enp.BJ_F32, mixed=True, graph=True,
                                    device_loop=device_loop)
        assert st["status"] == enp.ENP_OK and st["lambda"] == 1.0, st
        res.append((u.cpu().numpy(), st))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1]["stages"] == res[1][1]["stages"]
    assert res[0][1]["krylov_iterations"] == res[1][1]["krylov_iterations"]
