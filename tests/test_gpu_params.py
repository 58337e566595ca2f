"""dR/dtheta, the parameter adjoint and the torch.autograd.Function against the
oracle. theta = (D_1..D_m, c_in_1..c_in_{m-1}, phi_app_0..3). The GPU parameter
Jacobian is exact (forward-tangent coefficients), so it must match the oracle's
dual sweep to 1e-12 relative per parameter; the oracle's sweep is itself pinned
to central differences in test_oracle_pins.py."""
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


def _check_rows(g, ref):
    for j in range(ref.shape[0]):
        s = np.abs(ref[j]).max()
        if s == 0:
            assert np.abs(g[j]).max() == 0
        else:
            assert np.linalg.norm(g[j] - ref[j]) <= 1e-12 * np.linalg.norm(ref[j]), j


@pytest.mark.parametrize("cfg", ["cube_n3_p2", "cube_n2_p3", "channel_n1", "reactor_n1_p2"])
def test_param_jacobian_matches_oracle(cfg):
    enp = _enp()
    P = W.config(cfg)
    tags = [t.copy() for t in P.tags]
    tags[0][:] = W.INLET
    import dataclasses
    P = dataclasses.replace(P, tags=tags)
    op = enp.Operator(P)
    u = W.random_state(P, 2)
    g = op.param_jacobian(_cuda(u)).cpu().numpy()
    _check_rows(g, oracle.Oracle(P).param_jacobian(u))


def test_param_jacobian_full_size_config4():
    """cube24_p2 (746k DOFs): every parameter row against the oracle."""
    enp = _enp()
    P = W.config("cube24_p2")
    op = enp.Operator(P)
    u = W.random_state(P, 2)
    g = op.param_jacobian(_cuda(u)).cpu().numpy()
    _check_rows(g, oracle.Oracle(P).param_jacobian(u))


def test_param_vjp_and_autograd_function():
    import torch
    enp = _enp()
    P = W.config("cube_n3_p2")
    op = enp.Operator(P)
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    w = W.random_vector(P, 5)
    d = op.param_vjp(_cuda(u), _cuda(w))[0]
    ref = orc.param_jacobian(u) @ w
    assert np.abs(d - ref).max() <= 1e-12 * np.abs(ref).max()
    # autograd: R(u; theta) with backward = (J^T g, (dR/dtheta)^T g)
    fn = enp.residual_function(op)
    ut = _cuda(u).requires_grad_(True)
    th = torch.zeros(op.n_theta, dtype=torch.float64, device="cuda", requires_grad=True)
    r = fn(ut, th)
    r.backward(_cuda(w))
    jtw = orc.vjp_entries(u, w, np.arange(P.n_dof))
    assert np.linalg.norm(ut.grad.cpu().numpy() - jtw) <= 1e-12 * np.linalg.norm(jtw)
    assert np.abs(th.grad.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    # the forward value is R(u)
    assert np.linalg.norm(r.detach().cpu().numpy() - orc.residual(u)) <= 1e-12 * np.linalg.norm(
        orc.residual(u))


def test_param_jacobian_unsupported_in_2d():
    enp = _enp()
    op = enp.Operator(W.config("mms2d_n3"))
    with pytest.raises(enp.EnpError) as ei:
        op.param_jacobian(_cuda(W.random_state(W.config("mms2d_n3"), 1)))
    assert ei.value.status == enp.ENP_ERR_UNSUPPORTED


def test_param_vjp_total_sums_the_operating_points_on_the_device():
    """Batched autograd: one parameter vector shared by the batch gets the sum
    over operating points of <w_b, dR_b/dtheta>, formed in the library."""
    import dataclasses

    import torch
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 2
    phis = np.array([[0.2 * 38.92, 0.0, 0.0, 0.0], [0.5 * 38.92, 0.0, 0.0, 0.0]])
    op = enp.Operator(P, batch=B)
    op.set_phi_app(phis)
    us = [W.random_state(P, 30 + b) for b in range(B)]
    ws = [W.random_vector(P, 40 + b) for b in range(B)]
    u, w = _cuda(np.concatenate(us)), _cuda(np.concatenate(ws))
    per_point = op.param_vjp(u, w)
    total = op.param_vjp_total(u, w)
    assert np.array_equal(total, per_point[0] + per_point[1])
    ref = sum(oracle.Oracle(dataclasses.replace(P, bv_phi_app=list(phis[b]))).param_jacobian(us[b])
              @ ws[b] for b in range(B))
    assert np.abs(total - ref).max() <= 1e-12 * np.abs(ref).max()
    # the autograd Function's parameter gradient is that total
    fn = enp.residual_function(op)
    th = torch.zeros(op.n_theta, dtype=torch.float64, device="cuda", requires_grad=True)
    fn(u, th).backward(w)
    assert np.array_equal(th.grad.cpu().numpy(), total)
