"""Parity of the block-Jacobi preconditioner, FGMRES, Newton and c_m recovery
(through the C ABI) with the oracle.

* diagonal blocks of J(u): element by element against the oracle's assembled
  Jacobian, 1e-12 relative;
* block-Jacobi apply: against dense LU solves of the oracle's blocks. FP64:
  the Gauss-Jordan inverse differs from an LU solve by rounding amplified by
  the block condition number kappa, so the bound is 1e-14 * kappa_max (checked
  to be below 1e-9 on these meshes); FP32 storage 1e-5 * kappa_max; BF16 2e-2;
* FGMRES: against the sparse direct solve of J(u) x = b, to the Krylov
  tolerance times the condition estimate;
* Newton: the GPU solution against the oracle's direct-solve Newton solution;
* c_m: against Eq. substitution on the host.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cuda(x):
    import torch
    return torch.tensor(np.asarray(x), device="cuda")


BLOCK_CASES = ["cube_n3_p2", "cube_n2_p3", "channel_n1", "mms2d_n3", "reactor_n1_p2"]


def _prob(cfg):
    if cfg == "channel_n1":
        return W.config(cfg, p=2)
    if cfg == "channel_n1_p3":
        return W.config("channel_n1", p=3)
    if cfg == "cube_n2_p3_dirichlet":
        import dataclasses
        P = W.config("cube_n2_p3")
        return dataclasses.replace(P, tags=[np.full_like(t, W.DIRICHLET) for t in P.tags])
    return W.config(cfg)


@pytest.mark.parametrize("arith", ["f64", "df32"])
@pytest.mark.parametrize("cfg", BLOCK_CASES)
def test_block_diagonal_matches_oracle(cfg, arith):
    enp = _enp()
    P = _prob(cfg)
    dirv = W.random_dirichlet(P, 7)
    op = enp.Operator(P)
    op.set_arithmetic(enp.ARITH_DF32 if arith == "df32" else enp.ARITH_F64)
    op.set_sources(None, _cuda(dirv))
    orc = oracle.Oracle(P, dirichlet=dirv)
    u = W.random_state(P, 2)
    nb = P.n_fields * P.Np
    g = op.block_diagonal(_cuda(u)).cpu().numpy().reshape(P.E, nb, nb)
    ref = orc.block_diagonal(u)
    assert _rel(g, ref) < 1e-12


# block sizes 16, 54, 81, 128 and 192 (every shape of the FP32 register inversion) and
# 250 (p = 4, two fields: the two-CTA cluster inversion)
@pytest.mark.parametrize("cfg", ["cube_n3_p1", "cube_n3_p2", "cube_n2_p3", "channel_n1",
                                 "channel_n1_p3", "cube_n2_p4", "reactor_n1_p2",
                                 "cube_n2_p3_dirichlet"])
@pytest.mark.parametrize("storage,tol", [(0, 1e-14), (1, 1e-5), (2, 2e-2)])
def test_block_jacobi_apply_matches_oracle(cfg, storage, tol):
    enp = _enp()
    P = _prob(cfg)
    op = enp.Operator(P)
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    x = W.random_vector(P, 5)
    blocks = orc.block_diagonal(u)
    kappa = float(np.max(np.linalg.cond(blocks)))
    op.block_jacobi_setup(_cuda(u), storage)
    y = op.block_jacobi_apply(_cuda(x)).cpu().numpy()
    ref = orc.block_jacobi_apply(blocks, x)
    bound = tol * kappa if storage < 2 else tol
    if storage == 0:
        assert bound < 1e-9
    assert _rel(y, ref) < bound, (_rel(y, ref), kappa)


@pytest.mark.parametrize("cfg,precond", [("cube_n3_p2", True), ("channel_n1", True),
                                         ("mms2d_n3", False)])
def test_fgmres_matches_direct_solve(cfg, precond):
    enp = _enp()
    P = _prob(cfg)
    dirv = W.random_dirichlet(P, 7)
    op = enp.Operator(P)
    op.set_sources(None, _cuda(dirv))
    orc = oracle.Oracle(P, dirichlet=dirv)
    u = W.random_state(P, 2)
    b = W.random_vector(P, 6)
    ud, bd = _cuda(u), _cuda(b)
    if precond:
        op.block_jacobi_setup(ud, 0)
    x = _cuda(np.zeros(P.n_dof))
    st = op.fgmres_solve(ud, bd, x, restart=40, max_it=2000, rtol=1e-12)
    assert st["converged"] == 1
    ref = orc.linear_solve(u, b)
    # the true residual meets the tolerance; the error is bounded by cond(J) * rtol
    r = orc.jvp(u, x.cpu().numpy()) - b
    assert np.linalg.norm(r) <= 1.01e-12 * np.linalg.norm(b)
    assert _rel(x.cpu().numpy(), ref) < 1e-7


def test_fgmres_batched_matches_single():
    """Operating points of a batch are solved independently: each one's iterate
    is bit-for-bit the one a single solve gives (same reductions, same cycle
    structure; a converged point is frozen), and matches the direct solve."""
    import torch
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 2
    phis = np.array([[1.0, 0, 0, 0], [3.0, 0, 0, 0]])
    u = np.concatenate([W.random_state(P, 2), W.random_state(P, 3)])
    b = np.concatenate([W.random_vector(P, 6), 10 * W.random_vector(P, 7)])
    opts = dict(restart=80, max_it=3000, rtol=1e-10)
    singles, its = [], []
    for i in range(B):
        op1 = enp.Operator(dataclasses.replace(P, bv_phi_app=list(phis[i])))
        u1 = _cuda(u.reshape(B, -1)[i])
        op1.block_jacobi_setup(u1, 0)
        x1 = torch.zeros(P.n_dof, dtype=torch.float64, device="cuda")
        st1 = op1.fgmres_solve(u1, _cuda(b.reshape(B, -1)[i]), x1, **opts)
        singles.append(x1.cpu().numpy())
        its.append(st1["iterations"])
    op = enp.Operator(P, batch=B)
    op.set_phi_app(phis)
    ud = _cuda(u)
    op.block_jacobi_setup(ud, 0)
    x = torch.zeros(B * P.n_dof, dtype=torch.float64, device="cuda")
    st = op.fgmres_solve(ud, _cuda(b), x, **opts)
    assert st["converged"] == 1 and st["iterations"] == max(its)
    xs = x.cpu().numpy().reshape(B, -1)
    for i in range(B):
        np.testing.assert_array_equal(xs[i], singles[i])
        orc = oracle.Oracle(dataclasses.replace(P, bv_phi_app=list(phis[i])))
        ref = orc.linear_solve(u.reshape(B, -1)[i], b.reshape(B, -1)[i])
        assert _rel(xs[i], ref) < 1e-6


def test_fgmres_reports_non_convergence():
    enp = _enp()
    P = W.config("cube_n3_p2")
    op = enp.Operator(P)
    u = W.random_state(P, 2)
    x = _cuda(np.zeros(P.n_dof))
    st = op.fgmres_solve(_cuda(u), _cuda(W.random_vector(P, 6)), x, restart=5, max_it=3,
                         rtol=1e-14, raise_on_fail=False)
    assert st["status"] == enp.ENP_ERR_NOT_CONVERGED and st["converged"] == 0
    assert st["iterations"] == 3


def _newton_case(name):
    """Small nonlinear problems that need no symbolic sources: the reactor cube
    (inlet/outlet, Butler-Volmer electrodes, plate flow) and a 2D Dirichlet box
    with random smooth-amplitude sources."""
    if name == "reactor_cube":
        P = W.config("cube_n3_p2")
        return P, None, None
    P = W.config("mms2d_n4")
    src = 0.05 * W.random_sources(P, 31)
    dirv = W.random_dirichlet(P, 32, base=1.0, amp=0.05)
    return P, src, dirv


def _initial(P):
    u = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u[k] = P.c_in[k - 1]
    return u.reshape(-1)


@pytest.mark.parametrize("name", ["reactor_cube", "dirichlet_2d"])
@pytest.mark.parametrize("mixed", [False, True])
def test_newton_matches_oracle_newton(name, mixed):
    enp = _enp()
    P, src, dirv = _newton_case(name)
    orc = oracle.Oracle(P, src=src, dirichlet=dirv)
    u0 = _initial(P)
    ref, hist = orc.newton_solve(u0, rtol=1e-12, max_it=30)
    op = enp.Operator(P)
    if src is not None:
        op.set_sources(_cuda(src), _cuda(dirv))
    ud = _cuda(u0)
    st = op.newton_solve(ud, max_it=30, rtol=1e-10, krylov_rtol=1e-3 if not mixed else 1e-2,
                         bj_storage=0 if not mixed else 1, mixed=mixed)
    assert st["converged"] == 1, st
    assert st["residual_norm"] <= 1e-10 * st["initial_norm"]
    u = ud.cpu().numpy()
    # the oracle's residual at the GPU solution
    assert np.linalg.norm(orc.residual(u)) <= 2e-10 * np.linalg.norm(orc.residual(u0))
    assert _rel(u, ref) < 1e-8


def test_newton_reports_nonfinite_input():
    enp = _enp()
    P = W.config("cube_n2_p2")
    u = _initial(P)
    u[5] = np.nan
    op = enp.Operator(P)
    st = op.newton_solve(_cuda(u), raise_on_fail=False)
    assert st["status"] == enp.ENP_ERR_NONFINITE


def test_block_jacobi_singular_block_is_reported():
    enp = _enp()
    P = W.config("cube_n2_p2")
    u = _initial(P)
    u[3] = np.inf
    op = enp.Operator(P)
    with pytest.raises(enp.EnpError) as ei:
        op.block_jacobi_setup(_cuda(u), 0)
    assert ei.value.status == enp.ENP_ERR_NONFINITE


@pytest.mark.parametrize("cfg", ["channel_n2", "cube_n3_p2"])
def test_recover_cm_matches_substitution(cfg):
    enp = _enp()
    P = W.config(cfg)
    u = W.random_state(P, 4)
    op = enp.Operator(P)
    cm = op.recover_cm(_cuda(u)).cpu().numpy()
    ref = oracle.recover_cm(P, u)
    assert np.abs(cm - ref).max() <= 1e-15 * np.abs(ref).max()


def test_inner_product_matches_numpy():
    enp = _enp()
    P = W.config("channel_n2")
    op = enp.Operator(P)
    x, y = W.random_vector(P, 1), W.random_vector(P, 2)
    d = op.inner_product(_cuda(x), _cuda(y))[0]
    assert abs(d - float(np.dot(x, y))) <= 1e-13 * float(np.dot(np.abs(x), np.abs(y)))


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_shared_block_inverses(storage):
    """One set of block inverses for the whole batch (enp_set_shared_blocks):
    with identical operating points the apply equals the per-point apply bit
    for bit; with different states FGMRES preconditioned by the shared set
    reaches the per-point solutions."""
    import torch
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 2
    phis = np.array([[4.0, 0, 0, 0], [4.0, 0, 0, 0]])
    u1 = W.random_state(P, 2)
    x = np.concatenate([W.random_vector(P, 5), W.random_vector(P, 6)])
    ys = []
    for shared in (-1, 1):
        op = enp.Operator(P, batch=B)
        op.set_phi_app(phis)
        op.set_shared_blocks(shared)
        op.block_jacobi_setup(_cuda(np.concatenate([u1, u1])), storage)
        ys.append(op.block_jacobi_apply(_cuda(x)).cpu().numpy())
    np.testing.assert_array_equal(ys[0], ys[1])
    # different operating points: the shared set still preconditions FGMRES
    phis = np.array([[4.0, 0, 0, 0], [20.0, 0, 0, 0]])
    u = _cuda(np.concatenate([W.random_state(P, 2), W.random_state(P, 3)]))
    b = _cuda(x)
    sols = []
    for shared in (-1, 0):
        op = enp.Operator(P, batch=B)
        op.set_phi_app(phis)
        op.set_shared_blocks(shared)
        op.block_jacobi_setup(u, storage)
        xs = torch.zeros_like(b)
        st = op.fgmres_solve(u, b, xs, restart=40, max_it=3000, rtol=1e-10)
        assert st["converged"] == 1, st
        sols.append(xs.cpu().numpy())
    assert _rel(sols[1], sols[0]) < 1e-7
    with pytest.raises(enp.EnpError):
        op.set_shared_blocks(B)
