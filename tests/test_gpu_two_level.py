"""The two-level preconditioner: block-Jacobi plus a coarse correction on the
element-mean potential (through the C ABI).

* the coarse operator A0 = P^T J_PhiPhi(u) P, assembled on the GPU from seven
  coloured J v products, equals the same product formed from the oracle's
  assembled Jacobian, entry by entry, to 1e-12 of its largest entry, and has no
  entry outside the 7-point element stencil (the potential couples only
  face neighbours in the SIPG form of Sec. 3.3);
* FGMRES preconditioned by it reaches the tolerance on the true (oracle)
  residual and the direct-solve solution, in fewer iterations than with
  block-Jacobi alone, on one- to four-level hierarchies (grid-wide and
  one-block smoothing) and with FP32 vectors;
* with a singular coarse operator (no electrode fixes the potential) the
  coarsest level falls back to smoothing and FGMRES still converges;
* Newton with it reaches the oracle's Newton solution;
* argument errors are reported.
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _a0_oracle(orc, P, u):
    """P^T J_PhiPhi P from the oracle's assembled Jacobian (dense, E x E)."""
    import scipy.sparse as sp
    J = orc.jacobian(u).tocsr()
    nphi = P.E * P.Np
    Pm = sp.csr_matrix((np.ones(nphi), (np.arange(nphi), np.repeat(np.arange(P.E), P.Np))),
                       shape=(nphi, P.E))
    return (Pm.T @ J[:nphi, :nphi] @ Pm).toarray()


def _a0_dense(P, st):
    """Dense E x E matrix from the stencil rows [E][7] (self, -x, +x, -y, +y, -z, +z)."""
    nx, ny, nz = P.n_el
    A = np.zeros((P.E, P.E))
    off = [0, -1, 1, -nx, nx, -nx * ny, nx * ny]
    for K in range(P.E):
        ix, iy, iz = K % nx, (K // nx) % ny, K // (nx * ny)
        ok = [True, ix > 0, ix < nx - 1, iy > 0, iy < ny - 1, iz > 0, iz < nz - 1]
        for d in range(7):
            if ok[d]:
                A[K, K + off[d]] += st[K, d]
            else:
                assert st[K, d] == 0.0
    return A


@pytest.mark.parametrize("cfg,p,batch", [("channel_n2", 2, 1), ("cube_n3_p3", None, 1),
                                         ("reactor_n1_p2", None, 2)])
def test_coarse_operator_matches_oracle(cfg, p, batch):
    enp = _enp()
    P = W.config(cfg, p=p) if p else W.config(cfg)
    phis = [[1.17 + 0.5 * i, 0.0, 0.0, 0.0] for i in range(batch)]
    us = [W.random_state(P, 2 + i) for i in range(batch)]
    op = enp.Operator(P, batch=batch)
    if batch > 1:
        op.set_phi_app(np.array(phis))
    op.set_preconditioner(1)
    op.block_jacobi_setup(_cuda(np.concatenate(us)), 0)
    a0 = op.coarse_operator().cpu().numpy().reshape(batch, P.E, 7)
    for i in range(batch):
        Pi = dataclasses.replace(P, bv_phi_app=phis[i]) if batch > 1 else P
        ref = _a0_oracle(oracle.Oracle(Pi), Pi, us[i])
        got = _a0_dense(P, a0[i])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _solve(op, u, b, two_level, f32=False, restart=60, max_it=4000, rtol=1e-10):
    import torch
    op.set_preconditioner(1 if two_level else 0)
    ud = _cuda(u)
    op.block_jacobi_setup(ud, 0 if not f32 else 1)
    dt = torch.float32 if f32 else torch.float64
    x = torch.zeros(b.size, dtype=dt, device="cuda")
    st = op.fgmres_solve(ud.to(dt), _cuda(b).to(dt), x, restart=restart, max_it=max_it, rtol=rtol)
    return x.double().cpu().numpy(), st


# cube_n21_p1: 9261 cells on the finest coarse level, above the one-block
# V-cycle's 8192, so its smoothing runs grid-wide and the levels below in one block
@pytest.mark.parametrize("cfg,levels", [("cube_n5_p2", 1), ("cube_n9_p1", 2),
                                        ("cube_n18_p1", 3), ("cube_n21_p1", 4)])
def test_two_level_fgmres_converges_faster(cfg, levels):
    enp = _enp()
    P = W.config(cfg)
    nx = P.n_el[0]
    n_lev, m = 1, nx
    while m ** 3 > 128:  # coarsest grid: at most 128 cells, solved with its inverse
        m, n_lev = (m + 1) // 2, n_lev + 1
    assert n_lev == levels
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    b = W.random_vector(P, 6)
    op = enp.Operator(P)
    x1, st1 = _solve(op, u, b, False)
    x2, st2 = _solve(op, u, b, True)
    assert st1["converged"] == 1 and st2["converged"] == 1
    for x in (x1, x2):
        assert np.linalg.norm(orc.jvp(u, x) - b) <= 1.01e-10 * np.linalg.norm(b)
    assert _rel(x2, x1) < 1e-6
    assert st2["iterations"] < st1["iterations"], (st1["iterations"], st2["iterations"])
    if P.n_dof < 30000:
        assert _rel(x2, orc.linear_solve(u, b)) < 1e-6


def test_singular_coarse_operator_falls_back_to_smoothing():
    """Without electrodes no boundary condition fixes the potential: a uniform
    shift of Phi leaves every flux unchanged, so A0 has the constant vector in
    its kernel (checked) and J is singular. The coarsest level then falls back
    from its inverse to Gauss-Seidel smoothing, and FGMRES still solves a
    consistent system J x = b (b = J x_true) to the tolerance."""
    import torch
    enp = _enp()
    P = W.config("cube_n9_p1")
    P = dataclasses.replace(P, tags=[np.where(t >= W.ELECTRODE0, W.WALL, t).astype(np.uint8)
                                   for t in P.tags])
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    b = orc.jvp(u, W.random_vector(P, 6))
    op = enp.Operator(P)
    op.set_preconditioner(1)
    ud = _cuda(u)
    op.block_jacobi_setup(ud, 0)
    a0 = op.coarse_operator().cpu().numpy().reshape(P.E, 7)
    assert np.abs(a0.sum(axis=1)).max() <= 1e-12 * np.abs(a0).max()
    x = torch.zeros(P.n_dof, dtype=torch.float64, device="cuda")
    st = op.fgmres_solve(ud, _cuda(b), x, restart=60, max_it=4000, rtol=1e-10)
    assert st["converged"] == 1
    assert np.linalg.norm(orc.jvp(u, x.cpu().numpy()) - b) <= 1.01e-10 * np.linalg.norm(b)


def test_two_level_fgmres_f32():
    enp = _enp()
    P = W.config("cube_n9_p1")
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    b = W.random_vector(P, 6)
    op = enp.Operator(P)
    x, st = _solve(op, u, b, True, f32=True, rtol=1e-5)
    assert st["converged"] == 1
    assert np.linalg.norm(orc.jvp(u, x) - b) <= 1e-4 * np.linalg.norm(b)


@pytest.mark.parametrize("mixed", [False, True])
def test_two_level_newton_matches_oracle_newton(mixed):
    enp = _enp()
    P = W.config("cube_n3_p2")
    orc = oracle.Oracle(P)
    u0 = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u0[k] = P.c_in[k - 1]
    u0 = u0.reshape(-1)
    ref, _ = orc.newton_solve(u0, rtol=1e-12, max_it=30)
    op = enp.Operator(P)
    op.set_preconditioner(1)
    ud = _cuda(u0)
    st = op.newton_solve(ud, max_it=30, rtol=1e-10, krylov_rtol=1e-3 if not mixed else 1e-2,
                         bj_storage=0 if not mixed else 1, mixed=mixed)
    assert st["converged"] == 1, st
    assert _rel(ud.cpu().numpy(), ref) < 1e-8


def test_two_level_argument_errors():
    enp = _enp()
    op = enp.Operator(W.config("cube_n2_p2"))
    with pytest.raises(enp.EnpError) as ei:
        op.set_preconditioner(2)
    assert ei.value.status == enp.ENP_ERR_INVALID_ARG
    with pytest.raises(enp.EnpError) as ei:
        op.coarse_operator()  # not set up
    assert ei.value.status == enp.ENP_ERR_INVALID_ARG
    op2 = enp.Operator(W.config("mms2d_n3"))
    with pytest.raises(enp.EnpError) as ei:
        op2.set_preconditioner(1)
    assert ei.value.status == enp.ENP_ERR_UNSUPPORTED


@pytest.mark.parametrize("two_level", [0, 1])
def test_lagged_preconditioner_newton(two_level):
    """A preconditioner rebuilt every third Newton iteration (pc_lag = 3) still
    gives the oracle's Newton solution; the setups counted are ceil(its / 3)
    when every inner solve converged."""
    enp = _enp()
    P = W.config("cube_n3_p2")
    orc = oracle.Oracle(P)
    u0 = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u0[k] = P.c_in[k - 1]
    u0 = u0.reshape(-1)
    ref, _ = orc.newton_solve(u0, rtol=1e-12, max_it=30)
    op = enp.Operator(P)
    op.set_preconditioner(two_level)
    ud = _cuda(u0)
    st = op.newton_solve(ud, max_it=30, rtol=1e-10, krylov_rtol=1e-3, krylov_max_it=2000,
                         pc_lag=3)
    assert st["converged"] == 1, st
    assert st["setups"] == -(-st["iterations"] // 3)
    assert st["setup_seconds"] > 0 and st["krylov_seconds"] > 0
    assert _rel(ud.cpu().numpy(), ref) < 1e-8


def test_two_level_graph_equals_eager_batched():
    """The coarse correction is captured with the rest of a restart cycle: the
    graph-replayed batched FGMRES gives bit for bit the eager iterate."""
    import torch
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 2
    phis = np.array([[1.0, 0, 0, 0], [3.0, 0, 0, 0]])
    u = _cuda(np.concatenate([W.random_state(P, 2), W.random_state(P, 3)]))
    b = _cuda(np.concatenate([W.random_vector(P, 6), 10 * W.random_vector(P, 7)]))
    op = enp.Operator(P, batch=B)
    op.set_phi_app(phis)
    op.set_preconditioner(1)
    op.block_jacobi_setup(u, 0)
    xs, its = [], []
    for graph in (False, True):
        x = torch.zeros(B * P.n_dof, dtype=torch.float64, device="cuda")
        st = op.fgmres_solve(u, b, x, restart=30, max_it=600, rtol=1e-10, graph=graph)
        assert st["converged"] == 1
        xs.append(x.cpu().numpy())
        its.append(st["iterations"])
    np.testing.assert_array_equal(xs[0], xs[1])
