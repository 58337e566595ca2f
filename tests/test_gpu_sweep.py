"""The downwind block Gauss-Seidel sweep (through the C ABI).

* One application equals the solve of (D + L) z = r, with D and L taken from the
  oracle's assembled Jacobian: D the element-diagonal blocks, L every element's
  coupling to its upstream neighbour along the flow axis (x, the plate-flow
  axis of these workloads). FP64 storage, 1e-10 relative.
* FGMRES preconditioned by the sweep (and the two-level correction) reaches the
  tolerance on the true (oracle) residual in fewer iterations than with
  block-Jacobi (FP64), batched and graph-captured (a cycle captured before the
  sweep was switched on is not replayed after it).
* Newton with it reaches the oracle's Newton solution, FP64 and mixed.
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


def _lower_block_system(orc, P, u, axis=0, direction=1):
    """D + L from the assembled Jacobian: keep the entries whose column element
    is the row element or its upstream neighbour along `axis` for flow in
    `direction` (+1: the neighbour at the lower index, -1: at the higher)."""
    import scipy.sparse as sp
    J = orc.jacobian(u).tocoo()
    er = (J.row // P.Np) % P.E
    ec = (J.col // P.Np) % P.E
    stride = [1, P.n_el[0], P.n_el[0] * P.n_el[1]][axis]
    ia = (er // stride) % P.n_el[axis]
    has_up = ia > 0 if direction > 0 else ia < P.n_el[axis] - 1
    keep = (ec == er) | ((ec == er - direction * stride) & has_up)
    return sp.csr_matrix((J.data[keep], (J.row[keep], J.col[keep])), shape=J.shape)


GRADED = [np.array([0.0, 0.22, 0.61, 1.0]), np.array([0.0, 0.45, 0.7, 1.0]),
          np.array([0.0, 0.3, 0.52, 1.0])]


def _prob(cfg):
    if cfg == "cube_graded":
        return dataclasses.replace(W.config("cube_n3_p2"), coords=[c.copy() for c in GRADED])
    return W.config(cfg)


@pytest.mark.parametrize("cfg", ["reactor_n1_p2", "cube_n3_p2", "cube_graded", "channel_n1"])
def test_sweep_solves_the_lower_block_system(cfg):
    import scipy.sparse.linalg as spla
    enp = _enp()
    P = _prob(cfg)
    assert P.vel_params[0] == 0  # flow along x
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    r = W.random_vector(P, 5)
    op = enp.Operator(P)
    op.set_sweep(1)
    op.block_jacobi_setup(_cuda(u), enp.BJ_F64)
    z = op.block_jacobi_apply(_cuda(r)).cpu().numpy()
    ref = spla.spsolve(_lower_block_system(orc, P, u).tocsc(), r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


# constant velocities whose largest component points along -x, +y and -z, and
# plate flow with a negative mean speed (flow towards -x): the sweep's axis,
# direction and upstream face follow the flow
FLOWS = {"-x": (0, -1, [-1.0, 0.3, 0.2]), "+y": (1, 1, [0.2, 1.0, 0.1]),
         "-z": (2, -1, [0.1, 0.2, -1.0])}


@pytest.mark.parametrize("flow", ["-x", "+y", "-z", "plate-x"])
def test_sweep_follows_the_flow_direction(flow):
    import scipy.sparse.linalg as spla
    enp = _enp()
    P = W.config("cube_n3_p2")
    if flow == "plate-x":
        vp = list(P.vel_params)
        vp[4] = -vp[4]
        P = dataclasses.replace(P, vel_params=vp)
        axis, direction = 0, -1
    else:
        axis, direction, vel = FLOWS[flow]
        P = dataclasses.replace(P, vel_kind=W.VEL_CONSTANT, vel_params=vel + [0.0] * 5)
    orc = oracle.Oracle(P)
    u = W.random_state(P, 2)
    r = W.random_vector(P, 5)
    op = enp.Operator(P)
    op.set_sweep(1)
    op.block_jacobi_setup(_cuda(u), enp.BJ_F64)
    z = op.block_jacobi_apply(_cuda(r)).cpu().numpy()
    ref = spla.spsolve(_lower_block_system(orc, P, u, axis, direction).tocsc(), r)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("storage,tol", [(1, 1e-5), (2, 5e-2)])
@pytest.mark.parametrize("shared", [-1, 0])
def test_sweep_batched_storage_and_shared_blocks(storage, tol, shared):
    """Two operating points with different states in one batch, FP32 or BF16
    inverses, per point or one shared set (the inverses of point 0), FP64 and
    FP32 vectors: point b's sweep solves (D_s + L_b) z = r_b, with D_s the
    diagonal blocks of the point s whose inverses are stored and L_b point b's
    own upstream couplings."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 2
    phis = np.array([[4.0, 0, 0, 0], [20.0, 0, 0, 0]])
    us = [W.random_state(P, 2), W.random_state(P, 3)]
    rs = [W.random_vector(P, 5), W.random_vector(P, 6)]
    op = enp.Operator(P, batch=B)
    op.set_phi_app(phis)
    op.set_shared_blocks(shared)
    op.set_sweep(1)
    op.block_jacobi_setup(_cuda(np.concatenate(us)), storage)
    rd = _cuda(np.concatenate(rs))
    z = op.block_jacobi_apply(rd).cpu().numpy().reshape(B, -1)
    # FP32 vectors (the mixed inner solve's): the same system
    z32 = op.block_jacobi_apply_f32(rd.float()).double().cpu().numpy().reshape(B, -1)
    orcs = [oracle.Oracle(dataclasses.replace(P, bv_phi_app=list(phis[b]))) for b in range(B)]
    n = P.n_dof
    for b in range(B):
        s = b if shared < 0 else shared
        Ms = _lower_block_system(orcs[s], P, us[s]).tocoo()
        Mb = _lower_block_system(orcs[b], P, us[b]).tocoo()
        same = lambda M: (M.row // P.Np) % P.E == (M.col // P.Np) % P.E
        ds, db = same(Ms), same(Mb)
        M = sp.csr_matrix((np.concatenate([Ms.data[ds], Mb.data[~db]]),
                           (np.concatenate([Ms.row[ds], Mb.row[~db]]),
                            np.concatenate([Ms.col[ds], Mb.col[~db]]))), shape=(n, n))
        ref = spla.spsolve(M.tocsc(), rs[b])
        kappa = float(np.max(np.linalg.cond(orcs[s].block_diagonal(us[s]))))
        bound = tol * kappa if storage == 1 else tol
        assert np.linalg.norm(z[b] - ref) <= bound * np.linalg.norm(ref), (b, kappa)
        assert np.linalg.norm(z32[b] - ref) <= bound * np.linalg.norm(ref), (b, kappa)


def _fgmres(op, enp, u, b, sweep, f32=False, rtol=1e-10, graph=False):
    import torch
    op.set_sweep(1 if sweep else 0)
    op.set_preconditioner(1)
    op.block_jacobi_setup(u, enp.BJ_F32 if f32 else enp.BJ_F64)
    dt = torch.float32 if f32 else torch.float64
    x = torch.zeros(b.numel(), dtype=dt, device="cuda")
    st = op.fgmres_solve(u.to(dt), b.to(dt), x, restart=50, max_it=4000, rtol=rtol, graph=graph,
                         raise_on_fail=False)
    return x.double().cpu().numpy(), st


def test_sweep_fgmres_converges_in_fewer_iterations():
    enp = _enp()
    P = W.config("reactor_n2_p2")
    orc = oracle.Oracle(P)
    u = W.reactor_initial_state(P, [38.92 * 0.45])
    b = W.random_vector(P, 6)
    op = enp.Operator(P)
    op.set_phi_app(np.array([[38.92 * 0.45, 0, 0, 0]]))
    ud, bd = _cuda(u), _cuda(b)
    x1, st1 = _fgmres(op, enp, ud, bd, sweep=False)
    x2, st2 = _fgmres(op, enp, ud, bd, sweep=True)
    assert st1["converged"] == 1 and st2["converged"] == 1, (st1, st2)
    Pi = dataclasses.replace(P, bv_phi_app=[38.92 * 0.45, 0, 0, 0])
    orc = oracle.Oracle(Pi)
    for x in (x1, x2):
        assert np.linalg.norm(orc.jvp(u, x) - b) <= 1.01e-10 * np.linalg.norm(b)
    assert st2["iterations"] < st1["iterations"], (st1["iterations"], st2["iterations"])


def test_sweep_graph_equals_eager_batched():
    enp = _enp()
    P = W.config("reactor_n1_p2")
    B = 2
    phis = np.array([[4.0, 0, 0, 0], [20.0, 0, 0, 0]])
    u = _cuda(W.reactor_initial_state(P, phis[:, 0]))
    b = _cuda(np.concatenate([W.random_vector(P, 6), 10 * W.random_vector(P, 7)]))
    op = enp.Operator(P, batch=B)
    op.set_phi_app(phis)
    # a cycle captured without the sweep must not be replayed once it is on
    _, st0 = _fgmres(op, enp, u, b, sweep=False, graph=True)
    assert st0["converged"] == 1
    xs = []
    for graph in (False, True):
        x, st = _fgmres(op, enp, u, b, sweep=True, graph=graph)
        assert st["converged"] == 1
        xs.append(x)
    np.testing.assert_array_equal(xs[0], xs[1])
    # each point as it is alone
    for i in range(B):
        op1 = enp.Operator(dataclasses.replace(P, bv_phi_app=list(phis[i])))
        n = P.n_dof
        x1, _ = _fgmres(op1, enp, u[i * n:(i + 1) * n], b[i * n:(i + 1) * n], sweep=True)
        np.testing.assert_array_equal(xs[0][i * n:(i + 1) * n], x1)


@pytest.mark.parametrize("mixed", [False, True])
def test_sweep_newton_matches_oracle_newton(mixed):
    enp = _enp()
    P = W.config("cube_n3_p2")
    orc = oracle.Oracle(P)
    u0 = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u0[k] = P.c_in[k - 1]
    u0 = u0.reshape(-1)
    ref, _ = orc.newton_solve(u0, rtol=1e-12, max_it=30)
    op = enp.Operator(P)
    op.set_sweep(1)
    op.set_preconditioner(1)
    ud = _cuda(u0)
    st = op.newton_solve(ud, max_it=30, rtol=1e-10, krylov_rtol=1e-3 if not mixed else 1e-2,
                         bj_storage=0 if not mixed else 1, mixed=mixed)
    assert st["converged"] == 1, st
    assert np.linalg.norm(ud.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_sweep_argument_errors():
    enp = _enp()
    op = enp.Operator(W.config("cube_n2_p2"))
    for bad in (-1, 3):
        with pytest.raises(enp.EnpError) as ei:
            op.set_sweep(bad)
        assert ei.value.status == enp.ENP_ERR_INVALID_ARG
    op2 = enp.Operator(W.config("mms2d_n3"))
    with pytest.raises(enp.EnpError) as ei:
        op2.set_sweep(1)
    assert ei.value.status == enp.ENP_ERR_UNSUPPORTED
    op2.set_sweep(2)  # automatic: block-Jacobi on a 2D mesh


def _channel_line(n_along):
    """A plate-flow channel of n_along x 2 x 1 elements at p = 1."""
    n_el = [n_along, 2, 1]
    coords = W._linspace_coords(n_el, [n_along / 16.0, 1.0, 1.0])
    P = W.config("cube_n2_p2", p=1)
    return dataclasses.replace(P, n_el=n_el, coords=coords,
                               tags=W._reactor_tags(3, n_el, coords, 1.0 / 3.0, 2.0 / 3.0),
                               name="line")


@pytest.mark.parametrize("n_along,same_as", [(96, 0), (128, 1)])
def test_sweep_automatic_mode(n_along, same_as):
    """The default (2) picks block-Jacobi below 128 elements along the flow and
    the sweep from 128 on: its application equals that mode's bit for bit."""
    enp = _enp()
    P = _channel_line(n_along)
    u = _cuda(W.random_state(P, 2))
    r = _cuda(W.random_vector(P, 5))
    zs = {}
    for mode in (2, same_as, 1 - same_as):
        op = enp.Operator(P)
        if mode != 2:
            op.set_sweep(mode)
        op.block_jacobi_setup(u, enp.BJ_F64)
        zs[mode] = op.block_jacobi_apply(r).cpu().numpy()
    np.testing.assert_array_equal(zs[2], zs[same_as])
    assert np.linalg.norm(zs[2] - zs[1 - same_as]) > 0
