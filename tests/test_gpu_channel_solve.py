"""The three-species channel (the shape of the 64 x 32 x 16 channel workload,
z = (+1, -1, +2), Pe = 1e4, Butler-Volmer electrodes), reduced to 4 x 2 x 1
elements at p = 3: Newton to 1e-10 on the GPU against the oracle's Newton with
direct solves, in FP64 (native and double-float arithmetic for the residual and
J v) and mixed precision (FP32 inner operator and Krylov vectors, FP32 and
BF16-stored block inverses), with the two-level preconditioner, from c = c_in
and Phi = 0 and from the initial guess of Sec. 4.3."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

_REF = {}


def _enp():
    import paper_2112_09271_gb300 as enp
    enp.build()
    return enp


def _start(P):
    u = np.zeros((P.n_fields, P.E, P.Np))
    for k in range(1, P.n_fields):
        u[k] = P.c_in[k - 1]
    return u.reshape(-1)


def _reference(P):
    if "ref" not in _REF:
        orc = oracle.Oracle(P)
        _REF["ref"], _ = orc.newton_solve(_start(P), rtol=1e-12, max_it=40)
        _REF["orc"] = orc
    return _REF["ref"], _REF["orc"]


@pytest.mark.parametrize("variant", ["f64", "df32", "mixed_f32", "mixed_bf16", "mixed_guess"])
def test_channel_newton_matches_oracle_newton(variant):
    import torch
    enp = _enp()
    P = W.config("channel_n1")
    assert P.m == 3
    ref, orc = _reference(P)
    op = enp.Operator(P)
    op.set_preconditioner(1)
    if variant == "df32":
        op.set_arithmetic(enp.ARITH_DF32)
    mixed = variant.startswith("mixed")
    storage = {"mixed_bf16": enp.BJ_BF16}.get(variant, enp.BJ_F32 if mixed else enp.BJ_F64)
    u0 = _start(P)
    ud = torch.tensor(u0, device="cuda")
    if variant == "mixed_guess":
        gs = op.initial_guess(ud, krylov_rtol=1e-2, mixed=True, bj_storage=storage)
        assert gs["converged"] == 1, gs
    st = op.newton_solve(ud, max_it=40, rtol=1e-10, krylov_restart=50, krylov_max_it=4000,
                         krylov_rtol=1e-3, bj_storage=storage, mixed=mixed)
    assert st["converged"] == 1, st
    u = ud.cpu().numpy()
    assert np.linalg.norm(orc.residual(u)) <= 2e-10 * np.linalg.norm(orc.residual(u0))
    err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err < 1e-8, err
