"""The initial guess of Sec. 4.3 on the GPU (enp_initial_guess, through the C
ABI): constant concentrations at their inlet values and the potential from the
charge-conservation equation at those concentrations.

* Solved tightly (Newton to 1e-12, inner FGMRES to 1e-10), it equals the
  oracle's reading, Newton with direct solves on the potential block (itself
  pinned to the closed-form linear profile between Dirichlet faces), to 1e-9
  relative: on the plate reactor with Butler-Volmer electrodes (nonlinear in
  Phi), FP64 and mixed inner solves, one and two operating points, with and
  without the two-level preconditioner.
* The concentrations are exactly c^in afterwards.
* With the paper's loose inner tolerance (1e-2) Newton still reaches its
  outer tolerance.
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


@pytest.mark.parametrize("two_level,mixed", [(0, False), (1, False), (1, True)])
def test_initial_guess_matches_oracle_on_the_reactor(two_level, mixed):
    enp = _enp()
    P = W.config("reactor_n1_p2")
    phis = [0.2 * 38.92, 0.6 * 38.92]
    B = len(phis)
    op = enp.Operator(P, batch=B)
    op.set_phi_app(np.array([[ph, 0, 0, 0] for ph in phis]))
    op.set_preconditioner(two_level)
    n_phi = P.E * P.Np
    u0 = np.concatenate([W.random_state(P, 7 + b) for b in range(B)])  # concentrations overwritten
    for b, ph in enumerate(phis):
        u0[b * P.n_dof:b * P.n_dof + n_phi] = 0.5 * ph
    ud = _cuda(u0)
    st = op.initial_guess(ud, rtol=1e-12, krylov_rtol=1e-10, mixed=mixed,
                          bj_storage=enp.BJ_F32 if mixed else enp.BJ_F64)
    assert st["converged"] == 1, st
    got = ud.cpu().numpy().reshape(B, -1)
    for b, ph in enumerate(phis):
        Pb = dataclasses.replace(P, bv_phi_app=[ph, 0, 0, 0])
        orc = oracle.Oracle(Pb)
        ref, _ = oracle.potential_initial_guess(orc, Pb, np.full(n_phi, 0.5 * ph))
        for k in range(1, P.n_fields):
            assert np.all(got[b, k * n_phi:(k + 1) * n_phi] == P.c_in[k - 1])
        err = np.linalg.norm(got[b, :n_phi] - ref[:n_phi]) / np.linalg.norm(ref[:n_phi])
        assert err <= 1e-9, (b, err)


def test_initial_guess_with_the_papers_inner_tolerance():
    enp = _enp()
    P = W.config("reactor_n2_p2")
    ph = 0.45 * 38.92
    op = enp.Operator(P)
    op.set_phi_app(np.array([[ph, 0, 0, 0]]))
    op.set_preconditioner(1)
    u = W.reactor_initial_state(P, [ph])
    ud = _cuda(u)
    st = op.initial_guess(ud, rtol=1e-8, krylov_rtol=1e-2)
    assert st["converged"] == 1, st
    orc = oracle.Oracle(dataclasses.replace(P, bv_phi_app=[ph, 0, 0, 0]))
    n_phi = P.E * P.Np
    r = orc.residual(ud.cpu().numpy())
    r0 = orc.residual(u)
    assert np.linalg.norm(r[:n_phi]) <= 1e-8 * np.linalg.norm(r0[:n_phi])
