"""Pins for the oracle's initial guess of Sec. 4.3 (constant concentrations at
their inlet values, the potential from the charge-conservation equation at those
concentrations), independent of its own Newton iteration:

* closed form: with the potential prescribed on the faces x = 0 and x = 1
  (DIRICHLET) and natural conditions elsewhere, the charge equation at constant
  concentrations is Laplace's equation with constant conductivity, whose
  solution is linear in x; SIPG is consistent, so the discrete solution is the
  interpolant of that line (nodes evaluated here, not by the oracle), on a
  uniform and on a graded mesh;
* the concentrations are exactly c_k^in and the species residual rows are not
  what is solved: only the potential rows vanish;
* with Butler-Volmer electrodes (the plate reactor of Sec. 5.2) the equation is
  nonlinear in Phi: the result zeroes the potential rows of the residual to
  rounding and differs from the Phi = phi_app / 2 start.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W

GRADED = [np.array([0.0, 0.22, 0.61, 1.0]), np.array([0.0, 0.45, 0.7, 1.0]),
          np.array([0.0, 0.3, 0.52, 1.0])]


def _dirichlet_x_problem(graded):
    P = W.config("cube_n3_p2")
    tags = [np.full_like(t, W.WALL) for t in P.tags]
    tags[0][:] = W.DIRICHLET
    tags[1][:] = W.DIRICHLET
    P = dataclasses.replace(P, tags=tags)
    if graded:
        P = dataclasses.replace(P, coords=[c.copy() for c in GRADED])
    return P


@pytest.mark.parametrize("graded", [False, True])
def test_initial_potential_is_the_linear_profile_between_dirichlet_faces(graded):
    P = _dirichlet_x_problem(graded)
    phi_lo, phi_hi = 0.3, 1.7
    line = lambda x: phi_lo + (phi_hi - phi_lo) * x  # the exact solution (x in [0, 1])
    orc0 = oracle.Oracle(P)
    _, xb = orc0.quad_points()
    dirv = np.zeros((P.n_fields, P.n_bfaces, P.Nfq))
    dirv[0] = line(xb[..., 0])
    for k in range(1, P.n_fields):
        dirv[k] = P.c_in[k - 1]
    orc = oracle.Oracle(P, dirichlet=dirv.reshape(-1))
    u, hist = oracle.potential_initial_guess(orc, P, np.zeros(P.E * P.Np))
    xn = orc.node_points()  # nodal coordinates, [E, Np, 3]
    n_phi = P.E * P.Np
    np.testing.assert_allclose(u[:n_phi], line(xn[..., 0]).reshape(-1), rtol=0, atol=1e-11)
    for k in range(1, P.n_fields):
        assert np.all(u[k * n_phi:(k + 1) * n_phi] == P.c_in[k - 1])
    assert hist[-1] <= 1e-12 * hist[0]


def test_initial_potential_with_butler_volmer_zeroes_the_charge_rows():
    P = W.config("reactor_n1_p2")
    phi_app = 0.3 * 38.92
    P = dataclasses.replace(P, bv_phi_app=[phi_app, 0.0, 0.0, 0.0])
    orc = oracle.Oracle(P)
    n_phi = P.E * P.Np
    start = np.full(n_phi, 0.5 * phi_app)
    u, hist = oracle.potential_initial_guess(orc, P, start)
    r = orc.residual(u)
    assert np.linalg.norm(r[:n_phi]) <= 1e-11 * hist[0]
    assert len(hist) > 2                      # nonlinear: several Newton steps
    assert np.linalg.norm(u[:n_phi] - start) > 1e-3 * np.linalg.norm(start)
    # the species rows are not solved for: at c = c_in they do not vanish
    assert np.linalg.norm(r[n_phi:]) > 1e-8
