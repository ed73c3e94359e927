"""Pins of the oracle's semilinear reaction term and time-step residual.

Expected values: the domain measure and the pinned mass matrix (constant
and linear reactions, which the rules integrate exactly), second-order
convergence of the quadrature to the exact integral of a cubic reaction of
a smooth field, and central differences for the Jacobian action.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import meshgen as mg
import oracle as O
from test_oracle_pins import _jittered

ELS = [O.P1_TRI, O.P2_TRI, O.P1_TET]
R_AC = [0.0, -0.3, 0.0, 0.3]  # eps^2 (u^3 - u), eps^2 = 0.3: the Allen-Cahn reaction


def _mass(el, m):
    return O.assemble_bilinear(el, m.cells, m.coords, np.zeros(1), O.CONSTANT, 1.0).to_scipy()


@pytest.mark.parametrize("el", ELS)
def test_constant_state_integrates_the_reaction_value(el):
    m = _jittered(el)
    u0 = 0.6
    r = [0.2, -1.1, 0.5, 0.9]
    N = O.reaction_load(el, m.cells, m.coords, np.full(m.n_nodes, u0), r)
    ru = r[0] + r[1] * u0 + r[2] * u0 ** 2 + r[3] * u0 ** 3
    assert N.sum() == pytest.approx(ru * 1.0, rel=1e-13)  # |domain| = 1
    assert np.allclose(N, ru * (_mass(el, m) @ np.ones(m.n_nodes)), rtol=0, atol=1e-14)


@pytest.mark.parametrize("el", ELS)
def test_linear_reaction_is_the_mass_matrix(el):
    m = _jittered(el)
    x = np.random.default_rng(3).uniform(-1, 1, m.n_nodes)
    N = O.reaction_load(el, m.cells, m.coords, x, [0.0, 2.5, 0.0, 0.0])
    assert np.allclose(N, 2.5 * (_mass(el, m) @ x), rtol=0, atol=1e-14)


def test_cubic_reaction_converges_to_the_exact_integral():
    # u = sin(pi x) sin(pi y) on the unit square; int (u^3 - u) = 16/(9 pi^2) - 4/pi^2
    exact = 16.0 / (9.0 * math.pi ** 2) - 4.0 / math.pi ** 2
    errs = []
    for n in (16, 32, 64):
        m = mg.jitter(mg.tri_grid(n), 3)
        u = np.sin(math.pi * m.coords[:, 0]) * np.sin(math.pi * m.coords[:, 1])
        N = O.reaction_load(O.P1_TRI, m.cells, m.coords, u, [0.0, -1.0, 0.0, 1.0])
        errs.append(abs(N.sum() - exact))
    rates = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(rates) > 1.8, (errs, rates)


@pytest.mark.parametrize("el", ELS)
def test_jacobian_action_matches_central_differences(el):
    m = _jittered(el)
    g = np.random.default_rng(5)
    xr = g.uniform(-1, 1, m.n_nodes)
    v = g.uniform(-1, 1, m.n_nodes)
    r = [0.1, -0.7, 0.4, 1.3]
    J = O.reaction_load(el, m.cells, m.coords, v, r, x_react=xr)
    eps = 1e-5
    fd = (O.reaction_load(el, m.cells, m.coords, xr + eps * v, r)
          - O.reaction_load(el, m.cells, m.coords, xr - eps * v, r)) / (2 * eps)
    # the cubic's third derivative leaves eps^2 r3 |v|^3 per point, about 1e-12 here
    assert np.allclose(J, fd, rtol=0, atol=1e-8 * np.abs(J).max())


def test_allen_cahn_backward_euler_step():
    # (1/dt) M (U1 - U0) + a^2 K U1 + N(U1) through one call: kappa = a^2, c = 1/dt, f = U0 / dt
    m = _jittered(O.P1_TRI, n=8)
    g = np.random.default_rng(7)
    U0, U1 = g.uniform(-1, 1, m.n_nodes), g.uniform(-1, 1, m.n_nodes)
    a2, dt = 0.02, 1e-3
    y, _ = O.semilinear_residual(O.P1_TRI, m.cells, m.coords, np.array([a2]), O.CONSTANT, 1.0 / dt, U1, R_AC,
                                 U0 / dt, O.PER_NODE)
    M = _mass(O.P1_TRI, m)
    K = O.assemble_bilinear(O.P1_TRI, m.cells, m.coords, np.array([1.0]), O.CONSTANT, 0.0).to_scipy()
    # the reaction load of eps^2 (u^3 - u): with U1 = constant 1 it vanishes, so check the linear part there
    ones = np.ones(m.n_nodes)
    y1, _ = O.semilinear_residual(O.P1_TRI, m.cells, m.coords, np.array([a2]), O.CONSTANT, 1.0 / dt, ones, R_AC,
                                  U0 / dt, O.PER_NODE)
    assert np.allclose(y1, (M @ (ones - U0)) / dt, rtol=0, atol=1e-10)
    N = O.reaction_load(O.P1_TRI, m.cells, m.coords, U1, R_AC)
    assert np.allclose(y, (M @ (U1 - U0)) / dt + a2 * (K @ U1) + N, rtol=0, atol=1e-9)
