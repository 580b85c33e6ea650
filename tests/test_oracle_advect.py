"""Pins of the oracle's radiation energy advection (the d_j(E v^j) term of
Eq. "radiation"; WENO5-Z states and the Rusanov flux of Sec. 2.2.2)."""
import math

import numpy as np
import pytest

import hydro_inputs as H
import oracle
from oracle import metrics


def _fluid(shape, vel, gamma=1.4, rho=1.0, p=1.0):
    W = np.zeros((5,) + shape)
    W[0], W[4] = rho, p
    for a in range(3):
        W[1 + a] = vel[a]
    return H.prim_to_cons(W, gamma)


def test_free_stream():
    shape = (5, 6, 7)
    U = _fluid(shape, (0.3, -0.2, 0.5))
    E = np.full(shape, 2.5)
    g = oracle.Grid(shape, 1.4, oracle.BC_PERIODIC)
    assert np.max(np.abs(g.rhs_E(U, E))) < 1e-12


def test_rusanov_flux_properties():
    """Consistency F(E, E, u, u) = E u; monotone (non-decreasing in E_L,
    non-increasing in E_R) for any face velocities, which needs the
    dissipation speed max(|u_L|, |u_R|)."""
    assert oracle.rusanov_E(2.0, 2.0, -0.3, -0.3) == pytest.approx(-0.6, rel=1e-15)
    rng = np.random.default_rng(4)
    for _ in range(200):
        EL, ER = rng.random(2) + 0.1
        uL, uR = rng.uniform(-2, 2, 2)
        F0 = oracle.rusanov_E(EL, ER, uL, uR)
        assert oracle.rusanov_E(EL + 1e-3, ER, uL, uR) >= F0 - 1e-15
        assert oracle.rusanov_E(EL, ER + 1e-3, uL, uR) <= F0 + 1e-15


@pytest.mark.parametrize("axis,u", [(0, 1.0), (0, -0.7), (1, 0.8), (2, -1.1)])
def test_fifth_order_flux_difference(axis, u):
    """Uniform velocity along one axis: the Rusanov flux with a = |u| is the
    upwind flux of the WENO5-Z state, so L_E converges at fifth order to the
    exact -u (E(x_{i+1/2}) - E(x_{i-1/2})) / h of GL-10 cell averages
    (observed 5.0)."""
    errs = []
    for n in (32, 64, 128):
        edges = np.linspace(0.0, 1.0, n + 1)
        E = metrics.gl10_cell_average_1d(lambda x: 1.0 + 0.3 * np.sin(2 * np.pi * x), edges)
        shape = [1, 1, 1]
        shape[2 - axis] = n
        vel = [0.0, 0.0, 0.0]
        vel[axis] = u
        U = _fluid(tuple(shape), vel)
        L = oracle.Grid(tuple(shape), 1.4, 0).rhs_E(U, E.reshape(shape)).ravel()
        Ef = 1.0 + 0.3 * np.sin(2 * np.pi * edges)
        errs.append(np.mean(np.abs(L + u * (Ef[1:] - Ef[:-1]) * n)))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) >= 4.8, orders


def test_conservation_in_a_periodic_box():
    shape = (6, 7, 8)
    rng = np.random.default_rng(3)
    W = np.stack([1 + 0.3 * rng.random(shape), 0.5 * rng.standard_normal(shape),
                  0.5 * rng.standard_normal(shape), 0.5 * rng.standard_normal(shape),
                  1 + 0.3 * rng.random(shape)])
    U = H.prim_to_cons(W, 1.4)
    E = 1.0 + rng.random(shape)
    g = oracle.Grid(shape, 1.4, oracle.BC_PERIODIC)
    E1 = g.advect_E(U, E, 0.01)
    assert np.sum(E1) == pytest.approx(np.sum(E), rel=1e-14)


def test_mirror_symmetry_between_reflecting_walls():
    """E even and u odd about the box centre stay so (E is a scalar: no flip
    at the wall; the normal velocity is)."""
    n = 40
    x = H.centres(n)
    U = _fluid((1, 1, n), (0.4 * np.sin(2 * np.pi * x), 0.0, 0.0))
    E = 1.0 + np.exp(-50 * (x - 0.5) ** 2) + 0.2 * np.cos(4 * np.pi * x)
    g = oracle.Grid((1, 1, n), 1.4, oracle.BC_REFLECT)
    E1 = g.advect_E(U, E.reshape(1, 1, n), 0.02)[0, 0]
    assert np.allclose(E1, E1[::-1], rtol=1e-13)
    assert not np.allclose(E1, E)


def test_translation_of_a_profile():
    """One period of translation at u = 1 on a periodic line returns the
    profile (within the scheme's error, 2e-3 at 128 cells and CFL 0.4)."""
    n = 128
    x = H.centres(n)
    E0 = 1.0 + 0.3 * np.sin(2 * np.pi * x)
    U = _fluid((1, 1, n), (1.0, 0.0, 0.0))
    g = oracle.Grid((1, 1, n), 1.4, 0)
    E = E0.reshape(1, 1, n).copy()
    steps = 320
    for _ in range(steps):
        E = g.advect_E(U, E, 1.0 / steps)
    assert np.max(np.abs(E[0, 0] - E0)) < 2e-3
