"""Unit pins for the oracle's minmod limiter and HLLC flux (CPU only).

Each check is a property of the exact mathematics, not a re-typing of the
oracle's formulas: consistency with the physical flux (Eq. "fluxes"), exact
resolution of stationary and moving contacts (the property that separates
HLLC from HLL), upwinding in the supersonic regimes, mirror symmetry and the
passive transport of the tangential components.  The contact speed and the
star-state energy are pinned through the whole scheme's convergence to exact
Riemann solutions (test_oracle_scheme.py).
"""
import math

import numpy as np
import pytest


def phys_flux(W, gamma):
    """Eq. "fluxes" (x-normal) written out from the primitives."""
    r, u, v, w, p = W
    E = p / (gamma - 1) + 0.5 * r * (u * u + v * v + w * w)
    return np.array([r * u, r * u * u + p, r * u * v, r * u * w, (E + p) * u])


def cons(W, gamma):
    r, u, v, w, p = W
    return np.array([r, r * u, r * v, r * w, p / (gamma - 1) + 0.5 * r * (u * u + v * v + w * w)])


@pytest.mark.parametrize("a,b,expect", [
    (1.0, 2.0, 1.0), (2.0, 1.0, 1.0), (-1.0, -2.0, -1.0), (-2.0, -1.0, -1.0),
    (1.0, -1.0, 0.0), (-1.0, 1.0, 0.0), (0.0, 1.0, 0.0), (1.0, 0.0, 0.0),
    (0.0, 0.0, 0.0), (3.0, 3.0, 3.0), (-3.0, -3.0, -3.0),
    (1e-200, 1e-200, 1e-200),            # sign test: no underflow of a*b
    (-1e-300, -2e-300, -1e-300),
])
def test_minmod_cases(orc, a, b, expect):
    assert orc.minmod(a, b) == expect


def _rng_state(g, gamma=1.4):
    r, p = np.exp(g.uniform(math.log(0.1), math.log(10), size=2))
    u, v, w = g.uniform(-1, 1, size=3)
    return np.array([r, u, v, w, p])


@pytest.mark.parametrize("seed", range(8))
def test_consistency_equal_states(orc, seed):
    g = np.random.default_rng(seed)
    W = _rng_state(g)
    np.testing.assert_allclose(orc.hllc(W, W, 1.4), phys_flux(W, 1.4), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("rhoL,rhoR", [(1.0, 0.125), (0.2, 5.0), (3.0, 3.0)])
def test_stationary_contact(orc, rhoL, rhoR):
    p = 0.7
    F = orc.hllc([rhoL, 0, 0.3, -0.2, p], [rhoR, 0, -0.1, 0.4, p], 1.4)
    np.testing.assert_allclose(F, [0, p, 0, 0, 0], atol=1e-14)


@pytest.mark.parametrize("u", [0.4, -0.4])
def test_moving_contact_resolved_exactly(orc, u):
    """Isolated contact (equal u and p): the exact flux is the upwind physical
    flux.  HLL smears it; HLLC must not."""
    gam = 1.4
    WL = np.array([1.0, u, 0.2, -0.3, 1.5])
    WR = np.array([0.25, u, -0.5, 0.1, 1.5])
    F = orc.hllc(WL, WR, gam)
    up = WL if u > 0 else WR
    np.testing.assert_allclose(F, phys_flux(up, gam), rtol=1e-13, atol=1e-14)


def test_supersonic_upwinding(orc):
    gam = 1.4
    WL = np.array([1.0, 3.0, 0.1, 0.2, 1.0])   # c ~ 1.18 < 3 : all waves right-going
    WR = np.array([0.5, 2.8, -0.1, 0.0, 0.8])
    np.testing.assert_allclose(orc.hllc(WL, WR, gam), phys_flux(WL, gam), rtol=1e-14)
    WL2 = np.array([1.0, -3.0, 0.1, 0.2, 1.0])
    WR2 = np.array([0.5, -2.8, -0.1, 0.0, 0.8])
    np.testing.assert_allclose(orc.hllc(WL2, WR2, gam), phys_flux(WR2, gam), rtol=1e-14)


@pytest.mark.parametrize("seed", range(8))
def test_mirror_symmetry(orc, seed):
    """Reflecting x -> -x swaps the states and flips the normal velocity; the
    normal momentum flux keeps its sign, every other flux component flips."""
    g = np.random.default_rng(100 + seed)
    WL, WR = _rng_state(g), _rng_state(g)
    flipu = np.array([1, -1, 1, 1, 1])
    F = orc.hllc(WL, WR, 1.4)
    Fm = orc.hllc(WR * flipu, WL * flipu, 1.4)
    np.testing.assert_allclose(Fm, F * np.array([-1, 1, -1, -1, -1]), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed", range(8))
def test_tangential_components_are_passive(orc, seed):
    """Swapping the two tangential velocities swaps the two tangential momentum
    fluxes and leaves the rest unchanged."""
    g = np.random.default_rng(200 + seed)
    WL, WR = _rng_state(g), _rng_state(g)
    sw = [0, 1, 3, 2, 4]
    F = orc.hllc(WL, WR, 1.4)
    Fs = orc.hllc(WL[sw], WR[sw], 1.4)
    np.testing.assert_allclose(Fs, F[sw], rtol=1e-14, atol=1e-15)
