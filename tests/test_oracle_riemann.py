"""Pins for the oracle's exact Riemann solver and the L1 metric (CPU only).

The exact solver is pinned by properties it must satisfy that do not reuse
its own formulas: Toro's tabulated Sod star state, the Rankine-Hugoniot jump
conditions across every shock it produces, isentropy and the Riemann
invariant across every rarefaction, and continuity of p and u at the contact.
The Gauss-Legendre rule is pinned by exact polynomial integration.
"""
import math

import numpy as np
import pytest

import hydro_inputs as H
from conftest import read_golden

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_sod_star_matches_textbook(orc):
    g = read_golden("toro_sod_star.txt")
    pb = H.sod()
    ps, us = orc.riemann_star(pb.WL, pb.WR, g["gamma"])
    assert ps == pytest.approx(g["p_star"], abs=6e-6)
    assert us == pytest.approx(g["u_star"], abs=6e-6)
    W = orc.riemann_sample(pb.WL, pb.WR, g["gamma"], [us - 1e-9, us + 1e-9])
    assert W[0, 0] == pytest.approx(g["rho_star_left"], abs=6e-6)
    assert W[1, 0] == pytest.approx(g["rho_star_right"], abs=6e-6)


def _rh_residuals(W1, W2, gamma):
    """Shock speed from the mass jump, then the relative mismatch of the
    momentum and energy jumps (Rankine-Hugoniot)."""
    r1, u1, p1 = W1
    r2, u2, p2 = W2
    S = (r2 * u2 - r1 * u1) / (r2 - r1)
    E1 = p1 / (gamma - 1) + 0.5 * r1 * u1 * u1
    E2 = p2 / (gamma - 1) + 0.5 * r2 * u2 * u2
    mom = (r2 * u2 * u2 + p2 - r1 * u1 * u1 - p1) - S * (r2 * u2 - r1 * u1)
    ene = ((E2 + p2) * u2 - (E1 + p1) * u1) - S * (E2 - E1)
    scale = max(abs(p1), abs(p2), abs(E1), abs(E2))
    return S, abs(mom) / scale, abs(ene) / scale


@pytest.mark.parametrize("seed", range(16))
def test_exact_solution_jump_conditions(orc, seed):
    pb = H.riemann_1d(seed)
    gam = pb.gamma
    ps, us = orc.riemann_star(pb.WL, pb.WR, gam)
    eps = 1e-10
    # sides: (far state, star state on that side, sign)
    far_l = orc.riemann_sample(pb.WL, pb.WR, gam, [-1e6])[0]
    far_r = orc.riemann_sample(pb.WL, pb.WR, gam, [1e6])[0]
    np.testing.assert_allclose(far_l, pb.WL, rtol=0, atol=0)
    np.testing.assert_allclose(far_r, pb.WR, rtol=0, atol=0)
    star_l = orc.riemann_sample(pb.WL, pb.WR, gam, [us - eps])[0]
    star_r = orc.riemann_sample(pb.WL, pb.WR, gam, [us + eps])[0]
    # contact: pressure and velocity continuous, both equal to the star values
    assert star_l[2] == pytest.approx(ps, rel=1e-12)
    assert star_r[2] == pytest.approx(ps, rel=1e-12)
    assert star_l[1] == pytest.approx(us, rel=1e-12, abs=1e-12)
    assert star_r[1] == pytest.approx(us, rel=1e-12, abs=1e-12)
    for far, star, side in ((pb.WL, star_l, -1), (pb.WR, star_r, +1)):
        if star[2] > far[2] * (1 + 1e-12):                   # shock
            S, rm, re = _rh_residuals(far, star, gam)
            assert rm < 1e-12 and re < 1e-12
            # the solution jumps exactly at the shock speed
            Wa = orc.riemann_sample(pb.WL, pb.WR, gam, [S - 1e-7, S + 1e-7])
            outer, inner = (Wa[0], Wa[1]) if side < 0 else (Wa[1], Wa[0])
            np.testing.assert_allclose(outer, far, rtol=1e-12)
            np.testing.assert_allclose(inner, star, rtol=1e-9)
        else:                                                # rarefaction
            c_far = math.sqrt(gam * far[2] / far[0])
            head = far[1] + side * c_far
            # isentropic: p / rho^gamma constant across the fan and in the star state
            s_far = far[2] / far[0] ** gam
            c_star = math.sqrt(gam * star[2] / star[0])
            tail = star[1] + side * c_star
            xs = np.linspace(min(head, tail), max(head, tail), 9)[1:-1]
            Wf = orc.riemann_sample(pb.WL, pb.WR, gam, xs)
            for W in np.vstack([Wf, star[None]]):
                assert W[2] / W[0] ** gam == pytest.approx(s_far, rel=1e-11)
                # generalised Riemann invariant u -/+ 2c/(gamma-1) carried from the far side
                c = math.sqrt(gam * W[2] / W[0])
                J = W[1] - side * 2 * c / (gam - 1)
                assert J == pytest.approx(far[1] - side * 2 * c_far / (gam - 1), rel=1e-11, abs=1e-11)
            # inside the fan the flow is sonic along the characteristic: u -/+ c = xi
            for xi, W in zip(xs, Wf):
                c = math.sqrt(gam * W[2] / W[0])
                assert W[1] + side * c == pytest.approx(xi, rel=1e-11, abs=1e-11)


def test_vacuum_data_rejected(orc):
    with pytest.raises(ValueError):
        orc.riemann_star((1.0, -10.0, 0.1), (1.0, 10.0, 0.1), 1.4)


def test_gl10_integrates_degree_19_exactly():
    from oracle.metrics import gl10_cell_average_1d
    edges = np.array([0.0, 0.3, 1.0, 2.5])
    f = lambda x: x ** 19 - 3 * x ** 7 + 2
    avg = gl10_cell_average_1d(f, edges)
    a, b = edges[:-1], edges[1:]
    F = lambda x: x ** 20 / 20 - 3 * x ** 8 / 8 + 2 * x
    np.testing.assert_allclose(avg, (F(b) - F(a)) / (b - a), rtol=1e-13)


def test_gl10_3d_average_of_separable_product():
    from oracle.metrics import gl10_cell_average_3d
    e = np.linspace(0, 1, 5)
    avg = gl10_cell_average_3d(lambda x, y, z: np.sin(2 * np.pi * x) * (y ** 2) * np.exp(z), e, e, e)
    a, b = e[:-1], e[1:]
    ax = (np.cos(2 * np.pi * a) - np.cos(2 * np.pi * b)) / (2 * np.pi) / (b - a)
    ay = (b ** 3 - a ** 3) / 3 / (b - a)
    az = (np.exp(b) - np.exp(a)) / (b - a)
    np.testing.assert_allclose(avg, az[:, None, None] * ay[None, :, None] * ax[None, None, :],
                               rtol=1e-12, atol=1e-15)
