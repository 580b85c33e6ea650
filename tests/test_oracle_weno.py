"""Pins of the oracle's second scheme (Sec. 2.2.2: WENO5-Z face states and
the HLL flux) against closed forms, exact results and invariants."""
import math

import numpy as np
import pytest

import hydro_inputs as H
import oracle
from oracle import metrics


def _cell_averages(f, n):
    return metrics.gl10_cell_average_1d(f, np.linspace(0.0, 1.0, n + 1))


# ---------------------------------------------------------------- WENO5-Z --

def test_weno5z_reproduces_linear_data():
    """Cell averages of a linear function: every candidate is exact and the
    indicators are equal, so the face value is the exact one."""
    for a, b in [(1.0, 0.25), (-3.0, 2.5), (7.0, -0.125)]:
        v = [a + b * i for i in range(5)]           # cell i spans [i - 1/2, i + 1/2]
        assert oracle.weno5z(v) == pytest.approx(a + b * 2.5, rel=1e-14, abs=1e-14)


def test_weno5z_symmetric_stencil_takes_the_linear_weights():
    """b0 = b2 for data mirror-symmetric about the middle cell, so tau5 = 0 and
    the weights are the linear ones: the fifth-order upwind value
    (2 v0 - 13 v1 + 47 v2 + 27 v3 - 3 v4) / 60."""
    for a, b, c in [(3, 5, 7), (-2, 4, 1), (10, -6, 0)]:
        v = [a, b, c, b, a]
        assert oracle.weno5z(v) == pytest.approx((-a + 14 * b + 47 * c) / 60.0, rel=1e-14)


def test_weno5z_fifth_order_on_smooth_data():
    """Face values from GL-10 cell averages of a smooth periodic function
    converge at fifth order in L1 (observed 5.3 and 5.6)."""
    def f(x):
        return np.sin(2 * np.pi * x) + 0.3 * np.cos(4 * np.pi * x)

    errs = []
    for n in (40, 80, 160):
        v = _cell_averages(f, n)
        e = [oracle.weno5z([v[(i + k) % n] for k in (-2, -1, 0, 1, 2)]) - f((i + 1) / n)
             for i in range(n)]
        errs.append(np.mean(np.abs(e)))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert orders[0] >= 5.0 and orders[1] >= 5.3, orders


def test_weno5z_step_takes_the_smooth_side():
    """Essentially non-oscillatory at a jump: the face inside the smooth side
    takes that side's value (the weight of the jump-crossing stencils is of
    order eps / b)."""
    assert abs(oracle.weno5z([0, 0, 0, 1, 1])) < 1e-20
    assert oracle.weno5z([0, 0, 1, 1, 1]) == pytest.approx(1.0, abs=1e-15)
    assert oracle.weno5z([2, 2, 2, -5, -5]) == pytest.approx(2.0, abs=1e-15)


# -------------------------------------------------------------------- HLL --

def _physical_flux(W, gamma):
    r, u, v, w, p = W
    E = p / (gamma - 1) + 0.5 * r * (u * u + v * v + w * w)
    return np.array([r * u, r * u * u + p, r * u * v, r * u * w, (E + p) * u])


@pytest.mark.parametrize("W", [(1.0, 0.3, -0.2, 0.1, 1.0), (0.125, -1.5, 0.0, 2.0, 0.1),
                               (4.0, 0.0, 0.0, 0.0, 7.0)])
def test_hll_consistency(W):
    """F_HLL(W, W) is the physical flux of W."""
    assert np.allclose(oracle.hll(W, W, 1.4), _physical_flux(W, 1.4), rtol=1e-14, atol=1e-14)


def test_hll_supersonic_upwinding():
    """All waves right-going: F = F_L; all left-going: F = F_R."""
    WL, WR = (1.0, 5.0, 0.1, 0.0, 1.0), (0.5, 4.5, 0.0, 0.2, 0.8)
    assert np.array_equal(oracle.hll(WL, WR, 1.4), _physical_flux(WL, 1.4))
    WL, WR = (1.0, -5.0, 0.1, 0.0, 1.0), (0.5, -4.5, 0.0, 0.2, 0.8)
    assert np.array_equal(oracle.hll(WL, WR, 1.4), _physical_flux(WR, 1.4))


def test_hll_smears_a_stationary_contact():
    """Resting contact (u = 0, equal p): the Davis bounds are -+c_max, so
    F_rho = -c_max (rho_R - rho_L) / 2, the momentum flux is p and the energy
    flux vanishes (E_L = E_R)."""
    g = 1.4
    rL, rR, p = 1.0, 0.25, 0.7
    F = oracle.hll((rL, 0, 0, 0, p), (rR, 0, 0, 0, p), g)
    cmax = max(math.sqrt(g * p / rL), math.sqrt(g * p / rR))
    assert F[0] == pytest.approx(-cmax * (rR - rL) / 2, rel=1e-14)
    assert F[1] == pytest.approx(p, rel=1e-14)
    assert F[2] == 0 and F[3] == 0 and abs(F[4]) < 1e-15


# ----------------------------------------------------------------- scheme --

def test_weno_scheme_preserves_a_uniform_state():
    U = H.prim_to_cons(np.broadcast_to(np.array([1.3, 0.4, -0.2, 0.7, 2.1])[:, None, None, None],
                                       (5, 5, 6, 7)).copy(), 1.4)
    g = oracle.Grid((5, 6, 7), 1.4, oracle.BC_PERIODIC, scheme=oracle.SCHEME_WENO5Z_HLL)
    assert np.max(np.abs(g.rhs(U))) < 1e-12


def test_weno_rhs_fifth_order_on_advected_profile():
    """Exact cell averages of rho = 1 + 0.2 sin(2 pi x) carried at u = 1 with
    p = 1: L(U) against the exact flux difference of the face values,
    -(F(x_{i+1/2}) - F(x_{i-1/2})) / h, converges at fifth order
    (observed 5.0)."""
    gam = 1.4
    errs = []
    for n in (32, 64, 128):
        rho = _cell_averages(lambda x: 1 + 0.2 * np.sin(2 * np.pi * x), n)
        U = np.zeros((5, 1, 1, n))
        U[0, 0, 0], U[1, 0, 0], U[4, 0, 0] = rho, rho, 1 / (gam - 1) + 0.5 * rho
        L = oracle.Grid((1, 1, n), gam, 0, scheme=oracle.SCHEME_WENO5Z_HLL).rhs(U)
        xf = np.arange(n + 1) / n
        mass = 1 + 0.2 * np.sin(2 * np.pi * xf)
        errs.append(np.mean(np.abs(L[0, 0, 0] + (mass[1:] - mass[:-1]) * n)))
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) >= 4.8, orders


def test_weno_conserves_totals_in_a_periodic_box():
    shape = (6, 7, 8)
    rng = np.random.default_rng(5)
    W = np.stack([1 + 0.3 * rng.random(shape), 0.2 * rng.standard_normal(shape),
                  0.2 * rng.standard_normal(shape), 0.2 * rng.standard_normal(shape),
                  1 + 0.3 * rng.random(shape)])
    U = H.prim_to_cons(W, 1.4)
    g = oracle.Grid(shape, 1.4, oracle.BC_PERIODIC, scheme=oracle.SCHEME_WENO5Z_HLL)
    before = g.totals(U)
    Uf, _, _ = g.run(U, 5, 0.4)
    assert np.allclose(g.totals(Uf), before, rtol=0, atol=1e-13 * np.abs(before).max())


def test_weno_mirror_symmetry_between_reflecting_walls():
    """A mirror-symmetric state between two reflecting walls stays symmetric:
    rho, E even and rho u odd under x -> 1 - x."""
    n = 40
    x = H.centres(n)
    W = np.zeros((5, 1, 1, n))
    W[0, 0, 0] = 1 + 0.5 * np.exp(-80 * (x - 0.5) ** 2)
    W[1, 0, 0] = 0.3 * np.sin(2 * np.pi * x)        # odd about 1/2
    W[4, 0, 0] = 1 + np.exp(-80 * (x - 0.5) ** 2)
    U = H.prim_to_cons(W, 1.4)
    g = oracle.Grid((1, 1, n), 1.4, oracle.BC_REFLECT, scheme=oracle.SCHEME_WENO5Z_HLL)
    Uf, _, _ = g.run(U, 30, 0.4)
    r = Uf[:, 0, 0, ::-1]
    assert np.allclose(Uf[0, 0, 0], r[0], rtol=1e-12)
    assert np.allclose(Uf[4, 0, 0], r[4], rtol=1e-12)
    assert np.allclose(Uf[1, 0, 0], -r[1], atol=1e-12)


def _acoustic(n, gam, t, amp=1e-6):
    """Right-going linear acoustic wave (Sec. 3.5 closed form, rho0 = P0 = 1):
    exact cell averages at time t."""
    cs = math.sqrt(gam)
    h = 1.0 / n
    x = np.arange(n) * h
    S = (np.cos(2 * np.pi * (x - cs * t)) - np.cos(2 * np.pi * (x + h - cs * t))) / (2 * np.pi * h)
    W = np.zeros((5, 1, 1, n))
    W[0, 0, 0], W[1, 0, 0], W[4, 0, 0] = 1 + amp * S, cs * amp * S, 1 + cs * cs * amp * S
    return H.prim_to_cons(W, gam)


def test_weno_acoustic_wave_convergence():
    """The convergence test of Sec. 3.5: an acoustic wave, same final time on
    every grid, CFL-limited steps.  With Heun in time the observed order is 2
    (the time error dominates at CFL 0.4), and at 32 cells WENO5-Z + HLL is
    more than 10x closer to the exact wave than PLM + HLLC."""
    gam = 5.0 / 3.0
    T = 0.5 / math.sqrt(gam)
    err = {}
    for scheme in (0, 1):
        for n in (32, 64, 128):
            g = oracle.Grid((1, 1, n), gam, 0, scheme=scheme)
            Uf, t, _ = g.run(_acoustic(n, gam, 0.0), 100000, 0.4, t_end=T)
            assert t == pytest.approx(T, rel=1e-14)
            err[scheme, n] = np.mean(np.abs(Uf[0, 0, 0] - _acoustic(n, gam, T)[0, 0, 0]))
    orders = [math.log2(err[1, n] / err[1, 2 * n]) for n in (32, 64)]
    assert min(orders) >= 1.9, orders
    assert err[1, 32] * 10 < err[0, 32]


def test_weno_sod_converges_to_the_exact_solution():
    """Sod (Sec. 3.1) at t = 0.2 against GL-10 averages of the exact Riemann
    solution: the density L1 error falls with resolution and is below PLM's."""
    pb = H.sod()
    errs = {}
    for scheme in (0, 1):
        for n in (100, 200):
            g = oracle.Grid((1, 1, n), pb.gamma, oracle.BC_OUTFLOW, scheme=scheme)
            Uf, t, _ = g.run(pb.U(n), 100000, 0.4, t_end=0.2)
            ref = metrics.exact_riemann_cell_averages(pb.WL, pb.WR, pb.gamma, n, t)
            errs[scheme, n] = metrics.l1_error(Uf[0].ravel(), ref[0], 1.0 / n)
    assert errs[1, 200] < 0.7 * errs[1, 100]
    assert errs[1, 100] < errs[0, 100] and errs[1, 200] < errs[0, 200]
    assert errs[1, 200] < 2.5e-3


def test_weno_needs_three_cells_per_active_axis():
    with pytest.raises(ValueError):
        oracle.Grid((1, 2, 8), 1.4, 0, scheme=oracle.SCHEME_WENO5Z_HLL)
