"""Pins for the oracle's whole stage update (CPU only).

  * exact 1D Riemann solutions: L1 (Eq. "l1_error", GL-10 cell averages)
    shrinks with resolution on seeded two-state problems;
  * the Sod tube of Sec. 3.1 against the paper's printed L1 bound (soft);
  * conservation of mass, momentum and energy on periodic domains;
  * mirror symmetry and the equivalence of the x, y and z sweeps;
  * a uniform state is a fixed point;
  * second-order convergence on smooth problems: the advected entropy wave and
    the linear acoustic wave of Sec. 3.5 (closed forms);
  * Heun's Butcher form equals the Shu-Osher form (algebraic identity);
  * the CFL rate of a fluid at rest is c * sum(1/dx).
"""
import math

import numpy as np
import pytest

import hydro_inputs as H
from conftest import read_golden
from oracle import metrics as M


def grid(orc, shape, gamma, bc, extent=(1.0, 1.0, 1.0)):
    return orc.Grid(shape, gamma, bc, extent)


# --------------------------------------------------------------------------
# exact Riemann solutions
# --------------------------------------------------------------------------

def admissible_seeds(orc, count, t_end=0.15):
    """Seeds whose exact waves stay inside [0.02, 0.98] until t_end."""
    out, seed = [], 0
    while len(out) < count:
        pb = H.riemann_1d(seed)
        lo, hi = orc.riemann_extent(pb.WL, pb.WR, pb.gamma)
        if 0.5 + lo * t_end >= 0.02 and 0.5 + hi * t_end <= 0.98:
            out.append(seed)
        seed += 1
    return out


def riemann_l1(orc, pb, n, t_end, cfl):
    g = grid(orc, (1, 1, n), pb.gamma, orc.BC_OUTFLOW)
    U, t, _ = g.run(pb.U(n), 10 ** 7, cfl, t_end=t_end)
    assert t == pytest.approx(t_end, rel=0, abs=1e-15)
    avg = M.exact_riemann_cell_averages(pb.WL, pb.WR, pb.gamma, n, t)
    W = orc.prim_from_cons(U, pb.gamma)[:, 0, 0]
    return [M.l1_error(W[c], avg[k], 1.0 / n) for c, k in ((0, 0), (1, 1), (4, 2))]


def test_riemann_problems_converge(orc):
    seeds = admissible_seeds(orc, 12)
    for seed in seeds:
        pb = H.riemann_1d(seed)
        errs = np.array([riemann_l1(orc, pb, n, 0.15, 0.4) for n in (100, 200, 400, 800)])
        scale = np.array([max(pb.WL[0], pb.WR[0]), 1.0, max(pb.WL[2], pb.WR[2])])
        rel = errs / scale
        # contacts bound the density rate (a smeared contact converges at
        # 1/2 for first-order and at most ~2/3 for second-order TVD schemes);
        # velocity and pressure are continuous across contacts
        for c, min_rate in ((0, 0.5), (1, 0.7), (2, 0.7)):
            assert np.all(np.diff(rel[:, c]) < 0), (seed, rel[:, c])
            rate = math.log2(rel[0, c] / rel[-1, c]) / 3.0
            assert rate >= min_rate, (seed, c, rate)
        assert rel[-1].max() < 0.02, (seed, rel[-1])


def test_sod_against_paper_bound(orc):
    g = read_golden("sod_paper.txt")
    pb = H.RiemannProblem((g["rho_left"], g["u_left"], g["p_left"]),
                          (g["rho_right"], g["u_right"], g["p_right"]), 1.4, g["x0"])
    l1_rho = riemann_l1(orc, pb, int(g["n_cells"]), g["t_final"], g["cfl"])[0]
    # PLM-minmod + HLLC against WENO5-Z + HLL: same order of magnitude
    assert l1_rho < 2.0 * g["l1_density_bound"]


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def random_smooth_state(shape, gamma, seed):
    g = np.random.default_rng(seed)
    nz, ny, nx = shape
    z = H.centres(nz)[:, None, None]
    y = H.centres(ny)[None, :, None]
    x = H.centres(nx)[None, None, :]
    full = shape

    def field(base, amp):
        a, b, c, ph = g.uniform(-1, 1, 4)
        return np.broadcast_to(base + amp * np.sin(2 * np.pi * (x + 2 * y * b + z * c) + 3 * ph)
                               + 0.3 * amp * np.cos(2 * np.pi * (2 * x * a - y + 3 * z)), full)

    W = np.stack([field(1.0, 0.3), field(0.2, 0.5), field(-0.1, 0.5), field(0.3, 0.5),
                  field(1.0, 0.3)])
    return H.prim_to_cons(W, gamma)


@pytest.mark.parametrize("shape", [(8, 12, 10), (1, 16, 14), (1, 1, 40)])
def test_conservation_periodic(orc, shape):
    gam = 5.0 / 3.0
    g = grid(orc, shape, gam, orc.BC_PERIODIC)
    U = random_smooth_state(shape, gam, 7)
    T0 = g.totals(U)
    U1, t, dts = g.run(U, 10, 0.4)
    T1 = g.totals(U1)
    scale = np.abs(T0) + np.sum(np.abs(U), axis=(1, 2, 3)) * np.prod(g.dxyz)
    assert np.all(np.abs(T1 - T0) <= 1e-13 * scale), (T0, T1)


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shape", [(1, 1, 12), (1, 7, 9), (5, 6, 7)])
def test_ghost_cells_equal_padded_domain(orc, bc, shape):
    """The boundary kinds by definition: two ghost layers per active axis that
    wrap (periodic), repeat the edge cell (outflow, zero gradient) or mirror
    the interior with the normal momentum negated (reflect).  The right-hand
    side on the interior must equal that of a domain padded explicitly with
    numpy.pad ('wrap', 'edge', 'symmetric'), whatever the padded domain's own
    boundary kind."""
    gam = 1.4
    U = random_smooth_state(shape, gam, 21 + bc)
    active = [n > 1 for n in shape]                   # (z, y, x)
    widths = [(0, 0)] + [(2, 2) if a else (0, 0) for a in active]
    mode = {0: "wrap", 1: "edge", 2: "symmetric"}[bc]
    P = np.pad(U, widths, mode=mode)
    if bc == 2:
        # negate the normal momentum inside the ghost slabs of each axis
        for ax, comp in ((3, 1), (2, 2), (1, 3)):     # x -> rho u, y -> rho v, z -> rho w
            if not active[ax - 1]:
                continue
            sl = [slice(None)] * 4
            sl[0] = comp
            for ghost in (slice(0, 2), slice(-2, None)):
                sl[ax] = ghost
                P[tuple(sl)] *= -1
    g = grid(orc, shape, gam, bc)
    gp = grid(orc, P.shape[1:], gam, orc.BC_PERIODIC)
    gp.dxyz = g.dxyz.copy()                          # identical cell widths
    L = g.rhs(U)
    Lp = gp.rhs(P)
    inner = tuple([slice(None)] + [slice(2, -2) if a else slice(None) for a in active])
    np.testing.assert_array_equal(L, Lp[inner])


def test_reflecting_box_conserves_mass_and_energy(orc):
    """Closed box with reflecting walls: no mass or energy crosses a wall."""
    gam = 1.4
    shape = (6, 7, 8)
    g = grid(orc, shape, gam, orc.BC_REFLECT)
    U = random_smooth_state(shape, gam, 5)
    T0 = g.totals(U)
    V, _, _ = g.run(U, 10, 0.4)
    T1 = g.totals(V)
    for f in (0, 4):
        assert abs(T1[f] - T0[f]) <= 1e-13 * abs(T0[f]), (f, T0[f], T1[f])


def test_uniform_state_is_fixed_point(orc):
    gam = 1.4
    for bc, vel in ((orc.BC_PERIODIC, (0.3, -0.2, 0.5)), (orc.BC_OUTFLOW, (0.3, -0.2, 0.5)),
                    (orc.BC_REFLECT, (0.0, 0.0, 0.0))):
        shape = (5, 6, 7)
        W = [np.full(shape, v) for v in (1.3, *vel, 0.8)]
        U = H.prim_to_cons(W, gam)
        L = grid(orc, shape, gam, bc).rhs(U)
        assert np.max(np.abs(L)) <= 1e-14 * np.max(np.abs(U)), bc


def test_mirror_symmetry_1d(orc):
    """A two-state problem and its mirror image (x -> 1 - x, u -> -u) stay
    mirror images of each other."""
    pb = H.riemann_1d(3)
    n = 128
    U = pb.U(n)
    Um = U[:, :, :, ::-1].copy()
    Um[1] *= -1
    g = grid(orc, (1, 1, n), pb.gamma, orc.BC_OUTFLOW)
    A, _, _ = g.run(U, 60, 0.4)
    B, _, _ = g.run(Um, 60, 0.4)
    B = B[:, :, :, ::-1].copy()
    B[1] *= -1
    np.testing.assert_allclose(A, B, rtol=1e-13, atol=1e-13)


def test_blast_symmetry_3d(orc):
    """Noise-free spherical blast with reflecting walls: symmetric under each
    axis reflection and under permutations of the axes."""
    n = 16
    U = H.blast_3d(n, noise=False, radius_cells=3.0)
    g = grid(orc, (n, n, n), 1.4, orc.BC_REFLECT)
    V, _, _ = g.run(U, 8, 0.3)
    rho = V[0]
    scale = np.max(np.abs(rho))
    assert np.max(np.abs(rho - rho[::-1, :, :])) <= 1e-13 * scale
    assert np.max(np.abs(rho - rho[:, ::-1, :])) <= 1e-13 * scale
    assert np.max(np.abs(rho - rho[:, :, ::-1])) <= 1e-13 * scale
    assert np.max(np.abs(rho - rho.transpose(1, 0, 2))) <= 1e-13 * scale
    assert np.max(np.abs(rho - rho.transpose(0, 2, 1))) <= 1e-13 * scale
    # x-momentum is odd under x reflection and maps to y-momentum under x<->y
    mx, my = V[1], V[2]
    assert np.max(np.abs(mx + mx[:, :, ::-1])) <= 1e-13 * np.max(np.abs(mx))
    assert np.max(np.abs(mx - my.transpose(0, 2, 1))) <= 1e-13 * np.max(np.abs(mx))
    E = V[4]
    assert np.max(np.abs(E - E.transpose(2, 1, 0))) <= 1e-13 * np.max(np.abs(E))


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_axis_sweeps_equivalent(orc, bc):
    """The same 1D problem laid along x, y or z gives the same result (the
    momentum component follows the axis)."""
    pb = H.riemann_1d(5)
    n = 64
    res = []
    for axis in range(3):
        U = pb.U(n, axis=axis)
        shape = U.shape[1:]
        g = grid(orc, shape, pb.gamma, bc)
        V, _, _ = g.run(U, 30, 0.4)
        V = V.reshape(5, n)
        res.append(V[[0, 1 + axis, 4]])
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], res[2])


def test_3d_periodic_translation_equivariance(orc):
    """Shifting the initial data by whole cells shifts the periodic solution."""
    gam = 5.0 / 3.0
    shape = (6, 8, 10)
    U = random_smooth_state(shape, gam, 11)
    g = grid(orc, shape, gam, orc.BC_PERIODIC)
    A, _, _ = g.run(U, 4, 0.4)
    B, _, _ = g.run(np.roll(U, (2, -3, 5), axis=(1, 2, 3)), 4, 0.4)
    np.testing.assert_array_equal(np.roll(A, (2, -3, 5), axis=(1, 2, 3)), B)


# --------------------------------------------------------------------------
# convergence on smooth solutions
# --------------------------------------------------------------------------

def test_acoustic_wave_second_order(orc):
    """Sec. 3.5 closed form: a small plane acoustic wave with P_A = c_s^2 rho_A,
    u_A = c_s rho_A / rho0 travels at c_s = sqrt(gamma P0 / rho0).  After one
    period the error in the density perturbation converges at second order."""
    gam, A = 1.4, 1e-6
    cs = math.sqrt(gam)
    T = 1.0 / cs
    errs = []
    for n in (128, 256, 512):
        e = np.linspace(0, 1, n + 1)
        s0 = M.gl10_cell_average_1d(lambda x: np.sin(2 * np.pi * x), e)
        W = (1 + A * s0, cs * A * s0, 0 * s0, 0 * s0, 1 + cs * cs * A * s0)
        U = H.prim_to_cons(W, gam).reshape(5, 1, 1, n)
        g = grid(orc, (1, 1, n), gam, orc.BC_PERIODIC)
        V, t, _ = g.run(U, 10 ** 6, 0.4, t_end=T)
        sT = M.gl10_cell_average_1d(lambda x: np.sin(2 * np.pi * (x - cs * T)), e)
        errs.append(M.l1_error((V[0, 0, 0] - 1) / A, sT, 1.0 / n))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) >= 1.8, (errs, rates)
    assert errs[-1] < 1e-3


def test_entropy_wave_second_order_2d(orc):
    """rho = 1 + 0.2 sin(2 pi (x + y)) advected at v = (1, 1), p = 1 is translated
    exactly; the L1 error against the GL-10 averaged exact solution drops at
    close to second order along the diagonal of a 2D grid."""
    gam = 1.4
    T = 0.25
    errs = []
    for n in (32, 64):
        W = H.entropy_wave((1, n, n), direction=(1, 1, 0))
        U = H.prim_to_cons(W, gam)
        g = grid(orc, (1, n, n), gam, orc.BC_PERIODIC)
        V, t, _ = g.run(U, 10 ** 6, 0.4, t_end=T)
        e = np.linspace(0, 1, n + 1)
        avg = M.gl10_cell_average_3d(
            lambda x, y, z: 1 + 0.2 * np.sin(2 * np.pi * ((x - T) + (y - T))), e, e,
            np.array([0.0, 1.0]))
        errs.append(M.l1_error(V[0], avg, 1.0 / n / n))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= 1.4, (errs, rate)


def test_entropy_wave_1d_order(orc):
    gam = 1.4
    T = 0.5
    errs = []
    for n in (64, 128, 256, 512):
        W = H.entropy_wave((1, 1, n), direction=(1, 0, 0))
        U = H.prim_to_cons(W, gam)
        g = grid(orc, (1, 1, n), gam, orc.BC_PERIODIC)
        V, t, _ = g.run(U, 10 ** 6, 0.4, t_end=T)
        e = np.linspace(0, 1, n + 1)
        avg = M.gl10_cell_average_1d(lambda x: 1 + 0.2 * np.sin(2 * np.pi * (x - T)), e)
        errs.append(M.l1_error(V[0, 0, 0], avg, 1.0 / n))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert rates[-1] >= 1.8, (errs, rates)


# --------------------------------------------------------------------------
# time integrator and time step
# --------------------------------------------------------------------------

def test_heun_equals_shu_osher(orc):
    gam = 1.4
    shape = (4, 6, 8)
    U = random_smooth_state(shape, gam, 3)
    g = grid(orc, shape, gam, orc.BC_PERIODIC)
    dt = 0.4 / g.max_rate(U)
    A = g.step(U, dt)
    B = g.step_heun(U, dt)
    assert np.max(np.abs(A - B)) <= 1e-14 * np.max(np.abs(U))
    # and the two stages compose to the step
    U1 = g.stage(1, U, U, dt)
    np.testing.assert_array_equal(g.stage(2, U, U1, dt), A)


def test_rate_of_fluid_at_rest(orc):
    gam = 1.4
    shape = (3, 4, 5)
    rho, p = 0.7, 2.2
    W = [np.full(shape, rho), *(np.zeros(shape),) * 3, np.full(shape, p)]
    U = H.prim_to_cons(W, gam)
    g = grid(orc, shape, gam, orc.BC_PERIODIC, extent=(1.0, 2.0, 0.5))
    c = math.sqrt(gam * p / rho)
    assert g.max_rate(U) == pytest.approx(c * (5 / 1.0 + 4 / 2.0 + 3 / 0.5), rel=1e-14)
    # inactive axes do not contribute
    g1 = grid(orc, (1, 1, 5), gam, orc.BC_PERIODIC)
    U1 = H.prim_to_cons([np.full((1, 1, 5), rho), *(np.zeros((1, 1, 5)),) * 3,
                         np.full((1, 1, 5), p)], gam)
    assert g1.max_rate(U1) == pytest.approx(c * 5, rel=1e-14)


def test_run_clips_to_final_time(orc):
    pb = H.sod()
    g = grid(orc, (1, 1, 64), 1.4, orc.BC_OUTFLOW)
    _, t, dts = g.run(pb.U(64), 10 ** 5, 0.4, t_end=0.05)
    assert t == 0.05 or abs(t - 0.05) < 1e-16
    assert dts[-1] <= dts[0] * 1.5
