"""Pins of the oracle's radiative heating / cooling exchange (Eq.
"heating-cooling", the test problem of Sec. 3.2): the ODE solution by
quadrature, conservation, the equilibrium fixed point and the stiff limit."""
import math

import numpy as np
import pytest

import hydro_inputs as H
import oracle

scipy_integrate = pytest.importorskip("scipy.integrate")


def _ode_time(pb, e0, Etot, e):
    """t(e) of de/dt = c kappa rho (E_tot - e - a (e / (rho c_v))^4) by adaptive
    quadrature (a library routine, independent of the oracle's Newton solve)."""
    c, kappa, a, cv = pb.params
    k, rcv = c * kappa * pb.rho, pb.rho * pb.cv
    val, _ = scipy_integrate.quad(lambda x: 1.0 / (k * (Etot - x - a * (x / rcv) ** 4)),
                                  e0, e, epsabs=0.0, epsrel=1e-12, limit=200)
    return val


@pytest.mark.parametrize("pb,t_end,final", [(H.heating(), 2e-8, 2e-4), (H.cooling(), 2e-8, 4e-2)])
def test_backward_euler_converges_to_the_ode_solution(pb, t_end, final):
    """N backward-Euler steps of dt = t_end / N reach a fluid energy e_N whose
    exact ODE time t(e_N) approaches t_end at first order in dt."""
    U0, Er0 = pb.state()
    e0 = float(U0[4].item())
    Etot = e0 + float(Er0.item())
    errs = []
    for N in (50, 100, 200):
        U, Er = U0, Er0
        for _ in range(N):
            U, Er, _ = oracle.rad_exchange(U, Er, t_end / N, *pb.params)
        errs.append(abs(_ode_time(pb, e0, Etot, float(U[4].item())) - t_end) / t_end)
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) >= 0.85, (errs, orders)
    assert errs[-1] < final, errs


@pytest.mark.parametrize("pb", [H.heating(), H.cooling()])
def test_exchange_conserves_energy_and_leaves_mass_and_momentum(pb):
    U, Er = pb.state((2, 3, 4), seed=3, spread=0.5)
    for dt in (1e-12, 1e-8, 1e-3, 1e6):
        U2, Er2, _ = oracle.rad_exchange(U, Er, dt, *pb.params)
        assert np.array_equal(U2[:4], U[:4])
        tot, tot2 = U[4] + Er, U2[4] + Er2
        assert np.all(np.abs(tot2 - tot) <= 4e-16 * tot)


def test_radiative_equilibrium_is_a_fixed_point():
    pb = H.HeatingCooling(T_fluid=3.4e6)            # fluid at the radiation temperature
    U, Er = pb.state((5,))
    U2, Er2, _ = oracle.rad_exchange(U, Er, 1e-3, *pb.params)
    assert np.allclose(U2[4], U[4], rtol=1e-14) and np.allclose(Er2, Er, rtol=1e-14)


@pytest.mark.parametrize("pb", [H.heating(), H.cooling()])
def test_large_steps_land_on_equilibrium_without_overshoot(pb):
    """Backward Euler on this monotone exchange: e' lies between e and the
    equilibrium energy for every dt, and dt -> infinity gives the equilibrium
    E_tot - e - a T(e)^4 = 0 (checked as a relative residual)."""
    U, Er = pb.state()
    c, kappa, a, cv = pb.params
    rcv = pb.rho * pb.cv
    e0 = float(U[4].item())
    Etot = e0 + float(Er.item())
    prev = e0
    for dt in (1e-12, 1e-10, 1e-8, 1e-6, 1e-3, 1e3, 1e9):
        U2, _, _ = oracle.rad_exchange(U, Er, dt, *pb.params)
        e = float(U2[4].item())
        heating = pb.T_fluid < pb.T_rad
        assert (prev <= e if heating else prev >= e)      # moves monotonically with dt
        prev = e
    resid = Etot - prev - a * (prev / rcv) ** 4       # = (e' - e) / (dt k) at dt = 1e9
    assert abs(resid) <= 1e-12 * Etot
    # radiation-dominated: the fluid settles at (nearly) the radiation
    # temperature; in the cooling case the fluid's energy raises it by 0.6 %
    assert prev / rcv == pytest.approx(pb.T_rad, rel=1e-2)
