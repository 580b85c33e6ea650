"""Order of accuracy of the CUDA path on the smooth 3D configuration.

The entropy wave rho = 1 + 0.2 sin(2 pi (x + y + z)), v = (1, 1, 1), p = 1,
gamma = 5/3 on the periodic unit cube is translated exactly by the Euler
equations (Eq. "conservative form": with uniform v and p the density is
advected).  Its exact cell averages at time T are
    1 + 0.2 sin(2 pi (x_c + y_c + z_c - 3 T)) (sin(pi h) / (pi h))^3,
a closed form, so the L1 error of the FP32 stage kernels at 64^3, 128^3 and
256^3 (the meshes of the smooth-flow configuration), all advanced to the same
final time with the CFL step clipped there, must fall at second order.
Minmod clips the extrema, so the rate sits a little under two."""
import math

import numpy as np
import pytest

import hydro_inputs as H

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")

GAMMA = 5.0 / 3.0
T_END = 0.02          # the 100-step time at 256^3 rounded down to 0.02


def _l1_density_error(n):
    W = H.entropy_wave((n, n, n), direction=(1, 1, 1))
    U = torch.tensor(H.prim_to_cons(W, GAMMA), dtype=torch.float32, device="cuda")
    m = hh.HardHydro((n, n, n), GAMMA, hh.HARD_BC_PERIODIC, dtype=torch.float32)
    mass0 = m.totals(U)[0]
    # enough steps to reach T_END: the signal rate is below 3 (1 + 1.5) n
    nsteps = int(math.ceil(T_END * 3 * 2.5 * n / 0.4)) + 5
    t, _, _ = m.advance(U, nsteps, 0.4, t_end=T_END)
    assert float(t) == pytest.approx(T_END, rel=1e-12)
    assert m.get_error() == hh.HARD_OK
    mass1 = m.totals(U)[0]
    h = 1.0 / n
    xc = H.centres(n)
    phase = xc[:, None, None] + xc[None, :, None] + xc[None, None, :] - 3.0 * T_END
    sinc = math.sin(math.pi * h) / (math.pi * h)
    exact = 1.0 + 0.2 * np.sin(2.0 * math.pi * phase) * sinc ** 3
    rho = U[0].double().cpu().numpy()
    return float(np.sum(np.abs(rho - exact)) * h ** 3), mass0, mass1


def test_entropy_wave_second_order_64_128_256():
    errs = []
    for n in (64, 128, 256):
        e, mass0, mass1 = _l1_density_error(n)
        # flux form: the FP32 update conserves mass to its rounding
        assert abs(mass1 - mass0) <= 1e-6 * abs(mass0), (n, mass0, mass1)
        errs.append(e)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(r >= 1.8 for r in rates), (errs, rates)
