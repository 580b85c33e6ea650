"""The windowed oracle (tests/oracle_window.py) against the oracle run on the
whole mesh: the noisy blast at 40^3 with reflecting walls, three steps of the
whole-mesh CFL schedule; interior, face, edge and corner cells and the blast
centre agree bit for bit (each cell's arithmetic is the same, only the cells
outside its dependence cone differ)."""
import numpy as np

import hydro_inputs as H
import oracle
import oracle_window

GAMMA = 1.4


def test_window_equals_whole_mesh():
    n, steps = 40, 3
    U0 = H.blast_3d(n, seed=2, gamma=GAMMA, radius_cells=3.0)
    g = oracle.Grid((n, n, n), GAMMA, oracle.BC_REFLECT)
    U, _, dts = g.run(U0, steps, 0.3)
    assert float(np.max(np.abs(U[1]))) > 0.0
    c0 = n // 2
    cells = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, c0, n - 1), (c0, c0, c0), (c0 - 1, c0 + 2, c0),
             (5, 11, 12), (12, 13, 27), (27, 27, 13), (1, 30, 38)]
    for c in cells:
        got = oracle_window.cell_after(U0, c, dts, GAMMA, 4 * steps)
        assert np.array_equal(got, U[(slice(None),) + c]), c


def test_window_too_small_is_refused():
    U0 = H.blast_3d(20, seed=2, gamma=GAMMA)
    try:
        oracle_window.cell_after(U0, (10, 10, 10), [1e-4] * 3, GAMMA, 8)
    except ValueError:
        return
    raise AssertionError("a window narrower than the dependence cone was accepted")
