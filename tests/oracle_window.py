"""The oracle's state of one cell after a few steps, computed on a window of
the mesh around it instead of the whole mesh: a two-stage PLM step reads two
cells per stage on each side, so after s steps a cell depends only on the
cells within 4 s of it.  A window face inside the mesh is given outflow
ghosts, whose error moves in by at most 4 cells per step and so does not
reach the centre of a window of half-width 4 s; a window face on a wall keeps
the wall's reflecting ghosts.  Used to check single cells of meshes too large
for the oracle to run whole (test infrastructure)."""
import numpy as np

import oracle


def window(c, n, half):
    """Index range [lo, hi) and oracle boundary kinds (low face, high face) of
    the window of 2 half + 1 cells around coordinate c on an axis of n cells
    with reflecting walls; a window that would cross a wall is moved inside
    and keeps that wall."""
    w = 2 * half + 1
    if c < half:
        return 0, w, oracle.BC_REFLECT, oracle.BC_OUTFLOW
    if c > n - 1 - half:
        return n - w, n, oracle.BC_OUTFLOW, oracle.BC_REFLECT
    return c - half, c + half + 1, oracle.BC_OUTFLOW, oracle.BC_OUTFLOW


def cell_after(U, c, dts, gamma, half):
    """State (5,) of cell c = (k, j, i) of the cubic mesh U (5, n, n, n) on the
    unit cube with reflecting walls after oracle steps of the sizes dts, from
    the window of half-width `half` (at least 4 len(dts)) around it."""
    n = U.shape[-1]
    if half < 4 * len(dts) or 2 * half + 1 > n:
        raise ValueError("the window must reach 4 cells per step and fit the mesh")
    rz, ry, rx = (window(int(v), n, half) for v in c)
    W = np.array(U[:, rz[0]:rz[1], ry[0]:ry[1], rx[0]:rx[1]], dtype=np.float64)
    g = oracle.Grid(W.shape[1:], gamma, [rx[2], rx[3], ry[2], ry[3], rz[2], rz[3]])
    g.dxyz = np.array([1.0 / n, 1.0 / n, 1.0 / n])
    for dt in dts:
        W = g.step(W, float(dt))
    return W[:, int(c[0]) - rz[0], int(c[1]) - ry[0], int(c[2]) - rx[0]]
