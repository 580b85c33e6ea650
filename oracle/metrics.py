"""Verification metric of the paper's examples (Sec. 3, Eq. "l1_error").

TEST INFRASTRUCTURE (see the package docstring).

    L1 = dV * sum_i | N_i - <A(x_i)> |

N_i is the numerical cell value, <A(x_i)> the cell average of the analytic
solution, taken with a 10-node Gauss-Legendre rule per cell (per axis for
tensor-product cells), as the paper prescribes for its L1 figures.
"""
from __future__ import annotations

import numpy as np

from . import riemann_sample

GL_NODES, GL_WEIGHTS = np.polynomial.legendre.leggauss(10)


def gl10_cell_average_1d(f, edges):
    """Average of f over each cell [edges[i], edges[i+1]] with 10-node GL.
    ``f`` maps an array of points to an array of values (any trailing shape)."""
    a, b = edges[:-1], edges[1:]
    half, mid = 0.5 * (b - a), 0.5 * (b + a)
    x = mid[:, None] + half[:, None] * GL_NODES[None, :]          # (ncell, 10)
    vals = np.asarray(f(x.ravel()))
    vals = vals.reshape(x.shape + vals.shape[1:])
    w = GL_WEIGHTS.reshape((1, 10) + (1,) * (vals.ndim - 2))
    return 0.5 * np.sum(w * vals, axis=1)


def gl10_cell_average_3d(f, edges_x, edges_y, edges_z):
    """Tensor-product 10x10x10 GL average of a scalar f(x, y, z) over each cell.
    Returns an array of shape (nz, ny, nx)."""
    def pts(e):
        a, b = e[:-1], e[1:]
        return 0.5 * (b + a)[:, None] + 0.5 * (b - a)[:, None] * GL_NODES[None, :]
    X, Y, Z = pts(edges_x), pts(edges_y), pts(edges_z)
    out = np.zeros((Z.shape[0], Y.shape[0], X.shape[0]))
    for qz in range(10):
        for qy in range(10):
            zz = Z[:, qz][:, None, None]
            yy = Y[:, qy][None, :, None]
            wzy = GL_WEIGHTS[qz] * GL_WEIGHTS[qy]
            for qx in range(10):
                xx = X[:, qx][None, None, :]
                out += wzy * GL_WEIGHTS[qx] * f(xx, yy, zz)
    return out / 8.0


def l1_error(numerical, averaged, dV):
    """Eq. "l1_error": dV * sum |N_i - <A(x_i)>|."""
    return float(dV * np.sum(np.abs(np.asarray(numerical) - np.asarray(averaged))))


def exact_riemann_cell_averages(WL3, WR3, gamma, n, t, x0=0.5, length=1.0, lib=None):
    """GL-10 cell averages of the exact 1D Riemann solution (rho, u, p) at time t
    on n uniform cells of [0, length], interface at x0.  Shape (3, n)."""
    edges = np.linspace(0.0, length, n + 1)

    def f(x):
        return riemann_sample(WL3, WR3, gamma, (x - x0) / t, lib=lib)

    return gl10_cell_average_1d(f, edges).T
