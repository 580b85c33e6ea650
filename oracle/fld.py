"""Flux-limited radiation diffusion, one implicit step (FP64, numpy / scipy).

TEST INFRASTRUCTURE (see the package docstring): only tests and the bench's
CPU legs use it.

What it computes (paper "HARD", Sec. 2.2.1 and 2.2.2): the diffusive part of
the radiation energy equation, Eq. "radiation" without the advection, work
and heating terms,

    dE/dt = div(D grad E),   D = c lambda / (kappa rho)      (Eq. "F_r"),
    lambda = (2 + R) / (6 + 3R + R^2),  R = |grad E| / (rho kappa E)
                                        (the Levermore limiter of Sec. 2.2.1),

discretised on the cell-centred mesh and advanced by one backward-Euler step
with D frozen at the old state (so the step is a linear solve, Eq.
"linear_equation" A u = f, which the paper hands to geometric multigrid):

    E' - dt sum_d [D_{i+1/2} (E'_{i+1} - E'_i) - D_{i-1/2} (E'_i - E'_{i-1})] / dx_d^2 = E.

Readings where the paper is silent:
  * face coefficient: the arithmetic mean of the two cells' D;
  * grad E for R: central differences with the boundary map of the hydro
    stage (periodic wrap; outflow and reflecting walls repeat or mirror the
    edge cell), |grad E| summed over the active axes;
  * boundaries: periodic faces couple across the wrap; outflow and reflecting
    faces carry no flux (the ghost equals the edge cell);
  * the linear system is solved exactly here (a sparse direct solve, a
    library primitive); the CUDA path iterates V-cycles to a tolerance.
"""
from __future__ import annotations

import numpy as np

BC_PERIODIC, BC_OUTFLOW, BC_REFLECT = 0, 1, 2


def flux_limiter(R):
    """Levermore's lambda(R) = (2 + R) / (6 + 3R + R^2)."""
    R = np.asarray(R, dtype=np.float64)
    return (2.0 + R) / (6.0 + 3.0 * R + R * R)


def _axes(shape):
    """(tensor axis, physical axis) of every active axis, x first."""
    nz, ny, nx = shape
    out = []
    for d, n in enumerate((nx, ny, nz)):
        if n > 1:
            out.append((2 - d, d))
    return out


def _neighbour(E, ax, step, periodic):
    """E shifted by one cell along tensor axis ax (+1: the next cell), with the
    edge cell repeated at a non-periodic boundary."""
    if periodic:
        return np.roll(E, -step, axis=ax)
    n = E.shape[ax]
    idx = np.clip(np.arange(n) + step, 0, n - 1)
    return np.take(E, idx, axis=ax)


def diffusion_coefficient(rho, E, c, kappa, dxyz, bc6):
    """Cell-centred D = c lambda(R) / (kappa rho) of the current state."""
    grad2 = np.zeros_like(E)
    for ax, d in _axes(E.shape):
        per = bc6[2 * d] == BC_PERIODIC
        g = (_neighbour(E, ax, +1, per) - _neighbour(E, ax, -1, per)) / (2.0 * dxyz[d])
        grad2 += g * g
    R = np.sqrt(grad2) / (rho * kappa * E)
    return c * flux_limiter(R) / (kappa * rho)


def fld_matrix(D, dt, dxyz, bc6):
    """Sparse A = I - dt div(D grad .) of the backward-Euler step (CSR)."""
    import scipy.sparse as sp
    shape = D.shape
    N = D.size
    idx = np.arange(N).reshape(shape)
    rows, cols, vals = [np.arange(N)], [np.arange(N)], [np.ones(N)]
    diag = np.zeros(shape)
    for ax, d in _axes(shape):
        per = bc6[2 * d] == BC_PERIODIC
        n = shape[ax]
        up = np.arange(n) + 1                         # the cell across the upper face
        valid = up < n
        if per:
            up = up % n
            valid = np.ones(n, dtype=bool)
        up = np.clip(up, 0, n - 1)
        Dn = np.take(D, up, axis=ax)
        w = 0.5 * (D + Dn) * dt / (dxyz[d] * dxyz[d])  # face weight dt D_f / dx^2
        mask_shape = [1, 1, 1]
        mask_shape[ax] = n
        w = w * valid.reshape(mask_shape)
        nb = np.take(idx, up, axis=ax)
        # the face couples cell i and its upper neighbour symmetrically
        rows += [idx.ravel(), nb.ravel()]
        cols += [nb.ravel(), idx.ravel()]
        vals += [-w.ravel(), -w.ravel()]
        diag += w
        diag += np.take(w, (np.arange(n) - 1) % n, axis=ax) if per else \
            np.concatenate([np.zeros_like(np.take(w, [0], axis=ax)),
                            np.take(w, np.arange(n - 1), axis=ax)], axis=ax)
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A


def fld_step(rho, E, dt, c, kappa, dxyz, bc6):
    """One backward-Euler step of the flux-limited diffusion: returns E'."""
    import scipy.sparse.linalg as spla
    rho = np.asarray(rho, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    D = diffusion_coefficient(rho, E, c, kappa, dxyz, bc6)
    A = fld_matrix(D, dt, dxyz, bc6)
    return spla.spsolve(A.tocsc(), E.ravel()).reshape(E.shape)
