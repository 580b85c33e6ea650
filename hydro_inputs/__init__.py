"""Seeded synthetic initial states for the hydro stage update.

This module is shared by the oracle-side tests and the CUDA-side tests, the
bench and the smoke check.  It holds no arithmetic of the numerical method:
it only draws seeded random parameters (numpy PCG64) and writes initial
primitive fields, converted to the conserved layout U[5][nz][ny][nx]
(rho, rho u, rho v, rho w, E) with the ideal-gas definition of the total
energy E = p/(gamma-1) + rho |v|^2 / 2 that defines the input.

Cell centres are x_i = (i + 1/2) dx on [0, L) along every axis; all domains
are the unit box unless stated.  The problems stand in for the paper's test
suite (Sec. 3): the Sod tube of Sec. 3.1, seeded two-state Riemann problems,
a smooth advected wave with acoustic modes (Sec. 3.5), a spherical blast, a
shear layer (the non-radiative analogue of Sec. 3.4's Kelvin-Helmholtz run)
and a batch of small piecewise-constant problems.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def centres(n, length=1.0):
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def prim_to_cons(W, gamma):
    """(rho, u, v, w, p) -> (rho, rho u, rho v, rho w, E); defines the input."""
    rho, u, v, w, p = (np.asarray(a, dtype=np.float64) for a in W)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E])


# --------------------------------------------------------------------------
# 1D two-state Riemann problems (seeded) and the Sod tube
# --------------------------------------------------------------------------

@dataclass
class RiemannProblem:
    WL: tuple                 # (rho, u, p) left of x0
    WR: tuple                 # (rho, u, p) right of x0
    gamma: float = 1.4
    x0: float = 0.5
    seed: int | None = None
    draws: int = 1            # how many draws the seed needed (vacuum rejection)

    def U(self, n, axis=0, length=1.0):
        """Conserved state on n cells, the jump along ``axis`` (0=x, 1=y, 2=z)."""
        x = centres(n, length)
        left = x <= self.x0
        rho = np.where(left, self.WL[0], self.WR[0])
        vel = np.where(left, self.WL[1], self.WR[1])
        p = np.where(left, self.WL[2], self.WR[2])
        zero = np.zeros(n)
        vs = [zero, zero, zero]
        vs[axis] = vel
        U = prim_to_cons((rho, *vs, p), self.gamma)         # (5, n)
        shape = [1, 1, 1]
        shape[2 - axis] = n
        return U.reshape((5, *shape)).copy()


def riemann_1d(seed, gamma=1.4):
    """Two-state problem: rho, p log-uniform in [0.1, 10], u uniform in [-1, 1].
    Draws that would create vacuum (2(cL+cR)/(gamma-1) <= uR-uL) are redrawn."""
    g = _rng(seed)
    draws = 0
    while True:
        draws += 1
        rl, rr, pl, pr = np.exp(g.uniform(math.log(0.1), math.log(10.0), size=4))
        ul, ur = g.uniform(-1.0, 1.0, size=2)
        cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
        if 2.0 * (cl + cr) / (gamma - 1.0) > ur - ul:
            return RiemannProblem((rl, ul, pl), (rr, ur, pr), gamma, 0.5, seed, draws)


def sod(gamma=1.4):
    """Sec. 3.1: (rho, v, p) = (1, 0, 1) for x <= 0.5, (0.125, 0, 0.1) beyond."""
    return RiemannProblem((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), gamma, 0.5)


# --------------------------------------------------------------------------
# Smooth 3D flow: entropy wave + acoustic modes (Sec. 3.5)
# --------------------------------------------------------------------------

# The 8 lowest integer wave vectors, one of each +-n pair, ordered by |n|^2
# then lexicographically (the reading of "the 8 lowest modes").
LOW_MODES = ((0, 0, 1), (0, 1, 0), (1, 0, 0), (0, 1, 1), (0, 1, -1), (1, 0, 1),
             (1, 0, -1), (1, 1, 0))


def acoustic_phases(seed, nmodes=8):
    return _rng(seed).uniform(0.0, 2.0 * math.pi, size=nmodes)


def smooth_3d(n, seed=0, gamma=5.0 / 3.0, amp=1e-3, acoustic=True, shape=None,
              dtype=np.float64):
    """rho = 1 + 0.2 sin(2 pi (x+y+z)), v = (1,1,1), p = 1, plus acoustic modes
    (Sec. 3.5 closed forms, rho0 = P0 = 1):  d rho = amp sin(2 pi n.x + phi),
    dp = c_s^2 d rho,  dv = n_hat c_s d rho / rho0,  c_s = sqrt(gamma P0/rho0).
    ``shape`` = (nz, ny, nx) overrides the cube n^3 (all on the unit box)."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    z = centres(nz)[:, None, None]
    y = centres(ny)[None, :, None]
    x = centres(nx)[None, None, :]
    full = (nz, ny, nx)
    rho = np.broadcast_to(1.0 + 0.2 * np.sin(2.0 * math.pi * (x + y + z)), full).copy()
    u = np.ones(full)
    v = np.ones(full)
    w = np.ones(full)
    p = np.ones(full)
    if acoustic:
        cs = math.sqrt(gamma)
        for m, phi in zip(LOW_MODES, acoustic_phases(seed)):
            kx, ky, kz = m
            norm = math.sqrt(kx * kx + ky * ky + kz * kz)
            drho = amp * np.sin(2.0 * math.pi * (kx * x + ky * y + kz * z) + phi)
            rho += drho
            p += cs * cs * drho
            u += kx / norm * cs * drho
            v += ky / norm * cs * drho
            w += kz / norm * cs * drho
    return prim_to_cons((rho, u, v, w, p), gamma).astype(dtype)


def entropy_wave(shape, direction=(1, 1, 1), amp=0.2, vel=1.0, t=0.0):
    """Exact advected density wave rho = 1 + amp sin(2 pi (k.(x - v t))),
    v = vel * k (component-wise), p = 1, returned as primitives (5, nz, ny, nx)
    sampled at cell centres (use for initial data; averages come from GL)."""
    nz, ny, nx = shape
    kx, ky, kz = direction
    z = centres(nz)[:, None, None]
    y = centres(ny)[None, :, None]
    x = centres(nx)[None, None, :]
    phase = kx * (x - vel * kx * t) + ky * (y - vel * ky * t) + kz * (z - vel * kz * t)
    full = (nz, ny, nx)
    rho = np.broadcast_to(1.0 + amp * np.sin(2.0 * math.pi * phase), full)
    return np.stack([rho, np.full(full, vel * kx), np.full(full, vel * ky),
                     np.full(full, vel * kz), np.ones(full)])


# --------------------------------------------------------------------------
# Spherical blast (3D) and 2D shear layer
# --------------------------------------------------------------------------

def blast_3d(n, seed=0, gamma=1.4, noise=True, e_total=1.0, radius_cells=4.0, p_amb=1e-5,
             dtype=np.float64, planes=None):
    """Ambient rho = 1 (+-1% seeded uniform noise), p = 1e-5, v = 0.  Total
    energy e_total spread equally over the cells whose centre lies within
    radius_cells * dx of the centre (0.5, 0.5, 0.5), added to the ambient
    internal energy.  ``planes=(k0, k1)`` returns only the z planes k0..k1-1
    of the same n^3 state (same noise, same energy density)."""
    x = centres(n)
    dx = 1.0 / n
    k0, k1 = (0, n) if planes is None else (int(planes[0]), int(planes[1]))
    nzs = k1 - k0
    rho = np.ones((nzs, n, n))
    if noise:
        # the generator's draws for the whole cube in z-plane order: planes
        # k0..k1-1 are the draws k0*n*n .. k1*n*n - 1
        g = _rng(seed)
        if k0:
            g.uniform(-1.0, 1.0, size=k0 * n * n)
        rho += 0.01 * g.uniform(-1.0, 1.0, size=(nzs, n, n))
    z = x[k0:k1]
    r2 = ((z[:, None, None] - 0.5) ** 2 + (x[None, :, None] - 0.5) ** 2
          + (x[None, None, :] - 0.5) ** 2)
    lim = (radius_cells * dx) ** 2 * (1.0 + 1e-12)
    inside = r2 <= lim
    if planes is None:
        n_in = int(inside.sum())
    else:
        # cells inside the sphere over the whole cube, plane by plane
        rxy = (x[:, None] - 0.5) ** 2 + (x[None, :] - 0.5) ** 2
        n_in = sum(int(np.count_nonzero((zz - 0.5) ** 2 + rxy <= lim)) for zz in x)
    zero = np.zeros((nzs, n, n))
    U = prim_to_cons((rho, zero, zero, zero, np.full((nzs, n, n), p_amb)), gamma)
    U[4] += np.where(inside, e_total / (n_in * dx ** 3), 0.0)
    return U.astype(dtype)


def shear_2d(n, seed=0, gamma=1.4, amp=0.01):
    """rho = 2 in |y - 0.5| < 0.25 else 1, u = +0.5 inside / -0.5 outside,
    p = 2.5, v = amp * sum_{m=1..4} a_m sin(2 pi m x + phi_m), a_m ~ U[-1, 1].
    Shape (5, 1, n, n)."""
    g = _rng(seed)
    a = g.uniform(-1.0, 1.0, size=4)
    phi = g.uniform(0.0, 2.0 * math.pi, size=4)
    x = centres(n)[None, :]
    y = centres(n)[:, None]
    inside = np.abs(y - 0.5) < 0.25
    rho = np.where(inside, 2.0, 1.0) * np.ones((n, n))
    u = np.where(inside, 0.5, -0.5) * np.ones((n, n))
    v = amp * sum(a[m] * np.sin(2.0 * math.pi * (m + 1) * x + phi[m]) for m in range(4))
    v = v * np.ones((n, n))
    U = prim_to_cons((rho, u, v, np.zeros((n, n)), np.full((n, n), 2.5)), gamma)
    return U.reshape(5, 1, n, n)


def shear_target(n, seed=0):
    """Target density of the shear-layer loss: 1.5 + 0.1 * (seeded sum of
    Fourier modes 1..4 in x and y).  Shape (1, n, n)."""
    g = _rng(seed + 7919)
    x = centres(n)[None, :]
    y = centres(n)[:, None]
    f = np.zeros((n, n))
    for m in range(1, 5):
        a, b = g.uniform(-1.0, 1.0, size=2)
        px, py = g.uniform(0.0, 2.0 * math.pi, size=2)
        f += 0.25 * (a * np.sin(2.0 * math.pi * m * x + px) + b * np.sin(2.0 * math.pi * m * y + py))
    return (1.5 + 0.1 * f).reshape(1, n, n)


# --------------------------------------------------------------------------
# Batch of independent small problems
# --------------------------------------------------------------------------

@dataclass
class BatchSpec:
    nx: np.ndarray
    ny: np.ndarray
    gamma: np.ndarray
    kind: np.ndarray          # 0 = two-state along x, 1 = four quadrants (2D)
    states: list = field(default_factory=list)   # per problem: list of (rho,u,v,p)

    @property
    def nprob(self):
        return int(self.nx.size)

    @property
    def cells(self):
        return self.nx.astype(np.int64) * self.ny.astype(np.int64)


def batch_spec(nprob=4096, seed=0, gamma=1.4, n1d=(64, 4096), n2d=(32, 256)):
    """Half 1D problems (n ~ U{64..4096}), half 2D square (side ~ U{32..256}).
    1D: two states split at x = 0.5.  2D: four quadrants split at (0.5, 0.5).
    rho, p log-uniform in [0.1, 10]; velocity components uniform in [-1, 1]."""
    g = _rng(seed)
    n_1d = nprob // 2
    nx = np.empty(nprob, dtype=np.int32)
    ny = np.empty(nprob, dtype=np.int32)
    kind = np.empty(nprob, dtype=np.int32)
    nx[:n_1d] = g.integers(n1d[0], n1d[1] + 1, size=n_1d)
    ny[:n_1d] = 1
    kind[:n_1d] = 0
    side = g.integers(n2d[0], n2d[1] + 1, size=nprob - n_1d)
    nx[n_1d:] = side
    ny[n_1d:] = side
    kind[n_1d:] = 1
    states = []
    for q in range(nprob):
        nstate = 2 if kind[q] == 0 else 4
        rho = np.exp(g.uniform(math.log(0.1), math.log(10.0), size=nstate))
        p = np.exp(g.uniform(math.log(0.1), math.log(10.0), size=nstate))
        u = g.uniform(-1.0, 1.0, size=nstate)
        v = g.uniform(-1.0, 1.0, size=nstate) if kind[q] == 1 else np.zeros(nstate)
        states.append([(rho[s], u[s], v[s], p[s]) for s in range(nstate)])
    return BatchSpec(nx, ny, np.full(nprob, gamma), kind, states)


def batch_problem_U(spec: BatchSpec, q: int):
    """Conserved initial state of problem q, shape (5, 1, ny, nx)."""
    nx, ny, gamma = int(spec.nx[q]), int(spec.ny[q]), float(spec.gamma[q])
    x = centres(nx)[None, :]
    y = centres(ny)[:, None]
    st = spec.states[q]
    if spec.kind[q] == 0:
        sel = np.where(x <= 0.5, 0, 1) * np.ones((ny, nx), dtype=np.int64)
    else:
        sel = (np.where(x <= 0.5, 0, 1) + 2 * np.where(y <= 0.5, 0, 1)) * np.ones((ny, nx), dtype=np.int64)
    arr = np.array(st)                                  # (nstate, 4)
    rho, u, v, p = (arr[sel, c] for c in range(4))
    U = prim_to_cons((rho, u, v, np.zeros_like(rho), p), gamma)
    return U.reshape(5, 1, ny, nx)


# --------------------------------------------------------------------------
# Radiative heating / cooling (Sec. 3.2), CGS units
# --------------------------------------------------------------------------

C_LIGHT = 2.99792458e10              # cm / s
K_BOLTZMANN = 1.380649e-16           # erg / K
M_U = 1.66053906660e-24              # g (atomic mass unit)
SIGMA_SB = 5.670374419e-5            # erg / (cm^2 s K^4)
A_RAD = 4.0 * SIGMA_SB / C_LIGHT     # radiation constant a = 4 sigma / c


@dataclass
class HeatingCooling:
    """Sec. 3.2: rho = 1e-7 g/cm^3, mu = 0.6, kappa = 0.4 cm^2/g, a uniform
    radiation field at T_r = 3.4e6 K and a fluid at T_f = 11 K (heating) or
    1.1e9 K (cooling).  gamma = 5/3 (monatomic ideal gas; the paper does not
    print it)."""
    T_fluid: float
    rho: float = 1e-7
    mu: float = 0.6
    kappa: float = 0.4
    T_rad: float = 3.4e6
    gamma: float = 5.0 / 3.0

    @property
    def cv(self):
        """Specific heat per unit mass, k_B / ((gamma - 1) mu m_u)."""
        return K_BOLTZMANN / ((self.gamma - 1.0) * self.mu * M_U)

    @property
    def params(self):
        """(c, kappa, a, c_v) of the exchange."""
        return (C_LIGHT, self.kappa, A_RAD, self.cv)

    def state(self, shape=(1, 1, 1), seed=None, spread=0.0):
        """Fluid at rest (U, 5 x shape) and radiation energy density Er (shape).
        With a seed, rho, T_f and T_r vary cell by cell by a log-uniform
        factor in [1/(1+spread), 1+spread] and the fluid moves at up to
        1e5 cm/s."""
        shape = tuple(shape)
        rho = np.full(shape, self.rho)
        Tf = np.full(shape, self.T_fluid)
        Tr = np.full(shape, self.T_rad)
        vel = np.zeros((3,) + shape)
        if seed is not None:
            g = _rng(seed)
            s = math.log1p(spread)
            rho = rho * np.exp(g.uniform(-s, s, shape))
            Tf = Tf * np.exp(g.uniform(-s, s, shape))
            Tr = Tr * np.exp(g.uniform(-s, s, shape))
            vel = g.uniform(-1e5, 1e5, (3,) + shape)
        e = rho * self.cv * Tf
        U = np.stack([rho, rho * vel[0], rho * vel[1], rho * vel[2],
                      e + 0.5 * rho * np.sum(vel * vel, axis=0)])
        return U, A_RAD * Tr ** 4


def heating():
    return HeatingCooling(T_fluid=11.0)


def cooling():
    return HeatingCooling(T_fluid=1.1e9)
