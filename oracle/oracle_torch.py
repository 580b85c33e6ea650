"""Small-size PyTorch FP64 transcription of the stage update, for autograd.

TEST INFRASTRUCTURE (see the package docstring).  The same scheme as
hard_oracle.c, written with torch operations on whole arrays so that
torch.autograd yields the reference gradient of a rollout with respect to the
initial state and to gamma.  Branches (minmod, Davis min/max, the HLLC
regions) are torch.where selections, so the gradient follows the branch the
forward pass took (the subgradient convention of the adjoint kernels).
Denominators of branches that are not selected are made safe, so no NaN or
inf reaches the gradient of a selected branch.

Pinned against the C oracle (tests/test_oracle_torch.py): forward values to
1e-13, and torch.autograd.gradcheck on tiny meshes.
"""
from __future__ import annotations

import torch

from . import BC_OUTFLOW, BC_PERIODIC, BC_REFLECT

ROT = ((1, 2, 3), (2, 1, 3), (3, 1, 2))      # normal, tangent 1, tangent 2 per axis


def ghost_map(n, bc_lo, bc_hi):
    """Source index and momentum sign of m in [-2, n+1] (the C oracle's map)."""
    idx, sign = [], []
    for m in range(-2, n + 2):
        if 0 <= m < n:
            idx.append(m); sign.append(1.0); continue
        bc = bc_lo if m < 0 else bc_hi
        if bc == BC_PERIODIC:
            idx.append(m % n); sign.append(1.0)
        elif bc == BC_OUTFLOW:
            idx.append(0 if m < 0 else n - 1); sign.append(1.0)
        else:
            idx.append(-1 - m if m < 0 else 2 * n - 1 - m); sign.append(-1.0)
    return torch.tensor(idx), torch.tensor(sign, dtype=torch.float64)


def prim(U, gamma):
    rho = U[0]
    u, v, w = U[1] / rho, U[2] / rho, U[3] / rho
    kin = 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, u, v, w, (gamma - 1.0) * (U[4] - kin)])


def minmod(a, b):
    same = ((a > 0) & (b > 0)) | ((a < 0) & (b < 0))
    pick = torch.where(a.abs() <= b.abs(), a, b)
    return torch.where(same, pick, torch.zeros_like(a))


def normal_flux(W, gamma):
    rho, un, t1, t2, p = W
    E = p / (gamma - 1.0) + 0.5 * rho * (un * un + t1 * t1 + t2 * t2)
    U = torch.stack([rho, rho * un, rho * t1, rho * t2, E])
    F = torch.stack([rho * un, rho * un * un + p, rho * un * t1, rho * un * t2, (E + p) * un])
    return U, F


def hllc(WL, WR, gamma):
    UL, FL = normal_flux(WL, gamma)
    UR, FR = normal_flux(WR, gamma)
    rL, uL, pL = WL[0], WL[1], WL[4]
    rR, uR, pR = WR[0], WR[1], WR[4]
    cL = torch.sqrt(gamma * pL / rL)
    cR = torch.sqrt(gamma * pR / rR)
    SL = torch.minimum(uL - cL, uR - cR)
    SR = torch.maximum(uL + cL, uR + cR)
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))
    left = Ss >= 0
    W = torch.where(left, WL, WR)
    UK = torch.where(left, UL, UR)
    FK = torch.where(left, FL, FR)
    SK = torch.where(left, SL, SR)
    r, u, p = W[0], W[1], W[4]
    sub = (SL < 0) & (SR > 0)                   # the star regions
    one = torch.ones_like(SK)
    den = torch.where(sub, SK - Ss, one)
    m = torch.where(sub, r * (SK - u), one)
    fac = r * (SK - u) / den
    Us = torch.stack([fac, fac * Ss, fac * W[2], fac * W[3],
                      fac * (UK[4] / r + (Ss - u) * (Ss + p / m))])
    Fstar = FK + SK * (Us - UK)
    F = torch.where(SL >= 0, FL, torch.where(SR <= 0, FR, Fstar))
    return F


def rhs(U, gamma, dxyz, bc6):
    """L(U) = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d over the active axes."""
    _, nz, ny, nx = U.shape
    n = (nx, ny, nz)
    L = torch.zeros_like(U)
    for d in range(3):
        if n[d] <= 1:
            continue
        dim = 3 - d                              # tensor dim of axis d
        idx, sign = ghost_map(n[d], bc6[2 * d], bc6[2 * d + 1])
        P = U.index_select(dim, idx)             # 2 ghost layers each side
        bshape = [1, 1, 1]
        bshape[dim - 1] = idx.numel()
        flip = torch.ones((5, *bshape), dtype=U.dtype)
        flip[1 + d] = sign.view(bshape)          # reflecting walls negate the normal momentum
        P = P * flip
        W = prim(P, gamma)
        q = [W.narrow(dim, k, n[d] + 1) for k in range(4)]   # cells m-2 .. m+1 around face m
        qL = q[1] + 0.5 * minmod(q[1] - q[0], q[2] - q[1])
        qR = q[2] - 0.5 * minmod(q[2] - q[1], q[3] - q[2])
        r = ROT[d]
        order = [0, r[0], r[1], r[2], 4]
        Fn = hllc(qL[order], qR[order], gamma)
        F = torch.empty_like(Fn)
        F[0], F[r[0]], F[r[1]], F[r[2]], F[4] = Fn[0], Fn[1], Fn[2], Fn[3], Fn[4]
        L = L - (F.narrow(dim, 1, n[d]) - F.narrow(dim, 0, n[d])) / dxyz[d]
    return L


def step(U, gamma, dt, dxyz, bc6):
    """One Shu-Osher (Heun) step with a fixed dt."""
    U1 = U + dt * rhs(U, gamma, dxyz, bc6)
    return 0.5 * U + 0.5 * (U1 + dt * rhs(U1, gamma, dxyz, bc6))


def rollout(U0, gamma, dts, dxyz, bc6):
    U = U0
    for dt in dts:
        U = step(U, gamma, float(dt), dxyz, bc6)
    return U
