"""Pins of the oracle's flux-limited diffusion step (Sec. 2.2.1-2.2.2):
limiter limits, the discrete operator's closed-form eigenvalues, conservation,
the maximum principle and the exactness of the gradient on linear data."""
import importlib.util
import os

import numpy as np
import pytest

pytest.importorskip("scipy.sparse")


def _fld():
    """The oracle module, or a planted copy when HARD_FLD_PATH names one."""
    path = os.environ.get("HARD_FLD_PATH")
    if not path:
        from oracle import fld
        return fld
    spec = importlib.util.spec_from_file_location("fld_planted", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


F = _fld()


def test_limiter_limits():
    """Optically thick: lambda -> 1/3 (Eddington); thin: lambda R -> 1 (the flux
    |F| = lambda c |grad E| / (kappa rho) tends to c E); monotone in between."""
    assert F.flux_limiter(0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    for R in (1e6, 1e9):
        assert F.flux_limiter(R) * R == pytest.approx(1.0, rel=2.0 / R)
    R = np.logspace(-6, 6, 200)
    assert np.all(np.diff(F.flux_limiter(R)) < 0)


@pytest.mark.parametrize("shape,bc", [((1, 1, 16), 0), ((1, 12, 10), 0), ((6, 8, 10), 0),
                                      ((5, 7, 9), 1), ((4, 6, 8), 2)])
def test_operator_symmetric_m_matrix(shape, bc):
    rng = np.random.default_rng(1)
    D = 0.5 + rng.random(shape)
    A = F.fld_matrix(D, 0.3, np.array([0.1, 0.2, 0.15]), [bc] * 6).toarray()
    assert np.allclose(A, A.T, rtol=0, atol=1e-15)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    assert np.allclose(A.sum(axis=1), 1.0, rtol=0, atol=1e-13)   # rows sum to the identity part


@pytest.mark.parametrize("shape,k", [((1, 1, 32), (3, 0, 0)), ((1, 16, 24), (2, 5, 0)),
                                     ((8, 12, 16), (1, 2, 3))])
def test_constant_coefficient_fourier_eigenvalue(shape, k):
    """Constant D on a periodic mesh: a Fourier mode is an eigenvector of
    A = I - dt div(D grad) with eigenvalue 1 + dt D sum_d 4 sin^2(pi k_d / n_d) / dx_d^2."""
    nz, ny, nx = shape
    dx = np.array([1.0 / nx, 0.7 / ny, 1.3 / nz])
    D0, dt = 0.37, 0.05
    A = F.fld_matrix(np.full(shape, D0), dt, dx, [0] * 6)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = np.cos(2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz))
    lam = 1.0
    for d, n in enumerate((nx, ny, nz)):
        if n > 1:
            lam += dt * D0 * 4.0 * np.sin(np.pi * k[d] / n) ** 2 / dx[d] ** 2
    assert np.allclose(A @ v.ravel(), lam * v.ravel(), rtol=0, atol=1e-12 * lam)


def _state(shape, seed):
    rng = np.random.default_rng(seed)
    rho = 1e-3 * (0.5 + rng.random(shape))
    E = 1e10 * (1.0 + 0.8 * rng.random(shape))
    return rho, E


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_step_conserves_and_obeys_the_maximum_principle(bc):
    shape = (6, 7, 9)
    rho, E = _state(shape, 2)
    dx = np.array([0.1, 0.1, 0.2])
    E1 = F.fld_step(rho, E, 1e-9, 3e10, 0.4, dx, [bc] * 6)
    assert np.sum(E1) == pytest.approx(np.sum(E), rel=1e-13)
    assert E.min() <= E1.min() and E1.max() <= E.max()
    assert np.std(E1) < np.std(E)                              # it smooths


def test_gradient_exact_on_linear_data():
    """Central differences are exact for E linear in x: in the interior
    D = c lambda(b / (rho kappa E)) / (kappa rho) with b the slope."""
    shape = (3, 4, 10)
    dx = np.array([0.1, 0.1, 0.1])
    x = (np.arange(10) + 0.5) * dx[0]
    b, c, kappa = 2.0e11, 3.0e10, 0.4
    E = np.broadcast_to(1e10 + b * x, shape).copy()
    rho = np.full(shape, 1e-3)
    D = F.diffusion_coefficient(rho, E, c, kappa, dx, [1] * 6)
    R = b / (rho * kappa * E)
    ref = c * F.flux_limiter(R) / (kappa * rho)
    assert np.allclose(D[:, :, 1:-1], ref[:, :, 1:-1], rtol=1e-13)


def test_face_coefficient_is_the_mean_of_its_cells():
    """The reading for the face coefficient: D_{i+1/2} = (D_i + D_{i+1}) / 2,
    so on three cells with zero-flux walls the couplings are
    -dt (D_0 + D_1) / (2 dx^2) and -dt (D_1 + D_2) / (2 dx^2)."""
    D = np.array([1.0, 4.0, 10.0]).reshape(1, 1, 3)
    dx, dt = 0.5, 0.2
    A = F.fld_matrix(D, dt, np.array([dx, 1.0, 1.0]), [1] * 6).toarray()
    w01, w12 = dt * 2.5 / dx ** 2, dt * 7.0 / dx ** 2
    expect = np.array([[1 + w01, -w01, 0.0], [-w01, 1 + w01 + w12, -w12], [0.0, -w12, 1 + w12]])
    assert np.allclose(A, expect, rtol=1e-15, atol=0)
