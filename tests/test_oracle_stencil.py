"""Pins of the oracle's finite-difference stencils (isotropic 9-point gradient and
Laplacian) against closed forms: the discrete Fourier symbols of the stencils on
periodic sinusoids, exactness on quadratic polynomials, and the zero-gradient
ghost at a wall."""
import numpy as np

import oracle
from paper_2603_22902_gb300 import workloads as W


def _case(nx, ny, bc):
    c = W.Case(name="st", nx=nx, ny=ny, N=2, phases=[W.phase(), W.phase()], sigma=np.zeros((2, 2)))
    c.bc = bc
    return c


def test_periodic_sinusoid_symbols():
    nx, ny = 24, 16
    k, l = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    chi = np.sin(k * X) * np.sin(l * Y)
    gx, gy, lap = oracle.stencil(_case(nx, ny, (0, 0, 0, 0)), chi)
    # symbols of sum_i w_i c_i chi(x + c_i) / c_s^2 and sum_i 2 w_i (chi(x + c_i) - chi) / c_s^2
    gx_ref = np.sin(k) * np.cos(k * X) * np.sin(l * Y) * (2.0 / 3.0 + np.cos(l) / 3.0)
    gy_ref = np.sin(l) * np.sin(k * X) * np.cos(l * Y) * (2.0 / 3.0 + np.cos(k) / 3.0)
    lap_ref = (4.0 / 3.0 * (np.cos(k) + np.cos(l) - 2.0) + 2.0 / 3.0 * (np.cos(k) * np.cos(l) - 1.0)) * chi
    assert np.abs(gx - gx_ref).max() < 1e-14
    assert np.abs(gy - gy_ref).max() < 1e-14
    assert np.abs(lap - lap_ref).max() < 1e-14


def test_exact_on_quadratics_interior():
    nx, ny = 9, 7
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    a, b, c2, d, e = 0.3, -0.7, 0.45, 1.1, -0.2
    chi = a * X ** 2 + b * X * Y + c2 * Y ** 2 + d * X + e * Y
    gx, gy, lap = oracle.stencil(_case(nx, ny, (1, 1, 1, 1)), chi)
    inner = (slice(1, -1), slice(1, -1))
    assert np.abs(gx[inner] - (2 * a * X + b * Y + d)[inner]).max() < 1e-12
    assert np.abs(gy[inner] - (b * X + 2 * c2 * Y + e)[inner]).max() < 1e-12
    assert np.abs(lap[inner] - (2 * a + 2 * c2)).max() < 1e-12


def test_wall_ghost_is_zero_gradient():
    nx, ny = 6, 8
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    gx, gy, lap = oracle.stencil(_case(nx, ny, (0, 0, 1, 2)), Y.copy())
    # interior: exact slope 1; boundary rows see a copied ghost: half the slope
    assert np.allclose(gy[1:-1], 1.0, atol=1e-14)
    assert np.allclose(gy[0], 0.5, atol=1e-14) and np.allclose(gy[-1], 0.5, atol=1e-14)
    assert np.allclose(gx, 0.0, atol=1e-14)
    # Laplacian of y at a boundary row: only the three inward neighbours differ by 1:
    # 6 (1/9 + 2/36) = 1
    assert np.allclose(lap[0], 1.0, atol=1e-14) and np.allclose(lap[-1], -1.0, atol=1e-14)
