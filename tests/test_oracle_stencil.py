"""Pins for the oracle's operator (Eq. (1)): coefficients, boundary rule, assembly."""
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import stencil
from conftest import golden_path


def _golden_coefficients():
    vals = []
    with open(golden_path("fd12_second_derivative.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(Fraction(line))
    return vals


def test_coefficients_match_textbook_table():
    assert stencil.fd2_coefficients_exact() == _golden_coefficients()


def test_coefficients_moment_conditions():
    # sum_m c_|m| m^(2k) over m = -6..6 is 2 for k = 1 (exact on x^2) and 0 for
    # k = 0, 2..6 (exact on every polynomial up to degree 13).
    c = stencil.fd2_coefficients_exact()
    for k in range(0, 7):
        s = c[0] * (1 if k == 0 else 0) + 2 * sum(c[m] * Fraction(m) ** (2 * k) for m in range(1, 7))
        assert s == (2 if k == 1 else 0), k


@pytest.mark.parametrize("n", [6, 7, 13, 20])
def test_odd_reflection_sine_modes(n):
    # With odd reflection the discrete sine modes are exact eigenvectors of the
    # 1D operator; any other ghost rule breaks this.
    D = stencil.second_difference_1d(n, stencil.BC_ODD)
    c = [float(x) for x in _golden_coefficients()]
    i = np.arange(n)
    for q in range(1, n + 1):
        s = np.sin(np.pi * q * (i + 1) / (n + 1))
        lam = c[0] + 2 * sum(c[m] * np.cos(m * np.pi * q / (n + 1)) for m in range(1, 7))
        np.testing.assert_allclose(D @ s, lam * s, atol=1e-12)


def test_matvec_sine_mode_3d():
    # The ghost-padded 3D matvec maps a product of sine modes to its eigenvalue
    # (V = Gamma = 0); pins the padding, the axis order and the -1/(2h^2) scale.
    nx, ny, nz, h = 7, 9, 11, 0.5
    qx, qy, qz = 2, 5, 3
    x = np.sin(np.pi * qx * (np.arange(nx) + 1) / (nx + 1))
    y = np.sin(np.pi * qy * (np.arange(ny) + 1) / (ny + 1))
    z = np.sin(np.pi * qz * (np.arange(nz) + 1) / (nz + 1))
    u = (z[:, None, None] * y[None, :, None] * x[None, None, :]).reshape(-1)
    c = [float(v) for v in _golden_coefficients()]

    def sym(q, n):
        return c[0] + 2 * sum(c[m] * np.cos(m * np.pi * q / (n + 1)) for m in range(1, 7))

    lam = -0.5 / h ** 2 * (sym(qx, nx) + sym(qy, ny) + sym(qz, nz))
    zero = np.zeros(nx * ny * nz)
    out = stencil.apply_A(u, nx, ny, nz, h, zero, zero, zero)
    np.testing.assert_allclose(out, lam * u, atol=1e-12)


def test_box_closed_form_spectrum():
    nx, ny, nz, h = 6, 7, 9, 0.5
    zero = np.zeros(nx * ny * nz)
    A = stencil.dense_A(nx, ny, nz, h, zero, zero, zero)
    ev = np.linalg.eigvalsh(A.real)
    np.testing.assert_allclose(ev, stencil.laplacian_box_eigenvalues(nx, ny, nz, h), atol=1e-12)


def test_dense_is_complex_symmetric_bitwise_and_sign_of_absorber():
    w = W.make_wire(7, 6, 9, 0.5, 3, 11)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    assert np.array_equal(A, A.T)
    # A = H - i Gamma: the imaginary part is exactly -diag(Gamma), Eq. (1).
    assert np.array_equal(A.imag, -np.diag(w.gamma_L + w.gamma_R))


def test_matvec_equals_dense_block():
    w = W.make_wire(8, 7, 10, 0.5, 4, 3)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((w.N, 5)) + 1j * rng.standard_normal((w.N, 5))
    for sigma in (0.0, -0.7, 1.3):
        Y = stencil.apply_A(X, w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R, sigma=sigma)
        np.testing.assert_allclose(Y, A @ X - sigma * X, rtol=0, atol=1e-12)


def test_zero_padding_is_separable():
    # bc=1: A is a Kronecker sum, so 3D eigenvalues are sums of the 1D ones.
    nx, ny, nz, h = 5, 6, 7, 0.5
    zero = np.zeros(nx * ny * nz)
    A = stencil.dense_A(nx, ny, nz, h, zero, zero, zero, bc=stencil.BC_ZERO)
    # 1D zero-padded operators built independently as banded Toeplitz matrices.
    c = [float(v) for v in _golden_coefficients()]

    def toeplitz(n):
        T = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                if abs(i - j) <= 6:
                    T[i, j] = c[abs(i - j)]
        return -0.5 / h ** 2 * np.linalg.eigvalsh(T)

    s = np.add.outer(np.add.outer(toeplitz(nz), toeplitz(ny)), toeplitz(nx)).reshape(-1)
    np.testing.assert_allclose(np.linalg.eigvalsh(A.real), np.sort(s), atol=1e-11)


def test_gershgorin_bounds_spectrum():
    w = W.make_wire(6, 6, 8, 0.5, 3, 5)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    g = stencil.gershgorin_norm(w.h, w.V, w.gamma_L, w.gamma_R)
    assert np.max(np.abs(np.linalg.eigvals(A))) <= g
    assert g >= np.max(np.sum(np.abs(A), axis=1)) - 1e-12
