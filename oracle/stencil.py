"""The operator A = H_KS - i Gamma (Eq. (1)) as a plain FP64 stencil and a dense matrix.

H_KS is represented only as a matrix-vector product formula, never stored
(Section 1): a real-space finite-difference kinetic term -1/2 nabla^2 plus a
local potential V(r).  The paper does not state the finite-difference order;
this build uses the 12th-order (radius-6) central second derivative.  Gamma =
Gamma_L + Gamma_R is diagonal, real and non-negative (Section 1).

Boundary condition (the paper is silent): odd reflection, i.e. psi = 0 on the
planes just outside the grid (index -1 and n) with ghost values
``u[-1-k] = -u[-1+k]`` and ``u[n+k] = -u[n-k]``.  ``bc=1`` is plain zero
padding (every ghost is 0).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

RADIUS = 6
BC_ODD = 0
BC_ZERO = 1


def fd2_coefficients_exact(radius: int = RADIUS):
    """Central second-derivative weights c_0..c_R as exact rationals.

    c_m = 2 (-1)^(m+1) (R!)^2 / (m^2 (R-m)! (R+m)!) for m >= 1 and
    c_0 = -2 sum_{m>=1} 1/m^2 (the closed form of the order-2R central
    difference, e.g. Fornberg 1988).
    """
    R = radius
    c = [Fraction(0)] * (R + 1)
    for m in range(1, R + 1):
        c[m] = Fraction(2 * (-1) ** (m + 1) * factorial(R) ** 2,
                        m * m * factorial(R - m) * factorial(R + m))
    c[0] = -2 * sum(Fraction(1, m * m) for m in range(1, R + 1))
    return c


def fd2_coefficients(radius: int = RADIUS) -> np.ndarray:
    return np.array([float(x) for x in fd2_coefficients_exact(radius)])


def ghost_index(j: int, n: int, bc: int):
    """Map a (possibly out-of-range) 1D index to (source index, sign) or None."""
    if 0 <= j < n:
        return j, 1.0
    if bc == BC_ZERO:
        return None
    if j == -1 or j == n:
        return None
    if j <= -2:
        return -2 - j, -1.0
    return 2 * n - j, -1.0


def second_difference_1d(n: int, bc: int = BC_ODD, radius: int = RADIUS) -> np.ndarray:
    """Dense n x n matrix of sum_m c_|m| u[i+m] with the chosen ghost rule (no 1/h^2)."""
    if n < radius - 1:
        raise ValueError("each axis needs at least radius-1 points for a single reflection")
    c = fd2_coefficients(radius)
    D = np.zeros((n, n))
    for i in range(n):
        for m in range(-radius, radius + 1):
            g = ghost_index(i + m, n, bc)
            if g is not None:
                src, sgn = g
                D[i, src] += sgn * c[abs(m)]
    return D


def diagonal(V, gamma_L, gamma_R) -> np.ndarray:
    """Local part of A: V(r) - i (Gamma_L + Gamma_R)(r) (Eq. (1))."""
    return np.asarray(V, dtype=np.float64) - 1j * (np.asarray(gamma_L, dtype=np.float64)
                                                   + np.asarray(gamma_R, dtype=np.float64))


def apply_A(u: np.ndarray, nx: int, ny: int, nz: int, h: float, V, gamma_L, gamma_R,
            sigma: float = 0.0, bc: int = BC_ODD) -> np.ndarray:
    """(A - sigma) u for one vector (length N) or a block (N x b), ghost-padded.

    The field is padded by ``radius`` ghost planes on each face (filled by the
    boundary rule), then the 13-point line stencil is summed along each axis.
    """
    u = np.asarray(u)
    single = u.ndim == 1
    U = u.reshape(nz, ny, nx, -1).astype(np.complex128)
    c = fd2_coefficients()
    R = RADIUS
    lap = np.zeros_like(U)
    for axis, n in ((0, nz), (1, ny), (2, nx)):
        src = np.moveaxis(U, axis, 0)
        pad = np.zeros((n + 2 * R,) + src.shape[1:], dtype=np.complex128)
        for jj in range(-R, n + R):
            g = ghost_index(jj, n, bc)
            if g is not None:
                pad[jj + R] = g[1] * src[g[0]]
        acc = np.zeros_like(src)
        for m in range(-R, R + 1):
            acc += c[abs(m)] * pad[R + m:R + m + n]
        lap += np.moveaxis(acc, 0, axis)
    d = diagonal(V, gamma_L, gamma_R).reshape(nz, ny, nx, 1)
    out = -0.5 / (h * h) * lap + (d - sigma) * U
    out = out.reshape(nx * ny * nz, -1)
    return out[:, 0] if single else out


def dense_A(nx: int, ny: int, nz: int, h: float, V, gamma_L, gamma_R, bc: int = BC_ODD) -> np.ndarray:
    """Dense complex-symmetric A as a Kronecker sum (x fastest in the flat index)."""
    Dx = second_difference_1d(nx, bc)
    Dy = second_difference_1d(ny, bc)
    Dz = second_difference_1d(nz, bc)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    L = (np.kron(Iz, np.kron(Iy, Dx)) + np.kron(Iz, np.kron(Dy, Ix)) + np.kron(Dz, np.kron(Iy, Ix)))
    return (-0.5 / (h * h)) * L + np.diag(diagonal(V, gamma_L, gamma_R))


def laplacian_box_eigenvalues(nx: int, ny: int, nz: int, h: float) -> np.ndarray:
    """All eigenvalues of -1/2 nabla^2_FD on the odd-reflection box (V = Gamma = 0).

    With odd reflection the sine modes sin(pi q (i+1)/(n+1)) are exact
    eigenvectors of the 1D stencil, with symbol c_0 + 2 sum_m c_m cos(m pi q/(n+1)).
    """
    c = fd2_coefficients()

    def axis(n):
        q = np.arange(1, n + 1)
        th = np.pi * q / (n + 1)
        s = c[0] + 2.0 * sum(c[m] * np.cos(m * th) for m in range(1, RADIUS + 1))
        return -0.5 / (h * h) * s

    ex, ey, ez = axis(nx), axis(ny), axis(nz)
    lam = (ez[:, None, None] + ey[None, :, None] + ex[None, None, :]).reshape(-1)
    return np.sort(lam)


def gershgorin_norm(h: float, V, gamma_L, gamma_R) -> float:
    """Gershgorin bound on |A|: 3 axes x (1/2h^2) sum_m |c_m| + max|V| + max Gamma.

    This is the scale of the relative-residual test ||A u - eps u|| / (||A||_G ||u||).
    """
    c = fd2_coefficients()
    kin = 3 * 0.5 / (h * h) * (abs(c[0]) + 2 * np.sum(np.abs(c[1:])))
    return float(kin + np.max(np.abs(V)) + np.max(np.asarray(gamma_L) + np.asarray(gamma_R)))
