"""Pins for the oracle's spectra, normalisation and windowed ARPACK solver."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, partition, stencil


def _dense(w):
    return stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)


@pytest.fixture(scope="module")
def small_wire():
    w = W.make_wire(6, 6, 12, 0.5, 3, 7)
    A = _dense(w)
    eps, U = eigen.dense_spectrum(A)
    return w, A, eps, U


def test_bilinear_orthonormal_and_residuals(small_wire):
    w, A, eps, U = small_wire
    np.testing.assert_allclose(U.T @ U, np.eye(w.N), atol=1e-10)
    r = eigen.residual_norms(lambda X: A @ X, eps, U)
    assert r.max() < 1e-11 * stencil.gershgorin_norm(w.h, w.V, w.gamma_L, w.gamma_R)


def test_imaginary_parts_bounded_by_absorber(small_wire):
    # Eq. (5): 0 <= -Im eps <= max Gamma.  Exactly, for an eigenvector u of
    # H - i Gamma with H real symmetric, Im eps = -u^H Gamma u / u^H u.
    w, A, eps, U = small_wire
    g = w.gamma_L + w.gamma_R
    assert np.all(eps.imag <= 1e-12) and np.all(-eps.imag <= g.max() + 1e-12)
    rq = -np.einsum("rk,r,rk->k", U.conj(), g, U).real / np.einsum("rk,rk->k", U.conj(), U).real
    np.testing.assert_allclose(eps.imag, rq, atol=1e-11)


def test_separable_spectrum_with_absorbers():
    # V and Gamma depend on z only: A = Tx + Ty + Az, so each eigenvalue is
    # lambda_x + lambda_y + mu_z with mu_z from the 1D complex-symmetric problem.
    w = W.separable_wire(5, 6, 14, 0.5, 3, 2)
    A = _dense(w)
    ev = np.linalg.eigvals(A)
    h = w.h
    Tx = -0.5 / h ** 2 * stencil.second_difference_1d(w.nx)
    Ty = -0.5 / h ** 2 * stencil.second_difference_1d(w.ny)
    plane = w.nx * w.ny
    vz = w.V[::plane]
    gz = (w.gamma_L + w.gamma_R)[::plane]
    Az = -0.5 / h ** 2 * stencil.second_difference_1d(w.nz) + np.diag(vz - 1j * gz)
    mu = np.linalg.eigvals(Az)
    lam = np.add.outer(np.add.outer(mu, np.linalg.eigvalsh(Ty)), np.linalg.eigvalsh(Tx)).reshape(-1)
    a = np.sort_complex(np.round(ev, 9))
    b = np.sort_complex(np.round(lam, 9))
    np.testing.assert_allclose(np.sort(ev.real), np.sort(lam.real), atol=1e-10)
    np.testing.assert_allclose(np.sort(ev.imag), np.sort(lam.imag), atol=1e-10)
    assert a.shape == b.shape


def test_degenerate_cluster_normalisation_matches_eigh():
    # V = Gamma = 0 on a cube: a real symmetric problem with exact degeneracies.
    # The cluster projectors sum_k U_k U_k^T are basis-independent and must match
    # those from the Hermitian solver.
    n, h = 6, 0.5
    zero = np.zeros(n ** 3)
    A = stencil.dense_A(n, n, n, h, zero, zero, zero).astype(np.complex128)
    eps, U = eigen.dense_spectrum(A)
    np.testing.assert_allclose(U.T @ U, np.eye(n ** 3), atol=1e-9)
    lam, Q = np.linalg.eigh(A.real)
    for g in eigen.clusters(eps, 1e-9):
        if len(g) < 2:
            continue
        P = eigen.cluster_projector(U, g)
        Pq = Q[:, g] @ Q[:, g].T
        np.testing.assert_allclose(P, Pq, atol=1e-8)


@pytest.mark.slow
def test_arpack_windows_union_equals_dense_lowest():
    # Eq. (3) + Eq. (4) + Algorithm 2: windows of Algorithm 1 sizes, shifts at the
    # middle of each run of the known spectrum (the paper's own placement with
    # foreknowledge, Section 3), requests inflated by 10%, merged.
    w = W.make_wire(6, 6, 16, 0.5, 4, 3)
    A = _dense(w)
    eps, U = eigen.dense_spectrum(A)
    n_r, p = 24, 4
    counts = partition.window_counts(n_r, p)
    sig, req = W.count_windows(eps.real[:n_r], counts)
    e_list, u_list = [], []
    for s, r in zip(sig, req):
        e, V = eigen.arpack_window(w, float(s), int(r), tol=1e-13, seed=1)
        e_list.append(e)
        u_list.append(V)
    e_all, U_all, _, holes = partition.combine(e_list, u_list)
    e_sel, U_sel = eigen.lowest_by_real(e_all, U_all, n_r)
    np.testing.assert_allclose(e_sel, eps[:n_r], rtol=0, atol=1e-10)
    assert not any(holes)
    # Degenerate partners (x <-> y symmetry of the wire) are compared through
    # cluster projectors sum_k U_k U_k^T, which do not depend on the basis.
    for g in eigen.clusters(eps[:n_r], 1e-9):
        P_dense = eigen.cluster_projector(U, g)
        P_win = eigen.cluster_projector(U_sel, g)
        np.testing.assert_allclose(P_win, P_dense, atol=1e-8)


def test_arpack_complex_shift_windows_are_the_nearest_eigenvalues():
    # Section 2's complex shifts: ARPACK 'SM' on A - sigma for sigma off the
    # real axis returns the eigenvalues nearest sigma in the complex plane,
    # which on a 20-bohr wire (the absorbers cover only its ends, so -Im eps
    # spreads over [0, 0.33]) differ between a shift near the axis and one
    # below it at the same real part
    w = W.make_wire(6, 6, 40, 0.5, 6, 3)
    eps, U = eigen.dense_spectrum(_dense(w))
    sets = []
    for s in (1.2 - 0.3j, 1.2 - 0.01j):
        idx = partition.complex_shift_window(eps, s, 6)
        d = np.sort(np.abs(eps - s))
        assert d[6] - d[5] > 0.1 * d[5]  # a clear cut
        e, V = eigen.arpack_window(w, s, 6, tol=1e-13, seed=1)
        np.testing.assert_allclose(np.sort_complex(e), np.sort_complex(eps[idx]), atol=1e-10)
        sets.append(set(int(i) for i in idx))
    assert sets[0] != sets[1]
