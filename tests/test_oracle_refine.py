"""Pins for the oracle's residual-correction sweep (Rayleigh-Ritz on span[U_g, R_u])."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, refine, stencil


@pytest.fixture(scope="module")
def wire():
    w = W.make_wire(6, 6, 12, 0.5, 3, 7)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps, U = eigen.dense_spectrum(A)
    an = stencil.gershgorin_norm(w.h, w.V, w.gamma_L, w.gamma_R)
    return w, A, eps, U, an


def test_exact_recovery_from_an_invariant_span(wire):
    # u'_k = u_k + d u_j(k) with j(k) far up the spectrum: span[U', R'] is the
    # invariant subspace of {u_k, u_j(k)}, so one Rayleigh-Ritz step returns the
    # exact pairs (the SM selection keeps the group's own eigenvalues)
    w, A, eps, U, an = wire
    n = 24
    U0 = U[:, :n] + 1e-3 * U[:, 200:200 + n]
    e0 = eps[:n] + 1e-6
    e1, U1, r1, sweeps = refine.refine(lambda X: A @ X, an, e0, U0, 1e-13, max_sweeps=1, group=8)
    assert sweeps == 1 and len(e1) == n
    assert np.max(np.abs(e1 - eps[:n])) < 1e-11
    assert r1.max() < 1e-13
    # same vectors: projectors sum_k u_k u_k^T per cluster of equal eigenvalues
    # (basis- and sign-independent; the 6 x 6 cross-section has degenerate pairs)
    for cl in eigen.clusters(eps[:n], 1e-9):
        P1, P0 = eigen.cluster_projector(U1, cl), eigen.cluster_projector(U[:, :n], cl)
        assert np.max(np.abs(P1 - P0)) < 1e-9 * max(1.0, np.max(np.abs(P0)))
    np.testing.assert_allclose(U1.T @ U1, np.eye(n), atol=1e-10)


def test_converged_pairs_are_a_fixed_point(wire):
    w, A, eps, U, an = wire
    n = 20
    e1, U1, r1, sweeps = refine.refine(lambda X: A @ X, an, eps[:n], U[:, :n], 1e-10, max_sweeps=3, group=8)
    assert sweeps == 0
    np.testing.assert_array_equal(e1, eps[:n])
    # a forced sweep (target below the rounding floor) keeps the same pairs
    e2, U2, r2, sweeps = refine.refine(lambda X: A @ X, an, eps[:n], U[:, :n], 0.0, max_sweeps=1, group=8)
    assert sweeps == 1 and len(e2) == n
    assert np.max(np.abs(e2 - eps[:n])) < 1e-11


def test_eigenvalue_error_is_quadratic_in_the_vector_error(wire):
    # the unconjugated pencil makes the Ritz values stationary at the
    # eigenvectors of the complex-symmetric A: error O(d^2), not O(d)
    w, A, eps, U, an = wire
    n = 16
    rng = np.random.default_rng(5)
    noise = (rng.standard_normal((w.N, n)) + 1j * rng.standard_normal((w.N, n))) / np.sqrt(w.N)
    errs = []
    for d in (1e-4, 1e-5):
        e1, U1, r1, _ = refine.refine(lambda X: A @ X, an, eps[:n] * (1 + d), U[:, :n] + d * noise, 0.0,
                                      max_sweeps=1, group=8)
        assert len(e1) == n
        errs.append(np.max(np.abs(e1 - eps[:n])))
    assert errs[0] < 1e-6
    assert errs[1] < errs[0] / 30.0


def test_groups_without_unconverged_pairs_are_untouched(wire):
    w, A, eps, U, an = wire
    n = 16
    U0 = np.array(U[:, :n], copy=True)
    U0[:, 10] += 1e-3 * U[:, 300]  # only the second group of 8 has an unconverged pair
    res = refine.relative_residuals(lambda X: A @ X, an, eps[:n], U0)
    e1, U1 = refine.rr_sweep(lambda X: A @ X, eps[:n], U0, res, 1e-10, group=8)
    np.testing.assert_array_equal(e1[:8], eps[:8])
    assert np.max(np.abs(e1[8:] - eps[8:n])) < 1e-11


def test_sweep_keeps_converged_pairs_and_bounds_the_residual(wire):
    # each group of 8 holds 4 exact eigenpairs (converged) and 4 pairs far from
    # convergence (random combinations of the 40 lowest eigenvectors with
    # shifted eigenvalues): whatever the Rayleigh-Ritz step returns, a group is
    # replaced only if it keeps as many converged pairs and its largest
    # residual grows at most tenfold; with every residual at rel_tol nothing
    # changes at all
    w, A, eps, U, an = wire
    n, tol = 16, 1e-10
    apply = lambda X: A @ X  # noqa: E731
    for seed in range(4):
        rng = np.random.default_rng(seed)
        C = rng.standard_normal((40, 8)) + 1j * rng.standard_normal((40, 8))
        R = U[:, :40] @ C
        R /= np.sqrt(np.sum(R * R, axis=0))[None, :]
        U0 = np.concatenate([U[:, 0:4], R[:, 0:4], U[:, 4:8], R[:, 4:8]], axis=1)
        e0 = np.concatenate([eps[0:4], eps[0:4] + 0.05, eps[4:8], eps[4:8] + 0.05])
        e0, U0 = eigen.sort_by_real(e0, U0)
        r0 = refine.relative_residuals(apply, an, e0, U0)
        assert np.sum(r0 <= tol) == 8
        e1, U1 = refine.rr_sweep(apply, e0, U0, r0, tol, group=8, eq_rtol=0.0, drop_tol=0.0, anorm=an, near_tol=1.0)
        r1 = refine.relative_residuals(apply, an, e1, U1)
        assert len(e1) == n
        assert np.sum(r1 <= tol) >= 8 and np.max(r1) <= 10.0 * np.max(r0) * (1 + 1e-12)
        # every group replaced or kept whole: the kept groups' pairs are returned unchanged
        e2, U2 = refine.rr_sweep(apply, e0, U0, np.zeros(n), tol, group=8, eq_rtol=0.0, drop_tol=0.0, anorm=an)
        np.testing.assert_array_equal(np.sort_complex(e2), np.sort_complex(e0))
        # groups far from convergence (largest residual above near_tol) are not swept
        e3, U3 = refine.rr_sweep(apply, e0, U0, r0, tol, group=8, eq_rtol=0.0, drop_tol=0.0, anorm=an,
                                 near_tol=0.5 * np.max(r0))
        np.testing.assert_array_equal(np.sort_complex(e3), np.sort_complex(e0))
