"""Residual-correction sweeps: Rayleigh-Ritz refinement of computed pairs (CPU FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 1 counts the subspace rotations of the Rayleigh-Ritz refinement, with
orthogonalisation, as the part of the Krylov cost that grows like N n_r^2;
Eq. (3) selects, per shift, the eigenvalues of smallest magnitude of the
shifted operator (ARPACK's SM), and Algorithm 2 combines pairs and scales them
to U^T U = I.  A correction sweep applies the same three ingredients to pairs
that are already computed.  The paper gives no further detail, so this module
fixes a reading:

* pairs ordered by real part are cut into groups of ``group`` consecutive
  pairs; a group whose pairs all have relative residual <= rel_tol is kept,
  and so is a group whose largest relative residual is above ``near_tol``
  (far from convergence: the sweep corrects pairs, it does not solve);
* otherwise, with U_g the group's vectors and R_u = A U_u - U_u diag(eps_u)
  the residuals of its unconverged pairs u, Q is a basis of span[U_g, R_u]
  (Householder QR here), sigma_g the middle of the group's real parts, and the
  n_g eigenvalues theta of smallest magnitude of the pencil
  Q^T (A - sigma_g) Q y = theta Q^T Q y give eps = sigma_g + theta and U = Q y.
  The pencil is the Rayleigh-Ritz step in the unconjugated product under which
  the eigenvectors of the complex-symmetric A are bi-orthogonal (Section 1);
  its eigenvalue error is quadratic in the vectors' error, where the Hermitian
  projection Q^H A Q of a non-Hermitian A gives a linear one.  The result does
  not depend on which basis of the span is used;
* a group keeps its Rayleigh-Ritz pairs unless they lower the number of the
  group's pairs at rel_tol or raise its largest relative residual more than
  tenfold; otherwise its previous pairs stay.  The sweep sharpens eigenvalues
  quadratically while a residual can stay level or rise a little (a vector
  error spread over all directions is not removed by one residual direction),
  so a rule on the residual alone would discard exactly those gains; far from
  convergence, though, the SM selection around sigma_g can pick directions
  away from pairs that had converged;
* all pairs then pass Algorithm 2 as one window (equal-eigenvalue projection,
  redundancy drop, v^T v = 1) and are ordered by real part.
"""
from __future__ import annotations

import numpy as np

from . import eigen, partition


def rr_sweep(apply_A, eps: np.ndarray, U: np.ndarray, res: np.ndarray, rel_tol: float, group: int = 16,
             eq_rtol: float = 1e-8, drop_tol: float = 1e-6, anorm: float | None = None, near_tol: float = 1e-3):
    """One sweep over the Re-sorted pairs (eps, U) with relative residuals res (relative to anorm;
    anorm None skips the rule that keeps a group's previous pairs)."""
    n = len(eps)
    eps_new = np.array(eps, dtype=np.complex128, copy=True)
    U_new = np.array(U, dtype=np.complex128, copy=True)
    for lo in range(0, n, group):
        g = list(range(lo, min(n, lo + group)))
        u = [k for k in g if not res[k] <= rel_tol]
        if not u or not np.max(res[g]) <= near_tol:
            continue
        R = apply_A(U[:, u]) - U[:, u] * eps[u][None, :]
        Q, _ = np.linalg.qr(np.concatenate([U[:, g], R], axis=1))
        sigma = 0.5 * (eps[g].real.min() + eps[g].real.max())
        K = Q.T @ (apply_A(Q) - sigma * Q)
        S = Q.T @ Q
        theta, Y = np.linalg.eig(np.linalg.solve(S, K))
        sel = np.argsort(np.abs(theta), kind="stable")[:len(g)]
        e, V = eigen.sort_by_real(theta[sel] + sigma, Q @ Y[:, sel])
        if anorm is not None:
            r_new = eigen.residual_norms(apply_A, e, V) / anorm
            r_old = res[g]
            if np.sum(r_new <= rel_tol) < np.sum(r_old <= rel_tol) or np.max(r_new) > 10.0 * np.max(r_old):
                continue
        eps_new[g] = e
        U_new[:, g] = V
    eps2, U2, _, _ = partition.combine([eps_new], [U_new], eq_rtol, drop_tol)
    return eigen.sort_by_real(eps2, U2)


def relative_residuals(apply_A, anorm: float, eps: np.ndarray, U: np.ndarray) -> np.ndarray:
    """||A u - eps u|| / (||A|| ||u||), the solver's convergence measure."""
    return eigen.residual_norms(apply_A, eps, U) / anorm


def refine(apply_A, anorm: float, eps: np.ndarray, U: np.ndarray, rel_tol: float, max_sweeps: int = 3,
           group: int = 16, eq_rtol: float = 1e-8, drop_tol: float = 1e-6, near_tol: float = 1e-3):
    """Sweeps until every pair is at rel_tol or max_sweeps ran; returns (eps, U, residuals, sweeps)."""
    res = relative_residuals(apply_A, anorm, eps, U)
    sweeps = 0
    while sweeps < max_sweeps and not np.all(res <= rel_tol):
        eps, U = rr_sweep(apply_A, eps, U, res, rel_tol, group, eq_rtol, drop_tol, anorm, near_tol)
        res = relative_residuals(apply_A, anorm, eps, U)
        sweeps += 1
    return eps, U, res, sweeps
