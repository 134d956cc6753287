"""Dense spectra, U^T U = I normalisation and the paper's windowed solver (CPU FP64).

* Eq. (1): (H_KS - i Gamma) U_k = eps_k U_k, eps_k complex.  Eigenvectors of a
  complex-symmetric matrix are bi-orthogonal under the unconjugated product
  (Section 1), so they can be scaled to U^T U = I.
* Eq. (3): each window j solves the shifted problem (A - E_S,j) U = (eps - E_S,j) U
  for the n_r,j eigenvalues closest to the shift, using ARPACK's 'SM'
  (smallest magnitude) selection on the shifted operator, with no inversion
  (Section 2, where the shift-plus-SM recipe is introduced).
* "Ordering" of eigenvalues always means ordering by real part (Section 2,
  footnote on the target set).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import stencil


def sort_by_real(eps: np.ndarray, U: np.ndarray | None = None):
    """Order eigenpairs by (Re, Im)."""
    idx = np.lexsort((eps.imag, eps.real))
    return (eps[idx], None if U is None else U[:, idx])


def clusters(eps_sorted: np.ndarray, rtol: float):
    """Group consecutive (Re-sorted) eigenvalues with |d eps| <= rtol * max(1, |eps|)."""
    groups = []
    cur = [0]
    for k in range(1, len(eps_sorted)):
        if abs(eps_sorted[k] - eps_sorted[cur[-1]]) <= rtol * max(1.0, abs(eps_sorted[k])):
            cur.append(k)
        else:
            groups.append(cur)
            cur = [k]
    if len(eps_sorted):
        groups.append(cur)
    return groups


def bilinear_normalise(eps_sorted: np.ndarray, U: np.ndarray, cluster_rtol: float = 1e-9):
    """Scale eigenvectors to U^T U = I (unconjugated product).

    Within a cluster of (numerically) equal eigenvalues, eigenvectors are
    first made bilinear-orthogonal by Gram-Schmidt with the projection
    v_k -= v_m (v_m^T v_k) / (v_m^T v_m); every vector is then divided by the
    principal square root of v^T v.
    """
    U = np.array(U, dtype=np.complex128, copy=True)
    for g in clusters(eps_sorted, cluster_rtol):
        for a, k in enumerate(g):
            for m in g[:a]:
                U[:, k] -= U[:, m] * (U[:, m] @ U[:, k])  # v_m already has v_m^T v_m = 1
            U[:, k] /= np.sqrt(U[:, k] @ U[:, k])
    return U


def dense_spectrum(A: np.ndarray, cluster_rtol: float = 1e-9):
    """All eigenpairs of the dense A (LAPACK zgeev), Re-sorted, with U^T U = I."""
    eps, U = np.linalg.eig(A)
    eps, U = sort_by_real(eps, U)
    return eps, bilinear_normalise(eps, U, cluster_rtol)


def residual_norms(apply_A, eps: np.ndarray, U: np.ndarray) -> np.ndarray:
    """||A u_k - eps_k u_k||_2 / ||u_k||_2 for each column."""
    AU = apply_A(U)
    R = AU - U * eps[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(U, axis=0)


def arpack_window(wire, sigma: complex, n_req: int, tol: float = 1e-12, seed: int = 0,
                  ncv: int | None = None, maxiter: int | None = None, bc: int = stencil.BC_ODD):
    """The paper's per-window solve: ARPACK 'SM' on x -> (A - sigma) x (Eq. (3)).

    sigma is real for the paper's windows; a complex sigma gives a window of
    the two-dimensional partition Section 2 names for strongly non-Hermitian
    problems.

    Returns eps (Re-sorted, shifted back by sigma) and eigenvectors scaled to
    unit 2-norm.  ARPACK's implicitly restarted Arnoldi applies the shifted
    operator only through matrix-vector products; nothing is inverted.
    """
    N = wire.N

    def mv(x):
        return stencil.apply_A(x, wire.nx, wire.ny, wire.nz, wire.h, wire.V,
                               wire.gamma_L, wire.gamma_R, sigma=sigma, bc=bc)

    op = spla.LinearOperator((N, N), matvec=mv, dtype=np.complex128)
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    theta, V = spla.eigs(op, k=n_req, which="SM", tol=tol, v0=v0, ncv=ncv, maxiter=maxiter)
    eps = theta + sigma
    eps, V = sort_by_real(eps, V)
    return eps, V / np.linalg.norm(V, axis=0)[None, :]


def lowest_by_real(eps: np.ndarray, U: np.ndarray, n_r: int):
    """The n_r pairs with smallest real part (the paper's target set, Section 2)."""
    eps, U = sort_by_real(eps, U)
    return eps[:n_r], U[:, :n_r]


def cluster_projector(U: np.ndarray, idx) -> np.ndarray:
    """P = sum_{k in idx} U_k U_k^T: basis-independent within a degenerate cluster."""
    Uc = U[:, list(idx)]
    return Uc @ Uc.T
