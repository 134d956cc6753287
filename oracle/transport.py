"""Transmission T(E) and its gradients (CPU FP64).

Section 1 defines G(E) = {E 1 - (H_KS - i Gamma)}^-1 and
T(E) = Tr{G(E) Gamma_R G^dagger(E) Gamma_L}; the eigenpairs of Eq. (1) are the
intermediate through which G is evaluated.  With U^T U = I the spectral form
is G(E) = sum_k U_k U_k^T / (E - eps_k) (exact when all N pairs are used).

Spectral T:  R = U^T Gamma_R conj(U), L = U^T Gamma_L conj(U), W = R o L
(elementwise), g_k = 1/(E - eps_k), T = sum_kl g_k W_kl conj(g_l).

Gradient with respect to the potential: dG = G dV G, so
dT/dV(r) = 2 Re[(G Gamma_R G^dagger Gamma_L G)_rr]; spectrally
(G Gamma_R G^dagger Gamma_L G) = U D R conj(D) L^T D U^T with D = diag(g).
dT/dE = -2 Re sum_kl g_k^2 W_kl conj(g_l) (U and eps do not depend on E).
"""
from __future__ import annotations

import numpy as np


def projections(U: np.ndarray, gamma_L, gamma_R):
    """R = U^T Gamma_R conj(U) and L = U^T Gamma_L conj(U) (both Hermitian)."""
    gR = np.asarray(gamma_R)[:, None]
    gL = np.asarray(gamma_L)[:, None]
    R = U.T @ (gR * U.conj())
    L = U.T @ (gL * U.conj())
    return R, L


def transmission_spectral(eps, U, gamma_L, gamma_R, E) -> np.ndarray:
    """T(E_e) from eigenpairs through the spectral Green's function."""
    R, L = projections(U, gamma_L, gamma_R)
    W = R * L
    E = np.atleast_1d(np.asarray(E, dtype=np.float64))
    out = np.empty(len(E))
    for e, En in enumerate(E):
        g = 1.0 / (En - eps)
        out[e] = np.real(g @ W @ g.conj())
    return out


def transmission_direct(A: np.ndarray, gamma_L, gamma_R, E) -> np.ndarray:
    """T(E) by dense inversion: T = sum_rs Gamma_L(r) |G_rs|^2 Gamma_R(s)."""
    N = A.shape[0]
    gL = np.asarray(gamma_L)
    gR = np.asarray(gamma_R)
    out = []
    for En in np.atleast_1d(E):
        G = np.linalg.inv(En * np.eye(N) - A)
        out.append(float(gL @ (np.abs(G) ** 2) @ gR))
    return np.array(out)


def grad_V_spectral(eps, U, gamma_L, gamma_R, E, dLdT) -> np.ndarray:
    """dL/dV(r) = sum_e dLdT_e * 2 Re[(U D_e R conj(D_e) L^T D_e U^T)_rr]."""
    R, L = projections(U, gamma_L, gamma_R)
    M = np.zeros_like(R)
    for En, w in zip(np.atleast_1d(E), np.atleast_1d(dLdT)):
        g = 1.0 / (En - eps)
        M += w * (g[:, None] * R * g.conj()[None, :]) @ (L.T * g[None, :])
    return 2.0 * np.real(np.einsum("ra,ac,rc->r", U, M, U))


def grad_E_spectral(eps, U, gamma_L, gamma_R, E) -> np.ndarray:
    """dT/dE_e = -2 Re sum_kl g_k^2 W_kl conj(g_l)."""
    R, L = projections(U, gamma_L, gamma_R)
    W = R * L
    out = []
    for En in np.atleast_1d(E):
        g = 1.0 / (En - eps)
        out.append(-2.0 * np.real((g * g) @ W @ g.conj()))
    return np.array(out)


def grad_V_direct(A: np.ndarray, gamma_L, gamma_R, E, dLdT) -> np.ndarray:
    """dL/dV(r) from the dense inverse: sum_e w_e 2 Re[(G Gamma_R G^dagger Gamma_L G)_rr]."""
    N = A.shape[0]
    gL = np.asarray(gamma_L)
    gR = np.asarray(gamma_R)
    out = np.zeros(N)
    for En, w in zip(np.atleast_1d(E), np.atleast_1d(dLdT)):
        G = np.linalg.inv(En * np.eye(N) - A)
        X = (G * gR[None, :]) @ G.conj().T @ (gL[:, None] * G)
        out += w * 2.0 * np.real(np.diag(X))
    return out
