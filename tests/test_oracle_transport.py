"""Pins for T(E) = Tr{G Gamma_R G^dagger Gamma_L} and its gradients (Section 1)."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, stencil, transport


def _dense(w):
    return stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)


@pytest.fixture(scope="module")
def tiny():
    w = W.make_wire(5, 5, 10, 0.5, 3, 9)
    A = _dense(w)
    eps, U = eigen.dense_spectrum(A)
    E = np.linspace(eps.real[0] - 0.1, eps.real[30], 7)
    return w, A, eps, U, E


def test_full_spectral_equals_direct_inverse(tiny):
    # (E - A)^-1 = U diag(1/(E - eps)) U^T when U^T U = I and all N pairs are used.
    w, A, eps, U, E = tiny
    t_s = transport.transmission_spectral(eps, U, w.gamma_L, w.gamma_R, E)
    t_d = transport.transmission_direct(A, w.gamma_L, w.gamma_R, E)
    np.testing.assert_allclose(t_s, t_d, rtol=1e-10)
    assert np.all(t_d >= 0)


def test_direct_trace_by_brute_force(tiny):
    # Tr{G Gamma_R G^dagger Gamma_L} with explicit matrices, written out.
    w, A, eps, U, E = tiny
    G = np.linalg.inv(E[2] * np.eye(w.N) - A)
    T = np.trace(G @ np.diag(w.gamma_R) @ G.conj().T @ np.diag(w.gamma_L))
    assert abs(T.imag) < 1e-12 * abs(T)
    np.testing.assert_allclose(transport.transmission_direct(A, w.gamma_L, w.gamma_R, E[2:3])[0], T.real, rtol=1e-12)


def test_separable_transmission_is_a_channel_sum():
    # Gamma and V depend on z only: T(E) = sum_q T_z(E - e_q) over transverse modes.
    w = W.separable_wire(5, 6, 12, 0.5, 3, 4)
    A = _dense(w)
    h = w.h
    plane = w.nx * w.ny
    vz, gl, gr = w.V[::plane], w.gamma_L[::plane], w.gamma_R[::plane]
    Az = -0.5 / h ** 2 * stencil.second_difference_1d(w.nz) + np.diag(vz - 1j * (gl + gr))
    ex = np.linalg.eigvalsh(-0.5 / h ** 2 * stencil.second_difference_1d(w.nx))
    ey = np.linalg.eigvalsh(-0.5 / h ** 2 * stencil.second_difference_1d(w.ny))
    eperp = np.add.outer(ey, ex).reshape(-1)
    E = np.array([-0.5, 0.3, 1.1])
    t3 = transport.transmission_direct(A, w.gamma_L, w.gamma_R, E)
    t1 = np.array([sum(transport.transmission_direct(Az, gl, gr, [En - e])[0] for e in eperp) for En in E])
    np.testing.assert_allclose(t3, t1, rtol=1e-10)


def test_adjoint_gradient_matches_direct_and_finite_differences(tiny):
    w, A, eps, U, E = tiny
    rng = np.random.default_rng(3)
    dLdT = rng.standard_normal(len(E))
    g_spec = transport.grad_V_spectral(eps, U, w.gamma_L, w.gamma_R, E, dLdT)
    g_dir = transport.grad_V_direct(A, w.gamma_L, w.gamma_R, E, dLdT)
    np.testing.assert_allclose(g_spec, g_dir, rtol=1e-9, atol=1e-12 * np.abs(g_dir).max())
    # central differences in V at a few grid points (dV = 1e-5 Ha)
    dv = 1e-5
    for r in rng.choice(w.N, size=6, replace=False):
        Ap = A.copy(); Ap[r, r] += dv
        Am = A.copy(); Am[r, r] -= dv
        tp = transport.transmission_direct(Ap, w.gamma_L, w.gamma_R, E)
        tm = transport.transmission_direct(Am, w.gamma_L, w.gamma_R, E)
        fd = dLdT @ (tp - tm) / (2 * dv)
        assert abs(fd - g_dir[r]) <= 1e-6 * max(1.0, np.abs(g_dir).max()), (r, fd, g_dir[r])


def test_energy_derivative_matches_finite_differences(tiny):
    w, A, eps, U, E = tiny
    n_r = 20  # truncated spectral T: U and eps do not depend on E, so dT/dE is exact
    e, Us = eps[:n_r], U[:, :n_r]
    d = transport.grad_E_spectral(e, Us, w.gamma_L, w.gamma_R, E)
    de = 1e-6
    tp = transport.transmission_spectral(e, Us, w.gamma_L, w.gamma_R, E + de)
    tm = transport.transmission_spectral(e, Us, w.gamma_L, w.gamma_R, E - de)
    np.testing.assert_allclose(d, (tp - tm) / (2 * de), rtol=1e-5, atol=1e-8)


def test_truncated_transmission_hermitian_structure(tiny):
    # R and L are Hermitian, so T is real for any subset of pairs.
    w, A, eps, U, E = tiny
    R, L = transport.projections(U[:, :15], w.gamma_L, w.gamma_R)
    np.testing.assert_allclose(R, R.conj().T, atol=1e-13)
    np.testing.assert_allclose(L, L.conj().T, atol=1e-13)
