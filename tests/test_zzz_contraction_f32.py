"""FP32 contractions of T(E) and its adjoint (SWI_CONTRACT_F32) against the oracle.

The FP32 form rounds U to complex64 and accumulates in FP32, so a result is
held to the forward error bound of its sums: a multiple of u = 2^-24 of the
sum of the MAGNITUDES of its terms, the multiple being the accumulation length
of the kernels plus a few roundings.
 - Projections: R_kl = sum_r gamma_r U_rk conj(U_rl) over the absorber's rows,
   summed in 256-row blocks, then up to (rows per chunk)/256 block sums, the
   chunk partials in FP64:  |dR_kl| <= (256 + 64 + 8) u Rt_kl with
   Rt = |U|^T Gamma_R |U| (the chunks of these grids hold at most 3,392 rows).
 - T_e = sum_kl g_k R_kl L_kl conj(g_l) in FP64 from those:
   |dT_e| <= 2 (328 u) S_e,  S_e = sum_kl |g_k| Rt_kl Lt_kl |g_l|;
   dT_e/dE_e the same with |g_k|^2.
 - dL/dV(r) = 2 Re sum_ac U_ra M_ac U_rc, M = sum_e w_e D R conj(D) L^T D:
   sums over l (n terms), e (nE), a (n) and c (n) on top of R and L:
   |d(dL/dV)_r| <= (2 * 328 + 3 n + nE + 16) u Qt_r,
   Qt_r = 2 sum_ac |U_ra| Mt_ac |U_rc|,  Mt = sum_e |w_e| |D| Rt |D| Lt^T |D|.
The tests allow twice these bounds (the FP32 errors seen in practice are one
to two orders of magnitude below them).  The file is named so that pytest
collects it after the other GPU tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, stencil, transport

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
PROJ = 256 + 64 + 8  # accumulation length of one projection entry (see above)


@pytest.fixture(scope="module")
def swi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1606_01139_gb300 as lib
    from paper_1606_01139_gb300 import build as b
    b.build()
    lib.load()
    return lib


def _ctx(swi, w):
    c = swi.Context(w.nx, w.ny, w.nz, w.h)
    c.set_potential(w.V)
    c.set_absorber(w.gamma_L, w.gamma_R)
    return c


def _bounds(eps, U, w, E, wts):
    """Magnitude sums S_e (T), S'_e (dT/dE) and Qt_r (dL/dV) of the FP32 error bounds."""
    Ua = np.abs(U)
    Rt, Lt = transport.projections(Ua, w.gamma_L, w.gamma_R)  # |U|^T Gamma |U| (real)
    Rt, Lt = Rt.real, Lt.real
    Wt = Rt * Lt
    S, Sd = [], []
    Mt = np.zeros_like(Rt)
    for En, we in zip(E, wts):
        ga = np.abs(1.0 / (En - eps))
        S.append(ga @ Wt @ ga)
        Sd.append((ga * ga) @ Wt @ ga)
        Mt += abs(we) * (ga[:, None] * Rt * ga[None, :]) @ (Lt.T * ga[None, :])
    Qt = 2.0 * np.sum((Ua @ Mt) * Ua, axis=1)
    return np.array(S), np.array(Sd), Qt


def _check(eps, U, w, E, wts, T, dV, dE):
    n, nE = U.shape[1], len(E)
    To = transport.transmission_spectral(eps, U, w.gamma_L, w.gamma_R, E)
    dEo = transport.grad_E_spectral(eps, U, w.gamma_L, w.gamma_R, E)
    dVo = transport.grad_V_spectral(eps, U, w.gamma_L, w.gamma_R, E, wts)
    S, Sd, Qt = _bounds(eps, U, w, E, wts)
    tol_T = 2.0 * (2 * PROJ * U32) * S + 1e-300
    tol_dE = 2.0 * (2 * PROJ * U32) * 2.0 * Sd * np.abs(wts) + 1e-300
    tol_dV = 2.0 * (2 * PROJ + 3 * n + nE + 16) * U32 * Qt + 1e-300
    assert np.all(np.abs(T - To) <= tol_T), np.max(np.abs(T - To) / tol_T)
    assert np.all(np.abs(dE - wts * dEo) <= tol_dE), np.max(np.abs(dE - wts * dEo) / tol_dE)
    assert np.all(np.abs(dV - dVo) <= tol_dV), np.max(np.abs(dV - dVo) / tol_dV)
    return To, dEo, dVo


@pytest.mark.parametrize("n", [40, 130])
def test_f32_transport_on_oracle_pairs(swi, n):
    # 40 pairs: one ragged 64 x 64 tile; 130 pairs: three tiles, the lower ones
    # formed from their upper mirrors
    w = W.make_wire(7, 6, 12, 0.5, 3, 9)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps_o, U_o = eigen.dense_spectrum(A)
    eps, U = eps_o[:n], U_o[:, :n]
    E = np.linspace(eps.real[0] - 0.2, eps.real[-1], 9)
    wts = np.random.default_rng(5).standard_normal(len(E))
    with _ctx(swi, w) as c:
        c.set_eigenpairs(eps, U)
        c.set_contraction(swi.CONTRACT_F32)
        T = c.transmission(E)
        dV, dE = c.grad(E, wts)
        To, dEo, dVo = _check(eps, U, w, E, wts, T, dV, dE)
        # back to the FP64-class products: the cached FP32 projections are dropped
        c.set_contraction(swi.CONTRACT_F64)
        T64 = c.transmission(E)
    np.testing.assert_allclose(T64, To, rtol=1e-11, atol=1e-13)


def test_f32_on_a_grid_larger_than_one_slab(swi):
    # 48 x 48 x 96 rows with 64 seeded pairs: the absorbers' FP32 row ranges
    # cover 55% of the grid each, and each projection is split into row chunks
    w = W.config_wire("wire_48x48x96")
    rng = np.random.default_rng(12)
    n = 64
    U = (rng.standard_normal((w.N, n)) + 1j * rng.standard_normal((w.N, n))) / np.sqrt(2.0 * w.N)
    eps = np.sort(rng.uniform(-1.0, 0.5, n)) - 1j * rng.uniform(0.01, 0.2, n)
    E = np.linspace(-1.1, 0.6, 33)
    wts = rng.standard_normal(len(E))
    with _ctx(swi, w) as c:
        c.set_eigenpairs(eps, U)
        c.set_contraction(swi.CONTRACT_F32)
        T = c.transmission(E)
        dV, dE = c.grad(E, wts)
    _check(eps, U, w, E, wts, T, dV, dE)


def test_f32_autograd_against_central_differences(swi):
    # torch.autograd through the FP32 contractions with all N pairs of a small
    # grid (the spectral G is then the inverse): central differences of the
    # dense-inverse T(E) (delta V = 1e-5 Ha) within the FP32 bounds
    import torch
    w = W.make_wire(6, 6, 8, 0.5, 2, 4)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps_o, U_o = eigen.dense_spectrum(A)
    E0 = np.array([-0.35, 0.2, 0.9, 1.6])
    wts = np.random.default_rng(3).standard_normal(len(E0))
    with _ctx(swi, w) as c:
        c.set_eigenpairs(eps_o, U_o)
        c.set_contraction(swi.CONTRACT_F32)
        fn = swi.transmission_function()
        V = torch.tensor(w.V, dtype=torch.float64, device="cuda", requires_grad=True)
        E = torch.tensor(E0, dtype=torch.float64, device="cuda", requires_grad=True)
        T = fn.apply(V, E, c)
        loss = (torch.tensor(wts, dtype=torch.float64, device="cuda") * T).sum()
        loss.backward()
        dV = V.grad.cpu().numpy()
        dE = E.grad.cpu().numpy()
        Tn = T.detach().cpu().numpy()
    _check(eps_o, U_o, w, E0, wts, Tn, dV, dE)
    S, Sd, Qt = _bounds(eps_o, U_o, w, E0, wts)
    n, nE = U_o.shape[1], len(E0)
    tol_dV = 2.0 * (2 * PROJ + 3 * n + nE + 16) * U32 * Qt

    def loss_direct(Vv, Ev):
        Av = stencil.dense_A(w.nx, w.ny, w.nz, w.h, Vv, w.gamma_L, w.gamma_R)
        return float(wts @ transport.transmission_direct(Av, w.gamma_L, w.gamma_R, Ev))

    d = 1e-5
    for r in (0, w.N // 2 + 3, w.N - 5):
        Vp, Vm = w.V.copy(), w.V.copy()
        Vp[r] += d
        Vm[r] -= d
        fd = (loss_direct(Vp, E0) - loss_direct(Vm, E0)) / (2 * d)
        assert abs(dV[r] - fd) <= tol_dV[r] + 1e-6 * max(1.0, abs(fd)), (r, dV[r], fd, tol_dV[r])


def test_f32_contraction_rejects_unknown_values(swi):
    w = W.make_wire(6, 6, 8, 0.5, 2, 4)
    with _ctx(swi, w) as c:
        with pytest.raises(swi.SwiError) as e:
            c.set_contraction(7)
        assert e.value.code == swi.SWI_EINVAL
