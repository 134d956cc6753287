"""Windows with complex shifts (the two-dimensional partition of Section 2) on the GPU.

A 20-bohr wire whose absorbers cover only its ends spreads -Im eps over
[0, 0.33] Ha, so windows at one real part and two imaginary parts select
different eigenvalues.  Each window must deliver the eigenvalues nearest its
shift (the oracle's partition.complex_shift_window over the dense spectrum)
and the merge their union, held to the checks of the real-shift solves:
eigenvalues within 1e-10 max(1, |eps|), explicit residuals below 1e-10
relative to ||A||_G, U^T U = I, degenerate clusters' projectors against the
oracle's.  The file is named so that pytest collects it after the other GPU
tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, partition, stencil

pytestmark = pytest.mark.gpu

EPS_TOL = 1e-10
RES_TOL = 1e-10
REL_TOL_SV = 2e-12
SHIFTS = [1.2 - 0.3j, 1.2 - 0.01j, 2.4 - 0.3j, 2.4 - 0.01j]  # increasing by (Re, Im)
REQS = [6, 6, 7, 7]


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


@pytest.fixture(scope="module")
def wire():
    w = W.make_wire(6, 6, 40, 0.5, 6, 3)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps_o, U_o = eigen.dense_spectrum(A)
    return w, eps_o, U_o


def _ctx(swi, w):
    c = swi.Context(w.nx, w.ny, w.nz, w.h)
    c.set_potential(w.V)
    c.set_absorber(w.gamma_L, w.gamma_R)
    return c


def test_complex_shift_grid_delivers_the_nearest_eigenvalues(swi, wire):
    w, eps_o, U_o = wire
    idx = set()
    per_window = []
    for s, r in zip(SHIFTS, REQS):
        d = np.sort(np.abs(eps_o - s))
        assert d[r] - d[r - 1] > 0.05 * d[r - 1]  # the cut is clear of ties
        sel = set(int(k) for k in partition.complex_shift_window(eps_o, s, r))
        per_window.append(sel)
        idx |= sel
    assert per_window[0] != per_window[1] and per_window[2] != per_window[3]
    idx = sorted(idx, key=lambda k: (eps_o[k].real, eps_o[k].imag))
    eps_x, U_x = eps_o[idx], U_o[:, idx]
    with _ctx(swi, w) as c:
        c.set_windows_complex(SHIFTS, REQS)
        info = c.solve(block=2, rel_tol=REL_TOL_SV, n_keep=0, max_matvecs=200000)
        eps, U = c.eigenpairs()
        res = c.residuals()
    assert info["status"] in ("SWI_OK", "SWI_HOLES"), info
    assert len(eps) == len(idx), (len(eps), len(idx))
    assert np.max(np.abs(eps - eps_x) / np.maximum(1.0, np.abs(eps_x))) <= EPS_TOL
    assert np.max(res) <= RES_TOL, np.max(res)
    G = U.T @ U
    n = len(eps)
    np.testing.assert_allclose(np.diag(G), np.ones(n), atol=1e-12)
    an = stencil.gershgorin_norm(w.h, w.V, w.gamma_L, w.gamma_R)
    r = np.asarray(res) * an * np.linalg.norm(U, axis=0)
    gap = np.abs(eps[:, None] - eps[None, :])
    off = ~np.eye(n, dtype=bool)
    same = gap <= 1e-9 * np.maximum(1.0, np.abs(eps))[:, None]
    assert np.all(np.abs(G[off & same]) <= 1e-10)
    bound = 4.0 * (r[:, None] + r[None, :]) / np.maximum(gap, 1e-300) + 1e-12
    assert np.all(np.abs(G[off & ~same]) <= bound[off & ~same])
    for cl in eigen.clusters(eps_x, 1e-9):
        P = eigen.cluster_projector(U, cl)
        Po = eigen.cluster_projector(U_x, cl)
        assert np.max(np.abs(P - Po)) <= 1e-8 * max(1.0, np.max(np.abs(Po)))


def test_complex_shifts_are_validated_and_limited_to_narrow_windows(swi, wire):
    w, eps_o, U_o = wire
    with _ctx(swi, w) as c:
        with pytest.raises(swi.SwiError) as e:
            c.set_windows_complex([1.2 - 0.01j, 1.2 - 0.3j], [4, 4])  # not increasing by (Re, Im)
        assert e.value.code == swi.SWI_EINVAL
        c.set_windows_complex([1.2 - 0.3j, 1.2 - 0.01j], [4, 4])
        with pytest.raises(swi.SwiError) as e:
            c.solve(block=4)  # wide blocks take real shifts only
        assert e.value.code == swi.SWI_EINVAL
        info = c.solve(block=2, rel_tol=1e-10, n_keep=0, max_matvecs=200000)
        assert info["status"] in ("SWI_OK", "SWI_HOLES"), info
        with pytest.raises(swi.SwiError) as e:
            c.fill_holes(0.0, 3.0)  # hole filling works on the real axis
        assert e.value.code == swi.SWI_EINVAL
        # real windows again
        c.set_windows([1.0, 2.0], [4, 4])
        info = c.solve(block=2, rel_tol=1e-10, n_keep=0, max_matvecs=200000)
        assert info["status"] in ("SWI_OK", "SWI_HOLES"), info
