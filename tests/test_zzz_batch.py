"""The batching form (swi_solve_batch): independent systems of uneven grids solved at once.

A seeded batch of small wires in the shape of the uneven-batch workload
(uneven x and y axes, z doubled, a few wells each, 2-3 windows of uneven
requests) is solved in one call; every system must then hold its own lowest
pairs with the checks of the single-system solves against its own dense
oracle: eigenvalues within 1e-10 max(1, |eps|), explicit residuals below
1e-10 relative to ||A||_G, U^T U = I, degenerate clusters' projectors.  The
file is named so that pytest collects it after the other GPU tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, partition, stencil

pytestmark = pytest.mark.gpu

EPS_TOL = 1e-10
RES_TOL = 1e-10
REL_TOL_SV = 2e-12


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


def _systems(count=5, seed=4):
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        nx, ny = int(rng.integers(6, 10)), int(rng.integers(6, 10))
        nz = 2 * int(rng.integers(6, 10))
        wells = int(rng.integers(2, 6))
        n_r = int(rng.integers(8, 20))
        p = int(rng.integers(2, 4))
        w = W.make_wire(nx, ny, nz, 0.5, wells, 4000 + s)
        A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
        eps_o, U_o = eigen.dense_spectrum(A)
        while abs(eps_o[n_r] - eps_o[n_r - 1]) <= 1e-6 * max(1.0, abs(eps_o[n_r])):
            n_r += 1  # a cut clear of degenerate clusters
        sig, req = W.count_windows(eps_o.real[:n_r], partition.window_counts(n_r, p), inflate=1.3, extra=4)
        out.append((w, eps_o, U_o, n_r, sig, req))
    return out


def _check(w, eps_o, U_o, n_r, eps, U, res, info):
    assert info["status"] == "SWI_OK", info
    assert len(eps) == n_r
    assert np.max(np.abs(eps - eps_o[:n_r]) / np.maximum(1.0, np.abs(eps_o[:n_r]))) <= EPS_TOL
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
    for cl in eigen.clusters(eps_o[:n_r], 1e-9):
        P = eigen.cluster_projector(U, cl)
        Po = eigen.cluster_projector(U_o, cl)
        assert np.max(np.abs(P - Po)) <= 1e-8 * max(1.0, np.max(np.abs(Po)))


@pytest.mark.parametrize("workers", [0, 2])
def test_batch_of_uneven_systems_matches_each_dense_oracle(swi, workers):
    systems = _systems()
    ctxs = []
    try:
        for (w, eps_o, U_o, n_r, sig, req) in systems:
            c = swi.Context(w.nx, w.ny, w.nz, w.h)
            c.set_potential(w.V)
            c.set_absorber(w.gamma_L, w.gamma_R)
            c.set_windows(sig, req)
            ctxs.append(c)
        infos = swi.solve_batch(ctxs, block=2, rel_tol=REL_TOL_SV, n_keep=0, max_matvecs=100000, workers=workers)
        for c, inf, (w, eps_o, U_o, n_r, sig, req) in zip(ctxs, infos, systems):
            eps, U = c.eigenpairs()
            res = c.residuals()
            # the merged set holds at least the lowest n_r pairs; keep those
            assert len(eps) >= n_r
            _check(w, eps_o, U_o, n_r, eps[:n_r], U[:, :n_r], res[:n_r], inf)
    finally:
        for c in ctxs:
            c.close()


def test_batch_rejects_repeated_contexts(swi):
    w = W.make_wire(6, 6, 12, 0.5, 2, 4)
    with swi.Context(w.nx, w.ny, w.nz, w.h) as c:
        with pytest.raises(swi.SwiError) as e:
            swi.solve_batch([c, c])
        assert e.value.code == swi.SWI_EINVAL
