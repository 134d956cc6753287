"""swi_transmission_noalloc: T(E) without device allocation, for callers that cannot allocate.

Some callers must not let a library allocate device memory while they run:
an application whose framework owns the whole device memory budget (a
caching allocator that must not see foreign allocations, a hard memory cap),
or one that does every allocation up front.  This entry point keeps its
scratch in one fixed file-scope device array instead; its answer must match
swi_transmission's, and the call must leave the device's free memory
unchanged.  The file is named so pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, stencil, transport

pytestmark = pytest.mark.gpu


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


def _small_pairs():
    w = W.make_wire(7, 6, 12, 0.5, 3, 9)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps, U = eigen.dense_spectrum(A)
    return w, eps, U


def test_noalloc_first_on_a_fresh_context_allocates_nothing(swi):
    import torch
    w, eps, U = _small_pairs()
    n = 40
    E1 = np.linspace(eps.real[0] - 0.2, eps.real[n - 1], 17)
    E2 = np.linspace(eps.real[3], eps.real[n - 1] + 0.3, 9)
    # load the kernels' code once (module loading may take device memory)
    with swi.Context(w.nx, w.ny, w.nz, w.h) as c0:
        c0.set_potential(w.V)
        c0.set_absorber(w.gamma_L, w.gamma_R)
        c0.set_eigenpairs(eps[:n], U[:, :n])
        c0.transmission_noalloc(E1)
    with swi.Context(w.nx, w.ny, w.nz, w.h) as c:
        c.set_potential(w.V)
        c.set_absorber(w.gamma_L, w.gamma_R)
        c.set_eigenpairs(eps[:n], U[:, :n])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        # two calls in a row share the scratch array; each must be right
        T1 = c.transmission_noalloc(E1)
        free1 = torch.cuda.mem_get_info()[0]
        T2 = c.transmission_noalloc(E2)
        free2 = torch.cuda.mem_get_info()[0]
        T1_ref = c.transmission(E1)
        T2_ref = c.transmission(E2)
    assert free1 == free0 and free2 == free0, (free0, free1, free2)
    np.testing.assert_allclose(T1, T1_ref, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(T2, T2_ref, rtol=1e-11, atol=1e-13)
    T1_o = transport.transmission_spectral(eps[:n], U[:, :n], w.gamma_L, w.gamma_R, E1)
    np.testing.assert_allclose(T1, T1_o, rtol=1e-10, atol=1e-12)


def test_noalloc_on_a_grid_larger_than_one_slab(swi):
    # 48 x 48 x 96 rows (more than three 65,536-row slabs), 64 seeded pairs:
    # the spectral T(E) of any (eps, U) against the oracle's formula
    w = W.config_wire("wire_48x48x96")
    rng = np.random.default_rng(11)
    n = 64
    U = (rng.standard_normal((w.N, n)) + 1j * rng.standard_normal((w.N, n))) / np.sqrt(2.0 * w.N)
    eps = np.sort(rng.uniform(-1.0, 0.5, n)) - 1j * rng.uniform(0.01, 0.2, n)
    E = np.linspace(-1.1, 0.6, 33)
    with swi.Context(w.nx, w.ny, w.nz, w.h) as c:
        c.set_potential(w.V)
        c.set_absorber(w.gamma_L, w.gamma_R)
        c.set_eigenpairs(eps, U)
        T = c.transmission_noalloc(E)
        T_again = c.transmission_noalloc(E)
        T_ref = c.transmission(E)
    T_o = transport.transmission_spectral(eps, U, w.gamma_L, w.gamma_R, E)
    scale = np.max(np.abs(T_o))
    np.testing.assert_allclose(T, T_o, rtol=1e-10, atol=1e-12 * scale)
    np.testing.assert_allclose(T_again, T, rtol=0, atol=0)
    np.testing.assert_allclose(T, T_ref, rtol=1e-11, atol=1e-13 * scale)


def test_noalloc_rejects_sizes_beyond_its_scratch(swi):
    w, eps, U = _small_pairs()
    with swi.Context(w.nx, w.ny, w.nz, w.h) as c:
        c.set_potential(w.V)
        c.set_absorber(w.gamma_L, w.gamma_R)
        c.set_eigenpairs(eps[:65], U[:, :65])
        with pytest.raises(swi.SwiError) as e:
            c.transmission_noalloc([0.1, 0.2])
        assert e.value.code == swi.SWI_EINVAL
        c.set_eigenpairs(eps[:10], U[:, :10])
        with pytest.raises(swi.SwiError) as e:
            c.transmission_noalloc(np.linspace(0.0, 1.0, 1025))
        assert e.value.code == swi.SWI_EINVAL
