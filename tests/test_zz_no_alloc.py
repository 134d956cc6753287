"""swi_transmission_noalloc: T(E) without device allocation, for callers that cannot allocate.

A caller recording work under CUDA stream capture, or living inside a
framework that owns the whole device memory budget, cannot let the library
call cudaMalloc during the call.  This entry point keeps its scratch in one
fixed device array instead; its answer must match swi_transmission's.  The
file is named so pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eigen, stencil

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


def test_noalloc_matches_transmission_on_two_calls(swi):
    w = W.make_wire(7, 6, 12, 0.5, 3, 9)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps, U = eigen.dense_spectrum(A)
    n = 40
    E1 = np.linspace(eps.real[0] - 0.2, eps.real[n - 1], 17)
    E2 = np.linspace(eps.real[3], eps.real[n - 1] + 0.3, 9)
    with swi.Context(w.nx, w.ny, w.nz, w.h) as c:
        c.set_potential(w.V)
        c.set_absorber(w.gamma_L, w.gamma_R)
        c.set_eigenpairs(eps[:n], U[:, :n])
        T1_ref = c.transmission(E1)
        T2_ref = c.transmission(E2)
        # two calls in a row share the scratch array; each must be right
        T1 = c.transmission_noalloc(E1)
        T2 = c.transmission_noalloc(E2)
    np.testing.assert_allclose(T1, T1_ref, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(T2, T2_ref, rtol=1e-11, atol=1e-13)


def test_noalloc_rejects_sizes_beyond_its_scratch(swi):
    w = W.make_wire(7, 6, 12, 0.5, 3, 9)
    A = stencil.dense_A(w.nx, w.ny, w.nz, w.h, w.V, w.gamma_L, w.gamma_R)
    eps, U = eigen.dense_spectrum(A)
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
