"""Write the Kohn-Sham spectrum estimate used to place windows (calls only oracle/).

The paper places its shifts with foreknowledge of the spectrum and suggests
estimating it from the lowest eigenvalues of H_KS alone (without i Gamma),
which approximate Re eps_k to first order (Section 2, Eq. (5)).  This
script computes the lowest `count` eigenvalues of the real symmetric H of a
workload with the oracle's stencil (Gamma = 0) and ARPACK's Lanczos driver,
and writes them, one per line, to tests/golden/<name>_ks_spectrum.txt.

    python tests/golden/make_wire_spectrum.py wire_48x48x96 460
"""
import os
import sys

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import stencil  # noqa: E402


def main(name: str, count: int):
    w = W.config_wire(name)
    zero = np.zeros(w.N)

    def mv(x):
        return stencil.apply_A(x, w.nx, w.ny, w.nz, w.h, w.V, zero, zero).real

    op = spla.LinearOperator((w.N, w.N), matvec=mv, dtype=np.float64)
    v0 = np.random.default_rng(0).standard_normal(w.N)
    lam = spla.eigsh(op, k=count, which="SA", tol=1e-10, v0=v0, return_eigenvectors=False)
    lam = np.sort(lam)
    out = os.path.join(HERE, f"{name}_ks_spectrum.txt")
    with open(out, "w") as f:
        f.write(f"# lowest {count} eigenvalues (Ha) of H_KS = -1/2 lap_FD + V (Gamma = 0) for {name};\n")
        f.write("# written by tests/golden/make_wire_spectrum.py (oracle stencil + ARPACK Lanczos)\n")
        for x in lam:
            f.write(f"{x:.12f}\n")
    print(out, lam[0], lam[-1])


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]))
