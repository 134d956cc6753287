"""The bench workload's window plan on CPU: 8 windows of equal eigenpair count
over the lowest 400 real parts of the 48x48x96 wire (the committed Kohn-Sham
spectrum), shift at the middle of each run of 50, requests ceil(50 x 1.1) + 2."""
import sys

import numpy as np

from conftest import ROOT


def test_plan_of_the_48x48x96_workload():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    cfg = W.CONFIGS[bench.WORKLOAD]
    sig, req, E, source = bench.plan(cfg)
    assert source == "ks_spectrum"
    n_req = int(np.ceil(50 * bench.INFLATE)) + bench.EXTRA
    assert len(sig) == cfg["p"] == 8 and list(req) == [n_req] * 8 and 52 <= n_req <= 60
    lam = bench.ks_spectrum(bench.WORKLOAD)[:cfg["n_r"]]
    per = cfg["n_r"] // cfg["p"]
    for j in range(cfg["p"]):
        run = lam[j * per:(j + 1) * per]
        assert run[0] <= sig[j] <= run[-1]  # inside its own run of 50
    assert np.all(np.diff(sig) > 0)
    assert len(E) == cfg["n_E"] and E[0] == lam[0] and E[-1] == lam[cfg["n_r"] - 1]
