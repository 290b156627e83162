"""The gamma-fit pipeline on GPU data against the same pipeline on oracle data (3x4 grid, exact
at chi = 64, truncated at chi = 16 and 21, 20 second-order steps, mid temperature).  These are
the tie-free bond dimensions of this grid (smallest relative gap at any cut 2.4e-6 and 8.9e-5;
chi = 8, 12, 14, 18, 20, 24 have exact ties at the cut, where several truncations are equally
correct and the two implementations may keep different states).

The GPU produces the exact <Z^2> itself (FP64 MPS at the exact bond bound).  The data agree with
the oracle within 1e-6 (the chi = 16 second-order run has a cut with relative gap ~2e-6, where
two correct FP64 truncations differ by ~eps/gap; see the parity tests), so gamma* (slope
d<Z^2>_gamma/dgamma ~ 1e-3) agrees within 1e-3."""
import numpy as np
import pytest

from oracle import model

pytestmark = pytest.mark.gpu


def test_gamma_pipeline_gpu_vs_oracle():
    from paper_2511_23438_gb300 import gamma
    from test_gamma import oracle_runs
    dtheta = model.TEMPERATURES["mid"]
    g_runs, g_exact = gamma.gpu_runs([(3, 4)], [16, 21], dtheta)
    o_runs, o_exact = oracle_runs([(3, 4)], [16, 21], dtheta)
    assert np.abs(g_exact[(3, 4)] - o_exact[(3, 4)]).max() < 1e-9
    for key in o_runs:
        for a, b in zip(g_runs[key], o_runs[key]):
            assert np.abs(a - b).max() < 1e-6, key
    g, o = gamma.analyse(g_runs, g_exact), gamma.analyse(o_runs, o_exact)
    for rg, ro in zip(g["rows"], o["rows"]):
        assert abs(rg["gamma_star"] - ro["gamma_star"]) < 1e-3
        assert rg["max_err_rescaled"] < rg["max_err_mps"]
    assert abs(g["a"] - o["a"]) < 1e-2 and abs(g["b"] - o["b"]) < 1e-3
