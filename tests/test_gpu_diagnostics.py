"""Discarded-component diagnostic on GPU runs against the same diagnostic on the oracle (3x4 grid,
chi = 16, the grid's tie-free bond dimension, 10 second-order steps, mid temperature): F_exact,
<Z^2> of the MPS, of the exact state and of the discarded component, and the off-diagonal term
agree within 1e-6 (the bound of the chi = 16 parity case, which has a cut with relative gap
2.4e-6)."""
import pytest

from oracle import model

pytestmark = pytest.mark.gpu


def test_orthogonal_component_gpu_vs_oracle(tmp_path):
    from paper_2511_23438_gb300 import diagnostics as dg
    from test_diagnostics import oracle_orthogonal_run
    theta = model.initial_theta(model.TEMPERATURES["mid"])
    g = dg.gpu_orthogonal_run(3, 4, 16, theta, 10, str(tmp_path))
    o = oracle_orthogonal_run(3, 4, 16, theta, 10)
    for rg, ro in zip(g, o):
        for k in ("F_exact", "F_mps", "z2_mps", "z2_exact", "z2_perp", "cross"):
            assert abs(rg[k] - ro[k]) < 1e-6, (k, rg[k], ro[k])
    assert g[-1]["F_exact"] < 1 - 1e-6
