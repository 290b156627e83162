"""The benchmark configuration itself: 6x8 grid (d = 16, 12 blocks), chi = 1024, split-precision
form, the launch configuration bench.py times.

The oracle cannot run a chi = 1024 truncation of this grid (one bond update is a dense 16384^2
SVD), so full size is checked two ways: (1) after the first X layer the state is still a product
of block states, which the oracle evolves exactly at this grid size, so <Z_tot>, <Z_tot^2> and
<X_tot> are compared value by value (bound 1e-5, the FP32 storage of the split form); (2) after a
whole second-order Trotter step (172 truncations at chi = 1024) the properties that hold at any
size: 0 < F <= 1, |<Z>| <= 1, <Z^2> >= <Z>^2, <Z^2> <= 1, unit norm (within the split form's
drift), no bond above chi, and the Schmidt values of a bond descending and
normalised.
"""
import numpy as np
import pytest

from oracle import model
from oracle import mps as omps

pytestmark = pytest.mark.gpu


def test_bench_configuration_6x8_chi1024_split():
    from paper_2511_23438_gb300 import build, lib as L
    build.build()
    L.load()
    theta = model.initial_theta(model.TEMPERATURES["mid"])
    alpha, phi = model.layer_angles(-1.0, 2.0, 0.25, 2)
    m = L.MPS(L.config(6, 8, 1024, theta, prec="split_bf16x3"))
    # (1) exact at full size: the X layer keeps the state a product of block states
    m.apply_layer(L.LAYER_X, alpha)
    o = m.observables()
    ref = omps.MPS(6, 8, 1, theta)
    ref.x_layer(alpha)
    z, z2, x, nrm = ref.observables()
    assert abs(o["Z"] - z) < 1e-5 and abs(o["Z2"] - z2) < 1e-5 and abs(o["X"] - x) < 1e-5, (o, z, z2, x)
    assert abs(o["norm"] - 1) < 1e-5
    # (2) one whole Trotter step at chi = 1024: invariants
    m2 = L.MPS(L.config(6, 8, 1024, theta, prec="split_bf16x3"))
    m2.step(-1.0, 2.0, 0.25, 2, 1)
    st = m2.stats()
    assert st["truncations"] == 172
    F = m2.fidelity()
    o = m2.observables()
    assert 0 < F <= 1 + 1e-12
    assert abs(o["Z"]) <= 1 and o["Z2"] <= 1 + 1e-6 and o["Z2"] >= o["Z"] ** 2 - 1e-6
    assert abs(o["norm"] - 1) < 5e-3
    dims = m2.bond_dims()
    assert max(dims) <= 1024 and min(dims) >= 1
    s = np.array(m2.singular_values(len(dims) // 2))
    assert np.all(np.diff(s) <= 1e-6 * s[0]) and np.all(s >= 0)
    assert abs(np.sum(s ** 2) - 1) < 5e-3
