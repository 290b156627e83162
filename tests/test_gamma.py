"""Fidelity rescaling of <Z_tot^2> (Sec. III, Eq. z2_tot_rescaled, Table gamma_scaling,
Table scaling_error_params): the host-side fits, pinned on data whose answers are known, and the
pipeline run end to end on the oracle's data at a size with an exact state."""
import math

import numpy as np

from oracle import model
from oracle import mps as omps
from paper_2511_23438_gb300 import gamma


def _synthetic(g0, steps=20, seed=1):
    rng = np.random.default_rng(seed)
    F = np.cumprod(1 - rng.uniform(0.001, 0.02, steps))
    ex = rng.uniform(0.1, 0.4, steps)
    return ex, ex * F ** (-g0), F


def test_exact_exponent_is_recovered():
    ex, z2, F = _synthetic(1.37)
    g, err = gamma.gamma_star(ex, z2, F)
    assert abs(g - 1.37) < 1e-7 and err < 1e-9
    assert np.allclose(gamma.gamma_tilde(ex, z2, F), 1.37, atol=1e-12)


def test_minimax_against_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(5):
        F = np.cumprod(1 - rng.uniform(0.001, 0.05, 20))
        ex = rng.uniform(0.05, 0.5, 20)
        z2 = ex * rng.uniform(0.6, 1.1, 20)
        g, err = gamma.gamma_star(ex, z2, F)
        grid = np.linspace(-2, 6, 160001)
        brute = min(gamma.max_abs_error(x, ex, z2, F) for x in grid[::16])
        fine = [gamma.max_abs_error(x, ex, z2, F) for x in np.linspace(g - 1e-3, g + 1e-3, 2001)]
        assert err <= brute + 1e-12 and err <= min(fine) + 1e-12


def test_gamma_tilde_undefined_points():
    t = gamma.gamma_tilde([0.2, 0.2, 0.2], [0.1, 0.3, 0.2], [1.0, 0.9, 0.8])
    assert math.isnan(t[0]) and abs(t[1] - math.log(2 / 3) / math.log(0.9)) < 1e-12 and t[2] == 0


def test_line_and_error_fits():
    chis = np.array([4, 8, 16, 32, 8, 16, 64])
    ns = np.array([12, 12, 12, 12, 16, 16, 16])
    x = np.log2(chis) / ns
    a, b = gamma.fit_gamma_line(chis, ns, 1.8252 * x - 0.13)
    assert abs(a - 1.8252) < 1e-12 and abs(b + 0.13) < 1e-12
    a0, b0 = gamma.fit_gamma_line(chis, ns, 2.588 * x, with_intercept=False)
    assert abs(a0 - 2.588) < 1e-12 and b0 == 0
    K, alpha = gamma.fit_error_scaling(chis, ns, 0.24 * chis ** (-24.4 / ns))
    assert abs(K - 0.24) < 1e-10 and abs(alpha + 24.4) < 1e-9


def test_bond_bound_matches_layout():
    from oracle import layout
    for g in [(3, 3), (3, 4), (4, 4), (4, 5), (5, 6), (6, 8), (7, 8)]:
        assert gamma.exact_bond_bound(*g) == max(layout.bond_bounds(*g))


def oracle_runs(grids, chis, dtheta, steps=20):
    theta = model.initial_theta(dtheta)
    runs, exact = {}, {}
    for (Lx, Ly) in grids:
        r = omps.run(Lx, Ly, gamma.exact_bond_bound(Lx, Ly), theta, -1.0, 2.0, 0.25, steps)
        assert max(abs(f - 1) for f in r["F"]) < 1e-12
        exact[(Lx, Ly)] = np.array(r["Z2"][1:])
        for chi in chis:
            t = omps.run(Lx, Ly, chi, theta, -1.0, 2.0, 0.25, steps)
            runs[((Lx, Ly), chi)] = (np.array(t["Z2"][1:]), np.array(t["F"][1:]))
    return runs, exact


def test_pipeline_on_oracle_data():
    runs, exact = oracle_runs([(3, 3)], [4, 8], model.TEMPERATURES["mid"])
    out = gamma.analyse(runs, exact)
    assert len(out["rows"]) == 2
    for r in out["rows"]:
        # gamma = 0 is in the bracket, so the minimax error cannot exceed the unrescaled one
        assert r["max_err_rescaled"] <= r["max_err_mps"] + 1e-12
        assert np.isfinite(r["gamma_star"])
