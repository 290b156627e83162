"""Rescaling of <Z_tot^2> by the MPS fidelity: fitting the exponent at sizes with exact data.

The paper (Sec. III, Eq. z2_tot_rescaled) rescales the truncated estimate as
<Z^2>_gamma = <Z^2>_MPS * F_MPS^gamma(n, chi), determines the optimal gamma* of each
(grid, chi) by minimising the maximum absolute error over the Trotter steps against exact data,
fits the linear ansatz gamma_fit = a log2(chi)/n + b (Table gamma_scaling), defines the
unconstrained exponent gamma~ = log(<Z^2>_ex / <Z^2>_MPS) / log F_MPS per data point, and fits
the remaining error as eps = K chi^(alpha/n) (Table scaling_error_params).

This module holds those host-side fits (plain NumPy on arrays) and a pipeline that produces the
data with the GPU library itself: on grids small enough, the FP64 MPS at chi equal to the
largest exact bond dimension is the exact state, so no separate exact simulator is needed.
"""
import math

import numpy as np


def gamma_tilde(z2_ex, z2_mps, F):
    """Per-point exponent that makes the rescaling exact; NaN where it is undefined
    (F = 1, or a ratio that is not positive)."""
    z2_ex, z2_mps, F = (np.asarray(a, dtype=float) for a in (z2_ex, z2_mps, F))
    out = np.full(z2_ex.shape, np.nan)
    ok = (F < 1) & (F > 0) & (z2_mps > 0) & (z2_ex > 0)
    out[ok] = np.log(z2_ex[ok] / z2_mps[ok]) / np.log(F[ok])
    return out


def max_abs_error(gamma, z2_ex, z2_mps, F):
    """max_s |<Z^2>_MPS(s) F(s)^gamma - <Z^2>_ex(s)|."""
    return float(np.max(np.abs(np.asarray(z2_mps) * np.power(np.asarray(F), gamma) - np.asarray(z2_ex))))


def gamma_star(z2_ex, z2_mps, F, lo=-2.0, hi=6.0, tol=1e-10):
    """The exponent minimising the maximum absolute error over the steps (Sec. III).

    Each term |z2 F^gamma - ex| is a monotone function of gamma minus a constant, in absolute
    value, so the maximum is unimodal in gamma: a scan of the bracket locates the minimum to one
    grid cell and golden-section search refines it."""
    f = lambda g: max_abs_error(g, z2_ex, z2_mps, F)
    grid = np.linspace(lo, hi, 801)
    vals = np.array([f(g) for g in grid])
    k = int(np.argmin(vals))
    a, b = grid[max(0, k - 1)], grid[min(len(grid) - 1, k + 1)]
    r = (math.sqrt(5) - 1) / 2
    c, d = b - r * (b - a), a + r * (b - a)
    fc, fd = f(c), f(d)
    while b - a > tol:
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - r * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + r * (b - a)
            fd = f(d)
    g = 0.5 * (a + b)
    return g, f(g)


def fit_gamma_line(chis, ns, gammas, with_intercept=True):
    """Least-squares fit gamma = a log2(chi)/n + b (b = 0 when with_intercept is False)."""
    x = np.log2(np.asarray(chis, dtype=float)) / np.asarray(ns, dtype=float)
    y = np.asarray(gammas, dtype=float)
    if with_intercept:
        A = np.stack([x, np.ones_like(x)], axis=1)
        (a, b), *_ = np.linalg.lstsq(A, y, rcond=None)
        return float(a), float(b)
    return float(np.dot(x, y) / np.dot(x, x)), 0.0


def fit_error_scaling(chis, ns, eps):
    """Least-squares fit of eps = K chi^(alpha/n): ln eps = ln K + alpha ln(chi)/n."""
    x = np.log(np.asarray(chis, dtype=float)) / np.asarray(ns, dtype=float)
    y = np.log(np.asarray(eps, dtype=float))
    A = np.stack([x, np.ones_like(x)], axis=1)
    (alpha, lnK), *_ = np.linalg.lstsq(A, y, rcond=None)
    return float(math.exp(lnK)), float(alpha)


def analyse(runs, exact, with_intercept=True):
    """runs: {(grid, chi): (z2_mps[s], F[s])}; exact: {grid: z2_ex[s]} (grid = (Lx, Ly)).

    Returns per-(grid, chi) gamma*, the errors before and after rescaling, gamma~ over all
    points, and the fits of gamma* and of the mean / max error after rescaling with gamma_fit."""
    rows = []
    for (grid, chi), (z2, F) in sorted(runs.items()):
        ex = np.asarray(exact[grid])
        g, err = gamma_star(ex, z2, F)
        rows.append(dict(grid=grid, n=grid[0] * grid[1], chi=chi, gamma_star=g, max_err_rescaled=err,
                         max_err_mps=float(np.max(np.abs(np.asarray(z2) - ex))),
                         gamma_tilde=gamma_tilde(ex, z2, F)))
    a, b = fit_gamma_line([r["chi"] for r in rows], [r["n"] for r in rows], [r["gamma_star"] for r in rows],
                          with_intercept)
    for r in rows:
        z2, F = runs[(r["grid"], r["chi"])]
        gfit = a * math.log2(r["chi"]) / r["n"] + b
        e = np.abs(np.asarray(z2) * np.power(np.asarray(F), gfit) - np.asarray(exact[r["grid"]]))
        r.update(gamma_fit=gfit, mean_err_fit=float(e.mean()), max_err_fit=float(e.max()))
    out = dict(rows=rows, a=a, b=b)
    usable = [r for r in rows if r["mean_err_fit"] > 0 and r["max_err_fit"] > 0]
    if len(usable) >= 2:
        out["K_mean"], out["alpha_mean"] = fit_error_scaling([r["chi"] for r in usable], [r["n"] for r in usable],
                                                             [r["mean_err_fit"] for r in usable])
        out["K_max"], out["alpha_max"] = fit_error_scaling([r["chi"] for r in usable], [r["n"] for r in usable],
                                                           [r["max_err_fit"] for r in usable])
    return out


def gpu_runs(grids, chis, dtheta, steps=20, J=-1.0, h=2.0, dt=0.25, order=2, stream=None):
    """Data for analyse() from the GPU library (FP64 form): <Z^2> and F after every step for each
    (grid, chi < exact bound), and the exact <Z^2> from the same library at chi = the grid's
    largest exact bond dimension (no truncation: the MPS is the exact state)."""
    from . import build, lib
    build.build()
    lib.load()
    theta = lib.initial_theta(J, h, dtheta)

    def run(Lx, Ly, chi):
        m = lib.MPS(lib.config(Lx, Ly, chi, theta, prec="fp64", J=J, h=h, dt=dt, order=order), stream=stream)
        z2, F = [], []
        for _ in range(steps):
            m.step(J, h, dt, order, 1)
            z2.append(m.observables()["Z2"])
            F.append(m.fidelity())
        m.close()
        return np.array(z2), np.array(F)

    runs, exact = {}, {}
    for (Lx, Ly) in grids:
        bound = exact_bond_bound(Lx, Ly)
        exact[(Lx, Ly)], F = run(Lx, Ly, bound)
        if np.max(np.abs(F - 1)) > 1e-12:
            raise RuntimeError("the run at chi = %d of %dx%d truncated: not exact" % (bound, Lx, Ly))
        for chi in chis:
            if chi < bound:
                runs[((Lx, Ly), chi)] = run(Lx, Ly, chi)
    return runs, exact


def exact_bond_bound(Lx, Ly):
    """Largest exact bond dimension of the grouped MPS of an Lx x Ly grid: over the bonds of the
    snake (blocks of ceil(Ly/2) and floor(Ly/2) qubits, the second row reversed), 2 to the
    smaller number of qubits on either side."""
    ks = []
    for r in range(Lx):
        k0, k1 = (Ly + 1) // 2, Ly // 2
        ks += [k0, k1] if r % 2 == 0 else [k1, k0]
    total, left, best = sum(ks), 0, 0
    for k in ks[:-1]:
        left += k
        best = max(best, min(left, total - left))
    return 1 << best
