"""SWAP routing of non-adjacent inter-block gates (route MPSGB_ROUTE_SWAP) against the oracle.

A gate between blocks p and q is applied by moving block q next to block p with two-site SWAP
updates, one two-site update carrying the gate's diagonal phase, and the moves back; every
two-site update is an SVD truncation (2 (q - p - 1) + 1 per gate).  The oracle takes the dense
two-site tensor and numpy.linalg.svd at every one of them (oracle.mps.MPS.zz_inter_swap).
FP64 form: 1e-9 on <Z_tot>, <Z_tot^2>, <X_tot> and relative on F, over 3x4 runs from the paper's
product state (truncating at chi = 16, exact at chi = 64) and two steps of a seeded random
canonical 5x6 MPS (d = 8, chi = 32); at chi = 64 the 3x4 run also equals the state vector and
the MPO route.  Split form: the tie-free 3x4 run at chi = 21 within SPLIT_SWAP_BOUND.
"""
import numpy as np
import pytest

from oracle import layout, model, mps
from oracle import statevector as sv

pytestmark = pytest.mark.gpu
TOL = 1e-9
TH_MID = model.initial_theta(model.TEMPERATURES["mid"])
# observables and |dF/F|, split form, 3x4 chi = 21, ten first-order steps: measured 7.1e-5 and
# 6.8e-5 on a GB300 (FP32 rounding through 140 two-site truncations of gaps down to 4e-5)
SPLIT_SWAP_BOUND = 3e-4


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def _gpu_run(L, Lx, Ly, chi, steps, order, prec="fp64"):
    m = L.MPS(L.config(Lx, Ly, chi, TH_MID, prec=prec, order=order, route=L.ROUTE_SWAP))
    rec = {"Z": [], "Z2": [], "X": [], "F": []}
    for i in range(steps + 1):
        if i:
            m.step(-1.0, 2.0, 0.25, order, 1)
        o = m.observables()
        for k in ("Z", "Z2", "X"):
            rec[k].append(o[k])
        rec["F"].append(m.fidelity())
    return {k: np.array(v) for k, v in rec.items()}, m


# first order from the product state is tie-free at these chi (relative gaps > 3e-5 at every cut);
# second-order runs of the uniform product state meet near-ties under SWAP routing (the permuted
# chains inherit the lattice symmetry), so the second order is covered exactly (chi = 64) and by
# the random 5x6 state
@pytest.mark.parametrize("chi,order", [(16, 1), (21, 1), (64, 2)])
def test_swap_route_3x4_against_oracle(L, chi, order):
    steps = 10
    o = mps.run(3, 4, chi, TH_MID, -1.0, 2.0, 0.25, steps, order=order, route="swap")
    if chi < 64:  # at chi = 64 only numerically zero values are dropped (no truncation to compare)
        assert o["min_cut_gap"] > 1e-5
    g, m = _gpu_run(L, 3, 4, chi, steps, order)
    for k in ("Z", "Z2", "X"):
        assert np.abs(g[k] - o[k]).max() < TOL, k
    assert np.abs(g["F"] / o["F"] - 1).max() < TOL
    _, inter = layout.schedule(3, 4)
    per_step = sum(2 * (gt[1] - gt[0] - 1) + 1 for gt in inter)
    assert m.stats()["truncations"] == steps * per_step
    if chi == 64:  # exact: equals the state vector (and hence the MPO route)
        ex, _ = sv.run(3, 4, TH_MID, -1.0, 2.0, 0.25, steps, order=order)
        for k in ("Z", "Z2", "X"):
            assert np.abs(g[k] - ex[k]).max() < TOL
        assert abs(g["F"][-1] - 1) < 1e-12


def test_swap_route_5x6_random_state(L, tmp_path):
    from test_gpu_parity import _random_canonical_blocks, _write_checkpoint
    chi = 32
    m = _random_canonical_blocks(5, 6, chi, seed=75)  # every cut separated by > 3e-5 s_0
    cfg = L.config(5, 6, chi, TH_MID, prec="fp64", route=L.ROUTE_SWAP)
    p = str(tmp_path / "swap.bin")
    _write_checkpoint(L, p, cfg, m)
    g = L.MPS.load_checkpoint(p)
    alpha, phi = model.layer_angles(-1.0, 2.0, 0.25, 2)
    intra, inter = layout.schedule(5, 6)
    for _ in range(2):
        m.x_layer(alpha)
        m.zz_intra(phi, intra)
        for gt in inter:
            m.zz_inter_swap(gt, phi)
        m.x_layer(alpha)
        g.step(-1.0, 2.0, 0.25, 2, 1)
    assert min(m.cut_gaps) > 1e-5
    z, z2, x, _ = m.observables()
    o = g.observables()
    err = max(abs(o["Z"] - z), abs(o["Z2"] - z2), abs(o["X"] - x))
    ferr = abs(g.fidelity() / m.F - 1)
    print("fp64 SWAP route vs oracle: max |d obs| %.2e, |dF/F| %.2e" % (err, ferr))
    assert err < TOL and ferr < TOL
    assert g.bond_dims() == m.bond_dims()


def test_swap_route_split_form_3x4(L):
    # the split form (complex64; at chi = 21 every contraction is below the tensor-core tile, so
    # this is its FP32 CUDA-core arithmetic with the complex64 Jacobi SVD) on the tie-free 3x4 run.
    # A random 5x6 state is not used here: SWAP truncation of its nearly flat spectra keeps
    # F ~ 1e-3 after one layer, and its near-ties at the cuts turn FP32 rounding into O(1e-3)
    # differences of the kept states, which says nothing about the implementation.
    steps = 10
    o = mps.run(3, 4, 21, TH_MID, -1.0, 2.0, 0.25, steps, order=1, route="swap")
    g, _ = _gpu_run(L, 3, 4, 21, steps, 1, prec="split_bf16x3")
    err = max(np.abs(g[k] - o[k]).max() for k in ("Z", "Z2", "X"))
    ferr = np.abs(g["F"] / o["F"] - 1).max()
    print("split SWAP route vs oracle (3x4, chi = 21): max |d obs| %.2e, |dF/F| %.2e" % (err, ferr))
    assert err < SPLIT_SWAP_BOUND and ferr < SPLIT_SWAP_BOUND
