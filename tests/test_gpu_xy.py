"""The XY workload (MODEL_XY on LATTICE_2D_SITES) against the oracle (oracle/xy.py).

Supplemental Material, section "XY Model": H_XY = (g/2) sum (X X + Y Y) on an open grid, one qubit
per site, the depth-7 Trotter step over the bond sets A..D, the initial state of Eq. xy_init
(|Neel>, Trotter steps of g dtau = 0.02 pi, the staggered Z phases pi/8) and the signal
<X_stag^2> of Eq. xy_signal.  Every two-qubit gate runs by SWAP routing with a two-site update
carrying the whole 4 x 4 gate.  FP64 form: 1e-9 on <Z_tot> (conserved: U(1)), <X_stag^2> and
relative on F, against the state vector at exact chi, and against the oracle's TEBD from seeded
random states (the U(1)-symmetric runs from |Neel> meet exact Schmidt-value ties at the chi cut).
Split form: exact chi against the state vector within SPLIT_XY_BOUND.
"""
import numpy as np
import pytest

from oracle import mps, xy

pytestmark = pytest.mark.gpu
TOL = 1e-9
# <X_stag^2>, <Z_tot> and 1 - F of the split form at exact chi (complex64 storage, FP32 Jacobi SVD
# of every two-site update)
SPLIT_XY_BOUND = 1e-4


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def _gpu_xy(L, Lx, Ly, chi, steps, prep, prec="fp64"):
    m = L.MPS(L.xy_config(Lx, Ly, chi, xy.G_PAPER, xy.DT_PAPER, prec=prec))
    m.step(xy.G_PAPER, 0.0, xy.DTAU_PAPER, 2, prep)
    m.apply_layer(L.LAYER_ZSTAG, np.pi / 8)
    rec = {"Z": [], "X2": [], "F": []}
    for i in range(steps + 1):
        if i:
            m.step(xy.G_PAPER, 0.0, xy.DT_PAPER, 2, 1)
        rec["Z"].append(m.observables()["Z"])
        rec["X2"].append(m.expect(L.X_STAG2))
        rec["F"].append(m.fidelity())
    return {k: np.array(v) for k, v in rec.items()}, m


@pytest.mark.parametrize("dims,prep", [((3, 3), 3), ((3, 4), 5), ((2, 4), 1)])
def test_exact_chi_equals_statevector(L, dims, prep):
    Lx, Ly = dims
    steps = 4
    ex, _ = xy.sv_run(Lx, Ly, steps, prep)
    g, m = _gpu_xy(L, Lx, Ly, 2 ** ((Lx * Ly) // 2), steps, prep)
    assert np.abs(g["Z"] - ex["Z"]).max() < TOL
    assert np.abs(g["X2"] - ex["X2"]).max() < TOL
    assert abs(g["F"][-1] - 1) < 1e-12
    assert abs(g["X2"][0] - ex["X2"][0]) < TOL and np.abs(g["X2"][1:] - g["X2"][0]).max() > 1e-3
    # every gate: 2 (q - p - 1) + 1 two-site truncations, seven sets per step
    sched = xy.schedule(Lx, Ly)
    per_step = sum(w_n * sum(2 * (q - p - 1) + 1 for (p, q, *_r) in sched[s])
                   for s, w_n in (("A", 2), ("B", 2), ("C", 2), ("D", 1)))
    assert m.stats()["truncations"] == (steps + prep) * per_step


@pytest.mark.parametrize("dims,chi,seed", [((3, 4), 16, 1), ((4, 4), 24, 2)])
def test_truncated_random_state_against_oracle(L, dims, chi, seed, tmp_path):
    from test_gpu_parity import _write_checkpoint
    Lx, Ly = dims
    r = mps.random_canonical(Lx, Ly, chi, seed, sites=xy.blocks(Lx, Ly))
    o = xy.XYMPS(Lx, Ly, chi)
    o.blocks, o.centre = r.blocks, r.centre
    cfg = L.xy_config(Lx, Ly, chi, xy.G_PAPER, xy.DT_PAPER)
    p = str(tmp_path / "xy_rand.bin")
    _write_checkpoint(L, p, cfg, o)
    g = L.MPS.load_checkpoint(p)
    assert abs(g.expect(L.X_STAG2) - o.x_stag2()) < TOL  # the signal of the loaded state
    sched = xy.schedule(Lx, Ly)
    for _ in range(2):
        o.step(xy.G_PAPER, xy.DT_PAPER, sched)
        g.step(xy.G_PAPER, 0.0, xy.DT_PAPER, 2, 1)
    assert min(o.cut_gaps) > 1e-4 and o.F < 1
    assert abs(g.expect(L.X_STAG2) - o.x_stag2()) < TOL
    assert abs(g.observables()["Z"] - o.observables()[0]) < TOL
    assert abs(g.fidelity() / o.F - 1) < TOL
    assert g.bond_dims() == o.bond_dims()


def test_split_form_exact_chi(L):
    Lx, Ly, steps, prep = 3, 4, 4, 3
    ex, _ = xy.sv_run(Lx, Ly, steps, prep)
    g, _ = _gpu_xy(L, Lx, Ly, 64, steps, prep, prec="split_bf16x3")
    ex2 = np.abs(g["X2"] - ex["X2"]).max()
    ez = np.abs(g["Z"] - ex["Z"]).max()
    print("split form XY 3x4 exact chi vs state vector: |d X2| %.2e, |d Z| %.2e, |1 - F| %.2e"
          % (ex2, ez, abs(1 - g["F"][-1])))
    assert ex2 < SPLIT_XY_BOUND and ez < SPLIT_XY_BOUND and abs(1 - g["F"][-1]) < SPLIT_XY_BOUND


def test_xy_rejects_tfim_layers(L):
    m = L.MPS(L.xy_config(3, 3, 8, xy.G_PAPER, xy.DT_PAPER))
    for layer in (L.LAYER_X, L.LAYER_ZZ):
        with pytest.raises(L.MpsgbError):
            m.apply_layer(layer, 0.1)
    with pytest.raises(L.MpsgbError):
        m.step(1.0, 0.0, 0.1, 1, 1)
