"""3D TFIM with one qubit per MPS site (LATTICE_3D_SITES) against the oracle.

Supplemental Material, section "3D Transverse Field Ising Model": open Lx x Ly x Lz cubic grid,
sites along a 3D snake (d = 2), the product state of Eq. initial_state with theta_min at the
cubic coordination 6, temperatures 0, pi/9, 2 pi/9.  Every lattice bond is an inter-site gate;
z-neighbours are up to 2 Lx Ly - 1 sites apart, so most gates span many bonds (MPO route) or move
a site far along the chain (SWAP route).  FP64 form: 1e-9 on <Z_tot>, <Z_tot^2>, <X_tot> and
relative on F against the exact state vector (exact chi) and the oracle's TEBD (truncating chi,
seeded random states: the uniform product state is symmetric and meets exact ties at the cut).
Split form: exact chi against the state vector, and the paper's 3 x 3 x 4 lattice at chi = 32
against the oracle, within SPLIT_3D_BOUND.
"""
import numpy as np
import pytest

from oracle import layout, model, mps
from oracle import statevector as sv

pytestmark = pytest.mark.gpu
TOL = 1e-9
TH3 = {k: model.initial_theta(v, coordination=model.COORDINATION_3D) for k, v in model.TEMPERATURES_3D.items()}
# observables and |dF/F| of the split form (complex64 storage, FP32 truncation core): measured on a
# GB300 at most 9.0e-5 (|d obs|, exact chi, five steps) and 7.6e-5 (|dF/F|, 3x3x4 chi = 32)
SPLIT_3D_BOUND = 3e-4


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def _gpu_run(L, dims, chi, theta, steps, order, prec="fp64", route=0):
    Lx, Ly, Lz = dims
    cfg = L.config(Lx, Ly, chi, theta, prec=prec, order=order, route=route, lattice=L.LATTICE_3D_SITES, Lz=Lz)
    m = L.MPS(cfg)
    rec = {"Z": [], "Z2": [], "X": [], "F": []}
    for i in range(steps + 1):
        if i:
            m.step(-1.0, 2.0, 0.25, order, 1)
        o = m.observables()
        for k in ("Z", "Z2", "X"):
            rec[k].append(o[k])
        rec["F"].append(m.fidelity())
    return {k: np.array(v) for k, v in rec.items()}, m


def test_initial_theta_and_schedule(L):
    for k, th in TH3.items():
        assert abs(L.initial_theta(-1.0, 2.0, model.TEMPERATURES_3D[k], lattice=L.LATTICE_3D_SITES) - th) < 1e-15
    cfg = L.config(3, 3, 32, TH3["mid"], lattice=L.LATTICE_3D_SITES, Lz=4)
    _, inter = layout.schedule_3d(3, 3, 4)
    assert L.schedule_gates(cfg) == [tuple(g) for g in inter]


@pytest.mark.parametrize("order", [1, 2])
def test_exact_chi_equals_statevector(L, order):
    # 2x2x3: 12 qubits, largest exact bond 2^6 = 64
    steps = 5
    ex, _ = sv.run(2, 2, TH3["mid"], -1.0, 2.0, 0.25, steps, order=order, Lz=3)
    g, m = _gpu_run(L, (2, 2, 3), 64, TH3["mid"], steps, order)
    for k in ("Z", "Z2", "X"):
        assert np.abs(g[k] - ex[k]).max() < TOL, k
    assert abs(g["F"][-1] - 1) < 1e-12
    _, inter = layout.schedule_3d(2, 2, 3)
    assert m.stats()["truncations"] == steps * sum(gt[1] - gt[0] for gt in inter)


def _evolve_random(L, dims, chi, seed, steps, tmp_path, prec="fp64", route="mpo", decay=None):
    """Seeded random canonical 3D MPS (generic input: the uniform product state meets exact
    Schmidt-value ties at the chi cut, from the lattice's symmetry), evolved by `steps`
    second-order steps by the oracle and on the GPU; returns (gpu obs+F, oracle obs+F, gap, both)."""
    from test_gpu_parity import _write_checkpoint
    Lx, Ly, Lz = dims
    m = mps.random_canonical(Lx, Ly, chi, seed, decay=decay, Lz=Lz)
    cfg = L.config(Lx, Ly, chi, TH3["mid"], prec=prec, route=L.ROUTE_SWAP if route == "swap" else L.ROUTE_MPO,
                   lattice=L.LATTICE_3D_SITES, Lz=Lz)
    p = str(tmp_path / ("rand3d_%s.bin" % prec))
    _write_checkpoint(L, p, cfg, m, dtype=np.complex128 if prec == "fp64" else np.complex64)
    g = L.MPS.load_checkpoint(p)
    alpha, phi = model.layer_angles(-1.0, 2.0, 0.25, 2)
    _, inter = layout.schedule_3d(Lx, Ly, Lz)
    for _ in range(steps):
        m.x_layer(alpha)
        for gt in inter:
            (m.zz_inter_swap if route == "swap" else m.zz_inter)(gt, phi)
        m.x_layer(alpha)
        g.step(-1.0, 2.0, 0.25, 2, 1)
    z, z2, x, _ = m.observables()
    o = g.observables()
    return (np.array([o["Z"], o["Z2"], o["X"], g.fidelity()]), np.array([z, z2, x, m.F]), min(m.cut_gaps),
            g, m)


@pytest.mark.parametrize("dims,chi,route", [((2, 3, 3), 16, "mpo"), ((3, 3, 4), 32, "mpo"), ((2, 3, 3), 16, "swap")])
def test_truncated_random_state_against_oracle(L, dims, chi, route, tmp_path):
    g, o, gap, gh, om = _evolve_random(L, dims, chi, 1, 2, tmp_path, route=route)
    assert gap > 1e-4 and o[3] < 1.0  # truncating, every cut separated
    assert np.abs(g[:3] - o[:3]).max() < TOL
    assert abs(g[3] / o[3] - 1) < TOL
    assert gh.bond_dims() == om.bond_dims()


def test_split_form_exact_chi_against_statevector(L):
    # 2x2x3, chi = 64 (no truncation beyond numerical zeros): FP32 rounding only
    steps = 5
    ex, _ = sv.run(2, 2, TH3["mid"], -1.0, 2.0, 0.25, steps, order=2, Lz=3)
    g, _ = _gpu_run(L, (2, 2, 3), 64, TH3["mid"], steps, 2, prec="split_bf16x3")
    err = max(np.abs(g[k] - ex[k]).max() for k in ("Z", "Z2", "X"))
    print("split form 2x2x3 exact chi vs state vector: max |d obs| %.2e, |1 - F| %.2e" % (err, abs(1 - g["F"][-1])))
    assert err < SPLIT_3D_BOUND and abs(1 - g["F"][-1]) < SPLIT_3D_BOUND


def test_split_form_3x3x4_random_state(L, tmp_path):
    # the paper's 3x3x4 lattice, chi = 32, a random state whose spectra fall off (decay 8), one step
    g, o, gap, _, _ = _evolve_random(L, (3, 3, 4), 32, 1, 1, tmp_path, prec="split_bf16x3", decay=8.0)
    err = np.abs(g[:3] - o[:3]).max()
    ferr = abs(g[3] / o[3] - 1)
    print("split form 3x3x4 chi = 32 vs FP64 oracle: max |d obs| %.2e, |dF/F| %.2e, gap %.1e" % (err, ferr, gap))
    assert err < SPLIT_3D_BOUND and ferr < SPLIT_3D_BOUND
