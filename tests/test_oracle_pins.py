"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
symmetries, a library routine (scipy.linalg.expm), brute force on a dense vector,
or values printed in the paper (tests/golden/).  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import layout, model, mps, rescale
from oracle import statevector as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TH_MID = model.initial_theta(model.TEMPERATURES["mid"])


# ------------------------------------------------------------------ model (Sec. II)
def test_theta_min_closed_form():
    # sin(theta_min) = h / (4 J) = -1/2  ->  theta_min = -pi/6 for J=-1, h=2
    assert abs(model.theta_min(-1.0, 2.0) + math.pi / 6) < 1e-15
    # mean-field energy per site at theta_min: -2 cos^2 + 2 sin = -3/2 - 1 = -5/2
    assert abs(model.mean_field_energy_per_site(model.theta_min()) + 2.5) < 1e-14
    # and it is the minimum (finite differences on both sides)
    t0 = model.theta_min()
    e0 = model.mean_field_energy_per_site(t0)
    for dt in (1e-3, -1e-3, 0.2, -0.2):
        assert model.mean_field_energy_per_site(t0 + dt) > e0


def test_temperature_presets():
    assert model.TEMPERATURES["low"] == 0.0
    assert abs(model.TEMPERATURES["mid"] - 2 * math.pi / 9) < 1e-15
    assert abs(model.TEMPERATURES["high"] - math.pi / 3) < 1e-15


def test_lattice_bonds_pbc_counts():
    # 2 bonds per site on a periodic square lattice with both sides >= 3
    for (Lx, Ly) in [(3, 3), (3, 4), (4, 4), (5, 6), (6, 8)]:
        bonds = model.lattice_bonds(Lx, Ly)
        assert len(bonds) == 2 * Lx * Ly
        deg = np.zeros(Lx * Ly, dtype=int)
        for a, b in bonds:
            deg[a] += 1
            deg[b] += 1
        assert np.all(deg == 4)
    # side of length 2: the wrap bond coincides with the inner one and is counted once
    assert len(model.lattice_bonds(2, 3)) == 3 + 6


# ------------------------------------------------------------------ layout (Sec. III, Fig. mps_drawing)
def test_layout_3x4_by_hand():
    blk = layout.blocks(3, 4)
    # snake: row 0 left->right, row 1 right->left, row 2 left->right
    assert [b["qubits"] for b in blk] == [[0, 1], [2, 3], [6, 7], [4, 5], [8, 9], [10, 11]]
    assert layout.bond_bounds(3, 4) == [4, 16, 64, 16, 4]
    nb, nintra, dist, ntr = layout.census(3, 4)
    # 24 bonds; 6 inside blocks; inter by hand: row bonds (1-2, 3-0) x3 rows at distance 1,
    # vertical r0-r1: cols 0,1 distance 3, cols 2,3 distance 1; r1-r2: cols 0,1 distance 1,
    # cols 2,3 distance 3; wrap r2-r0: distance 4 for all four columns
    assert (nb, nintra, dist, ntr) == (24, 6, {1: 10, 3: 4, 4: 4}, 38)


def test_layout_odd_row_split():
    blk = layout.blocks(3, 3)
    assert [b["d"] for b in blk] == [4, 2, 2, 4, 4, 2]
    assert blk[0]["qubits"] == [0, 1] and blk[1]["qubits"] == [2]


def test_schedule_is_sorted_and_complete():
    for (Lx, Ly) in [(3, 4), (4, 4), (5, 6)]:
        intra, inter = layout.schedule(Lx, Ly)
        keys = [(g[0], g[1], g[2], g[3]) for g in inter]
        assert keys == sorted(keys)
        assert sum(len(x) for x in intra) + len(inter) == len(model.lattice_bonds(Lx, Ly))


# ------------------------------------------------------------------ state vector (Sec. II)
def _dense_ops(Lx, Ly):
    n = Lx * Ly
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)

    def site(op, q):
        m = np.ones((1, 1), dtype=complex)
        for k in range(n):
            m = np.kron(m, op if k == q else np.eye(2))
        return m

    HX = sum(site(X, q) for q in range(n))
    HZZ = sum(site(Z, a) @ site(Z, b) for a, b in model.lattice_bonds(Lx, Ly))
    return HX, HZZ


@pytest.mark.parametrize("order", [1, 2])
def test_statevector_equals_expm_product(order):
    # library reduction: each Trotter step equals the product of scipy expm of the layer Hamiltonians
    Lx, Ly, J, h, dt, steps = 3, 3, -1.0, 2.0, 0.25, 4
    HX, HZZ = _dense_ops(Lx, Ly)
    if order == 2:
        UX = scipy.linalg.expm(-1j * dt * h * HX / 2)
        U = UX @ scipy.linalg.expm(-1j * dt * J * HZZ) @ UX
    else:
        U = scipy.linalg.expm(-1j * dt * J * HZZ) @ scipy.linalg.expm(-1j * dt * h * HX)
    rec, psi = sv.run(Lx, Ly, TH_MID, J, h, dt, steps, order=order)
    ref = sv.product_state(9, TH_MID)
    for _ in range(steps):
        ref = U @ ref
    assert np.abs(psi - ref).max() < 1e-12


def test_second_order_trotter_converges_as_dt_squared():
    Lx, Ly, J, h, T = 3, 3, -1.0, 2.0, 1.0
    HX, HZZ = _dense_ops(Lx, Ly)
    exact = scipy.linalg.expm(-1j * T * (J * HZZ + h * HX)) @ sv.product_state(9, TH_MID)
    errs = []
    for nstep in (10, 20):
        _, psi = sv.run(Lx, Ly, TH_MID, J, h, T / nstep, nstep, order=2)
        errs.append(np.linalg.norm(psi - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("order", [1, 2])
def test_statevector_J0_closed_form(order):
    # J = 0: every qubit precesses about X; <Z>(s) = cos(theta) cos(2 h s dt), <X> = sin(theta)
    Lx, Ly, h, dt, steps = 3, 4, 2.0, 0.25, 6
    n = Lx * Ly
    rec, _ = sv.run(Lx, Ly, TH_MID, 0.0, h, dt, steps, order=order)
    s = np.arange(steps + 1)
    zc = math.cos(TH_MID) * np.cos(2 * h * s * dt)
    assert np.abs(rec["Z"] - zc).max() < 1e-12
    assert np.abs(rec["Z2"] - (1.0 / n + (1 - 1.0 / n) * zc ** 2)).max() < 1e-12
    assert np.abs(rec["X"] - math.sin(TH_MID)).max() < 1e-12


@pytest.mark.parametrize("grid", [(3, 3), (3, 4), (4, 4)])
def test_statevector_h0_closed_form(grid):
    # h = 0: diagonal circuit; <X_j> = sin(theta) Re[(cos 2Jt + i cos(theta) sin 2Jt)^4], t = s dt
    Lx, Ly = grid
    n, J, dt, steps = Lx * Ly, -1.0, 0.25, 5
    rec, _ = sv.run(Lx, Ly, TH_MID, J, 0.0, dt, steps, order=2)
    t = np.arange(steps + 1) * dt
    ct = math.cos(TH_MID)
    xc = math.sin(TH_MID) * np.real((np.cos(2 * J * t) + 1j * ct * np.sin(2 * J * t)) ** 4)
    assert np.abs(rec["X"] - xc).max() < 1e-12
    assert np.abs(rec["Z"] - ct).max() < 1e-12
    assert np.abs(rec["Z2"] - (1.0 / n + (1 - 1.0 / n) * ct ** 2)).max() < 1e-12


def test_statevector_translation_invariance():
    Lx, Ly = 3, 4
    n = Lx * Ly
    _, psi = sv.run(Lx, Ly, TH_MID, -1.0, 2.0, 0.25, 5, order=2)
    p = np.abs(psi) ** 2
    z = sv._z_values(n).astype(float)
    per_site = z @ p
    assert np.ptp(per_site) < 1e-12


# ------------------------------------------------------------------ MPS TEBD (Sec. III)
@pytest.mark.parametrize("grid,order", [((3, 4), 1), ((3, 4), 2), ((3, 3), 2), ((4, 4), 2)])
def test_mps_exact_chi_equals_statevector(grid, order):
    Lx, Ly = grid
    chi = max(layout.bond_bounds(Lx, Ly))
    steps = 4 if grid != (4, 4) else 2
    rec, psi = sv.run(Lx, Ly, TH_MID, -1.0, 2.0, 0.25, steps, order=order)
    r = mps.run(Lx, Ly, chi, TH_MID, -1.0, 2.0, 0.25, steps, order=order)
    for k in ("Z", "Z2", "X"):
        assert np.abs(r[k] - rec[k]).max() < 1e-10
    assert abs(r["F"][-1] - 1.0) < 1e-12
    v = r["mps"].to_statevector()
    assert abs(np.vdot(psi, v)) ** 2 > 1 - 1e-10


def test_mps_J0_is_exact_at_chi_1():
    Lx, Ly, h, dt, steps = 3, 4, 2.0, 0.25, 5
    r = mps.run(Lx, Ly, 1, TH_MID, 0.0, h, dt, steps, order=2)
    s = np.arange(steps + 1)
    assert np.abs(r["Z"] - math.cos(TH_MID) * np.cos(2 * h * s * dt)).max() < 1e-12
    assert np.all(r["F"] == 1.0)
    assert r["bond_dims"] == [1] * 5


@pytest.mark.parametrize("chi", [5, 10])
def test_mps_z2_symmetry_under_truncation(chi):
    # P = prod X commutes with every gate; truncation is covariant under the local unitary P,
    # so theta -> pi - theta flips <Z_tot> and keeps <Z^2>, <X>, F, even at chi < bound --
    # provided no singular values are tied at a cut (then several truncations are correct).
    a = mps.run(3, 4, chi, TH_MID, -1.0, 2.0, 0.25, 3, order=2)
    b = mps.run(3, 4, chi, math.pi - TH_MID, -1.0, 2.0, 0.25, 3, order=2)
    assert a["min_cut_gap"] > 1e-9 and b["min_cut_gap"] > 1e-9
    assert a["F"][-1] < 0.99
    assert np.abs(a["Z"] + b["Z"]).max() < 1e-9
    assert np.abs(a["Z2"] - b["Z2"]).max() < 1e-9
    assert np.abs(a["F"] - b["F"]).max() < 1e-9
    c = mps.run(3, 4, 8, math.pi / 2, -1.0, 2.0, 0.25, 3, order=2)
    assert np.abs(c["Z"]).max() < 1e-9


def test_mps_norm_conservation_and_fidelity_identity():
    r = mps.run(3, 4, 8, TH_MID, -1.0, 2.0, 0.25, 4, order=1)
    f = r["fidelities"]
    kept = r["kept_norms"]
    total = kept / f
    assert np.abs(total - 1.0).max() < 1e-12  # unitary gates on a unit-norm state
    assert abs(np.prod(f) - r["F"][-1]) < 1e-14 * len(f)
    assert abs(np.prod(kept) - r["F"][-1]) < 1e-11  # second accumulator agrees
    assert r["F"][-1] < 0.999  # truncation really happened


def _random_canonical_mps(Lx, Ly, dims, seed):
    rng = np.random.default_rng(seed)
    m = mps.MPS(Lx, Ly, 1 << 30, 0.3)
    ds = [b["d"] for b in m.layout]
    bd = [1] + dims + [1]
    m.blocks = [(rng.standard_normal((bd[i], ds[i], bd[i + 1]))
                 + 1j * rng.standard_normal((bd[i], ds[i], bd[i + 1]))) for i in range(len(ds))]
    m.centre = len(ds) - 1
    m.move_centre(0)
    m.blocks[0] /= np.linalg.norm(m.blocks[0])
    return m


def _dense_mps_order(m):
    t = m.blocks[0]
    for b in m.blocks[1:]:
        t = np.tensordot(t, b, axes=([t.ndim - 1], [0]))
    return t.reshape(-1)


@pytest.mark.parametrize("gate_idx", [3, 6, 8, 10, 12])
def test_mps_gate_truncation_equals_bruteforce(gate_idx):
    # brute force: apply the gate to the dense vector and truncate bonds p..q-1 one after the other
    # by SVD of the full reshaped vector (Eckart-Young, sequentially) with renormalisation.
    Lx, Ly, chi = 3, 4, 6
    m = _random_canonical_mps(Lx, Ly, [4, 10, 12, 10, 4], seed=gate_idx)
    m.chi = chi
    _, inter = layout.schedule(Lx, Ly)
    g = inter[gate_idx]
    p, q, _, _, ti, tj = g
    ds = [b["d"] for b in m.layout]
    psi = _dense_mps_order(m).reshape(ds)
    phi = -0.25
    zi = mps.MPS._zdiag(int(math.log2(ds[p])), ti)
    zj = mps.MPS._zdiag(int(math.log2(ds[q])), tj)
    shape = [1] * len(ds)
    shape[p] = ds[p]
    zz = zi.reshape(shape)
    shape = [1] * len(ds)
    shape[q] = ds[q]
    zz = zz * zj.reshape(shape)
    psi = psi * np.exp(-1j * phi * zz)
    fs = []
    for bond in range(p, q):
        left = int(np.prod(ds[: bond + 1]))
        M = psi.reshape(left, -1)
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        k = min(chi, int(np.count_nonzero(s > s[0] * max(M.shape) * np.finfo(float).eps)))
        fs.append(np.sum(s[:k] ** 2) / np.sum(s ** 2))
        psi = (U[:, :k] * (s[:k] / np.sqrt(np.sum(s[:k] ** 2)))) @ Vh[:k]
    m.zz_inter(g, phi)
    assert min(m.fidelities) < 0.999  # the sweep really truncated
    got = _dense_mps_order(m)
    assert np.abs(got - psi.reshape(-1)).max() < 1e-12
    assert np.allclose(m.fidelities, fs, rtol=0, atol=1e-13)


@pytest.mark.parametrize("gate_idx", [3, 6, 10, 12])
def test_mps_swap_route_equals_bruteforce(gate_idx):
    # brute force of SWAP routing on the dense vector (axes = MPS positions): move block q left by
    # exchanging neighbouring axes, truncating the bond between them after each exchange by the SVD
    # of the whole reshaped vector, apply the phase to the adjacent pair, truncate that bond, and
    # exchange back with truncation.  Block distance k gives 2 (k - 1) + 1 truncations.
    Lx, Ly, chi = 3, 4, 6
    m = _random_canonical_mps(Lx, Ly, [4, 10, 12, 10, 4], seed=100 + gate_idx)
    m.chi = chi
    _, inter = layout.schedule(Lx, Ly)
    g = inter[gate_idx]
    p, q, _, _, ti, tj = g
    ds = [b["d"] for b in m.layout]
    psi = _dense_mps_order(m).reshape(ds)
    order = list(range(len(ds)))  # which original block sits at each position
    phi = -0.25
    fs = []

    def truncate(psi, bond):
        dims = psi.shape
        left = int(np.prod(dims[: bond + 1]))
        M = psi.reshape(left, -1)
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        k = min(chi, int(np.count_nonzero(s > s[0] * max(M.shape) * np.finfo(float).eps)))
        fs.append(np.sum(s[:k] ** 2) / np.sum(s ** 2))
        return ((U[:, :k] * (s[:k] / np.sqrt(np.sum(s[:k] ** 2)))) @ Vh[:k]).reshape(dims)

    def exchange(psi, pos):
        perm = list(range(psi.ndim))
        perm[pos], perm[pos + 1] = perm[pos + 1], perm[pos]
        order[pos], order[pos + 1] = order[pos + 1], order[pos]
        return np.transpose(psi, perm)

    for pos in range(q - 1, p, -1):
        psi = truncate(exchange(psi, pos), pos)
    assert order[p + 1] == q
    zi = mps.MPS._zdiag(int(math.log2(ds[p])), ti)
    zj = mps.MPS._zdiag(int(math.log2(ds[q])), tj)
    shape = [1] * len(ds)
    shape[p] = ds[p]
    zz = zi.reshape(shape)
    shape = [1] * len(ds)
    shape[p + 1] = ds[q]
    psi = truncate(psi * np.exp(-1j * phi * zz * zj.reshape(shape)), p)
    for pos in range(p + 1, q):
        psi = truncate(exchange(psi, pos), pos)
    assert order == list(range(len(ds)))
    m.zz_inter_swap(g, phi)
    assert len(m.fidelities) == 2 * (q - p - 1) + 1
    assert min(m.fidelities) < 0.999  # the route really truncated
    got = _dense_mps_order(m)
    assert np.abs(got - psi.reshape(-1)).max() < 1e-12
    assert np.allclose(m.fidelities, fs, rtol=0, atol=1e-13)
    assert [b["qubits"] for b in m.layout] == [b["qubits"] for b in layout.blocks(Lx, Ly)]


@pytest.mark.parametrize("grid,order", [((3, 4), 1), ((3, 4), 2), ((3, 3), 2)])
def test_mps_swap_route_exact_chi_equals_statevector(grid, order):
    # at chi >= every bond bound (also of the permuted chains met while swapping) nothing is cut:
    # SWAP routing reproduces the state vector like the MPO route
    Lx, Ly = grid
    chi = 1 << 12
    rec, psi = sv.run(Lx, Ly, TH_MID, -1.0, 2.0, 0.25, 3, order=order)
    r = mps.run(Lx, Ly, chi, TH_MID, -1.0, 2.0, 0.25, 3, order=order, route="swap")
    for k in ("Z", "Z2", "X"):
        assert np.abs(r[k] - rec[k]).max() < 1e-10
    assert abs(r["F"][-1] - 1.0) < 1e-12
    v = r["mps"].to_statevector()
    assert abs(np.vdot(psi, v)) ** 2 > 1 - 1e-10


def test_mps_observables_and_spectra_against_dense():
    Lx, Ly = 3, 4
    m = _random_canonical_mps(Lx, Ly, [4, 9, 11, 7, 3], seed=7)
    m.move_centre(3)
    v = m.to_statevector()
    z, z2, x, _ = sv.observables(v, Lx * Ly)
    z_, z2_, x_, norm = m.observables()
    assert abs(norm - 1) < 1e-12
    assert abs(z - z_) < 1e-12 and abs(z2 - z2_) < 1e-12 and abs(x - x_) < 1e-12
    ds = [b["d"] for b in m.layout]
    dense = _dense_mps_order(m)
    for bond in range(len(ds) - 1):
        left = int(np.prod(ds[: bond + 1]))
        s_ref = np.linalg.svd(dense.reshape(left, -1), compute_uv=False)
        s = m.singular_values(bond)
        k = len(s)
        assert np.abs(s - s_ref[:k]).max() < 1e-12
        assert np.all(s_ref[k:] < 1e-12)


# ------------------------------------------------------------------ rescaling (Sec. III)
def test_gamma_table_matches_paper_golden():
    with open(os.path.join(GOLDEN, "gamma_scaling.json")) as fh:
        gold = json.load(fh)
    for t in ("low", "mid", "high"):
        assert rescale.GAMMA_TABLE[t] == (gold[t]["a"], gold[t]["b"])
    # mid, chi = 1024, n = 48: 1.8252 * 10 / 48
    assert abs(rescale.gamma_fit("mid", 1024, 48) - 1.8252 * 10 / 48) < 1e-15
    assert abs(rescale.gamma_fit("high", 2, 1) - (1.641 - 0.1298)) < 1e-15


def test_gamma_table_3d_matches_paper_golden():
    with open(os.path.join(GOLDEN, "gamma_scaling_3d.json")) as fh:
        gold = json.load(fh)
    for t in ("low", "mid", "high"):
        assert rescale.GAMMA_TABLE_3D[t] == (gold[t]["a"], gold[t]["b"])
    # mid, chi = 256, n = 36 (the paper's 3x3x4 lattice): 2.153 * 8 / 36
    assert abs(rescale.gamma_fit("mid", 256, 36, three_d=True) - 2.153 * 8 / 36) < 1e-15


def test_rescaling_limits():
    # F -> 1 leaves observables unchanged; gamma = 1 reduces Eq. z2_tot_rescaled to F scaling
    assert rescale.rescale_z(0.3, 1.0) == 0.3
    assert rescale.rescale_z2(0.2, 1.0, 0.7) == 0.2
    assert abs(rescale.rescale_z2(0.2, 0.5, 1.0) - 0.1) < 1e-16


def test_per_qubit_initial_angles():
    # Eq. initial_state with one angle per qubit: <Z_j> = cos(theta_j), <X_j> = sin(theta_j)
    rng = np.random.default_rng(3)
    th = rng.uniform(-1, 1, 12)
    m = mps.MPS(3, 4, 4, th)
    v = m.to_statevector()
    assert np.allclose(v, sv.product_state(12, th), atol=1e-15)
    z, z2, x, _ = m.observables()
    assert abs(z - np.mean(np.cos(th))) < 1e-14 and abs(x - np.mean(np.sin(th))) < 1e-14
    zz = (np.sum(np.cos(th)) ** 2 - np.sum(np.cos(th) ** 2) + 12) / 144
    assert abs(z2 - zz) < 1e-14
