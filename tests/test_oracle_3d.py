"""Pins of the oracle's 3D TFIM variant (Supplemental Material, section "3D Transverse Field Ising
Model"): open Lx x Ly x Lz cubic grid, one qubit per MPS site along a 3D snake, the product state
of Eq. initial_state, theta_min with the cubic coordination 6, temperatures 0, pi/9, 2 pi/9.

The lattice is pinned by brute force over coordinates (all pairs at Manhattan distance 1), the
state vector by scipy's expm of the dense layer Hamiltonians built from those pairs, and the MPS
by the state vector at exact chi.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import layout, model, mps
from oracle import statevector as sv

TH3_MID = model.initial_theta(model.TEMPERATURES_3D["mid"], coordination=model.COORDINATION_3D)


def _coords(Lx, Ly, Lz):
    # qubit (x, y, z) -> index (z Lx + x) Ly + y, as the lattice's documented numbering
    return {(z * Lx + x) * Ly + y: (x, y, z) for x in range(Lx) for y in range(Ly) for z in range(Lz)}


def _bruteforce_bonds(Lx, Ly, Lz):
    c = _coords(Lx, Ly, Lz)
    out = []
    for a, b in itertools.combinations(sorted(c), 2):
        if sum(abs(u - v) for u, v in zip(c[a], c[b])) == 1:
            out.append((a, b))
    return sorted(out)


@pytest.mark.parametrize("dims", [(2, 2, 2), (2, 3, 4), (3, 3, 4), (4, 2, 3)])
def test_bonds_equal_bruteforce_and_count(dims):
    Lx, Ly, Lz = dims
    b = model.lattice_bonds_3d(Lx, Ly, Lz)
    assert b == _bruteforce_bonds(Lx, Ly, Lz)
    # open cubic grid: 3 n - (Ly Lz + Lx Lz + Lx Ly) bonds
    assert len(b) == 3 * Lx * Ly * Lz - (Ly * Lz + Lx * Lz + Lx * Ly)


@pytest.mark.parametrize("dims", [(2, 2, 2), (2, 3, 4), (3, 3, 4), (3, 4, 2)])
def test_snake_is_a_hamiltonian_path(dims):
    Lx, Ly, Lz = dims
    blks = layout.blocks_3d(Lx, Ly, Lz)
    c = _coords(Lx, Ly, Lz)
    qs = [b["qubits"][0] for b in blks]
    assert sorted(qs) == list(range(Lx * Ly * Lz)) and all(b["d"] == 2 for b in blks)
    for a, b in zip(qs, qs[1:]):  # consecutive sites are lattice neighbours
        assert sum(abs(u - v) for u, v in zip(c[a], c[b])) == 1
    assert c[qs[0]] == (0, 0, 0)


def test_schedule_3d_is_complete_and_sorted():
    Lx, Ly, Lz = 3, 3, 4
    intra, inter = layout.schedule_3d(Lx, Ly, Lz)
    assert all(not v for v in intra)
    assert len(inter) == len(model.lattice_bonds_3d(Lx, Ly, Lz))
    assert inter == sorted(inter, key=lambda g: (g[0], g[1], g[2], g[3]))
    home = layout.qubit_home(0, 0, layout.blocks_3d(Lx, Ly, Lz))
    for (p, q, qi, qj, ti, tj) in inter:
        assert p < q and ti == 0 and tj == 0 and home[qi][0] == p and home[qj][0] == q
    # the nearest neighbours along the snake are adjacent sites; z-neighbours span up to 2 Lx Ly - 1
    dist = [g[1] - g[0] for g in inter]
    assert dist.count(1) == Lx * Ly * Lz - 1 and max(dist) == 2 * Lx * Ly - 1


def test_theta_min_3d_closed_form():
    # sin theta_min = h / (6 J) = -1/3 at J = -1, h = 2; the mean-field energy of a bulk site
    # (three bonds per site) is stationary and minimal there
    t = model.theta_min(-1.0, 2.0, model.COORDINATION_3D)
    assert abs(math.sin(t) + 1.0 / 3.0) < 1e-15
    e = lambda th: model.mean_field_energy_per_site(th, -1.0, 2.0, model.COORDINATION_3D)
    assert abs(e(t) - (-3.0 * (8.0 / 9.0) - 2.0 / 3.0)) < 1e-14
    for dt_ in (1e-3, -1e-3, 0.3, -0.3):
        assert e(t + dt_) > e(t)
    assert model.TEMPERATURES_3D == {"low": 0.0, "mid": math.pi / 9, "high": 2 * math.pi / 9}


def _dense(Lx, Ly, Lz):
    n = Lx * Ly * Lz
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)

    def site(op, q):  # qubit 0 is the most significant bit
        return np.kron(np.kron(np.eye(2 ** q), op), np.eye(2 ** (n - q - 1)))

    HX = sum(site(X, q) for q in range(n))
    HZZ = sum(site(Z, a) @ site(Z, b) for a, b in _bruteforce_bonds(Lx, Ly, Lz))
    return HX, HZZ


@pytest.mark.parametrize("order", [1, 2])
def test_statevector_3d_equals_expm_product(order):
    Lx, Ly, Lz, J, h, dt, steps = 2, 2, 2, -1.0, 2.0, 0.25, 3
    HX, HZZ = _dense(Lx, Ly, Lz)
    if order == 2:
        UX = scipy.linalg.expm(-1j * dt * h * HX / 2)
        U = UX @ scipy.linalg.expm(-1j * dt * J * HZZ) @ UX
    else:
        U = scipy.linalg.expm(-1j * dt * J * HZZ) @ scipy.linalg.expm(-1j * dt * h * HX)
    rec, psi = sv.run(Lx, Ly, TH3_MID, J, h, dt, steps, order=order, Lz=Lz)
    ref = sv.product_state(8, TH3_MID)
    for _ in range(steps):
        ref = U @ ref
    assert np.abs(psi - ref).max() < 1e-12


@pytest.mark.parametrize("dims,order", [((2, 2, 3), 2), ((2, 2, 3), 1), ((2, 3, 2), 2)])
def test_mps_3d_exact_chi_equals_statevector(dims, order):
    Lx, Ly, Lz = dims
    chi = max(layout.bond_bounds(0, 0, layout.blocks_3d(Lx, Ly, Lz)))
    rec, psi = sv.run(Lx, Ly, TH3_MID, -1.0, 2.0, 0.25, 3, order=order, Lz=Lz)
    r = mps.run(Lx, Ly, chi, TH3_MID, -1.0, 2.0, 0.25, 3, order=order, Lz=Lz)
    for k in ("Z", "Z2", "X"):
        assert np.abs(r[k] - rec[k]).max() < 1e-10
    assert abs(r["F"][-1] - 1.0) < 1e-12
    assert abs(np.vdot(psi, r["mps"].to_statevector())) ** 2 > 1 - 1e-10


def test_mps_3d_truncated_norm_and_fidelity_identity():
    # below the exact chi: F is the product of the truncation fidelities and the state stays
    # normalised; at chi = 1 with J = 0 the product state evolves exactly (no entanglement)
    r = mps.run(2, 3, 4, TH3_MID, -1.0, 2.0, 0.25, 2, order=2, Lz=3)
    assert r["F"][-1] < 1.0 and abs(r["F"][-1] - np.prod(r["fidelities"])) < 1e-14
    assert abs(np.linalg.norm(r["mps"].to_statevector()) - 1.0) < 1e-12
    z = mps.run(2, 3, 1, TH3_MID, 0.0, 2.0, 0.25, 3, order=2, Lz=3)
    ex, _ = sv.run(2, 3, TH3_MID, 0.0, 2.0, 0.25, 3, order=2, Lz=3)
    assert np.abs(z["Z"] - ex["Z"]).max() < 1e-12 and abs(z["F"][-1] - 1) < 1e-12
