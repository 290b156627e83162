"""Pins of the oracle's XY-model workload (Supplemental Material, section "XY Model"; oracle/xy.py).

The gate and the Trotter step are pinned by scipy's expm of Hamiltonians built here from Pauli
matrices and brute-force coordinates, the signal by a dense matrix, the initial state by its
closed-form values, U(1) by the conservation of Z_tot, the second-order step by its dt^2
convergence, and the MPS by the state vector at exact chi.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg

from oracle import layout, xy

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.diag([1.0, -1.0]).astype(complex)


def _site(op, q, n):
    return np.kron(np.kron(np.eye(2 ** q), op), np.eye(2 ** (n - q - 1)))


def _coords_bonds(Lx, Ly):
    # nearest neighbours by brute force over coordinates, each with its set: horizontal bonds
    # starting on an even / odd column are A / B, vertical ones starting on an even / odd row C / D
    out = []
    for (r1, c1), (r2, c2) in itertools.combinations([(r, c) for r in range(Lx) for c in range(Ly)], 2):
        if abs(r1 - r2) + abs(c1 - c2) != 1:
            continue
        if r1 == r2:
            s = "A" if min(c1, c2) % 2 == 0 else "B"
        else:
            s = "C" if min(r1, r2) % 2 == 0 else "D"
        out.append((r1 * Ly + c1, r2 * Ly + c2, s))
    return sorted(out)


@pytest.mark.parametrize("dims", [(2, 2), (3, 4), (4, 4), (5, 6)])
def test_bonds_and_sets(dims):
    Lx, Ly = dims
    b = xy.bonds(Lx, Ly)
    assert sorted(b) == _coords_bonds(Lx, Ly)
    assert len(b) == Lx * (Ly - 1) + (Lx - 1) * Ly
    for s in "ABCD":  # the bonds of one set do not overlap (their gates commute)
        qs = [q for (j, k, t) in b if t == s for q in (j, k)]
        assert len(qs) == len(set(qs))


@pytest.mark.parametrize("dims", [(2, 3), (3, 3), (4, 4)])
def test_snake_and_schedule(dims):
    Lx, Ly = dims
    blks = xy.blocks(Lx, Ly)
    qs = [b["qubits"][0] for b in blks]
    assert sorted(qs) == list(range(Lx * Ly))
    for a, c in zip(qs, qs[1:]):  # consecutive sites are lattice neighbours
        ra, ca = divmod(a, Ly)
        rc, cc = divmod(c, Ly)
        assert abs(ra - rc) + abs(ca - cc) == 1
    sched = xy.schedule(Lx, Ly)
    assert sum(len(v) for v in sched.values()) == len(xy.bonds(Lx, Ly))
    home = layout.qubit_home(0, 0, blks)
    for s, gates in sched.items():
        for (p, q, j, k, _, _) in gates:
            assert p < q and home[j][0] == p and home[k][0] == q
    # horizontal bonds are adjacent on the snake, vertical ones span up to 2 Ly - 1 sites
    assert all(q - p == 1 for s in "AB" for (p, q, *_ ) in sched[s])
    assert max(q - p for s in "CD" for (p, q, *_) in sched[s]) == 2 * Ly - 1


@pytest.mark.parametrize("theta", [0.0, 0.1, -0.7, 1.3])
def test_gate_is_expm(theta):
    H = np.kron(X, X) + np.kron(Y, Y)
    assert np.abs(xy.gate(theta) - scipy.linalg.expm(-1j * theta * H)).max() < 1e-14


def _dense_layers(Lx, Ly, g):
    n = Lx * Ly
    Hs = {s: np.zeros((2 ** n, 2 ** n), dtype=complex) for s in "ABCD"}
    for (j, k, s) in _coords_bonds(Lx, Ly):
        Hs[s] += 0.5 * g * (_site(X, j, n) @ _site(X, k, n) + _site(Y, j, n) @ _site(Y, k, n))
    return Hs


def test_trotter_step_equals_expm_product():
    Lx, Ly, g, dt = 2, 3, 1.0, 0.05 * np.pi
    Hs = _dense_layers(Lx, Ly, g)
    E = {s: scipy.linalg.expm(-1j * dt * Hs[s] / 2) for s in "ABC"}
    U = E["A"] @ E["B"] @ E["C"] @ scipy.linalg.expm(-1j * dt * Hs["D"]) @ E["C"] @ E["B"] @ E["A"]
    rng = np.random.default_rng(3)
    psi = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    assert np.abs(xy.sv_step(psi, Lx, Ly, g, dt) - U @ psi).max() < 1e-12


def test_second_order_convergence():
    # error of one time T = 0.4 against exp(-i T H_XY): halving dt divides it by ~4
    Lx, Ly, g, T = 2, 3, 1.0, 0.4
    Hs = _dense_layers(Lx, Ly, g)
    exact = scipy.linalg.expm(-1j * T * sum(Hs.values())) @ xy.sv_neel(Lx, Ly)
    psi0 = xy.sv_zstag(xy.sv_neel(Lx, Ly), Lx, Ly, 0.0)
    errs = []
    for nstep in (4, 8):
        psi = psi0
        for _ in range(nstep):
            psi = xy.sv_step(psi, Lx, Ly, g, T / nstep)
        errs.append(np.linalg.norm(psi - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_neel_closed_forms_and_u1():
    Lx, Ly = 3, 4
    n = Lx * Ly
    psi = xy.sv_neel(Lx, Ly)
    z, x2, nrm = xy.sv_observables(psi, Lx, Ly)
    # Neel: Z_j = -(-1)^j, checkerboard with as many + as -: Z_tot = 0; Z-basis product state:
    # <X_j X_k> = delta_jk, so X^2 = 1/n; the Z phases keep both
    assert abs(z) < 1e-15 and abs(x2 - 1.0 / n) < 1e-15 and abs(nrm - 1) < 1e-15
    psi = xy.sv_zstag(psi, Lx, Ly, np.pi / 8)
    z2, x22, _ = xy.sv_observables(psi, Lx, Ly)
    assert abs(z2) < 1e-15 and abs(x22 - 1.0 / n) < 1e-15
    # U(1): X X + Y Y conserves sum_j Z_j, exactly at every step
    rec, _ = xy.sv_run(Lx, Ly, 4, 3)
    assert np.abs(rec["Z"]).max() < 1e-13
    assert np.abs(rec["X2"][1:] - 1.0 / n).max() > 1e-3  # the signal moves


def test_signal_equals_dense_second_moment():
    Lx, Ly = 2, 2
    n = 4
    M = sum(xy.stag_sign(Ly, j) * _site(X, j, n) for j in range(n))
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    _, x2, nrm = xy.sv_observables(psi, Lx, Ly)
    assert abs(x2 - np.vdot(psi, M @ M @ psi).real / (n * n * nrm)) < 1e-14
    assert [xy.stag_sign(2, j) for j in range(4)] == [1, -1, -1, 1]


@pytest.mark.parametrize("dims,prep", [((3, 3), 3), ((2, 4), 5), ((3, 4), 1)])
def test_mps_exact_chi_equals_statevector(dims, prep):
    Lx, Ly = dims
    chi = 2 ** ((Lx * Ly) // 2)
    steps = 3
    ex, psi = xy.sv_run(Lx, Ly, steps, prep)
    r = xy.run(Lx, Ly, chi, steps, prep)
    assert np.abs(r["Z"] - ex["Z"]).max() < 1e-12
    assert np.abs(r["X2"] - ex["X2"]).max() < 1e-12
    assert abs(r["F"][-1] - 1) < 1e-12
    assert abs(abs(np.vdot(psi, r["mps"].to_statevector())) - 1) < 1e-10


def test_mps_truncated_fidelity_identity():
    r = xy.run(3, 4, 6, 2, 3)
    assert r["F"][-1] < 1 and abs(r["F"][-1] - np.prod(r["fidelities"])) < 1e-14
    assert abs(np.linalg.norm(r["mps"].to_statevector()) - 1) < 1e-12
