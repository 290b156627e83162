"""GPU path (CUDA library through the C ABI) against the CPU oracle.

Element-by-element parity of gauge-invariant quantities on the same inputs:
observables <Z_tot>, <Z_tot^2>, <X_tot> (Eq. Z_tot, Eq. z2_tot), F_MPS (product of
truncation fidelities, Sec. III) and Schmidt spectra.  Tolerance of the FP64 form:
1e-9 absolute on observables and spectra (relative to s_0), 1e-9 relative on F.
Cases are tie-free at the chi cut (the oracle records the smallest relative gap);
where singular values tie, several truncations are equally correct.
"""
import math
import os
import struct

import numpy as np
import pytest

from oracle import layout, model, mps
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

TOL = 1e-9
TH_MID = model.initial_theta(model.TEMPERATURES["mid"])


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def run_gpu(L, Lx, Ly, chi, theta, J, h, dt, steps, order, prec="fp64"):
    m = L.MPS(L.config(Lx, Ly, chi, theta, prec=prec, J=J, h=h, dt=dt, order=order))
    rec = {"Z": [], "Z2": [], "X": [], "F": [], "norm": []}

    def record():
        o = m.observables()
        for k in ("Z", "Z2", "X", "norm"):
            rec[k].append(o[k])
        rec["F"].append(m.fidelity())

    record()
    for _ in range(steps):
        m.step(J, h, dt, order, 1)
        record()
    return {k: np.array(v) for k, v in rec.items()}, m


def assert_parity(g, o, tol=TOL, upto=None):
    sl = slice(0, upto)
    for k in ("Z", "Z2", "X"):
        err = np.abs(g[k][sl] - o[k][sl]).max()
        assert err < tol, (k, err)
    ferr = np.abs(g["F"][sl] / o["F"][sl] - 1).max()
    assert ferr < tol, ("F", ferr)
    assert np.abs(g["norm"] - 1).max() < 1e-10


@pytest.mark.parametrize("chi,order,tol", [(16, 1, TOL), (21, 2, TOL), (64, 1, TOL), (64, 2, TOL)])
def test_c1_3x4_parity(L, chi, order, tol):
    # 3x4 grid, d = 4, 20 steps, dtheta = 2 pi/9; chi = 64 is exact, the others truncate
    # with every cut well separated (relative gap > 5e-5)
    o = mps.run(3, 4, chi, TH_MID, -1.0, 2.0, 0.25, 20, order=order)
    assert o["min_cut_gap"] > 5e-5
    g, m = run_gpu(L, 3, 4, chi, TH_MID, -1.0, 2.0, 0.25, 20, order)
    assert_parity(g, o, tol=tol)
    if chi == 64:
        ex, _ = sv.run(3, 4, TH_MID, -1.0, 2.0, 0.25, 20, order=order)
        for k in ("Z", "Z2", "X"):
            assert np.abs(g[k] - ex[k]).max() < TOL
        assert abs(g["F"][-1] - 1) < 1e-12
    st = m.stats()
    assert st["truncations"] == 20 * 38


def test_c1_paper_config_near_tie(L):
    # the paper's second-order 3x4 run at chi = 16 has a near-tie at one cut (relative gap
    # 2.4e-6); rounding differences are amplified by 1/gap, so the bound here is 1e-6
    o = mps.run(3, 4, 16, TH_MID, -1.0, 2.0, 0.25, 20, order=2)
    g, _ = run_gpu(L, 3, 4, 16, TH_MID, -1.0, 2.0, 0.25, 20, 2)
    assert o["min_cut_gap"] > 1e-6
    assert_parity(g, o, tol=1e-6)


def assert_spectra_equal(s, s_ref, tol=TOL):
    """Schmidt spectra equal value by value to tol * s_0, every value down to the last one the
    oracle resolves; values present on one side only (numerically zero on the other) must be
    below tol * s_0 as well."""
    s = np.asarray(s, dtype=np.float64)
    s_ref = np.asarray(s_ref, dtype=np.float64)
    n = min(len(s), len(s_ref))
    assert np.abs(s[:n] - s_ref[:n]).max() < tol * s_ref[0], (np.abs(s[:n] - s_ref[:n]).max(), s_ref[0])
    assert np.all(np.abs(s[n:]) < tol * s_ref[0]) and np.all(np.abs(s_ref[n:]) < tol * s_ref[0])


def _random_canonical_blocks(Lx, Ly, chi, seed, decay=None, centre=0):
    """Seeded random canonical MPS from the oracle (see oracle.mps.random_canonical)."""
    return mps.random_canonical(Lx, Ly, chi, seed, decay=decay, centre=centre)


def _write_checkpoint(L, path, cfg, m, dtype=np.complex128):
    # layout of mpsgb_save: magic, config, {real bytes, blocks, centre, 0}, F, 5 counters,
    # bond dims, then every block (left, d, right) row-major complex128 (FP64 form) or complex64
    with open(path, "wb") as fh:
        fh.write(b"MPSGBv2\0")
        fh.write(bytes(cfg))
        fh.write(struct.pack("4i", 8 if dtype == np.complex128 else 4, len(m.blocks), m.centre, 0))
        fh.write(struct.pack("d", 1.0))
        fh.write(struct.pack("5q", 0, 0, 0, 0, 0))
        fh.write(struct.pack("%di" % (len(m.blocks) - 1), *[b.shape[2] for b in m.blocks[:-1]]))
        for b in m.blocks:
            fh.write(np.ascontiguousarray(b, dtype=dtype).tobytes())


@pytest.mark.parametrize("chi", [32, 64])
def test_c2_5x6_parity_random_state(L, chi, tmp_path):
    # 5x6 grid (rows split 3 + 3, d = 8, 10 blocks), generic input: a seeded random canonical
    # MPS at chi, evolved by two second-order steps on both sides
    m = _random_canonical_blocks(5, 6, chi, seed=chi)
    cfg = L.config(5, 6, chi, TH_MID)
    p = str(tmp_path / "rand.bin")
    _write_checkpoint(L, p, cfg, m)
    g = L.MPS.load_checkpoint(p)
    o0 = g.observables()
    z, z2, x, nrm = m.observables()
    assert abs(o0["Z"] - z) < TOL and abs(o0["Z2"] - z2) < TOL and abs(o0["X"] - x) < TOL
    alpha, phi = model.layer_angles(-1.0, 2.0, 0.25, 2)
    intra, inter = layout.schedule(5, 6)
    for _ in range(2):
        m.x_layer(alpha)
        m.zz_intra(phi, intra)
        for gt in inter:
            m.zz_inter(gt, phi)
        m.x_layer(alpha)
        g.step(-1.0, 2.0, 0.25, 2, 1)
    assert min(m.cut_gaps) > 1e-4
    z, z2, x, _ = m.observables()
    o = g.observables()
    assert abs(o["Z"] - z) < TOL and abs(o["Z2"] - z2) < TOL and abs(o["X"] - x) < TOL
    assert abs(g.fidelity() / m.F - 1) < TOL
    for bond in range(9):
        assert_spectra_equal(g.singular_values(bond), m.singular_values(bond))


def test_odd_row_split_and_spectra(L):
    # 3x3 grid: rows split 2 + 1 (d = 4 and 2); Schmidt spectra at every bond
    o = mps.run(3, 3, 7, TH_MID, -1.0, 2.0, 0.25, 4, order=2, record_spectra=True)
    assert o["min_cut_gap"] > 1e-4
    g, m = run_gpu(L, 3, 3, 7, TH_MID, -1.0, 2.0, 0.25, 4, 2)
    assert_parity(g, o, tol=TOL)
    for bond, s_ref in enumerate(o["spectra"][-1]):
        # every Schmidt value, including those far below sqrt(eps) s_0 (the truncation takes
        # the SVD of the centre block itself, never a Gram matrix)
        assert_spectra_equal(m.singular_values(bond), s_ref)


def test_closed_forms_on_gpu(L):
    # J = 0: <Z>(s) = cos(theta) cos(2 h s dt), F = 1, bonds stay 1
    g, m = run_gpu(L, 3, 4, 4, TH_MID, 0.0, 2.0, 0.25, 6, 2)
    s = np.arange(7)
    assert np.abs(g["Z"] - math.cos(TH_MID) * np.cos(2 * 2.0 * s * 0.25)).max() < TOL
    assert np.abs(g["X"] - math.sin(TH_MID)).max() < TOL
    assert np.all(g["F"] == 1.0) and m.bond_dims() == [1] * 5
    # h = 0: diagonal circuit; <X_j> = sin(theta) Re[(cos 2Jt + i cos(theta) sin 2Jt)^4]
    g, _ = run_gpu(L, 3, 4, 64, TH_MID, -1.0, 0.0, 0.25, 5, 2)
    t = np.arange(6) * 0.25
    ct = math.cos(TH_MID)
    xc = math.sin(TH_MID) * np.real((np.cos(-2 * t) + 1j * ct * np.sin(-2 * t)) ** 4)
    assert np.abs(g["X"] - xc).max() < TOL
    assert np.abs(g["Z"] - ct).max() < TOL


def test_z2_symmetry_on_gpu(L):
    a, _ = run_gpu(L, 3, 4, 5, TH_MID, -1.0, 2.0, 0.25, 3, 2)
    b, _ = run_gpu(L, 3, 4, 5, math.pi - TH_MID, -1.0, 2.0, 0.25, 3, 2)
    assert np.abs(a["Z"] + b["Z"]).max() < TOL
    assert np.abs(a["F"] - b["F"]).max() < TOL


def test_layers_equal_step(L):
    # apply_layer(X), apply_layer(ZZ), apply_layer(X) == one second-order step
    cfg = L.config(3, 4, 16, TH_MID)
    a = L.MPS(cfg)
    b = L.MPS(cfg)
    a.step(-1.0, 2.0, 0.25, 2, 2)
    for _ in range(2):
        b.apply_layer(L.LAYER_X, 0.25)
        b.apply_layer(L.LAYER_ZZ, -0.25)
        b.apply_layer(L.LAYER_X, 0.25)
    oa, ob = a.observables(), b.observables()
    # step() fuses X(alpha) with the in-block ZZ phases into one unitary: rounding differs
    for k in ("Z", "Z2", "X"):
        assert abs(oa[k] - ob[k]) < 1e-10
    assert abs(a.fidelity() - b.fidelity()) < 1e-10


def test_checkpoint_roundtrip(L, tmp_path):
    cfg = L.config(3, 4, 16, TH_MID)
    a = L.MPS(cfg)
    a.step(-1.0, 2.0, 0.25, 2, 3)
    p = str(tmp_path / "ck.bin")
    a.save(p)
    b = L.MPS.load_checkpoint(p)
    assert b.bond_dims() == a.bond_dims() and b.fidelity() == a.fidelity()
    a.step(-1.0, 2.0, 0.25, 2, 2)
    b.step(-1.0, 2.0, 0.25, 2, 2)
    oa, ob = a.observables(), b.observables()
    for k in ("Z", "Z2", "X"):
        assert oa[k] == ob[k]  # bit-identical resume in the FP64 form
    assert a.fidelity() == b.fidelity()


def test_truncate_whole_chain(L, tmp_path):
    # generic input (seeded random canonical MPS, 3x4, bonds at their bounds) re-compressed to
    # chi = 8: F and observables equal the sequential SVD compression of the dense vector
    m = _random_canonical_blocks(3, 4, 64, seed=11)
    cfg = L.config(3, 4, 64, TH_MID)
    p = str(tmp_path / "rand34.bin")
    _write_checkpoint(L, p, cfg, m)
    g = L.MPS.load_checkpoint(p)
    ds = [b.shape[1] for b in m.blocks]
    v = m.blocks[0]
    for b in m.blocks[1:]:
        v = np.tensordot(v, b, axes=([v.ndim - 1], [0]))
    v = v.reshape(-1)
    F = 1.0
    for bond in range(len(ds) - 1):
        M = v.reshape(int(np.prod(ds[: bond + 1])), -1)
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        k = min(8, len(s))
        F *= np.sum(s[:k] ** 2) / np.sum(s ** 2)
        v = ((U[:, :k] * (s[:k] / np.sqrt(np.sum(s[:k] ** 2)))) @ Vh[:k]).reshape(-1)
    g.truncate(8)
    assert abs(g.fidelity() / F - 1) < TOL
    assert max(g.bond_dims()) <= 8
    order = [q for b in m.layout for q in b["qubits"]]
    z, z2, x, _ = sv.observables(np.transpose(v.reshape((2,) * 12), np.argsort(order)).reshape(-1), 12)
    o = g.observables()
    assert abs(o["Z"] - z) < TOL and abs(o["Z2"] - z2) < TOL and abs(o["X"] - x) < TOL


def test_batch_step_equals_individual(L):
    cfgs = [L.config(3, 4, 16, TH_MID), L.config(3, 3, 6, TH_MID + 0.3), L.config(4, 4, 12, TH_MID - 0.2, order=1)]
    solo = []
    for c in cfgs:
        m = L.MPS(c)
        m.step(c.J, c.h, c.dt, c.trotter_order, 3)
        solo.append((m.observables(), m.fidelity()))
    ms = [L.MPS(c) for c in cfgs]
    L.batch_step(ms, 3)
    for m, (o, F) in zip(ms, solo):
        oo = m.observables()
        for k in ("Z", "Z2", "X"):
            assert abs(oo[k] - o[k]) < 1e-12
        assert abs(m.fidelity() - F) < 1e-13


def test_error_paths(L):
    m = L.MPS(L.config(3, 4, 16, TH_MID))
    with pytest.raises(L.MpsgbError) as e:
        m.apply_layer(L.LAYER_X, float("nan"))
    assert e.value.status == -1
    with pytest.raises(L.MpsgbError):
        m.singular_values(7)
    with pytest.raises(L.MpsgbError):
        m.truncate(0)
    with pytest.raises(L.MpsgbError):
        L.MPS.load_checkpoint("/nonexistent/ck.bin")
    # the handle stays usable after rejected calls
    m.step(-1.0, 2.0, 0.25, 2, 1)
    assert abs(m.observables()["norm"] - 1) < 1e-10
