"""Discarded-component diagnostic (Sec. III, Fig. orthogonal): the host-side pieces pinned on
the CPU (checkpoint reader, contraction, Z_tot^2 diagonal, the split of the exact state) and the
diagnostic run end to end on the oracle's MPS and exact state vector."""
import struct

import numpy as np

from oracle import model
from oracle import mps as omps
from oracle import statevector as osv
from paper_2511_23438_gb300 import diagnostics as dg


def test_z2_diagonal_against_explicit_operator():
    n = 5
    Z = np.diag([1.0, -1.0])
    tot = np.zeros((1 << n, 1 << n))
    for q in range(n):
        op = np.array([[1.0]])
        for p in range(n):
            op = np.kron(op, Z if p == q else np.eye(2))
        tot += op
    assert np.allclose(np.diag((tot / n) @ (tot / n)), dg.z2_diagonal(n), atol=1e-15)


def test_to_vector_against_einsum():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((1, 4, 3)) + 1j * rng.standard_normal((1, 4, 3))
    B = rng.standard_normal((3, 2, 5)) + 1j * rng.standard_normal((3, 2, 5))
    C = rng.standard_normal((5, 4, 1)) + 1j * rng.standard_normal((5, 4, 1))
    ref = np.einsum("aib,bjc,ckd->ijk", A, B, C).reshape(-1)
    assert np.allclose(dg.to_vector([A, B, C]), ref, atol=1e-13)


def _write_checkpoint(path, Lx, Ly, blocks, F, real_bytes, config_size=80):
    dims = [b.shape[2] for b in blocks[:-1]]
    dt = np.complex128 if real_bytes == 8 else np.complex64
    cfg = struct.pack("2i", Lx, Ly) + bytes(config_size - 8)
    with open(path, "wb") as fh:
        fh.write(dg.MAGIC + cfg + struct.pack("4i", real_bytes, len(blocks), 0, 0) + struct.pack("d", F)
                 + struct.pack("5q", 1, 2, 3, 4, 5) + struct.pack("%di" % len(dims), *dims))
        for b in blocks:
            fh.write(np.ascontiguousarray(b.astype(dt)).tobytes())


def test_checkpoint_reader_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    ks = dg.block_qubits(3, 3)
    assert ks == [2, 1, 1, 2, 2, 1]
    dims = [2, 3, 4, 3, 2]
    blocks = []
    for b, k in enumerate(ks):
        l = 1 if b == 0 else dims[b - 1]
        r = 1 if b == len(ks) - 1 else dims[b]
        blocks.append(rng.standard_normal((l, 1 << k, r)) + 1j * rng.standard_normal((l, 1 << k, r)))
    for rb in (8, 4):
        p = str(tmp_path / ("c%d.bin" % rb))
        _write_checkpoint(p, 3, 3, blocks, 0.75, rb)
        c = dg.read_checkpoint(p, config_size=80)
        assert c["F"] == 0.75 and c["dims"] == dims and (c["Lx"], c["Ly"]) == (3, 3)
        tol = 1e-15 if rb == 8 else 1e-6
        for a, b in zip(c["blocks"], blocks):
            assert a.shape == b.shape and np.abs(a - b).max() <= tol * max(1, np.abs(b).max())


def test_split_identity_and_limits():
    rng = np.random.default_rng(4)
    n = 6
    zd = dg.z2_diagonal(n)
    a = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    e = a + 0.3 * (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n))
    r = dg.split_discarded(a, e, zd)
    assert 0 < r["F_exact"] < 1
    assert abs(r["F_exact"] * r["z2_mps"] + (1 - r["F_exact"]) * r["z2_perp"] + r["cross"] - r["z2_exact"]) < 1e-13
    r1 = dg.split_discarded(a, 2j * a, zd)
    assert abs(r1["F_exact"] - 1) < 1e-14 and abs(r1["z2_with_perp"] - r1["z2_exact"]) < 1e-13


def oracle_orthogonal_run(Lx, Ly, chi, theta, steps):
    """The same diagnostic on the oracle: its MPS at chi and its exact state vector."""
    alpha, phi = model.layer_angles(-1.0, 2.0, 0.25, 2)
    from oracle import layout
    intra, inter = layout.schedule(Lx, Ly)
    m = omps.MPS(Lx, Ly, chi, theta)
    n = Lx * Ly
    psi = osv.product_state(n, theta)
    energy = osv.zz_energy(Lx, Ly)
    zd = dg.z2_diagonal(n)
    out = []
    for _ in range(steps):
        m.x_layer(alpha)
        m.zz_intra(phi, intra)
        for g in inter:
            m.zz_inter(g, phi)
        m.x_layer(alpha)
        psi = osv.x_layer(osv.zz_layer(osv.x_layer(psi, n, alpha), energy, phi), n, alpha)
        r = dg.split_discarded(m.to_statevector(), psi, zd)
        r["F_mps"] = m.F
        out.append(r)
    return out


def test_diagnostic_on_oracle_data():
    theta = model.initial_theta(model.TEMPERATURES["mid"])
    rows = oracle_orthogonal_run(3, 3, 4, theta, 10)
    ex, _ = osv.run(3, 3, theta, -1.0, 2.0, 0.25, 10)
    for s, r in enumerate(rows):
        assert abs(r["z2_exact"] - ex["Z2"][s + 1]) < 1e-12  # the split sees the exact <Z^2>
        assert 0 < r["F_exact"] <= 1 + 1e-12 and 0 < r["F_mps"] <= 1 + 1e-12
        assert abs(r["F_exact"] * r["z2_mps"] + (1 - r["F_exact"]) * r["z2_perp"] + r["cross"] - r["z2_exact"]) < 1e-12
    assert rows[-1]["F_exact"] < 1 - 1e-6  # chi = 4 truncates this grid
