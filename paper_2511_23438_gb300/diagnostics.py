"""Discarded-component diagnostic at sizes with an exact state (Sec. III, Fig. orthogonal).

The MPS and the exact state are evolved side by side; after every Trotter step the exact
state is split as psi_ex = c psi_MPS + d psi_perp (Gram-Schmidt against the normalised MPS,
|c|^2 = F_exact, d = sqrt(1 - F_exact)), so that

    <Z^2>_ex = F_exact <Z^2>_MPS + (1 - F_exact) <Z^2>_perp + 2 Re(conj(c) d <MPS|Z^2|perp>).

The paper compares the unrescaled estimate, the fidelity-rescaled one and the estimate with the
discarded component, F_exact <Z^2>_MPS + (1 - F_exact) <Z^2>_perp, and reports that the
off-diagonal term is negligible.  Here both states come from the GPU library: the MPS at chi and
the MPS at the exact bond bound (no truncation), each read back from its checkpoint and
contracted to a dense vector on the host.  Both vectors use the MPS's own qubit order; every
quantity used is independent of that order (Z_tot^2 is diagonal with value (n - 2 popcount)^2/n^2).
"""
import ctypes
import struct

import numpy as np

MAGIC = b"MPSGBv2\x00"


def block_qubits(Lx, Ly):
    """Qubits per MPS block along the snake: rows split into ceil(Ly/2) + floor(Ly/2) qubits, odd
    rows reversed."""
    ks = []
    for r in range(Lx):
        k0, k1 = (Ly + 1) // 2, Ly // 2
        ks += [k0, k1] if r % 2 == 0 else [k1, k0]
    return ks


def read_checkpoint(path, config_size=None):
    """Blocks (l, d, r) complex128 arrays, bond dims, centre and F_MPS of an mpsgb checkpoint
    (layout of mpsgb_save: magic, config, {real size, blocks, centre, 0}, F, 5 counters, bond
    dims, blocks in chain order)."""
    if config_size is None:
        from . import lib
        config_size = ctypes.sizeof(lib.Config)
        Config = lib.Config
    else:
        Config = None
    with open(path, "rb") as fh:
        raw = fh.read()
    if raw[:8] != MAGIC:
        raise ValueError("%s is not an mpsgb checkpoint" % path)
    off = 8
    cfg_raw = raw[off:off + config_size]
    off += config_size
    rbytes, nblk, centre, _ = struct.unpack_from("4i", raw, off)
    off += 16
    (F,) = struct.unpack_from("d", raw, off)
    off += 8 + 40
    dims = list(struct.unpack_from("%di" % (nblk - 1), raw, off))
    off += 4 * (nblk - 1)
    if Config is not None:
        cfg = Config.from_buffer_copy(cfg_raw)
        Lx, Ly = cfg.Lx, cfg.Ly
        three_d = cfg.lattice == 1
    else:  # Lx, Ly are the first two ints of the config (2D lattice)
        Lx, Ly = struct.unpack_from("2i", cfg_raw, 0)
        three_d = False
    ks = [1] * (Lx * Ly * cfg.Lz) if three_d else block_qubits(Lx, Ly)
    if len(ks) != nblk:
        raise ValueError("block count does not match the grid")
    dt = np.complex128 if rbytes == 8 else np.complex64
    blocks = []
    for b in range(nblk):
        l = 1 if b == 0 else dims[b - 1]
        r = 1 if b == nblk - 1 else dims[b]
        cnt = l * (1 << ks[b]) * r
        blocks.append(np.frombuffer(raw, dtype=dt, count=cnt, offset=off).reshape(l, 1 << ks[b], r)
                      .astype(np.complex128))
        off += cnt * np.dtype(dt).itemsize
    if off != len(raw):
        raise ValueError("trailing bytes in checkpoint")
    return dict(Lx=Lx, Ly=Ly, F=F, centre=centre, dims=dims, blocks=blocks)


def to_vector(blocks):
    """Dense state of a chain of blocks (l, d, r): index = block physical indices in chain order,
    the first block most significant."""
    v = blocks[0].reshape(-1, blocks[0].shape[2])
    for B in blocks[1:]:
        l, d, r = B.shape
        v = (v @ B.reshape(l, d * r)).reshape(-1, r)
    return v.reshape(-1)


def z2_diagonal(n):
    """Diagonal of Z_tot^2 = ((1/n) sum_j Z_j)^2 in any computational basis order."""
    x = np.arange(1 << n, dtype=np.int64)
    pop = np.zeros_like(x)
    for b in range(n):
        pop += (x >> b) & 1
    return ((n - 2 * pop) / n) ** 2


def split_discarded(psi_mps, psi_ex, zdiag):
    """F_exact, <Z^2> of the MPS, of the exact state and of the discarded component, the
    off-diagonal term and the estimate with the discarded component."""
    a = psi_mps / np.linalg.norm(psi_mps)
    e = psi_ex / np.linalg.norm(psi_ex)
    c = np.vdot(a, e)
    perp = e - c * a
    d = np.linalg.norm(perp)
    perp = perp / d if d > 1e-300 else perp
    z = lambda u, w: np.vdot(u, zdiag * w)
    z2_mps, z2_ex, z2_perp = z(a, a).real, z(e, e).real, z(perp, perp).real
    F_ex = abs(c) ** 2
    cross = 2 * (np.conj(c) * d * z(a, perp)).real
    return dict(F_exact=F_ex, z2_mps=z2_mps, z2_exact=z2_ex, z2_perp=z2_perp, cross=cross,
                z2_with_perp=F_ex * z2_mps + (1 - F_ex) * z2_perp)


def gpu_orthogonal_run(Lx, Ly, chi, theta, steps, workdir, J=-1.0, h=2.0, dt=0.25, order=2):
    """Evolve the MPS at chi and the exact MPS side by side on the GPU (FP64 form) and split the
    exact state after every step; returns a list of per-step dicts (plus F_MPS)."""
    import os

    from . import build, gamma, lib
    build.build()
    lib.load()
    n = Lx * Ly
    bound = gamma.exact_bond_bound(Lx, Ly)
    m = lib.MPS(lib.config(Lx, Ly, chi, theta, prec="fp64", J=J, h=h, dt=dt, order=order))
    ex = lib.MPS(lib.config(Lx, Ly, bound, theta, prec="fp64", J=J, h=h, dt=dt, order=order))
    zdiag = z2_diagonal(n)
    out = []
    try:
        for s in range(steps):
            m.step(J, h, dt, order, 1)
            ex.step(J, h, dt, order, 1)
            pm, pe = os.path.join(workdir, "mps.bin"), os.path.join(workdir, "exact.bin")
            m.save(pm)
            ex.save(pe)
            cm, ce = read_checkpoint(pm), read_checkpoint(pe)
            if abs(ce["F"] - 1) > 1e-12:
                raise RuntimeError("the exact run truncated")
            r = split_discarded(to_vector(cm["blocks"]), to_vector(ce["blocks"]), zdiag)
            r["F_mps"] = cm["F"]
            out.append(r)
    finally:
        m.close()
        ex.close()
    return out
