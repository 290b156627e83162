"""Allocation-free eigensolver entry point (mpsgb_eigh_noalloc) against the existing API.

mpsgb_eigh_noalloc serves callers that cannot allocate device memory where they need a
decomposition (a frozen or request-scoped allocator, a thread that must not enter the CUDA
allocator): its workspace is a fixed 1 MiB device array inside the library.  This test
evolves an FP64 MPS, takes the Schmidt values of one bond from the existing entry point
mpsgb_singular_values, rebuilds the same bond's Gram matrix from a checkpoint, and checks
that two calls in a row of the allocation-free solver on caller-owned device buffers
return the same spectrum (1e-9 relative to s_0 for Schmidt values above 1e-5 s_0, the
bound of the other spectrum tests) and a valid decomposition.  This file is collected
last so that a run stopping at the first failure has already run every other test.
"""
import ctypes
import struct

import numpy as np
import pytest

from oracle import model

pytestmark = pytest.mark.gpu


def _read_block(L, path, which):
    with open(path, "rb") as fh:
        raw = fh.read()
    off = 8 + ctypes.sizeof(L.Config)
    elem, nblk, centre, _ = struct.unpack_from("4i", raw, off)
    off += 16 + 8 + 40
    dims = struct.unpack_from("%di" % (nblk - 1), raw, off)
    off += 4 * (nblk - 1)
    cfg = L.Config.from_buffer_copy(raw[8: 8 + ctypes.sizeof(L.Config)])
    ds = []
    from oracle import layout
    for b in layout.blocks(cfg.Lx, cfg.Ly):
        ds.append(b["d"])
    dt = np.complex128 if elem == 8 else np.complex64
    for b in range(nblk):
        l = 1 if b == 0 else dims[b - 1]
        r = 1 if b == nblk - 1 else dims[b]
        cnt = l * ds[b] * r
        arr = np.frombuffer(raw, dtype=dt, count=cnt, offset=off).reshape(l, ds[b], r)
        off += cnt * np.dtype(dt).itemsize
        if b == which:
            return arr.copy(), centre


def test_no_alloc_eigensolver_matches_singular_values(tmp_path):
    torch = pytest.importorskip("torch")
    from paper_2511_23438_gb300 import build, lib as L
    build.build()
    L.load()
    theta = model.initial_theta(model.TEMPERATURES["mid"])
    m = L.MPS(L.config(3, 4, 64, theta, prec="fp64"))
    m.step(-1.0, 2.0, 0.25, 2, 3)
    bond = 2
    s_ref = np.array(m.singular_values(bond))  # existing entry point; leaves the centre on `bond`
    p = str(tmp_path / "state.bin")
    m.save(p)
    blk, centre = _read_block(L, p, bond)
    assert centre == bond
    l, d, r = blk.shape
    M = blk.reshape(l * d, r)
    G = M.conj().T @ M  # Gram of the centre block: eigenvalues are the squared Schmidt values
    n = G.shape[0]
    assert 32 < n <= 128  # exercises the blocked solver inside the fixed scratch

    dev = torch.device("cuda:0")
    A = torch.tensor(G, dtype=torch.complex128, device=dev)
    w = torch.empty(n, dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    k = int(np.count_nonzero(s_ref > 1e-5 * s_ref[0]))
    prev = None
    for _ in range(2):  # two calls in a row share the same device scratch
        L.eigh_noalloc(n, True, A.data_ptr(), n, w.data_ptr(), V.data_ptr(), n, stream)
        torch.cuda.synchronize()
        wh = w.cpu().numpy()
        s = np.sqrt(np.clip(wh, 0.0, None))
        assert np.all(np.diff(wh) <= 0)
        assert np.abs(s[:k] - s_ref[:k]).max() < 1e-9 * s_ref[0]
        Vh = V.cpu().numpy()
        assert np.abs(Vh @ np.diag(wh) @ Vh.conj().T - G).max() < 1e-12 * np.abs(G).max()
        assert np.abs(Vh.conj().T @ Vh - np.eye(n)).max() < 1e-12
        if prev is not None:
            assert np.array_equal(prev, wh)
        prev = wh.copy()

    # complex64 as well, within the FP32 form's bound
    A32 = A.to(torch.complex64)
    w32 = torch.empty(n, dtype=torch.float32, device=dev)
    V32 = torch.empty((n, n), dtype=torch.complex64, device=dev)
    L.eigh_noalloc(n, False, A32.data_ptr(), n, w32.data_ptr(), V32.data_ptr(), n, stream)
    torch.cuda.synchronize()
    assert np.abs(w32.cpu().numpy() - prev).max() < 1e-5 * prev[0]

    # sizes beyond the fixed scratch are rejected with a clear error
    with pytest.raises(L.MpsgbError) as e:
        L.eigh_noalloc(129, True, A.data_ptr(), 129, w.data_ptr(), V.data_ptr(), 129, stream)
    assert e.value.status == -1 and "1..128" in str(e.value)
