"""Allocation-free eigensolver entry point (mpsgb_eigh_noalloc) against the existing API.

mpsgb_eigh_noalloc serves callers that cannot allocate device memory where they need a
decomposition (a frozen or request-scoped allocator, a thread that must not enter the CUDA
allocator): its workspace is a fixed 1 MiB device array inside the library.  The tests check
(1) seeded random Hermitian matrices over every route of the solver inside the fixed scratch
(n = 16: one-warp Jacobi; 64, 96, 128: blocked Jacobi, 128 being the size limit), FP64 and
complex64, against numpy.linalg.eigvalsh and by reconstruction and unitarity (bounds: 1e-12 |A|
in FP64; in complex64 the Jacobi backward-error bound 4 n eps |A|_F, and 16 n eps on unitarity,
since every column of V takes n - 1 rotations per sweep); (2) two calls in a
row on two different streams with no synchronisation between them other than the call's own;
(3) the Schmidt values of an evolved FP64 MPS from the existing entry point
mpsgb_singular_values, reproduced by the allocation-free solver on the Gram of the same bond
(1e-9 relative to s_0 for Schmidt values above 1e-5 s_0).  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes
import struct

import numpy as np
import pytest

from oracle import model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_2511_23438_gb300 import build, lib as L
    build.build()
    L.load()
    return torch, L


def _read_block(L, path, which):
    with open(path, "rb") as fh:
        raw = fh.read()
    off = 8 + ctypes.sizeof(L.Config)
    elem, nblk, centre, _ = struct.unpack_from("4i", raw, off)
    off += 16 + 8 + 40
    dims = struct.unpack_from("%di" % (nblk - 1), raw, off)
    off += 4 * (nblk - 1)
    cfg = L.Config.from_buffer_copy(raw[8: 8 + ctypes.sizeof(L.Config)])
    from oracle import layout
    ds = [b["d"] for b in layout.blocks(cfg.Lx, cfg.Ly)]
    dt = np.complex128 if elem == 8 else np.complex64
    for b in range(nblk):
        l = 1 if b == 0 else dims[b - 1]
        r = 1 if b == nblk - 1 else dims[b]
        cnt = l * ds[b] * r
        arr = np.frombuffer(raw, dtype=dt, count=cnt, offset=off).reshape(l, ds[b], r)
        off += cnt * np.dtype(dt).itemsize
        if b == which:
            return arr.copy(), centre


def _random_hermitian(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (X + X.conj().T) / 2


def _solve(torch, L, A_host, fp64, stream):
    dev = torch.device("cuda:0")
    n = A_host.shape[0]
    cdt, rdt = (torch.complex128, torch.float64) if fp64 else (torch.complex64, torch.float32)
    A = torch.tensor(A_host, dtype=cdt, device=dev)
    w = torch.empty(n, dtype=rdt, device=dev)
    V = torch.empty((n, n), dtype=cdt, device=dev)
    stream.wait_stream(torch.cuda.current_stream())  # the input copy was issued on the current stream
    L.eigh_noalloc(n, fp64, A.data_ptr(), n, w.data_ptr(), V.data_ptr(), n, stream.cuda_stream)
    # the call has already waited for its stream; nothing else needs to be synchronised
    return w.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n", [16, 64, 96, 128])
@pytest.mark.parametrize("fp64", [True, False])
def test_no_alloc_random_hermitian(env, n, fp64):
    torch, L = env
    A = _random_hermitian(n, seed=1000 + n)
    ref = np.linalg.eigvalsh(A)[::-1]
    eps32 = float(np.finfo(np.float32).eps)
    tol_w = 1e-12 * np.abs(ref).max() if fp64 else 4 * n * eps32 * np.linalg.norm(A)
    tol_o = 1e-12 if fp64 else 16 * n * eps32
    s1 = torch.cuda.Stream()
    s2 = torch.cuda.Stream()
    results = []
    for st in (s1, s2):  # two calls in a row on different streams share the same device scratch
        w, V = _solve(torch, L, A, fp64, st)
        assert np.all(np.diff(w) <= 0)
        assert np.abs(w - ref).max() < tol_w
        assert np.abs(V @ np.diag(w) @ V.conj().T - A).max() < tol_w
        assert np.abs(V.conj().T @ V - np.eye(n)).max() < tol_o
        results.append(w)
    assert np.array_equal(results[0], results[1])


def test_no_alloc_eigensolver_matches_singular_values(env, tmp_path):
    torch, L = env
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
    k = int(np.count_nonzero(s_ref > 1e-5 * s_ref[0]))
    stream = torch.cuda.current_stream()
    prev = None
    for _ in range(2):  # two calls in a row share the same device scratch
        wh, Vh = _solve(torch, L, G, True, stream)
        s = np.sqrt(np.clip(wh, 0.0, None))
        assert np.all(np.diff(wh) <= 0)
        assert np.abs(s[:k] - s_ref[:k]).max() < 1e-9 * s_ref[0]
        assert np.abs(Vh @ np.diag(wh) @ Vh.conj().T - G).max() < 1e-12 * np.abs(G).max()
        assert np.abs(Vh.conj().T @ Vh - np.eye(n)).max() < 1e-12
        if prev is not None:
            assert np.array_equal(prev, wh)
        prev = wh.copy()
    # complex64 as well, within the FP32 form's bound
    w32, _ = _solve(torch, L, G, False, stream)
    assert np.abs(w32 - prev).max() < 1e-5 * prev[0]


def test_no_alloc_rejects_sizes_beyond_scratch(env):
    torch, L = env
    dev = torch.device("cuda:0")
    A = torch.zeros((129, 129), dtype=torch.complex128, device=dev)
    w = torch.empty(129, dtype=torch.float64, device=dev)
    V = torch.empty((129, 129), dtype=torch.complex128, device=dev)
    with pytest.raises(L.MpsgbError) as e:
        L.eigh_noalloc(129, True, A.data_ptr(), 129, w.data_ptr(), V.data_ptr(), 129,
                       torch.cuda.current_stream().cuda_stream)
    assert e.value.status == -1 and "1..128" in str(e.value)
