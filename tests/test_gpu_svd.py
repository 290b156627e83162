"""One-sided Jacobi SVD of the FP64 form's truncation (C-ABI kernel self-test) against LAPACK.

The FP64 form truncates every spanned bond by the SVD of the centre block (Sec. III), computed on
the GPU by Jacobi rotations of the rows of its conjugate transpose; the spectra it produces must
match numpy.linalg.svd value by value down to the rounding floor, without the sqrt(eps) loss of a
Gram matrix.  Seeded complex matrices with singular values graded over twelve decades, wide, tall
and square, one CTA per problem and the cooperative-grid form (p q >= 2^18); rank-deficient
inputs (exact zero singular values).  Bounds: |s - s_LAPACK| <= 1e-13 s_0 (FP64) / 1e-5 s_0
(complex64, about 8 eps sqrt(q) at q = 1024), residual and orthogonality 1e-12 (FP64); in
complex64 the residual 2e-5 and orthogonality 1e-4 (every rotation of a sweep touches the rows of
U once, so their unitarity error grows with rows x sweeps x eps); the Gram-eigenvector
preconditioning keeps the FP64 sweep count at ten or fewer.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def graded(p, q, seed, decades=12.0, rank=None):
    rng = np.random.default_rng(seed)
    k = min(p, q)
    Ua, _ = np.linalg.qr(rng.standard_normal((p, k)) + 1j * rng.standard_normal((p, k)))
    Va, _ = np.linalg.qr(rng.standard_normal((q, k)) + 1j * rng.standard_normal((q, k)))
    s = np.logspace(0, -decades, k)
    if rank is not None:
        s[rank:] = 0
    return (Ua * s) @ Va.conj().T


@pytest.mark.parametrize("p,q", [(7, 20), (20, 8), (64, 64), (128, 512), (256, 1024), (130, 700)])
@pytest.mark.parametrize("fp64", [True, False])
def test_jacobi_svd_matches_lapack(L, p, q, fp64):
    X = graded(p, q, seed=p * 31 + q)
    s, r = L.svd_selftest(X, fp64=fp64)
    ref = np.linalg.svd(X, compute_uv=False)
    k = min(p, q)
    tol = 1e-13 if fp64 else 1e-5
    assert 1 <= r["sweeps"] <= (10 if fp64 else 20), r
    assert np.all(np.diff(s) <= 0)
    assert np.abs(s[:k] - ref).max() < tol * ref[0], np.abs(s[:k] - ref).max()
    assert np.all(s[k:] < tol * ref[0])
    assert r["residual"] < (1e-12 if fp64 else 2e-5), r
    assert r["orth_u"] < (1e-12 if fp64 else 1e-4), r
    assert r["orth_v"] < (1e-12 if fp64 else 1e-4), r


def test_jacobi_svd_rank_deficient(L):
    X = graded(96, 300, seed=5, decades=3.0, rank=40)
    s, r = L.svd_selftest(X, fp64=True)
    ref = np.linalg.svd(X, compute_uv=False)
    assert int(r["rank"]) == 40
    assert np.abs(s[:96] - ref).max() < 1e-13 * ref[0]
    assert r["residual"] < 1e-12 and r["orth_u"] < 1e-12 and r["orth_v"] < 1e-12
