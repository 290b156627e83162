"""Hermitian eigensolver of the truncation core, checked on its own (C-ABI self-test).

The truncation core (Gram matrix, then H = Gs^H E Gs) needs A = V diag(w) V^H with V unitary
to working precision.  Three seeded spectra cover what the core meets: graded Gram matrices
(Schmidt spectra over many decades), rank-deficient Gram matrices (exact zero eigenvalues) and
a matrix whose eigenvalue 1 has multiplicity n - 2(n/8) inside the spectrum.  Sizes straddle
the switch from the Jacobi solvers (n <= 64) to the Householder-tridiagonal solver (n >= 65).
A backward-stable solver gives residual and loss of orthogonality of order n * eps, so the
bounds are 1e-12 (FP64) and 5e-5 (FP32) at n <= 512; the sizes of the 6x8, chi = 1024 cores
(n = 1024 and 2048, complex64: the split form's solves) are checked at 5e-5 as well.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


@pytest.mark.parametrize("n", [24, 40, 64, 65, 200, 512])
@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("fp64", [True, False])
def test_eigensolver_spectra(L, n, kind, fp64):
    r = L.eig_selftest(n, fp64=fp64, seed=1000 + 7 * n + kind, kind=kind)
    tol = 1e-12 if fp64 else 5e-5
    assert r["sweeps"] >= 1, r
    assert r["sorted"] == 1.0, r
    assert r["residual"] < tol, r
    assert r["orthogonality"] < tol, r


@pytest.mark.parametrize("n", [1024, 2048])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_eigensolver_bench_sizes_fp32(L, n, kind):
    r = L.eig_selftest(n, fp64=False, seed=2000 + n + kind, kind=kind)
    assert r["sweeps"] == 1, r
    assert r["sorted"] == 1.0, r
    assert r["residual"] < 5e-5, r
    assert r["orthogonality"] < 5e-5, r
