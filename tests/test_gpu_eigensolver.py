"""Hermitian eigensolver of the truncation core, checked on its own (C-ABI self-test).

The truncation core (Gram matrix, then H = Gs^H E Gs) needs A = V diag(w) V^H with V unitary
to working precision.  Three seeded spectra cover what the core meets: graded Gram matrices
(Schmidt spectra over many decades), rank-deficient Gram matrices (exact zero eigenvalues) and
a matrix whose eigenvalue 1 has multiplicity n - 2(n/8) inside the spectrum.  Sizes straddle
the switch from the Jacobi solvers (n <= 64) to the Householder-tridiagonal solver (n >= 65).
A backward-stable solver gives residual and loss of orthogonality of order n * eps, so the
bounds are 1e-12 (FP64) and 5e-5 (FP32) at n <= 512.
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
