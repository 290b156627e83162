"""Bounded device waits: a grid barrier that runs out returns MPSGB_ETIMEDOUT, the kernel
finishes and the CUDA context stays usable.

The Householder reduction of the eigensolver (n >= 65) synchronises its CTAs with grid barriers
whose waits are bounded by a cycle limit.  The test lowers that limit to one cycle, so the first
CTA to reach a barrier gives up at once (the other CTAs have not arrived yet): the barrier records
its error word, the kernel runs to its end without waiting, and the call reports ETIMEDOUT.
Nothing here faults or hangs the GPU: every access of the reduction stays inside its own matrix
whatever the values, and every wait ends after the limit.  With the default limit restored the
same calls succeed again on the same context.
"""
import numpy as np
import pytest

from oracle import model

pytestmark = pytest.mark.gpu
TH_MID = model.initial_theta(model.TEMPERATURES["mid"])


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


def test_eigensolver_barrier_timeout_is_reported(L):
    ok = L.eig_selftest(256, fp64=False, seed=3)
    assert ok["sweeps"] == 1 and ok["residual"] < 1e-5
    prev = L.set_wait_limit(1)
    try:
        bad = L.eig_selftest(256, fp64=False, seed=3)
    finally:
        L.set_wait_limit(prev)
    assert bad["sweeps"] == -2  # the eigensolver's status for a timed-out grid barrier
    again = L.eig_selftest(256, fp64=False, seed=3)
    assert again["sweeps"] == 1 and abs(again["residual"] - ok["residual"]) < 1e-6


def test_engine_returns_etimedout_and_context_survives(L, tmp_path):
    from test_gpu_parity import _random_canonical_blocks, _write_checkpoint
    # 5x6 grid, chi = 64: every truncation core is 128 x 128 and goes through the reduction
    m = _random_canonical_blocks(5, 6, 64, seed=9)
    cfg = L.config(5, 6, 64, TH_MID, prec="fp32")
    p = str(tmp_path / "rand_fp32.bin")
    _write_checkpoint(L, p, cfg, m, dtype=np.complex64)
    ref = L.MPS.load_checkpoint(p)
    ref.step(-1.0, 2.0, 0.25, 2, 1)
    o_ref = ref.observables()

    g = L.MPS.load_checkpoint(p)
    prev = L.set_wait_limit(1)
    try:
        with pytest.raises(L.MpsgbError) as e:
            g.step(-1.0, 2.0, 0.25, 2, 1)
    finally:
        L.set_wait_limit(prev)
    assert e.value.status == -3 and "timed out" in str(e.value)
    # the failed handle can still be queried and destroyed; the context is intact
    g.observables()
    del g
    h = L.MPS.load_checkpoint(p)
    h.step(-1.0, 2.0, 0.25, 2, 1)
    o = h.observables()
    for k in ("Z", "Z2", "X"):
        assert o[k] == o_ref[k]
    assert h.fidelity() == ref.fidelity()
