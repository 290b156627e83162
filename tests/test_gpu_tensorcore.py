"""Tensor-core split-precision path (tcgen05 + TMA) through the C ABI.

The GEMM self-test compares the tcgen05 kernel with the FP32 CUDA-core GEMM on
seeded data (ragged sizes spanning several 128 x 64 tiles, all op(A)/op(B) modes).
With 2-term BF16 splits (16 significant bits) every real product carries a relative
error of about 2^-16, so the bound on max|diff| / max|ref| is 2e-4; with TF32 splits (22
bits) 2e-5.  The split forms (SPLIT_BF16X3, SPLIT_TF32X3) are then checked end to end against
the FP64 oracle and the FP32 form.
"""
import numpy as np
import pytest

from oracle import model, mps

pytestmark = pytest.mark.gpu
TH_MID = model.initial_theta(model.TEMPERATURES["mid"])


@pytest.fixture(scope="module")
def L():
    from paper_2511_23438_gb300 import build, lib
    build.build()
    lib.load()
    return lib


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (64, 64, 64), (200, 130, 300), (1000, 70, 129),
                                   (256, 512, 2048), (2048, 2048, 1024)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("tf32", [False, True])
def test_tc_gemm_matches_cuda_cores(L, M, N, K, mode, tf32):
    # 2-term splits: 16 significant bits (BF16) or 22 (TF32), so about 2^-16 or 2^-21 relative
    # error per real product; the FP32 CUDA-core reference accumulates its own rounding
    err = L.tc_gemm_selftest(M, N, K, mode, seed=M * 7 + N * 13 + K + mode, tf32=tf32)
    assert err < (2e-5 if tf32 else 2e-4), err


def _evolve_random_state(L, prec, chi, steps, tmp_path, seed=5):
    """Seeded random canonical MPS on the 5x6 grid, evolved by `steps` second-order steps on the
    GPU (precision `prec`) and by the oracle; returns both (Z, Z2, X, F) after the last step."""
    from test_gpu_parity import _random_canonical_blocks, _write_checkpoint
    from oracle import layout
    m = _random_canonical_blocks(5, 6, chi, seed=seed)
    cfg = L.config(5, 6, chi, TH_MID, prec=prec)
    p = str(tmp_path / ("rand_%s.bin" % prec))
    _write_checkpoint(L, p, cfg, m, dtype=np.complex128 if prec == "fp64" else np.complex64)
    g = L.MPS.load_checkpoint(p)
    alpha, phi = model.layer_angles(-1.0, 2.0, 0.25, 2)
    intra, inter = layout.schedule(5, 6)
    for _ in range(steps):
        m.x_layer(alpha)
        m.zz_intra(phi, intra)
        for gt in inter:
            m.zz_inter(gt, phi)
        m.x_layer(alpha)
        g.step(-1.0, 2.0, 0.25, 2, 1)
    z, z2, x, _ = m.observables()
    o = g.observables()
    return np.array([o["Z"], o["Z2"], o["X"], g.fidelity()]), np.array([z, z2, x, m.F]), min(m.cut_gaps)


# bounds per form (max |d obs| over <Z_tot>, <Z_tot^2>, <X_tot>; |dF/F|) for the test below: its
# measured values on a GB300 times about 3.5: split BF16X3 8.5e-7 / 1.25e-4 (F carries the 2^-16
# relative error of the BF16-split Grams and cores), split TF32X3 7.4e-7 / 3.3e-5, FP32 2.0e-7 / 1.0e-6
FORM_BOUND = {"split_bf16x3": (3e-6, 4e-4), "split_tf32x3": (3e-6, 1.2e-4), "fp32": (7e-7, 4e-6)}


@pytest.mark.parametrize("prec", ["split_bf16x3", "split_tf32x3", "fp32"])
def test_reduced_precision_forms_against_oracle(L, prec, tmp_path):
    # 5x6 grid, d = 8, chi = 64 (block-sized contractions on the tensor cores in the split form),
    # generic input (seeded random canonical MPS), two second-order steps
    before = L.launch_count()
    g, ref, gap = _evolve_random_state(L, prec, 64, 2, tmp_path)
    assert L.launch_count() > before and gap > 1e-4
    err = np.abs(g[:3] - ref[:3]).max()
    ferr = abs(g[3] / ref[3] - 1)
    print("%s vs FP64 oracle: max |d obs| %.2e, |dF/F| %.2e" % (prec, err, ferr))
    assert err < FORM_BOUND[prec][0] and ferr < FORM_BOUND[prec][1]


def test_split_form_on_a_stream_equals_default_stream(L, tmp_path):
    # on a stream of its own the library records the Cholesky factorisations as CUDA graphs and
    # replays them; the legacy default stream cannot be captured and runs the same launches one by
    # one.  The results agree to the form's rounding (the Householder reduction sums partial dot
    # products across CTAs with atomics, so their last bits may come in another order)
    torch = pytest.importorskip("torch")
    from test_gpu_parity import _random_canonical_blocks, _write_checkpoint
    m = _random_canonical_blocks(5, 6, 64, seed=5)
    cfg = L.config(5, 6, 64, TH_MID, prec="split_bf16x3")
    p = str(tmp_path / "stream.bin")
    _write_checkpoint(L, p, cfg, m, dtype=np.complex64)
    a = L.MPS.load_checkpoint(p)
    s = torch.cuda.Stream()
    b = L.MPS.load_checkpoint(p, stream=s.cuda_stream)
    for _ in range(2):
        a.step(-1.0, 2.0, 0.25, 2, 1)
        b.step(-1.0, 2.0, 0.25, 2, 1)
    oa, ob = a.observables(), b.observables()
    for k in ("Z", "Z2", "X"):
        assert abs(oa[k] - ob[k]) < 1e-6
    assert abs(a.fidelity() / b.fidelity() - 1) < 1e-6
    assert b.counters()["chol_ok"] > 0
