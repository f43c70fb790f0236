"""Precision study: the forward and the inverse 2-D DFT on tensor cores (BF16
hi/lo split products, TF32) against the FP32 SIMT path and the FP64 oracle."""
import json
import os

import numpy as np
import pytest

import oracle
import parity as PA
from paper_2202_13926_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = ("fp32", "tc_bf16x3", "tc_tf32")


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_13926_gb300 import fsr
    h = fsr.Handle(0)
    yield h
    h.close()


def _run(h, img, mask, **kw):
    dev = torch.device("cuda:0")
    out = h.reconstruct(torch.from_numpy(img).to(dev), torch.from_numpy(mask).to(dev), **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("mode", MODES)
def test_transform_selects_dc_then_the_cosine_pair(handle, mode):
    """All pixels known, rho = 1, gamma = 1, no frequency weighting: W is
    1024 delta, so every interior support of 128 + A cos(2 pi (3 y + 5 x)/32)
    selects DC (index 0) and then the conjugate pair (3,5), (29,27) (indices
    101 and 955, lower first).  A wrong operand layout in the tensor-core
    transform would select something else."""
    from paper_2202_13926_gb300 import fsr
    H = W = 96
    yy, xx = np.mgrid[0:H, 0:W]
    f = (128 + 60.0 * np.cos(2 * np.pi * (3 * yy + 5 * xx) / 32 + 0.4)).astype(np.float32)
    mask = np.ones((H, W), np.uint8)
    dev = torch.device("cuda:0")
    nb = (H // 4) * (W // 4)
    seq = torch.full((nb * 3,), -1, dtype=torch.int16, device=dev)
    handle.reconstruct(torch.from_numpy(f).to(dev), torch.from_numpy(mask).to(dev), iters=3, rho=1.0,
                       gamma=1.0, freq_weight=False, precision=mode, seq_out=seq)
    torch.cuda.synchronize()
    s = seq.cpu().numpy().reshape(H // 4, W // 4, 3)
    inner = s[4:20, 4:20].reshape(-1, 3)          # supports entirely inside the image
    assert np.all(inner[:, 0] == 0), mode
    assert np.all(inner[:, 1] == 101) and np.all(inner[:, 2] == 955), mode


@pytest.mark.parametrize("mode,tol", [("fp32", 2e-3), ("tc_bf16x3", 2e-2), ("tc_tf32", 0.5)])
def test_inverse_transform_recovers_the_cosine(handle, mode, tol):
    """One unknown pixel per 4 x 4 block (rows 1 mod 4, columns 2 mod 4),
    rho = 1, gamma = 1, no frequency weighting, K = 3, f = 128 + A cos of
    frequency (3, 5).  In an interior support the lost grid only couples
    frequencies 8 apart, so the picks are DC, (3,5), (29,27), each projection
    is exact and the model equals f: the unknown pixels come back from the
    inverse transform (on tensor cores in the TC modes, from the sparse
    accumulation in FP32) within the mode's rounding."""
    H = W = 96
    yy, xx = np.mgrid[0:H, 0:W]
    f = (128 + 60.0 * np.cos(2 * np.pi * (3 * yy + 5 * xx) / 32 + 0.4)).astype(np.float32)
    mask = np.ones((H, W), np.uint8)
    mask[1::4, 2::4] = 0
    got = _run(handle, f, mask, iters=3, rho=1.0, gamma=1.0, freq_weight=False, precision=mode)
    inner = np.zeros((H, W), bool)
    inner[16:80, 16:80] = True                      # blocks whose supports lie inside the image
    sel = inner & (mask == 0)
    err = np.abs(got[sel] - f[sel].astype(np.float64))
    assert err.max() <= tol, (mode, err.max())


def test_precision_study_on_1080p_quarter_sampling(handle):
    """The 1080p quarter-sampling frame in FP32-SIMT, BF16x3 and TF32 transform
    modes; each against the FP64 oracle (whole frame)."""
    img, mask = synth.fhd_quarter_case()
    r = oracle.fsr_image_blocks(img, mask, K=100, rho=PA.RHO)
    ref = oracle.assemble_image(r["target"], 1080, 1920, 4)
    rows = {}
    for mode in MODES:
        got = _run(handle, img, mask, iters=100, precision=mode)
        unk = mask == 0
        rows[mode] = {
            "psnr_db": PA.psnr(got, img),
            "psnr_oracle_db": PA.psnr(ref, img),
            "dpsnr_db": PA.psnr(got, img) - PA.psnr(ref, img),
            "max_abs_vs_oracle": float(np.max(np.abs(got - ref))),
            "rms_vs_oracle_unknown": float(np.sqrt(np.mean((got - ref)[unk] ** 2))),
            "frac_within_0.5": PA.frac_within(got, ref),
        }
        assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64))
    print("precision study:", json.dumps(rows, indent=1))
    out = os.environ.get("FSR_PRECISION_REPORT")
    if out:
        with open(out, "w") as fh:
            json.dump(rows, fh, indent=1)
    assert rows["fp32"]["frac_within_0.5"] >= PA.FRAC_MIN
    # Every mode meets the PSNR part of the acceptance bar.  The share of
    # pixels within 0.5 grey levels depends on the transform's precision: the
    # hi/lo split carries 16 significant bits of each operand (two 8-bit BF16
    # mantissas), TF32 11, against FP32's 24, so near-ties of the greedy
    # selection flip more often; the floors below sit a little under the
    # measured shares (BF16x3 0.9937, TF32 0.7407), and the RMS difference at
    # the unknown pixels is bounded per mode a little above the measured
    # values (FP32 0.026, BF16x3 0.120, TF32 0.817 grey levels), so a
    # regression in either tensor-core transform fails here.
    floors = {"fp32": (PA.FRAC_MIN, 0.05), "tc_bf16x3": (0.990, 0.2), "tc_tf32": (0.70, 1.0)}
    for mode, (frac_min, rms_max) in floors.items():
        assert abs(rows[mode]["dpsnr_db"]) <= PA.PSNR_TOL_DB, mode
        assert rows[mode]["frac_within_0.5"] >= frac_min, mode
        assert rows[mode]["rms_vs_oracle_unknown"] <= rms_max, mode
