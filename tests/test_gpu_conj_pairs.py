"""The conjugate-pair ablation (FSR_UPDATE_CONJ_PAIR: the original FSR's real
model, the selected component and its conjugate updated together; not the
paper's Eqs. 11-12) against the oracle run with ``conj_pairs=True``."""
import numpy as np
import pytest

import oracle
import parity as PA
from paper_2202_13926_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fsr_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_13926_gb300 import fsr
    return fsr


@pytest.fixture(scope="module")
def handle(fsr_mod):
    h = fsr_mod.Handle(0)
    yield h
    h.close()


def _run(handle, img, mask, K, precision="fp32", seq=False):
    dev = torch.device("cuda:0")
    n = -(-img.shape[0] // 4) * -(-img.shape[1] // 4)
    seq_t = torch.full((n * max(K, 1),), -7, dtype=torch.int16, device=dev) if seq else None
    out = handle.reconstruct(torch.from_numpy(np.ascontiguousarray(img)).to(dev),
                             torch.from_numpy(np.ascontiguousarray(mask)).to(dev),
                             iters=K, precision=precision, seq_out=seq_t, update="conj_pair")
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    if seq:
        return o, seq_t.cpu().numpy().reshape(-1, max(K, 1))[:, :K]
    return o


def _oracle(img, mask, K, threads=0):
    r = oracle.fsr_image_blocks(img, mask, B=4, L=14, K=K, conj_pairs=True, threads=threads, rho=PA.RHO)
    return oracle.assemble_image(r["target"], img.shape[0], img.shape[1], 4), r


def test_fp32_matches_the_oracle(handle):
    img, mask = synth.small_case()
    got = _run(handle, img, mask, 100)
    ref, r = _oracle(img, mask, 100)
    assert np.max(np.abs(r["im_target"][np.isfinite(r["im_target"])])) <= 1e-6   # the model is real
    assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64))
    assert PA.frac_within(got, ref) >= PA.FRAC_MIN
    assert abs(PA.psnr(got, img) - PA.psnr(ref, img)) <= PA.PSNR_TOL_DB


def test_fp64_selection_sequences(handle):
    img, mask = synth.small_case(seed=5)
    got, seq = _run(handle, img, mask, 80, precision="fp64", seq=True)
    ref, r = _oracle(img, mask, 80)
    n_hard, n_tie = PA.sequence_mismatches(seq, r["seq"], r["margin"])
    assert n_hard == 0, (n_hard, n_tie)
    assert np.max(np.abs(got - ref)) <= 1e-3


@pytest.mark.parametrize("H,W", [(1, 1), (5, 7), (37, 53), (70, 9)])
def test_ragged_sizes(handle, H, W):
    img = synth.sinusoid_image(H, W, seed=H * 5 + W)
    mask = synth.iid_mask(H, W, seed=H + 2 * W, missing=0.6)
    got, seq = _run(handle, img, mask, 24, precision="fp64", seq=True)
    ref, r = _oracle(img, mask, 24)
    n_hard, _ = PA.sequence_mismatches(seq, r["seq"], r["margin"])
    assert n_hard == 0
    assert np.max(np.abs(got - ref)) <= 1e-3


def test_empty_supports_and_batch_form(fsr_mod, handle):
    fsr = fsr_mod
    H, W = 96, 120
    img = synth.sinusoid_image(H, W, seed=81)
    m = synth.macroblock_mask(H, W, seed=82, lost=0.5, mb=32)
    ref, r = _oracle(img, m, 30)
    assert r["n_empty"] > 0
    fsr.fsr_empty_blocks(handle.ptr)
    single = _run(handle, img, m, 30)
    assert fsr.fsr_empty_blocks(handle.ptr) == r["n_empty"]
    assert PA.frac_within(single, ref) >= PA.FRAC_MIN
    dev = torch.device("cuda:0")
    ti, tm = torch.from_numpy(img).to(dev), torch.from_numpy(m).to(dev)
    to = torch.full_like(ti, -1.0)
    p = fsr.make_params(iters=30, update="conj_pair")
    fsr.fsr_reconstruct_batch(handle.ptr, [fsr.image_desc(ti, tm, to, 30)], p)
    torch.cuda.synchronize()
    assert np.array_equal(to.cpu().numpy().astype(np.float64), single)


def test_fhd_quarter_full_frame(handle):
    """1920 x 1080 quarter sampling at K = 100, every block against the oracle."""
    img, mask = synth.fhd_quarter_case()
    got = _run(handle, img, mask, 100)
    ref, _ = _oracle(img, mask, 100)
    assert PA.frac_within(got, ref) >= PA.FRAC_MIN
    assert abs(PA.psnr(got, img) - PA.psnr(ref, img)) <= PA.PSNR_TOL_DB


def test_unsupported_combinations(fsr_mod, handle):
    fsr = fsr_mod
    img, mask = synth.small_case()
    dev = torch.device("cuda:0")
    ti, tm = torch.from_numpy(img).to(dev), torch.from_numpy(mask).to(dev)
    for kw in (dict(block=8, border=12), dict(block=4, border=6), dict(precision="tc_bf16x3")):
        with pytest.raises(fsr.FsrError) as e:
            handle.reconstruct(ti, tm, update="conj_pair", **kw)
        assert e.value.code == fsr.FSR_ERR_UNSUPPORTED, kw
    with pytest.raises(fsr.FsrError) as e:
        handle.reconstruct(ti, tm, update=2)
    assert e.value.code == fsr.FSR_ERR_INVALID_ARG
