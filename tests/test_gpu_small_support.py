"""Supports smaller than 32 (S = B + 2L in {4, 8, 16, 24}; the support-size
study of Sec. IV): the small-support kernels against the FP64 oracle, which
takes any S."""
import numpy as np
import pytest

import oracle
import parity as PA
from paper_2202_13926_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(24, 4), (24, 8), (16, 4), (16, 2), (16, 8), (8, 4), (8, 2), (4, 4), (4, 2)]   # (S, B)


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


def _run(handle, img, mask, S, B, K, precision="fp32", seq=False):
    dev = torch.device("cuda:0")
    n = -(-img.shape[0] // B) * -(-img.shape[1] // B)
    seq_t = torch.full((n * max(K, 1),), -7, dtype=torch.int16, device=dev) if seq else None
    out = handle.reconstruct(torch.from_numpy(np.ascontiguousarray(img)).to(dev),
                             torch.from_numpy(np.ascontiguousarray(mask)).to(dev),
                             block=B, border=(S - B) // 2, iters=K, precision=precision, seq_out=seq_t)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    if seq:
        return o, seq_t.cpu().numpy().reshape(-1, max(K, 1))[:, :K]
    return o


def _oracle(img, mask, S, B, K):
    r = oracle.fsr_image_blocks(img, mask, B=B, L=(S - B) // 2, K=K, rho=PA.RHO)
    return oracle.assemble_image(r["target"], img.shape[0], img.shape[1], B), r


@pytest.mark.parametrize("S,B", CASES)
def test_fp32_matches_the_oracle(handle, S, B):
    img, mask = synth.small_case()
    got = _run(handle, img, mask, S, B, 100)
    ref, _ = _oracle(img, mask, S, B, 100)
    assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64))
    frac = PA.frac_within(got, ref)
    assert frac >= PA.FRAC_MIN, (S, B, frac)
    dpsnr = abs(PA.psnr(got, img) - PA.psnr(ref, img))
    assert dpsnr <= PA.PSNR_TOL_DB, (S, B, dpsnr)


@pytest.mark.parametrize("S", [4, 8, 16, 24])
def test_fp32_full_1080p_frame_matches_the_oracle(handle, S):
    """The whole 1920 x 1080 quarter-sampling frame at K = 100, B = 4, in the
    launch configuration of the support-size sweep, against the oracle on
    every block.  The frame has far more blocks than the grid has resident
    warps (at most 64 warps per SM; the group kernel puts 32 / S blocks on a
    warp), so every warp runs its work loop many times: the per-block state
    reset and the tile-buffer parity flip between blocks are compared with
    the oracle here, not only the first block of each warp."""
    img, mask = synth.fhd_quarter_case()
    B = 4
    nblocks = -(-img.shape[0] // B) * -(-img.shape[1] // B)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks_per_warp = 32 // S if S in (4, 8, 16) else 1
    assert nblocks > 64 * sms * blocks_per_warp, (nblocks, sms)
    got = _run(handle, img, mask, S, B, 100)
    ref, r = _oracle(img, mask, S, B, 100)
    assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64))
    frac = PA.frac_within(got, ref)
    dpsnr = abs(PA.psnr(got, img) - PA.psnr(ref, img))
    print(f"S = {S}: within 0.5 {frac:.5f}, dPSNR {dpsnr:.2e} dB")
    if S != 4:
        assert frac >= PA.FRAC_MIN, (S, frac)
        assert dpsnr <= PA.PSNR_TOL_DB, (S, dpsnr)
        return
    # S = 4 (4 known pixels per support): many blocks meet a step where the
    # best component and the best one that is not its conjugate are closer
    # than FP32 can tell apart; there either pick is Eq. (8) evaluated to
    # FP32 precision.  The bar holds on the other blocks.
    near = (r["margin_nc"] < PA.FP32_NEAR_TIE).any(axis=1)
    keep = ~PA.block_pixels(near, img.shape[0], img.shape[1], B)
    frac_k = PA.frac_within(got[keep], ref[keep])
    dpsnr_k = abs(PA.psnr(got[keep], img[keep]) - PA.psnr(ref[keep], img[keep]))
    print(f"S = 4: {near.mean():.4f} of the blocks with an FP32 near tie; elsewhere within 0.5 {frac_k:.5f}, "
          f"dPSNR {dpsnr_k:.2e} dB")
    assert frac_k >= PA.FRAC_MIN, frac_k
    assert dpsnr_k <= PA.PSNR_TOL_DB, dpsnr_k


def test_fp64_full_1080p_frame_sequences_at_S4(handle):
    """The FP64 debug path at S = 4 on the whole 1080p quarter-sampling frame.
    With 4 known pixels per support the weighted residual of many blocks
    reaches the rounding floor of FP64 well before K = 100; from there the
    selection follows rounding noise on either side (measured: 51 of 129,600
    blocks leave the oracle's sequence at such a late step with a wide
    relative gap between noise-level objectives; their outputs differ by at
    most 5.4e-5 grey levels).  Sequences equal the oracle's up to the tie
    class, or the block's output agrees with the oracle's to 1e-3 grey
    levels like every block with the oracle's sequence."""
    img, mask = synth.fhd_quarter_case()
    H, W = img.shape
    got, seq = _run(handle, img, mask, 4, 4, 100, precision="fp64", seq=True)
    ref, r = _oracle(img, mask, 4, 4, 100)
    diff = seq.astype(np.int64) != r["seq"].astype(np.int64)
    rows = np.nonzero(diff.any(axis=1))[0]
    hard = [b for b in rows if r["margin"][b, int(np.argmax(diff[b]))] >= PA.TIE_MARGIN]
    print(f"S = 4 FP64: {rows.size - len(hard)} blocks leave the oracle's sequence at a tie, {len(hard)} at "
          "the rounding floor")
    flags = np.zeros(diff.shape[0], bool)
    flags[hard] = True
    hard_px = PA.block_pixels(flags, H, W, 4)
    assert np.max(np.abs(got - ref)[hard_px], initial=0.0) <= 1e-3
    same = PA.same_sequence_pixels(seq, r["seq"], H, W, 4)
    assert np.max(np.abs(got - ref)[same]) <= 1e-3


@pytest.mark.parametrize("S,B", CASES)
def test_fp64_selection_sequences(handle, S, B):
    img, mask = synth.small_case(seed=4)
    got, seq = _run(handle, img, mask, S, B, 60, precision="fp64", seq=True)
    ref, r = _oracle(img, mask, S, B, 60)
    n_hard, n_tie = PA.sequence_mismatches(seq, r["seq"], r["margin"])
    assert n_hard == 0, (S, B, n_hard, n_tie)
    same = PA.same_sequence_pixels(seq, r["seq"], img.shape[0], img.shape[1], B)
    assert np.max(np.abs(got - ref)[same]) <= 1e-3


@pytest.mark.parametrize("H,W", [(1, 1), (5, 7), (37, 53), (70, 9)])
def test_ragged_sizes_and_edges(handle, H, W):
    img = synth.sinusoid_image(H, W, seed=H * 7 + W)
    mask = synth.iid_mask(H, W, seed=H + W, missing=0.6)
    for S, B in ((24, 4), (16, 4), (8, 2), (4, 4), (4, 2)):
        got, seq = _run(handle, img, mask, S, B, 20, precision="fp64", seq=True)
        ref, r = _oracle(img, mask, S, B, 20)
        assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64))
        n_hard, _ = PA.sequence_mismatches(seq, r["seq"], r["margin"])
        assert n_hard == 0, (H, W, S, B)
        same = PA.same_sequence_pixels(seq, r["seq"], H, W, B)
        assert np.max(np.abs(got - ref)[same], initial=0.0) <= 1e-3


def test_empty_supports_and_batch_form(fsr_mod, handle):
    """Large holes leave 16 x 16 supports without known pixels (counted like
    the oracle, output 0); the batch form equals the single-image form."""
    fsr = fsr_mod
    H, W = 96, 120
    img = synth.sinusoid_image(H, W, seed=71)
    m = synth.macroblock_mask(H, W, seed=72, lost=0.5, mb=32)
    ref, r = _oracle(img, m, 16, 4, 30)
    assert r["n_empty"] > 0
    fsr.fsr_empty_blocks(handle.ptr)
    single = _run(handle, img, m, 16, 4, 30)
    assert fsr.fsr_empty_blocks(handle.ptr) == r["n_empty"]
    assert PA.frac_within(single, ref) >= PA.FRAC_MIN
    dev = torch.device("cuda:0")
    items = []
    for i, (hh, ww) in enumerate([(H, W), (40, 56)]):
        im = img if i == 0 else synth.sinusoid_image(hh, ww, seed=73)
        mk = m if i == 0 else synth.iid_mask(hh, ww, seed=74, missing=0.5)
        ti, tm = torch.from_numpy(im).to(dev), torch.from_numpy(mk).to(dev)
        items.append((im, mk, ti, tm, torch.full_like(ti, -1.0)))
    p = fsr.make_params(block=4, border=6, iters=30)
    fsr.fsr_reconstruct_batch(handle.ptr, [fsr.image_desc(ti, tm, to, 30) for _, _, ti, tm, to in items], p)
    torch.cuda.synchronize()
    for im, mk, ti, tm, to in items:
        alone = _run(handle, im, mk, 16, 4, 30)
        assert np.array_equal(to.cpu().numpy().astype(np.float64), alone)


def test_unsupported_support_sizes_are_rejected(fsr_mod, handle):
    fsr = fsr_mod
    img, mask = synth.small_case()
    dev = torch.device("cuda:0")
    ti, tm = torch.from_numpy(img).to(dev), torch.from_numpy(mask).to(dev)
    for kw in (dict(block=4, border=8), dict(block=2, border=11), dict(block=16, border=0),
               dict(block=4, border=6, precision="tc_tf32")):
        with pytest.raises(fsr.FsrError) as e:
            handle.reconstruct(ti, tm, **kw)
        assert e.value.code == fsr.FSR_ERR_UNSUPPORTED, kw


@pytest.mark.parametrize("S,B", [(16, 4), (16, 2), (16, 8), (4, 4), (4, 2), (8, 4), (24, 4)])
def test_fp32_batch_of_ragged_images_with_mixed_K(fsr_mod, handle, S, B):
    """A batch of ragged images with different K (the S = 16 and S = 4
    kernels pair two blocks per warp, also across images with different K):
    every image equals its single-image call bit for bit, and the oracle."""
    fsr = fsr_mod
    dev = torch.device("cuda:0")
    specs = [((67, 75), 40), ((1, 1), 13), ((37, 21), 0), ((53, 71), 25)]
    items = []
    for i, ((H, W), K) in enumerate(specs):
        img = synth.sinusoid_image(H, W, seed=90 + i)
        mk = synth.iid_mask(H, W, seed=95 + i, missing=0.5)
        ti, tm = torch.from_numpy(img).to(dev), torch.from_numpy(mk).to(dev)
        items.append((img, mk, K, ti, tm, torch.full_like(ti, -1.0)))
    p = fsr.make_params(block=B, border=(S - B) // 2, iters=40)
    fsr.fsr_reconstruct_batch(handle.ptr, [fsr.image_desc(ti, tm, to, K) for _, _, K, ti, tm, to in items], p)
    torch.cuda.synchronize()
    gots, refs = [], []
    for img, mk, K, ti, tm, to in items:
        got = to.cpu().numpy().astype(np.float64)
        assert np.array_equal(got, _run(handle, img, mk, S, B, K)), (img.shape, K)
        assert np.array_equal(got[mk == 1], img[mk == 1].astype(np.float64))
        ref, _ = _oracle(img, mk, S, B, K)
        gots.append(got.ravel())
        refs.append(ref.ravel())
    # the acceptance share of tests/parity.py, at least one pixel on these
    # few thousand pixels (as for the ragged sizes of the S = 32 tests)
    got_all, ref_all = np.concatenate(gots), np.concatenate(refs)
    n_out = int(np.sum(np.abs(got_all - ref_all) > PA.GREY_TOL))
    assert n_out <= max(1, int((1 - PA.FRAC_MIN) * got_all.size)), (S, B, n_out, got_all.size)
