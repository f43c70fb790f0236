"""Batch form: one persistent launch over many images with per-image K.

Every block is computed by one warp with the arithmetic of the single-image
path, so batch results must equal single-image results bit for bit, for
every schedule, for graph replays, and match the oracle within the
acceptance bar of tests/parity.py."""
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


SPECS = [  # H, W, K, mask kind
    (64, 96, 30, "iid"), (37, 53, 50, "mb"), (128, 128, 100, "quarter"),
    (16, 300, 20, "iid"), (200, 40, 0, "iid"), (5, 7, 12, "iid"),
]


def _mask(kind, H, W, seed):
    if kind == "iid":
        return synth.iid_mask(H, W, seed, 0.6)
    if kind == "mb":
        return synth.macroblock_mask(H, W, seed, 0.3)
    return synth.quarter_mask(H, W, seed)


def _make(specs, seed=0, B=4):
    dev = torch.device("cuda:0")
    items = []
    for i, (H, W, K, kind) in enumerate(specs):
        img = synth.sinusoid_image(H, W, seed + 17 * i)
        mask = _mask(kind, H, W, seed + 17 * i + 1)
        n = -(-H // B) * -(-W // B)
        items.append(dict(img=img, mask=mask, K=K,
                          d_img=torch.from_numpy(img).to(dev), d_mask=torch.from_numpy(mask).to(dev),
                          d_out=torch.full((H, W), -3.0, device=dev),
                          d_seq=torch.full((max(n * K, 1),), -9, dtype=torch.int16, device=dev)))
    return items


def _descs(fsr, items):
    return [fsr.image_desc(it["d_img"], it["d_mask"], it["d_out"], it["K"],
                           it["d_seq"] if it["K"] > 0 else None) for it in items]


def _single(fsr, h, it, precision):
    dev = torch.device("cuda:0")
    out = torch.empty_like(it["d_img"])
    seq = torch.full_like(it["d_seq"], -9)
    fsr.fsr_reconstruct(h.ptr, it["d_img"], it["d_mask"],
                        fsr.make_params(iters=it["K"], precision=precision,
                                        seq_out=seq if it["K"] > 0 else None), out)
    torch.cuda.synchronize(dev)
    return out.cpu().numpy(), seq.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_single(fsr_mod, handle, precision):
    fsr = fsr_mod
    items = _make(SPECS, seed=1)
    fsr.fsr_reconstruct_batch(handle.ptr, _descs(fsr, items), fsr.make_params(precision=precision))
    torch.cuda.synchronize()
    for it in items:
        out, seq = _single(fsr, handle, it, precision)
        assert np.array_equal(it["d_out"].cpu().numpy(), out)
        if it["K"] > 0:
            assert np.array_equal(it["d_seq"].cpu().numpy(), seq)


def test_graph_plan_replays_identically(fsr_mod, handle):
    fsr = fsr_mod
    items = _make(SPECS, seed=2)
    plan = fsr.fsr_batch_create(handle.ptr, _descs(fsr, items), fsr.make_params())
    try:
        fsr.fsr_batch_launch(plan, handle=handle.ptr)
        torch.cuda.synchronize()
        first = [it["d_out"].cpu().numpy().copy() for it in items]
        for it in items:
            it["d_out"].fill_(-1.0)
        fsr.fsr_batch_launch(plan, handle=handle.ptr)
        fsr.fsr_batch_launch(plan, handle=handle.ptr)
        torch.cuda.synchronize()
        for it, f in zip(items, first):
            assert np.array_equal(it["d_out"].cpu().numpy(), f)
            assert np.array_equal(f, _single(fsr, handle, it, "fp32")[0])
    finally:
        fsr.fsr_batch_destroy(plan)


def test_every_schedule_gives_identical_results(fsr_mod, handle):
    fsr = fsr_mod
    items = _make(SPECS[:4], seed=3)
    ref = None
    saved = fsr.fsr_get_schedule(handle.ptr)
    try:
        for warps in (16, 12, 8):
            for chunk in (1, 3, 8):
                fsr.fsr_set_schedule(handle.ptr, warps, chunk)
                for it in items:
                    it["d_out"].fill_(-2.0)
                fsr.fsr_reconstruct_batch(handle.ptr, _descs(fsr, items), fsr.make_params())
                torch.cuda.synchronize()
                outs = [it["d_out"].cpu().numpy().copy() for it in items]
                if ref is None:
                    ref = outs
                for a, b in zip(outs, ref):
                    assert np.array_equal(a, b), (warps, chunk)
    finally:
        fsr.fsr_set_schedule(handle.ptr, *saved)
    with pytest.raises(fsr.FsrError) as e:
        fsr.fsr_set_schedule(handle.ptr, 12, 1, block=8)   # not instantiated for B = 8
    assert e.value.code == fsr.FSR_ERR_UNSUPPORTED


def test_autotune_writes_and_reads_cache(fsr_mod, tmp_path):
    fsr = fsr_mod
    cache = str(tmp_path / "sched.txt")
    items = _make(SPECS[:3], seed=4)
    with fsr.Handle(0, schedule_cache=cache) as h:
        (warps, chunk), ms = fsr.fsr_autotune_batch(h.ptr, _descs(fsr, items), fsr.make_params())
        assert ms > 0 and fsr.fsr_get_schedule(h.ptr) == (warps, chunk)
    text = open(cache).read()
    assert f"|0|4|{warps}|{chunk}" in text
    with fsr.Handle(0, schedule_cache=cache) as h2:
        assert fsr.fsr_get_schedule(h2.ptr) == (warps, chunk)


def test_batch_rejects_bad_images(fsr_mod, handle):
    fsr = fsr_mod
    items = _make(SPECS[:2], seed=5)
    d = _descs(fsr, items)
    d[1].iters = -4
    with pytest.raises(fsr.FsrError) as e:
        fsr.fsr_reconstruct_batch(handle.ptr, d, fsr.make_params())
    assert e.value.code == fsr.FSR_ERR_INVALID_ARG and "image 1" in str(e.value)
    d = _descs(fsr, items)
    d[0].out = d[0].img
    with pytest.raises(fsr.FsrError) as e:
        fsr.fsr_reconstruct_batch(handle.ptr, d, fsr.make_params())
    assert e.value.code == fsr.FSR_ERR_INVALID_ARG
    with pytest.raises(fsr.FsrError):
        fsr.fsr_reconstruct_batch(handle.ptr, [], fsr.make_params())


def test_mixed_batch_48_images_full_size(fsr_mod, handle):
    """48 images (12 each of 256x256, 1280x720, 1920x1080, 3840x2160), masks
    alternating i.i.d. 10-90 % loss and 5-20 % lost 16x16 macroblocks, K in
    {50, 100, 200}: one graph-captured launch; sampled blocks of every image
    against the oracle."""
    fsr = fsr_mod
    dev = torch.device("cuda:0")
    items = synth.batch_case()
    descs = []
    for it in items:
        it["d_img"] = torch.from_numpy(it["img"]).to(dev)
        it["d_mask"] = torch.from_numpy(it["mask"]).to(dev)
        it["d_out"] = torch.empty_like(it["d_img"])
        descs.append(fsr.image_desc(it["d_img"], it["d_mask"], it["d_out"], it["K"]))
    plan = fsr.fsr_batch_create(handle.ptr, descs, fsr.make_params())
    try:
        fsr.fsr_batch_launch(plan, handle=handle.ptr)
        torch.cuda.synchronize()
    finally:
        fsr.fsr_batch_destroy(plan)
    rng = np.random.default_rng(12)
    got_all, ref_all, truth_all = [], [], []
    for it in items:
        H, W = it["img"].shape
        nbx, nby = -(-W // 4), -(-H // 4)
        ids = np.unique(np.concatenate([[0, nbx * nby - 1], rng.choice(nbx * nby, 100, replace=False)]))
        r = oracle.fsr_image_blocks(it["img"], it["mask"], K=it["K"], block_ids=ids, rho=PA.RHO)
        out = it["d_out"].cpu().numpy()
        assert np.array_equal(out[it["mask"] == 1], it["img"][it["mask"] == 1])
        for s, b in enumerate(ids):
            by, bx = divmod(int(b), nbx)
            got_all.append(out[by * 4:by * 4 + 4, bx * 4:bx * 4 + 4].ravel())
            ref_all.append(r["target"][s].ravel())
            truth_all.append(it["img"][by * 4:by * 4 + 4, bx * 4:bx * 4 + 4].ravel())
    got = np.concatenate(got_all).astype(np.float64)
    ref = np.concatenate(ref_all)
    truth = np.concatenate(truth_all).astype(np.float64)
    frac = PA.frac_within(got, ref)
    dpsnr = abs(PA.psnr(got, truth) - PA.psnr(ref, truth))
    print(f"mixed batch: {got.size} sampled pixels, within 0.5 {frac:.5f}, dPSNR {dpsnr:.5f} dB")
    assert frac >= PA.FRAC_MIN, frac
    assert dpsnr <= PA.PSNR_TOL_DB, dpsnr


def test_multichannel_frame_equals_per_channel_calls(fsr_mod, handle):
    """A (3, H, W) frame in one batch launch equals three single-image calls."""
    dev = torch.device("cuda:0")
    H, W = 72, 112
    planes = np.stack([synth.sinusoid_image(H, W, seed=60 + c) for c in range(3)])
    mask = synth.iid_mask(H, W, seed=63, missing=0.5)
    ti = torch.from_numpy(planes).to(dev)
    tm = torch.from_numpy(mask).to(dev)
    out = handle.reconstruct_channels(ti, tm, iters=40)
    torch.cuda.synchronize()
    for c in range(3):
        one = handle.reconstruct(ti[c].contiguous(), tm, iters=40)
        torch.cuda.synchronize()
        assert torch.equal(out[c], one), c


@pytest.mark.parametrize("per_channel_masks", [False, True])
def test_multichannel_frame_matches_the_oracle(fsr_mod, handle, per_channel_masks):
    """Three planes of a 1/f^2 frame (one quarter-sampling mask for all
    planes, or one per plane) reconstructed in one batch launch: every plane
    equals the oracle run on that plane within the acceptance bar."""
    dev = torch.device("cuda:0")
    H, W, K = 270, 328, 60
    planes = np.stack([synth.pink_image(H, W, seed=160 + c) for c in range(3)])
    if per_channel_masks:
        masks = np.stack([synth.quarter_mask(H, W, seed=170 + c) for c in range(3)])
    else:
        masks = synth.quarter_mask(H, W, seed=170)
    out = handle.reconstruct_channels(torch.from_numpy(planes).to(dev), torch.from_numpy(masks).to(dev),
                                      iters=K)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    for c in range(3):
        m = masks[c] if per_channel_masks else masks
        r = oracle.fsr_image_blocks(planes[c], m, K=K, rho=PA.RHO)
        ref = oracle.assemble_image(r["target"], H, W, 4)
        assert np.array_equal(got[c][m == 1], planes[c][m == 1].astype(np.float64)), c
        assert PA.frac_within(got[c], ref) >= PA.FRAC_MIN, c
        assert abs(PA.psnr(got[c], planes[c]) - PA.psnr(ref, planes[c])) <= PA.PSNR_TOL_DB, c
