"""Support tiles (step a1): the single-image kernels bring each block's 32 x 32
support in by two TMA tile copies when img and mask are 16-byte aligned and
the row pitch is a multiple of 16, and by plain loads otherwise.  Pixels
outside the image are unknown on both paths (zero fill of the copies, bounds
tests of the loads), so the two must agree bit for bit; the bounded wait on
the copies must report a timeout through the status word without faulting."""
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


def _pitched(img, mask, P):
    """Device copies of img/mask inside rows of P elements (views of width W)."""
    dev = torch.device("cuda:0")
    H, W = img.shape
    bi = torch.full((H, P), np.nan, device=dev)
    bm = torch.full((H, P), 1, dtype=torch.uint8, device=dev)   # garbage beyond the width
    bo = torch.full((H, P), -5.0, device=dev)
    bi[:, :W] = torch.from_numpy(img).to(dev)
    bm[:, :W] = torch.from_numpy(mask).to(dev)
    return bi[:, :W], bm[:, :W], bo


def _run(fsr, h, img, mask, P, **kw):
    ti, tm, bo = _pitched(img, mask, P)
    H, W = img.shape
    B = kw.get("block", 4)
    K = kw.get("iters", 30)
    n = -(-H // B) * -(-W // B)
    seq = torch.full((n * max(K, 1),), -7, dtype=torch.int16, device=ti.device)
    fsr.fsr_reconstruct(h.ptr, ti, tm, fsr.make_params(seq_out=seq if K > 0 else None, **kw), bo[:, :W])
    fsr.fsr_check_status(h.ptr)
    assert torch.all(bo[:, W:] == -5.0)   # nothing beyond the width is written
    return bo[:, :W].cpu().numpy(), seq.cpu().numpy()


def _pitches(W):
    tile = -(-W // 16) * 16 + 16          # multiple of 16: tile copies
    plain = W + 1 if (W + 1) % 16 else W + 2   # not a multiple of 16: plain loads
    return tile, plain


@pytest.mark.parametrize("H,W,B", [
    (1, 1, 4), (5, 7, 4), (3, 40, 2), (37, 53, 4), (70, 9, 8), (33, 31, 16), (129, 200, 4), (64, 96, 4),
])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tile_copies_equal_plain_loads(fsr_mod, handle, H, W, B, precision):
    img = synth.sinusoid_image(H, W, seed=7 * H + W)
    mask = synth.iid_mask(H, W, seed=H + 3 * W + B, missing=0.55)
    tile_p, plain_p = _pitches(W)
    kw = dict(block=B, border=(32 - B) // 2, iters=30, precision=precision)
    a, sa = _run(fsr_mod, handle, img, mask, tile_p, **kw)
    b, sb = _run(fsr_mod, handle, img, mask, plain_p, **kw)
    assert np.array_equal(a, b)
    assert np.array_equal(sa, sb)
    assert np.array_equal(a[mask == 1], img[mask == 1])


def test_tile_copies_match_the_oracle_at_image_edges(fsr_mod, handle):
    """Blocks whose supports hang over every edge and corner of the image:
    the zero fill of the copies must act as 'unknown' exactly as the oracle's
    rule for pixels outside the image."""
    H, W = 48, 80
    img = synth.sinusoid_image(H, W, seed=21)
    mask = synth.iid_mask(H, W, seed=22, missing=0.5)
    got, seq = _run(fsr_mod, handle, img, mask, 96, iters=40, precision="fp64")
    r = oracle.fsr_image_blocks(img, mask, K=40, rho=PA.RHO)
    ref = oracle.assemble_image(r["target"], H, W, 4)
    n_hard, _ = PA.sequence_mismatches(seq.reshape(-1, 40), r["seq"], r["margin"])
    assert n_hard == 0
    assert np.max(np.abs(got.astype(np.float64) - ref)) <= 1e-3


def test_tile_wait_timeout_is_reported_and_the_handle_recovers(fsr_mod, handle):
    fsr = fsr_mod
    img, mask = synth.small_case(seed=31)     # 128 x 128: tile copies
    dev = torch.device("cuda:0")
    ti, tm = torch.from_numpy(img).to(dev), torch.from_numpy(mask).to(dev)
    good = handle.reconstruct(ti, tm, iters=20)
    handle.check_status()
    fsr.fsr_inject_tile_wait_fault(handle.ptr)
    out = torch.full_like(ti, -9.0)
    fsr.fsr_reconstruct(handle.ptr, ti, tm, fsr.make_params(iters=20), out)
    with pytest.raises(fsr.FsrError) as e:
        handle.check_status()
    assert e.value.code == fsr.FSR_ERR_TIMEOUT
    assert "tile" in str(e.value)
    assert torch.any(out == -9.0)             # the warps stopped before writing
    handle.check_status()                     # the word was cleared
    again = handle.reconstruct(ti, tm, iters=20)
    handle.check_status()
    assert torch.equal(again, good)
