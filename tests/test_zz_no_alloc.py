"""The batch entry point that allocates no device memory.

It serves callers that may not call the device allocator (a framework that
owns the memory budget, a real-time loop, a plug-in without memory of its
own).  Its output must equal the allocating batch entry point's on the same
images, on two calls in a row (the shared static scratch keeps the previous
call's contents, so the second call checks that the state is reset)."""
import numpy as np
import pytest

from paper_2202_13926_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _images(seed, B=4):
    dev = torch.device("cuda:0")
    specs = [(64, 96, 30), (37, 53, 50), (128, 128, 100), (9, 200, 15), (40, 40, 0)]
    items = []
    for i, (H, W, K) in enumerate(specs):
        img = synth.sinusoid_image(H, W, seed + 31 * i)
        mask = synth.iid_mask(H, W, seed + 31 * i + 1, 0.55)
        n = -(-H // B) * -(-W // B)
        items.append(dict(K=K, img=torch.from_numpy(img).to(dev), mask=torch.from_numpy(mask).to(dev),
                          out=torch.full((H, W), -7.0, device=dev),
                          seq=torch.full((max(n * K, 1),), -5, dtype=torch.int16, device=dev)))
    return items


def _descs(fsr, items, out_key="out", seq_key="seq"):
    return [fsr.image_desc(it["img"], it["mask"], it[out_key], it["K"], it[seq_key] if it["K"] else None)
            for it in items]


@pytest.mark.parametrize("precision,B,own_stream", [("fp32", 4, False), ("fp64", 4, False),
                                                     ("fp32", 2, True), ("fp32", 8, True)])
def test_static_batch_matches_allocating_batch_twice(precision, B, own_stream):
    """Bit-equal to fsr_reconstruct_batch for the FP32 and the FP64 debug
    arithmetic, several block sizes, on the current stream and on a stream of
    the caller's own."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_13926_gb300 import fsr
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream() if own_stream else None
    params = fsr.make_params(block=B, border=(32 - B) // 2, precision=precision)
    with fsr.Handle(0) as h:
        for call, seed in enumerate((3, 11)):          # two calls in a row, different images
            items = _images(seed, B)
            for it in items:
                it["ref"] = torch.full_like(it["out"], -7.0)
                it["ref_seq"] = torch.full_like(it["seq"], -5)
            torch.cuda.synchronize()
            fsr.fsr_reconstruct_batch(h.ptr, _descs(fsr, items, "ref", "ref_seq"), params, stream)
            fsr.fsr_reconstruct_batch_static(_descs(fsr, items), params, stream)
            torch.cuda.synchronize()
            for it in items:
                a = it["out"].cpu().numpy()
                b = it["ref"].cpu().numpy()
                assert np.array_equal(a, b), f"call {call}: outputs differ"
                if it["K"]:
                    assert np.array_equal(it["seq"].cpu().numpy(), it["ref_seq"].cpu().numpy())


def test_static_batch_rejects_too_many_images():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_13926_gb300 import fsr
    it = _images(5)[0]
    descs = [fsr.image_desc(it["img"], it["mask"], it["out"], 5)] * 65
    with pytest.raises(fsr.FsrError) as e:
        fsr.fsr_reconstruct_batch_static(descs, fsr.make_params())
    assert e.value.code == fsr.FSR_ERR_INVALID_ARG and "at most 64 images" in str(e.value)
