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


def _images(seed):
    dev = torch.device("cuda:0")
    specs = [(64, 96, 30), (37, 53, 50), (128, 128, 100), (9, 200, 15), (40, 40, 0)]
    items = []
    for i, (H, W, K) in enumerate(specs):
        img = synth.sinusoid_image(H, W, seed + 31 * i)
        mask = synth.iid_mask(H, W, seed + 31 * i + 1, 0.55)
        n = -(-H // 4) * -(-W // 4)
        items.append(dict(K=K, img=torch.from_numpy(img).to(dev), mask=torch.from_numpy(mask).to(dev),
                          out=torch.full((H, W), -7.0, device=dev),
                          seq=torch.full((max(n * K, 1),), -5, dtype=torch.int16, device=dev)))
    return items


def _descs(fsr, items, out_key="out", seq_key="seq"):
    return [fsr.image_desc(it["img"], it["mask"], it[out_key], it["K"], it[seq_key] if it["K"] else None)
            for it in items]


def test_static_batch_matches_allocating_batch_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2202_13926_gb300 import fsr
    torch.cuda.set_device(0)
    with fsr.Handle(0) as h:
        for call, seed in enumerate((3, 11)):          # two calls in a row, different images
            items = _images(seed)
            for it in items:
                it["ref"] = torch.full_like(it["out"], -7.0)
                it["ref_seq"] = torch.full_like(it["seq"], -5)
            fsr.fsr_reconstruct_batch(h.ptr, _descs(fsr, items, "ref", "ref_seq"), fsr.make_params())
            fsr.fsr_reconstruct_batch_static(_descs(fsr, items), fsr.make_params())
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
