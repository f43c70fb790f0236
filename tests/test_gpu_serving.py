"""Serving form: continuous batching of a request stream with admission by
device memory.  Each result must equal the same frame reconstructed alone."""
import numpy as np
import pytest

from paper_2202_13926_gb300 import serving, synth

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


def _frames(specs, seed):
    frames = []
    for i, (H, W, kind) in enumerate(specs):
        img = synth.pink_image(H, W, seed + i)
        mask = synth.quarter_mask(H, W, seed + 50 + i) if kind == "q" else \
            synth.macroblock_mask(H, W, seed + 50 + i, 0.15)
        frames.append((torch.from_numpy(img).pin_memory(), torch.from_numpy(mask).pin_memory()))
    return frames


def _alone(fsr, h, img, mask, K):
    dev = torch.device("cuda:0")
    out = torch.empty(img.shape, device=dev)
    fsr.fsr_reconstruct(h.ptr, img.to(dev), mask.to(dev), fsr.make_params(iters=K), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_results_alone_equal_results_in_the_mix(fsr_mod, handle):
    fsr = fsr_mod
    frames = _frames([(120, 200, "q"), (64, 64, "mb"), (200, 96, "q"), (33, 257, "mb")], seed=3)
    Ks = [50, 100, 20, 70, 0, 100, 50, 30]
    with fsr.Server(handle, pool_bytes=64 << 20, max_inflight=8, streams=2) as srv:
        tickets = {}
        for j, K in enumerate(Ks):
            img, mask = frames[j % len(frames)]
            tickets[srv.submit(img, mask, K)] = (j % len(frames), K)
        got = {}
        while len(got) < len(Ks):
            for t, ms, out in srv.poll(wait_ms=100):
                assert ms > 0
                got[t] = out.numpy().copy()
        stats = srv.stats()
    assert stats["completed"] == len(Ks) and stats["launches"] >= 1
    for t, (f, K) in tickets.items():
        img, mask = frames[f]
        assert np.array_equal(got[t], _alone(fsr, handle, img, mask, K)), (t, K)


def test_admission_respects_the_memory_budget(fsr_mod, handle):
    fsr = fsr_mod
    frames = _frames([(400, 400, "q")], seed=4)       # 1.44 MB per request in the pool
    pool = 4 << 20
    with fsr.Server(handle, pool_bytes=pool, max_inflight=64, streams=2) as srv:
        for _ in range(12):
            srv.submit(frames[0][0], frames[0][1], 40)
        n = 0
        outs = []
        while n < 12:
            r = srv.poll(wait_ms=200)
            n += len(r)
            outs += [o.numpy() for _, _, o in r]
        st = srv.stats()
        assert st["peak_pool_bytes"] <= pool
        ref = _alone(fsr, handle, frames[0][0], frames[0][1], 40)
        assert all(np.array_equal(o, ref) for o in outs)
        big = torch.zeros((1200, 1200), dtype=torch.float32)
        with pytest.raises(fsr.FsrError) as e:            # larger than the whole pool
            srv.submit(big, torch.zeros((1200, 1200), dtype=torch.uint8), 10)
        assert e.value.code == fsr.FSR_ERR_INVALID_ARG


def test_one_slot_serialises_but_completes(fsr_mod, handle):
    fsr = fsr_mod
    frames = _frames([(64, 80, "q"), (48, 48, "mb")], seed=5)
    with fsr.Server(handle, pool_bytes=16 << 20, max_inflight=1, streams=1) as srv:
        for j in range(6):
            srv.submit(*frames[j % 2], 25)
        n = 0
        while n < 6:
            n += len(srv.poll(wait_ms=200))
        assert srv.stats()["launches"] == 6


def test_poisson_stream_reports_latencies(fsr_mod, handle):
    fsr = fsr_mod
    frames = _frames([(180, 320, "q"), (90, 160, "mb")], seed=6)
    arr = serving.poisson_arrivals(150.0, 1.0, seed=7)
    rng = np.random.default_rng(8)
    kinds = rng.integers(0, 2, arr.size)
    iters = rng.choice([50, 100], arr.size)
    with fsr.Server(handle, pool_bytes=128 << 20, max_inflight=32, streams=2) as srv:
        res = serving.run_stream(srv, frames, arr, kinds, iters)
    s = serving.summarize(res, ["320x180", "160x90"], [0.0576, 0.0144])
    assert s["failed"] == 0 and s["requests"] == arr.size
    assert 0 < s["p50_ms"] <= s["p99_ms"]


def test_short_and_long_classes_equal_results_alone(fsr_mod, handle):
    """Frames above 1920 x 1088 pixels go to the long class (other streams),
    smaller ones to the high-priority stream; the server's S = 32 launches
    run short-lived CTAs.  Every result equals the frame reconstructed alone."""
    fsr = fsr_mod
    frames = _frames([(1100, 2000, "q"), (90, 130, "mb"), (1090, 1930, "mb"), (57, 75, "q")], seed=21)
    Ks = [30, 40, 20, 10, 25, 35]
    with fsr.Server(handle, pool_bytes=256 << 20, max_inflight=8, streams=2) as srv:
        tickets = {}
        for j, K in enumerate(Ks):
            img, mask = frames[j % len(frames)]
            tickets[srv.submit(img, mask, K)] = (j % len(frames), K)
        got = {}
        while len(got) < len(Ks):
            for t, ms, out in srv.poll(wait_ms=100):
                assert ms > 0
                got[t] = out.numpy().copy()
    for t, (f, K) in tickets.items():
        img, mask = frames[f]
        assert np.array_equal(got[t], _alone(fsr, handle, img, mask, K)), (t, K)
