"""Serving form: continuous batching of a request stream with admission by
device memory.  Each result must equal the same frame reconstructed alone,
and the FP64 oracle within the acceptance bar of tests/parity.py."""
import time

import numpy as np
import pytest

import oracle
import parity as PA
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


def _oracle_image(img, mask, K, support=32, B=4):
    img = np.asarray(img, np.float32)
    mask = np.asarray(mask, np.uint8)
    r = oracle.fsr_image_blocks(img, mask, B=B, L=(support - B) // 2, K=K, rho=PA.RHO)
    return oracle.assemble_image(r["target"], img.shape[0], img.shape[1], B)


def _check_oracle(results):
    """results: [(img, mask, K, got)] of one test.  Known pixels bit-exact in
    every result; over all pixels of the test together: the acceptance share
    within 0.5 grey levels (at least one pixel allowed on small totals) and
    PSNR within 0.01 dB of the oracle's."""
    gots, refs, truths = [], [], []
    for img, mask, K, got in results:
        img = np.asarray(img, np.float32)
        mask = np.asarray(mask, np.uint8)
        got = np.asarray(got, np.float64)
        assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64)), "known pixels changed"
        gots.append(got.ravel())
        refs.append(_oracle_image(img, mask, K).ravel())
        truths.append(img.astype(np.float64).ravel())
    g, r, t = np.concatenate(gots), np.concatenate(refs), np.concatenate(truths)
    n_out = int(np.sum(np.abs(g - r) > PA.GREY_TOL))
    assert n_out <= max(1, int((1 - PA.FRAC_MIN) * g.size)), (n_out, g.size)
    dpsnr = abs(PA.psnr(g, t) - PA.psnr(r, t))
    assert dpsnr <= PA.PSNR_TOL_DB, dpsnr


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
    _check_oracle([(frames[f][0].numpy(), frames[f][1].numpy(), K, got[t]) for t, (f, K) in tickets.items()])


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
        _check_oracle([(frames[0][0].numpy(), frames[0][1].numpy(), 40, outs[0])])
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
    _check_oracle([(frames[f][0].numpy(), frames[f][1].numpy(), K, got[t]) for t, (f, K) in tickets.items()])


def test_request_admitted_mid_flight_overlaps_and_shares_a_launch(fsr_mod, handle):
    """Continuous batching: a long-class request (2.2 MP, K = 2000, about
    0.1 s of the whole GPU) is launched first; while it runs, a short-class
    request (720p, K = 100) and then a burst of five more are submitted.  The short requests
    are admitted and launched while the long one is still on the device
    (they complete before it), the burst joins one launch while the slot of
    the short class is busy (fewer launches than requests), and every result
    equals the oracle's and the same frame reconstructed alone."""
    fsr = fsr_mod
    long_img = synth.pink_image(1100, 2000, 31)
    long_mask = synth.quarter_mask(1100, 2000, 32)
    lt = (torch.from_numpy(long_img).pin_memory(), torch.from_numpy(long_mask).pin_memory())
    shorts = _frames([(720, 1280, "q"), (64, 96, "mb"), (80, 72, "q"), (48, 130, "q"), (96, 64, "mb"),
                      (33, 45, "q")], seed=33)
    short_K = [100, 40, 30, 50, 20, 60]
    with fsr.Server(handle, pool_bytes=256 << 20, max_inflight=16, streams=2) as srv:
        t_long = srv.submit(lt[0], lt[1], 2000)
        while srv.stats()["launches"] < 1:      # the long request is on the device
            time.sleep(0.001)
        launches0 = srv.stats()["launches"]
        t_first = srv.submit(*shorts[0], short_K[0])
        while srv.stats()["launches"] < launches0 + 1:   # the first short launch runs
            time.sleep(0.0002)
        burst = [srv.submit(*shorts[j], short_K[j]) for j in range(1, len(shorts))]
        order, got = [], {}
        while len(got) < 2 + len(burst):
            for t, ms, out in srv.poll(wait_ms=100):
                assert ms > 0
                order.append(t)
                got[t] = out.numpy().copy()
        st = srv.stats()
    short_tickets = [t_first] + burst
    assert order[-1] == t_long, order                     # every short request finished first
    n_short_launches = st["launches"] - launches0
    assert n_short_launches < len(short_tickets), (n_short_launches, len(short_tickets))
    _check_oracle([(shorts[j][0].numpy(), shorts[j][1].numpy(), short_K[j], got[t])
                   for j, t in enumerate(short_tickets)])
    for j, t in enumerate(short_tickets):
        assert np.array_equal(got[t], _alone(fsr, handle, shorts[j][0], shorts[j][1], short_K[j])), j
    assert np.array_equal(got[t_long], _alone(fsr, handle, lt[0], lt[1], 2000))


@pytest.mark.parametrize("support", [32, 16])
def test_frame_stream_outputs_match_the_oracle(fsr_mod, handle, support):
    """Frame streaming with the copies overlapped (the path of the bench's
    frame-stream measurement): eight different 1080p quarter-sampled frames
    submitted at once, eight in flight, outputs written to reused pinned
    buffers; each frame equals the oracle within the acceptance bar."""
    fsr = fsr_mod
    n, K = 8, 40
    frames = [synth.fhd_quarter_case(seed=60 + i) for i in range(n)]
    host = [(torch.from_numpy(f).pin_memory(), torch.from_numpy(m).pin_memory()) for f, m in frames]
    outs = [torch.full((1080, 1920), -1.0, dtype=torch.float32).pin_memory() for _ in range(n)]
    with fsr.Server(handle, pool_bytes=1 << 30, max_inflight=8, streams=2, block=4,
                    border=(support - 4) // 2) as srv:
        res = serving.stream_frames(srv, host, K, outs)
    assert np.all(res["latency_ms"] > 0)
    for (img, mask), out in zip(frames, outs):
        got = out.numpy().astype(np.float64)
        assert np.array_equal(got[mask == 1], img[mask == 1].astype(np.float64))
        ref = _oracle_image(img, mask, K, support=support)
        assert PA.frac_within(got, ref) >= PA.FRAC_MIN
        assert abs(PA.psnr(got, img) - PA.psnr(ref, img)) <= PA.PSNR_TOL_DB
