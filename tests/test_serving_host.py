"""Host logic of the serving measurement (no GPU): Poisson arrivals, the
submit/poll driver against a fake engine, and the per-class summary."""
import numpy as np

from paper_2202_13926_gb300 import serving


def test_poisson_arrivals_rate_and_order():
    t = serving.poisson_arrivals(120.0, 50.0, seed=3)
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 50.0
    assert abs(t.size / 50.0 - 120.0) < 120.0 * 0.05          # ~6000 arrivals, 5 % band
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 120.0) < 0.05 / 120.0
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05      # exponential gaps: CV = 1
    assert np.array_equal(t, serving.poisson_arrivals(120.0, 50.0, seed=3))


class _FakeEngine:
    """Completes every request a fixed delay (by K) after its submission;
    the latency it reports is that delay, as the native engine reports
    submit-to-output times."""

    def __init__(self, delay_by_k):
        self.delay_by_k, self.pending, self.next = delay_by_k, [], 0

    def submit(self, img, mask, iters):
        import time
        t = self.next
        self.next += 1
        d = self.delay_by_k[iters]
        self.pending.append((t, time.perf_counter() + d, d))
        return t

    def poll(self, wait_ms=0):
        import time
        time.sleep(wait_ms / 1000.0)
        now = time.perf_counter()
        done = [(t, 1000.0 * d, None) for t, due, d in self.pending if due <= now]
        self.pending = [p for p in self.pending if p[1] > now]
        return done


def test_run_stream_and_summary():
    arr = np.linspace(0.0, 0.3, 31)
    kinds = np.arange(31) % 3
    iters = np.where(kinds == 2, 100, 50)
    eng = _FakeEngine({50: 0.002, 100: 0.02})
    res = serving.run_stream(eng, [(None, None)] * 3, arr, kinds, iters, poll_ms=1)
    lat = res["latency_ms"]
    assert not np.isnan(lat).any()
    assert np.allclose(lat[iters == 50], 2.0) and np.allclose(lat[iters == 100], 20.0)
    assert res["wall_s"] >= 0.3
    s = serving.summarize(res, ["a", "b", "c"], {0: 1.0, 1: 2.0, 2: 8.0})
    assert s["requests"] == 31 and s["failed"] == 0
    assert s["per_class"]["a"]["p99_ms"] == 2.0 and s["per_class"]["c"]["p50_ms"] == 20.0
    assert s["per_class"]["a"]["n"] + s["per_class"]["b"]["n"] + s["per_class"]["c"]["n"] == 31
    mp = sum({0: 1.0, 1: 2.0, 2: 8.0}[k] for k in kinds)
    assert abs(s["sustained_mp_s"] - mp / res["wall_s"]) < 1e-9


def test_stream_frames_cycles_the_output_buffers():
    """Frame streaming submits every frame at t = 0 and hands the output
    buffers out in turn."""
    class _Recorder(_FakeEngine):
        def __init__(self):
            super().__init__({7: 0.001})
            self.outs = []

        def submit(self, img, mask, iters, out=None):
            self.outs.append(out)
            return super().submit(img, mask, iters)

    eng = _Recorder()
    res = serving.stream_frames(eng, [("i%d" % i, "m%d" % i) for i in range(5)], 7, ["a", "b"])
    assert eng.outs == ["a", "b", "a", "b", "a"]
    assert np.allclose(res["latency_ms"], 1.0) and np.array_equal(res["kinds"], np.arange(5))
