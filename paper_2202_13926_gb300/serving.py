"""Poisson request streams for the serving form (fsr_server_*).

The engine (admission by device memory, continuous batching, streams) is
native; this module only generates arrival times, submits frames at those
times and collects the latencies the engine reports.
"""
from __future__ import annotations

import time

import numpy as np


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from start) of a Poisson process."""
    rng = np.random.default_rng(seed)
    n = max(1, int(rate_hz * duration_s * 1.5) + 16)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    return t[t < duration_s]


def run_stream(server, frames, arrivals, kinds, iters, poll_ms: int = 1):
    """Submit frames[kinds[i]] with K = iters[i] at arrivals[i]; wait for all.

    frames: list of (img, mask) host tensors; returns dict with per-request
    latency (ms), kind, K, completion order and the wall time of the stream.
    """
    n = len(arrivals)
    lat = np.full(n, np.nan)
    ticket_of = {}
    t0 = time.perf_counter()
    i = 0
    done = 0
    while done < n:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            img, mask = frames[kinds[i]]
            t = server.submit(img, mask, int(iters[i]))
            ticket_of[t] = i
            i += 1
        wait = 0
        if i < n:
            wait = max(0, min(poll_ms, int((arrivals[i] - (time.perf_counter() - t0)) * 1000)))
        elif done < n:
            wait = 20
        for t, ms, _out in server.poll(wait_ms=wait):
            lat[ticket_of[t]] = ms
            done += 1
    wall = time.perf_counter() - t0
    return dict(latency_ms=lat, kinds=np.asarray(kinds), iters=np.asarray(iters), wall_s=wall)


class _CycledOutputs:
    """Hands the output buffers out in turn (a client that consumes each
    result before its buffer comes round again)."""

    def __init__(self, server, outs):
        self.server, self.outs, self.i = server, outs, 0

    def submit(self, img, mask, iters):
        out = self.outs[self.i % len(self.outs)]
        self.i += 1
        return self.server.submit(img, mask, iters, out=out)

    def poll(self, wait_ms=0):
        return self.server.poll(wait_ms)


def stream_frames(server, frames, iters, outs):
    """Frame streaming: every frame of ``frames`` (pinned host tensors) is
    submitted at t = 0 with K = ``iters``; the server overlaps the copies in,
    the launches and the copies out of the frames in flight.  Frame i is
    written to outs[i % len(outs)]; returns the run_stream result."""
    n = len(frames)
    return run_stream(_CycledOutputs(server, outs), frames, np.zeros(n), np.arange(n), np.full(n, int(iters)))


def summarize(res, kind_names, frame_megapixels):
    lat = res["latency_ms"]
    out = {"requests": int(lat.size), "failed": int(np.sum(lat < 0)),
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "wall_s": res["wall_s"]}
    mp = float(sum(frame_megapixels[k] for k in res["kinds"]))
    out["sustained_mp_s"] = mp / res["wall_s"]
    out["sustained_fps"] = lat.size / res["wall_s"]
    per = {}
    for k, name in enumerate(kind_names):
        sel = res["kinds"] == k
        if sel.any():
            per[name] = {"n": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                         "p99_ms": float(np.percentile(lat[sel], 99))}
    out["per_class"] = per
    return out
