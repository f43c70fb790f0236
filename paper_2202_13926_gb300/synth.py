"""Seeded synthetic images and sampling masks.

These stand in for the paper's test images (100 grayscale natural images at
1200 x 1200 with quarter sampling, Sec. IV), which are not available here.
The module holds no step of the reconstruction method: it only draws inputs,
and both the CUDA path and the oracle are fed from it.

Images are float32 in [0, 255]; masks are uint8 with 1 = known pixel.
"""
from __future__ import annotations

import numpy as np


def _edges(rng, H, W, n, lo=-60.0, hi=60.0):
    """Sum of ``n`` random straight step edges (random point, angle, height)."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.zeros((H, W))
    for _ in range(n):
        py, px = rng.uniform(0, H), rng.uniform(0, W)
        ang = rng.uniform(0, np.pi)
        h = rng.uniform(lo, hi)
        side = (xx - px) * np.sin(ang) - (yy - py) * np.cos(ang) > 0
        out += np.where(side, h, 0.0)
    return out


def sinusoid_image(H: int, W: int, seed: int, n_sin: int = 20, n_edges: int = 3) -> np.ndarray:
    """Sum of ``n_sin`` random 2-D sinusoids (amplitude 0-40 each) around mid
    grey, plus a linear gradient and ``n_edges`` random step edges, clipped to
    [0, 255]."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.full((H, W), 128.0)
    for _ in range(n_sin):
        a = rng.uniform(0, 40)
        fy, fx = rng.uniform(-0.25, 0.25, 2)
        ph = rng.uniform(0, 2 * np.pi)
        img += a * np.sin(2 * np.pi * (fy * yy + fx * xx) + ph)
    gy, gx = rng.uniform(-40, 40, 2)
    img += gy * (yy / max(H - 1, 1) - 0.5) + gx * (xx / max(W - 1, 1) - 0.5)
    img += _edges(rng, H, W, n_edges)
    return np.clip(img, 0, 255).astype(np.float32)


def pink_image(H: int, W: int, seed: int, n_edges: int = 8) -> np.ndarray:
    """Noise with a 1/f^2 power spectrum (natural-image statistics), scaled to
    [0, 255], with ``n_edges`` random step edges, clipped to [0, 255]."""
    rng = np.random.default_rng(seed)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f = np.sqrt(fy * fy + fx * fx)
    f[0, 0] = 1.0
    spec = (rng.standard_normal(f.shape) + 1j * rng.standard_normal(f.shape)) / f
    spec[0, 0] = 0.0
    img = np.fft.irfft2(spec, s=(H, W))
    img = (img - img.min()) / max(img.max() - img.min(), 1e-12) * 255.0
    img = img + _edges(rng, H, W, n_edges, -50.0, 50.0)
    return np.clip(img, 0, 255).astype(np.float32)


def iid_mask(H: int, W: int, seed: int, missing: float = 0.5) -> np.ndarray:
    """Each pixel independently missing with probability ``missing``."""
    rng = np.random.default_rng(seed)
    return (rng.random((H, W)) >= missing).astype(np.uint8)


def quarter_mask(H: int, W: int, seed: int) -> np.ndarray:
    """Quarter sampling: one random pixel of every 2 x 2 cell is known."""
    rng = np.random.default_rng(seed)
    ch, cw = -(-H // 2), -(-W // 2)
    pick = rng.integers(0, 4, size=(ch, cw))
    m = np.zeros((ch * 2, cw * 2), np.uint8)
    m[0::2, 0::2] = pick == 0
    m[0::2, 1::2] = pick == 1
    m[1::2, 0::2] = pick == 2
    m[1::2, 1::2] = pick == 3
    return np.ascontiguousarray(m[:H, :W])


def macroblock_mask(H: int, W: int, seed: int, lost: float = 0.1, mb: int = 16) -> np.ndarray:
    """Whole ``mb`` x ``mb`` macroblocks lost with probability ``lost``; the
    last row/column of macroblocks is clipped to the image."""
    rng = np.random.default_rng(seed)
    gh, gw = -(-H // mb), -(-W // mb)
    keep = rng.random((gh, gw)) >= lost
    m = np.repeat(np.repeat(keep, mb, axis=0), mb, axis=1)[:H, :W]
    return np.ascontiguousarray(m.astype(np.uint8))


# --- the workloads -----------------------------------------------------------

def small_case(seed: int = 1):
    """128 x 128 sinusoid image, i.i.d. mask with 50 % missing."""
    img = sinusoid_image(128, 128, seed)
    mask = iid_mask(128, 128, seed + 1000, 0.5)
    return img, mask


def fhd_quarter_case(seed: int = 2, H: int = 1080, W: int = 1920):
    """1920 x 1080 1/f^2 image with quarter sampling (25 % known)."""
    img = pink_image(H, W, seed)
    mask = quarter_mask(H, W, seed + 1000)
    return img, mask


BATCH_SIZES = ((256, 256), (720, 1280), (1080, 1920), (2160, 3840))
BATCH_KS = (50, 100, 200)


def batch_case(seed: int = 3, per_size: int = 12, sizes=BATCH_SIZES):
    """Images of mixed sizes (``per_size`` each), masks alternating between
    i.i.d. loss of 10-90 % and lost 16 x 16 macroblocks (5-20 %), with a
    per-image iteration count drawn from {50, 100, 200}.

    Returns a list of dicts with keys img, mask, K.
    """
    rng = np.random.default_rng(seed)
    items = []
    idx = 0
    for (H, W) in sizes:
        for j in range(per_size):
            s = int(rng.integers(0, 2**31 - 1))
            img = pink_image(H, W, s)
            if (idx % 2) == 0:
                mask = iid_mask(H, W, s + 1, float(rng.uniform(0.1, 0.9)))
            else:
                mask = macroblock_mask(H, W, s + 1, float(rng.uniform(0.05, 0.2)))
            K = int(rng.choice(BATCH_KS))
            items.append(dict(img=img, mask=mask, K=K))
            idx += 1
    return items
