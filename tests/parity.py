"""Shared helpers of the GPU parity tests: acceptance metrics and the
tie-class rule for comparing selection sequences.

Acceptance of the FP32 path against the FP64 oracle (written in the tests):
  * |gpu - oracle| <= 0.5 grey levels on >= 99.9 % of the pixels,
  * PSNR against the ground-truth image within 0.01 dB of the oracle's,
  * known pixels bit-exact.
FP64 debug path: identical selection sequences, except at a step where the
oracle's relative gap between the best and second-best objective is below
1e-12 ("tie class": the two choices are equal to rounding).
"""
from __future__ import annotations

import numpy as np

GREY_TOL = 0.5
FRAC_MIN = 0.999
PSNR_TOL_DB = 0.01
TIE_MARGIN = 1e-12
# rho-hat as the library receives it: fsr_params carries it as a binary32
# (0.7 -> 0.699999988...); the oracle is given the same value, so that both
# compute the spatial weights of Eq. (5) from one parameter (with rho = 0.7
# in binary64 the weights differ by up to ~4e-7 relative, enough to swap two
# objectives 4e-8 apart)
RHO = float(np.float32(0.7))
# relative gap between the best component and the best one that is not its
# conjugate below which FP32 arithmetic cannot tell the two apart (the FP32
# spectrum carries a few units of 2^-24 relative error per iteration)
FP32_NEAR_TIE = 3e-6


def psnr(x, truth, mask=None):
    d = np.asarray(x, np.float64) - np.asarray(truth, np.float64)
    if mask is not None:
        d = d[mask]
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0 else 10.0 * np.log10(255.0 ** 2 / mse)


def frac_within(a, b, tol=GREY_TOL):
    return float(np.mean(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)) <= tol))


def sequence_mismatches(seq_gpu, seq_ref, margin_ref):
    """Blocks whose sequences differ at a step that is not a tie.

    Returns (n_hard, n_tie): counts of blocks whose first differing step has
    an oracle margin >= TIE_MARGIN (hard) or below it (tie class)."""
    seq_gpu = np.asarray(seq_gpu).astype(np.int64)
    seq_ref = np.asarray(seq_ref).astype(np.int64)
    diff = seq_gpu != seq_ref
    rows = np.nonzero(diff.any(axis=1))[0]
    n_hard = n_tie = 0
    for r in rows:
        first = int(np.argmax(diff[r]))
        if margin_ref[r, first] < TIE_MARGIN:
            n_tie += 1
        else:
            n_hard += 1
    return n_hard, n_tie


def same_sequence_pixels(seq_gpu, seq_ref, H, W, B):
    """H x W flags: pixels of target blocks whose selection sequences are
    identical on both sides (a tie-class divergence legitimately changes the
    values of its block; value comparisons of the FP64 path use these)."""
    same = np.all(np.asarray(seq_gpu).astype(np.int64) == np.asarray(seq_ref).astype(np.int64), axis=1)
    nbx, nby = -(-W // B), -(-H // B)
    blocks = same.reshape(nby, nbx)
    return np.kron(blocks, np.ones((B, B), bool))[:H, :W]


def block_pixels(flags, H, W, B):
    """H x W booleans: the pixels of the target blocks whose flag is set
    (flags in raster order of the blocks)."""
    nbx, nby = -(-W // B), -(-H // B)
    blocks = np.asarray(flags, bool).reshape(nby, nbx)
    return np.kron(blocks, np.ones((B, B), bool))[:H, :W]
