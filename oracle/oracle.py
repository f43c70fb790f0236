"""ctypes wrapper of the plain FP64 C oracle (``fsr_oracle.c``).

Test infrastructure only (tests, smoke check, CPU baseline of the benchmark).
Each wrapper names the part of the paper its C routine follows:
  spatial_weight  Sec. II, Eq. (5)
  freq_weight     Sec. II, Eq. (9)
  dft2_real       the 2-D DFT F2 of Eq. (7)
  fsr_block       Sec. II, Eqs. (2), (5)-(12) on one support block
  fsr_image_blocks Sec. III-A tiling, Eq. (13), plus the write-back of Sec. II
  fsr_image_reuse the sequential form that re-uses reconstructed pixels, which
                  Sec. II leaves out (blocks in raster order; reading stated in
                  fsr_oracle.c)
With ``conj_pairs`` the two block routines run the ablation of the original
FSR's real model (the selected component and its conjugate updated together),
which is not the paper's Eqs. (11)-(12).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfsr_oracle.so")
_lock = threading.Lock()
_default = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    src = os.path.join(_HERE, "fsr_oracle.c")
    hdr = os.path.join(_HERE, "fsr_oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("K", ctypes.c_int), ("rho", ctypes.c_double),
                ("gamma", ctypes.c_double), ("freq_weight", ctypes.c_int),
                ("conj_pairs", ctypes.c_int)]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


class _BlockOut(ctypes.Structure):
    _fields_ = [(n, _DP) for n in ("w", "R0re", "R0im", "Wre", "Wim")] + \
               [("seq", _IP)] + \
               [(n, _DP) for n in ("pre", "pim", "margin", "margin_nc", "Rhre", "Rhim",
                                   "Gre", "Gim", "gre", "gim")] + \
               [("g_need", ctypes.POINTER(ctypes.c_ubyte))]


def _dp(a):
    return a.ctypes.data_as(_DP) if a is not None else None


class OracleLib:
    """One loaded copy of the oracle library (the default build, or a variant
    compiled from modified source by the mutation tests)."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.fsr_oracle_spatial_weight.argtypes = [ctypes.c_int, ctypes.c_double, _DP]
        lib.fsr_oracle_freq_weight.argtypes = [ctypes.c_int, _DP]
        lib.fsr_oracle_dft2_real.argtypes = [ctypes.c_int, _DP, _DP, _DP]
        lib.fsr_oracle_block.argtypes = [ctypes.POINTER(_Params), _DP,
                                         ctypes.POINTER(ctypes.c_ubyte),
                                         ctypes.POINTER(_BlockOut)]
        lib.fsr_oracle_block.restype = ctypes.c_int
        lib.fsr_oracle_block_scaled.argtypes = [ctypes.POINTER(_Params), _DP, _DP, ctypes.POINTER(_BlockOut)]
        lib.fsr_oracle_block_scaled.restype = ctypes.c_int
        lib.fsr_oracle_image_reuse.argtypes = [
            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_ubyte),
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_long, _DP, ctypes.c_int, _DP, _IP, _DP]
        lib.fsr_oracle_image_reuse.restype = ctypes.c_long
        lib.fsr_oracle_image_blocks.argtypes = [
            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_ubyte),
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(_Params), ctypes.c_long, ctypes.POINTER(ctypes.c_long),
            ctypes.c_int, _DP, _DP, _IP, _DP, _DP]
        lib.fsr_oracle_image_blocks.restype = ctypes.c_long
        lib.fsr_oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def max_threads(self) -> int:
        return int(self.lib.fsr_oracle_max_threads())

    def spatial_weight(self, S: int, rho: float) -> np.ndarray:
        """Eq. (5) on every pixel of an S x S support (centre (S-1)/2)."""
        out = np.empty((S, S), np.float64)
        self.lib.fsr_oracle_spatial_weight(S, rho, _dp(out))
        return out

    def freq_weight(self, S: int) -> np.ndarray:
        """Eq. (9)."""
        out = np.empty((S, S), np.float64)
        self.lib.fsr_oracle_freq_weight(S, _dp(out))
        return out

    def dft2_real(self, x: np.ndarray) -> np.ndarray:
        """Unnormalised 2-D DFT, e^{-j2pi(km+ln)/S}, of a real S x S array."""
        x = np.ascontiguousarray(x, np.float64)
        S = x.shape[0]
        re = np.empty((S, S)); im = np.empty((S, S))
        self.lib.fsr_oracle_dft2_real(S, _dp(x), _dp(re), _dp(im))
        return re + 1j * im

    def fsr_block(self, f: np.ndarray, known: np.ndarray, K: int, rho: float = 0.7,
                  gamma: float = 0.5, freq_weight: bool = True,
                  history: bool = False, conj_pairs: bool = False, scale=None) -> dict:
        """FSR of one S x S support block (Sec. II).

        Returns w, R0, W, seq (u*S+v per iteration, -1 if skipped), p, margin,
        G, g (complex, all pixels), skipped, and with ``history`` the residual
        spectra R^(nu) for nu = 0..K.  With ``scale`` (S x S, >= 0) the weight
        of Eq. (5) is scale * w0 and ``known`` is ignored (the pixels with
        scale 0 are the unknown ones).
        """
        f = np.ascontiguousarray(f, np.float64)
        S = f.shape[0]
        if scale is not None:
            scale = np.ascontiguousarray(scale, np.float64)
            assert scale.shape == (S, S)
            known = (scale > 0).astype(np.uint8)
        known = np.ascontiguousarray(known, np.uint8)
        assert f.shape == (S, S) and known.shape == (S, S)
        P = _Params(S, K, rho, gamma, int(bool(freq_weight)), int(bool(conj_pairs)))
        arrs = {n: np.empty((S, S)) for n in ("w", "R0re", "R0im", "Wre", "Wim",
                                                "Gre", "Gim", "gre", "gim")}
        seq = np.empty(max(K, 1), np.int32)
        pre = np.empty(max(K, 1)); pim = np.empty(max(K, 1)); margin = np.empty(max(K, 1))
        o = _BlockOut()
        for n, a in arrs.items():
            setattr(o, n, _dp(a))
        margin_nc = np.empty(max(K, 1))
        o.seq = seq.ctypes.data_as(_IP)
        o.pre, o.pim, o.margin, o.margin_nc = _dp(pre), _dp(pim), _dp(margin), _dp(margin_nc)
        if history:
            Rhre = np.empty((K + 1, S, S)); Rhim = np.empty((K + 1, S, S))
            o.Rhre, o.Rhim = _dp(Rhre), _dp(Rhim)
        if scale is not None:
            r = self.lib.fsr_oracle_block_scaled(ctypes.byref(P), _dp(f), _dp(scale), ctypes.byref(o))
        else:
            r = self.lib.fsr_oracle_block(ctypes.byref(P), _dp(f),
                                         known.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                         ctypes.byref(o))
        if r < 0:
            raise ValueError("oracle rejected the block arguments")
        res = dict(
            w=arrs["w"], R0=arrs["R0re"] + 1j * arrs["R0im"],
            W=arrs["Wre"] + 1j * arrs["Wim"], seq=seq[:K].copy(),
            p=(pre + 1j * pim)[:K].copy(), margin=margin[:K].copy(), margin_nc=margin_nc[:K].copy(),
            G=arrs["Gre"] + 1j * arrs["Gim"], g=arrs["gre"] + 1j * arrs["gim"],
            skipped=bool(r == 1))
        if history:
            res["R_hist"] = Rhre + 1j * Rhim
        return res

    def fsr_image_blocks(self, img: np.ndarray, mask: np.ndarray, B: int = 4, L: int = 14,
                         K: int = 100, rho: float = 0.7, gamma: float = 0.5,
                         freq_weight: bool = True, block_ids=None,
                         threads: int = 0, conj_pairs: bool = False) -> dict:
        """FSR of selected target blocks of an image (Sec. III-A tiling).

        Returns ``target`` (n, B, B) float64 (NaN outside the image), ``seq``
        (n, K) int32, ``margin`` (n, K), ``n_empty``, the ``block_ids`` used
        and ``im_target`` (n, B, B): Im g at the unknown target pixels, a
        diagnostic of the complex model (the output is Re g; Eq. 11).
        """
        img = np.ascontiguousarray(img, np.float32)
        mask = np.ascontiguousarray(mask, np.uint8)
        H, Wd = img.shape
        assert mask.shape == (H, Wd)
        nbx, nby = -(-Wd // B), -(-H // B)
        if block_ids is None:
            ids = None
            n = nbx * nby
        else:
            ids = np.ascontiguousarray(block_ids, np.int64)
            n = ids.size
        target = np.empty((n, B, B))
        im_target = np.empty((n, B, B))
        seq = np.empty((n, max(K, 1)), np.int32)
        margin = np.empty((n, max(K, 1)))
        margin_nc = np.empty((n, max(K, 1)))
        P = _Params(B + 2 * L, K, rho, gamma, int(bool(freq_weight)), int(bool(conj_pairs)))
        r = self.lib.fsr_oracle_image_blocks(
            img.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), H, Wd, Wd, B, L,
            ctypes.byref(P), n,
            ids.ctypes.data_as(ctypes.POINTER(ctypes.c_long)) if ids is not None else None,
            int(threads), _dp(target), _dp(im_target), seq.ctypes.data_as(_IP), _dp(margin), _dp(margin_nc))
        if r < 0:
            raise ValueError("oracle rejected the image arguments")
        return dict(target=target, seq=seq[:, :K], margin=margin[:, :K], margin_nc=margin_nc[:, :K],
                    n_empty=int(r), block_ids=np.arange(n) if ids is None else ids, im_target=im_target)


    def fsr_image_reuse(self, img: np.ndarray, mask: np.ndarray, B: int = 4, L: int = 14,
                        K: int = 100, delta: float = 0.5, rho: float = 0.7, gamma: float = 0.5,
                        freq_weight: bool = True, nblocks: int = 0, given=None, threads: int = 0) -> dict:
        """The sequential form that re-uses reconstructed pixels: blocks in
        raster order, unknown pixels of earlier targets enter later supports
        with their reconstruction and the weight delta * rho^dist.

        Returns ``out`` (H, W) float64 (the first ``nblocks`` blocks, all when
        0; NaN on unknown pixels of later blocks), ``seq`` and ``margin``
        (nblocks, K), ``n_empty``.  With ``given`` (H, W) the re-used values
        come from that reconstruction instead of the routine's own earlier
        results (every block on its own, ``threads`` OpenMP threads).
        """
        img = np.ascontiguousarray(img, np.float32)
        mask = np.ascontiguousarray(mask, np.uint8)
        H, Wd = img.shape
        assert mask.shape == (H, Wd)
        nall = -(-Wd // B) * -(-H // B)
        n = nall if nblocks <= 0 else min(int(nblocks), nall)
        out = np.empty((H, Wd))
        seq = np.empty((n, max(K, 1)), np.int32)
        margin = np.empty((n, max(K, 1)))
        P = _Params(B + 2 * L, K, rho, gamma, int(bool(freq_weight)), 0)
        r = self.lib.fsr_oracle_image_reuse(
            img.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), H, Wd, Wd, B, L,
            ctypes.byref(P), float(delta), n,
            _dp(np.ascontiguousarray(given, np.float64)) if given is not None else None, int(threads),
            _dp(out), seq.ctypes.data_as(_IP), _dp(margin))
        if r < 0:
            raise ValueError("oracle rejected the image arguments")
        return dict(out=out, seq=seq[:, :K], margin=margin[:, :K], n_empty=int(r))


def assemble_image(target: np.ndarray, H: int, Wd: int, B: int) -> np.ndarray:
    """Place the (nby*nbx, B, B) target blocks of all blocks into an H x Wd image."""
    nbx, nby = -(-Wd // B), -(-H // B)
    full = target.reshape(nby, nbx, B, B).transpose(0, 2, 1, 3).reshape(nby * B, nbx * B)
    return np.ascontiguousarray(full[:H, :Wd])


def default() -> OracleLib:
    """The oracle built from ``fsr_oracle.c`` as committed."""
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
    return _default


def build_variant(source_text: str, out_dir: str, name: str) -> OracleLib:
    """Compile ``source_text`` (a modified copy of ``fsr_oracle.c``) into
    ``out_dir`` and load it; used only to check that the pins catch planted
    mistakes."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, name + ".c")
    with open(src, "w") as fh:
        fh.write(source_text)
    so = os.path.join(out_dir, "lib" + name + ".so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", "-fopenmp", "-I", _HERE, src, "-o", so, "-lm"],
                   check=True)
    return OracleLib(so)


def source_text() -> str:
    with open(os.path.join(_HERE, "fsr_oracle.c")) as fh:
        return fh.read()


def max_threads() -> int:
    return default().max_threads()


def spatial_weight(*a, **k):
    return default().spatial_weight(*a, **k)


def freq_weight(*a, **k):
    return default().freq_weight(*a, **k)


def dft2_real(*a, **k):
    return default().dft2_real(*a, **k)


def fsr_block(*a, **k):
    return default().fsr_block(*a, **k)


def fsr_image_blocks(*a, **k):
    return default().fsr_image_blocks(*a, **k)


def fsr_image_reuse(*a, **k):
    return default().fsr_image_reuse(*a, **k)
