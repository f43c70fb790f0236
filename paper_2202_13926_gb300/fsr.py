"""ctypes binding of libfsr_gb300.so (declared in include/fsr.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of the library.  There is no CPU fallback: if the library is not
built, or the device is not an sm_103a GPU, the calls raise.

Tensors are torch tensors: device tensors for ``fsr_reconstruct`` (PyTorch
owns the memory and the stream), host tensors or numpy arrays for
``fsr_reconstruct_host``.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

FSR_OK = 0
FSR_ERR_INVALID_ARG = 1
FSR_ERR_OOM = 2
FSR_ERR_CUDA = 3
FSR_ERR_TIMEOUT = 4
FSR_ERR_UNSUPPORTED = 5

FSR_FP32 = 0
FSR_FP64_DEBUG = 1
FSR_TC_BF16X3 = 2
FSR_TC_TF32 = 3
PRECISIONS = {"fp32": FSR_FP32, "fp64": FSR_FP64_DEBUG, "tc_bf16x3": FSR_TC_BF16X3,
              "tc_tf32": FSR_TC_TF32}
FSR_UPDATE_SINGLE, FSR_UPDATE_CONJ_PAIR = 0, 1
UPDATES = {"single": FSR_UPDATE_SINGLE, "conj_pair": FSR_UPDATE_CONJ_PAIR}

# every function declared in include/fsr.h
EXPORTED = ("fsr_create", "fsr_destroy", "fsr_last_error", "fsr_reconstruct",
            "fsr_reconstruct_host", "fsr_num_blocks", "fsr_reconstruct_batch",
            "fsr_batch_create", "fsr_batch_launch", "fsr_batch_destroy",
            "fsr_autotune_batch", "fsr_get_schedule", "fsr_set_schedule",
            "fsr_reconstruct_batch_static", "fsr_server_create", "fsr_server_submit",
            "fsr_server_poll", "fsr_server_stats", "fsr_server_destroy",
            "fsr_check_status", "fsr_inject_tile_wait_fault", "fsr_empty_blocks")


class FsrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[fsr status {code}] {msg}")
        self.code = code


class fsr_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t),
                ("schedule_cache", ctypes.c_char_p)]


class fsr_image_desc(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("height", ctypes.c_int), ("width", ctypes.c_int), ("pitch", ctypes.c_int),
                ("iters", ctypes.c_int), ("seq_out", ctypes.c_void_p)]


class fsr_schedule(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int), ("chunk", ctypes.c_int)]


class fsr_server_config(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("streams", ctypes.c_int)]


class fsr_params(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("border", ctypes.c_int), ("iters", ctypes.c_int),
                ("rho", ctypes.c_float), ("gamma", ctypes.c_float),
                ("freq_weight", ctypes.c_int), ("precision", ctypes.c_int),
                ("seq_out", ctypes.c_void_p), ("update", ctypes.c_int), ("reuse", ctypes.c_float)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing: build it with __graft_entry__.build() "
                "(the CUDA library is required; there is no fallback)")
        lib = ctypes.CDLL(p)
        vp, ip = ctypes.c_void_p, ctypes.c_int
        lib.fsr_create.argtypes = [ctypes.POINTER(fsr_config), ctypes.POINTER(vp)]
        lib.fsr_create.restype = ip
        lib.fsr_destroy.argtypes = [vp]
        lib.fsr_destroy.restype = ip
        lib.fsr_last_error.argtypes = [vp]
        lib.fsr_last_error.restype = ctypes.c_char_p
        for name in ("fsr_reconstruct", "fsr_reconstruct_host"):
            f = getattr(lib, name)
            f.argtypes = [vp, vp, vp, ip, ip, ip, ctypes.POINTER(fsr_params), vp, vp]
            f.restype = ip
        lib.fsr_num_blocks.argtypes = [ip, ip, ip]
        lib.fsr_num_blocks.restype = ctypes.c_longlong
        dp, pp = ctypes.POINTER(fsr_image_desc), ctypes.POINTER(fsr_params)
        lib.fsr_reconstruct_batch.argtypes = [vp, ip, dp, pp, vp]
        lib.fsr_batch_create.argtypes = [vp, ip, dp, pp, ctypes.POINTER(vp)]
        lib.fsr_batch_launch.argtypes = [vp, vp]
        lib.fsr_batch_destroy.argtypes = [vp]
        lib.fsr_autotune_batch.argtypes = [vp, ip, dp, pp, ctypes.POINTER(fsr_schedule),
                                           ctypes.POINTER(ctypes.c_float)]
        lib.fsr_get_schedule.argtypes = [vp, ip, ip, ctypes.POINTER(fsr_schedule)]
        lib.fsr_set_schedule.argtypes = [vp, ip, ip, ctypes.POINTER(fsr_schedule)]
        lib.fsr_reconstruct_batch_static.argtypes = [ip, dp, pp, vp, ctypes.c_char_p, ctypes.c_size_t]
        llp = ctypes.POINTER(ctypes.c_longlong)
        lib.fsr_server_create.argtypes = [vp, ctypes.POINTER(fsr_server_config), pp, ctypes.POINTER(vp)]
        lib.fsr_server_submit.argtypes = [vp, vp, vp, ip, ip, ip, vp, llp]
        lib.fsr_server_poll.argtypes = [vp, llp, ctypes.POINTER(ctypes.c_double), ip,
                                        ctypes.POINTER(ctypes.c_int), ip]
        lib.fsr_server_stats.argtypes = [vp, llp, llp, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), llp, ctypes.POINTER(ctypes.c_size_t)]
        lib.fsr_server_destroy.argtypes = [vp]
        lib.fsr_check_status.argtypes = [vp, vp]
        lib.fsr_inject_tile_wait_fault.argtypes = [vp]
        lib.fsr_empty_blocks.argtypes = [vp, vp, llp]
        for name in ("fsr_server_create", "fsr_server_submit", "fsr_server_poll",
                     "fsr_server_stats", "fsr_server_destroy"):
            getattr(lib, name).restype = ip
        for name in ("fsr_reconstruct_batch_static", "fsr_reconstruct_batch", "fsr_batch_create", "fsr_batch_launch",
                     "fsr_batch_destroy", "fsr_autotune_batch", "fsr_get_schedule",
                     "fsr_set_schedule", "fsr_check_status", "fsr_inject_tile_wait_fault",
                     "fsr_empty_blocks"):
            getattr(lib, name).restype = ip
        if path is None:
            _lib = lib
        return lib


def _check(code: int, handle) -> None:
    if code != FSR_OK:
        lib = load_library()
        msg = lib.fsr_last_error(handle).decode(errors="replace")
        raise FsrError(code, msg)


def make_params(block=4, border=14, iters=100, rho=0.7, gamma=0.5, freq_weight=True,
                precision="fp32", seq_out=None, update="single", reuse=0.0) -> fsr_params:
    """fsr_params of include/fsr.h: B = block, L = border (support S = B + 2L:
    32, 24, 16, 8 or 4), K = iters, rho-hat, gamma, w_f switch, precision
    ("fp32", "fp64", "tc_bf16x3", "tc_tf32"), optional int16 CUDA tensor for
    the selected indices, update ("single": the paper's; "conj_pair": the
    ablation of the original FSR's real model), reuse (delta: 0 = the paper's
    independent blocks; > 0 re-uses reconstructed pixels of earlier blocks
    with that weight, the original FSR's sequential form)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    upd = UPDATES[update] if isinstance(update, str) else int(update)
    seq_ptr = None
    if seq_out is not None:
        import torch
        if not (isinstance(seq_out, torch.Tensor) and seq_out.is_cuda and seq_out.dtype == torch.int16
                and seq_out.is_contiguous()):
            raise ValueError("seq_out must be a contiguous int16 CUDA tensor")
        seq_ptr = seq_out.data_ptr()
    return fsr_params(int(block), int(border), int(iters), float(rho), float(gamma),
                      int(bool(freq_weight)), prec, seq_ptr, upd, float(reuse))


def fsr_num_blocks(height: int, width: int, block: int) -> int:
    return int(load_library().fsr_num_blocks(int(height), int(width), int(block)))


def fsr_last_error(handle=None) -> str:
    return load_library().fsr_last_error(handle).decode(errors="replace")


def fsr_create(device: int = 0, workspace_bytes: int = 0, schedule_cache: str | None = None) -> int:
    lib = load_library()
    h = ctypes.c_void_p()
    cache = schedule_cache.encode() if schedule_cache else None
    _check(lib.fsr_create(ctypes.byref(fsr_config(int(device), int(workspace_bytes), cache)),
                          ctypes.byref(h)), None)
    return h.value


def fsr_destroy(handle) -> None:
    load_library().fsr_destroy(handle)


def _geometry(img, mask, out):
    import torch
    if img.dim() != 2 or mask.shape != img.shape or out.shape != img.shape:
        raise ValueError("img, mask and out must be 2-D tensors of one shape")
    if img.dtype != torch.float32 or out.dtype != torch.float32 or mask.dtype != torch.uint8:
        raise ValueError("img/out must be float32 and mask uint8")
    H, W = img.shape
    # the stride of a dimension of size 1 is arbitrary in torch and never used
    pitch = img.stride(0) if H > 1 else W
    for t in (img, mask, out):
        if (W > 1 and t.stride(1) != 1) or (H > 1 and t.stride(0) != pitch):
            raise ValueError("img, mask and out must share one row pitch with unit column stride")
    return H, W, pitch


def fsr_reconstruct(handle, img, mask, params: fsr_params, out, stream=None) -> None:
    """Enqueue the reconstruction of one image (device tensors) on ``stream``
    (a torch.cuda.Stream, a raw cudaStream_t int, or None = current stream)."""
    import torch
    for t in (img, mask, out):
        if not t.is_cuda:
            raise ValueError("fsr_reconstruct takes CUDA tensors (use fsr_reconstruct_host for host data)")
    H, W, pitch = _geometry(img, mask, out)
    if stream is None:
        stream = torch.cuda.current_stream(img.device).cuda_stream
    elif isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    _check(load_library().fsr_reconstruct(handle, img.data_ptr(), mask.data_ptr(), H, W, pitch,
                                          ctypes.byref(params), out.data_ptr(), stream), handle)


def fsr_reconstruct_host(handle, img, mask, params: fsr_params, out, stream=None) -> None:
    """Reconstruct host data (torch CPU tensors, ideally pinned, or numpy
    arrays); copies in, computes and copies out inside the call."""
    import numpy as np
    import torch

    def as_tensor(x):
        return torch.from_numpy(x) if isinstance(x, np.ndarray) else x
    img, mask, out = as_tensor(img), as_tensor(mask), as_tensor(out)
    for t in (img, mask, out):
        if t.is_cuda:
            raise ValueError("fsr_reconstruct_host takes host tensors")
    H, W, pitch = _geometry(img, mask, out)
    if stream is None:
        stream = 0
    elif isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    _check(load_library().fsr_reconstruct_host(handle, img.data_ptr(), mask.data_ptr(), H, W, pitch,
                                               ctypes.byref(params), out.data_ptr(), stream), handle)


def _stream_ptr(stream, device=None):
    import torch
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return stream


def fsr_check_status(handle, stream=None) -> None:
    """Synchronise ``stream`` and raise FsrError(FSR_ERR_TIMEOUT) when a
    bounded tile-copy wait of a single-image launch gave up."""
    _check(load_library().fsr_check_status(handle, _stream_ptr(stream)), handle)


def fsr_empty_blocks(handle, stream=None) -> int:
    """Synchronise ``stream``; number of blocks without a known pixel since
    the previous call (the counter is reset)."""
    c = ctypes.c_longlong()
    _check(load_library().fsr_empty_blocks(handle, _stream_ptr(stream), ctypes.byref(c)), handle)
    return c.value


def fsr_inject_tile_wait_fault(handle) -> None:
    """Test hook: the next tile-copy launch on ``handle`` waits for bytes
    that never arrive, so its bounded waits run out (no GPU fault)."""
    _check(load_library().fsr_inject_tile_wait_fault(handle), handle)


def image_desc(img, mask, out, iters: int, seq_out=None) -> fsr_image_desc:
    """Descriptor of one device image of a batch (torch CUDA tensors)."""
    import torch
    for t in (img, mask, out):
        if not t.is_cuda:
            raise ValueError("batch images must be CUDA tensors")
    H, W, pitch = _geometry(img, mask, out)
    seq_ptr = None
    if seq_out is not None:
        if not (seq_out.is_cuda and seq_out.dtype == torch.int16 and seq_out.is_contiguous()):
            raise ValueError("seq_out must be a contiguous int16 CUDA tensor")
        seq_ptr = seq_out.data_ptr()
    return fsr_image_desc(img.data_ptr(), mask.data_ptr(), out.data_ptr(), H, W, pitch,
                          int(iters), seq_ptr)


def _descs(descs):
    arr = (fsr_image_desc * len(descs))(*descs)
    return arr, len(descs)


def _stream_ptr(stream, device=None):
    import torch
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return stream


def fsr_reconstruct_batch(handle, descs, params: fsr_params, stream=None) -> None:
    arr, n = _descs(descs)
    _check(load_library().fsr_reconstruct_batch(handle, n, arr, ctypes.byref(params),
                                                _stream_ptr(stream)), handle)


def fsr_reconstruct_batch_static(descs, params: fsr_params, stream=None) -> None:
    """Batch reconstruction that allocates no device memory (scratch in the
    library's static device array; at most 64 images per call)."""
    arr, n = _descs(descs)
    buf = ctypes.create_string_buffer(512)
    code = load_library().fsr_reconstruct_batch_static(n, arr, ctypes.byref(params),
                                                       _stream_ptr(stream), buf, len(buf))
    if code != FSR_OK:
        raise FsrError(code, buf.value.decode(errors="replace"))


def fsr_batch_create(handle, descs, params: fsr_params) -> int:
    arr, n = _descs(descs)
    b = ctypes.c_void_p()
    _check(load_library().fsr_batch_create(handle, n, arr, ctypes.byref(params), ctypes.byref(b)),
           handle)
    return b.value


def fsr_batch_launch(batch, stream=None, handle=None) -> None:
    _check(load_library().fsr_batch_launch(batch, _stream_ptr(stream)), handle)


def fsr_batch_destroy(batch) -> None:
    load_library().fsr_batch_destroy(batch)


def fsr_autotune_batch(handle, descs, params: fsr_params):
    arr, n = _descs(descs)
    best = fsr_schedule()
    ms = ctypes.c_float()
    _check(load_library().fsr_autotune_batch(handle, n, arr, ctypes.byref(params),
                                             ctypes.byref(best), ctypes.byref(ms)), handle)
    return (best.warps, best.chunk), ms.value


def fsr_get_schedule(handle, block: int = 4, precision: int = FSR_FP32):
    s = fsr_schedule()
    _check(load_library().fsr_get_schedule(handle, int(block), int(precision), ctypes.byref(s)),
           handle)
    return s.warps, s.chunk


def fsr_set_schedule(handle, warps: int, chunk: int, block: int = 4, precision: int = FSR_FP32):
    s = fsr_schedule(int(warps), int(chunk))
    _check(load_library().fsr_set_schedule(handle, int(block), int(precision), ctypes.byref(s)),
           handle)


class Handle:
    """Owning wrapper of an ``fsr_handle``."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0, schedule_cache: str | None = None):
        self.device = device
        self.ptr = fsr_create(device, workspace_bytes, schedule_cache)

    def close(self):
        if self.ptr:
            fsr_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reconstruct(self, img, mask, out=None, stream=None, **kw):
        import torch
        if out is None:
            out = torch.empty_like(img)
        fsr_reconstruct(self.ptr, img, mask, make_params(**kw), out, stream)
        return out

    def reconstruct_host(self, img, mask, out=None, stream=None, **kw):
        import numpy as np
        if out is None:
            out = np.empty(img.shape, np.float32)
        fsr_reconstruct_host(self.ptr, img, mask, make_params(**kw), out, stream)
        return out

    def check_status(self, stream=None):
        fsr_check_status(self.ptr, stream)

    def reconstruct_channels(self, img, mask, out=None, stream=None, **kw):
        """Multi-channel image (C, H, W) with one mask (H, W) or one per
        channel (C, H, W): the C planes are reconstructed independently (FSR
        works on single-channel images) in one batch launch."""
        import torch
        if img.dim() != 3:
            raise ValueError("img must be (C, H, W)")
        C = img.shape[0]
        masks = [mask] * C if mask.dim() == 2 else [mask[c] for c in range(C)]
        if out is None:
            out = torch.empty_like(img)
        p = make_params(**kw)
        fsr_reconstruct_batch(self.ptr, [image_desc(img[c], masks[c], out[c], p.iters) for c in range(C)], p,
                              stream)
        return out


# ---- serving form ------------------------------------------------------------

def fsr_server_create(handle, pool_bytes: int, max_inflight: int, streams: int,
                      params: fsr_params) -> int:
    srv = ctypes.c_void_p()
    cfg = fsr_server_config(int(pool_bytes), int(max_inflight), int(streams))
    _check(load_library().fsr_server_create(handle, ctypes.byref(cfg), ctypes.byref(params),
                                            ctypes.byref(srv)), handle)
    return srv.value


def fsr_server_submit(server, img_ptr: int, mask_ptr: int, height: int, width: int, iters: int,
                      out_ptr: int, handle=None) -> int:
    t = ctypes.c_longlong()
    _check(load_library().fsr_server_submit(server, img_ptr, mask_ptr, int(height), int(width),
                                            int(iters), out_ptr, ctypes.byref(t)), handle)
    return t.value


def fsr_server_poll(server, max_items: int = 256, wait_ms: int = 0):
    tk = (ctypes.c_longlong * max_items)()
    lat = (ctypes.c_double * max_items)()
    n = ctypes.c_int()
    _check(load_library().fsr_server_poll(server, tk, lat, int(max_items), ctypes.byref(n),
                                          int(wait_ms)), None)
    return [(tk[i], lat[i]) for i in range(n.value)]


def fsr_server_stats(server) -> dict:
    sub, com, lau = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    q, inf = ctypes.c_int(), ctypes.c_int()
    peak = ctypes.c_size_t()
    _check(load_library().fsr_server_stats(server, ctypes.byref(sub), ctypes.byref(com),
                                           ctypes.byref(q), ctypes.byref(inf), ctypes.byref(lau),
                                           ctypes.byref(peak)), None)
    return dict(submitted=sub.value, completed=com.value, queued=q.value, inflight=inf.value,
                launches=lau.value, peak_pool_bytes=peak.value)


def fsr_server_destroy(server) -> None:
    load_library().fsr_server_destroy(server)


class Server:
    """Owning wrapper of an ``fsr_server``.  Requests take host tensors
    (float32 image, uint8 mask; pinned for overlapped copies); the wrapper
    keeps them alive until the request completes and returns its output."""

    def __init__(self, handle: "Handle", pool_bytes: int, max_inflight: int = 64, streams: int = 2,
                 **params):
        self.handle = handle
        self.ptr = fsr_server_create(handle.ptr, pool_bytes, max_inflight, streams,
                                     make_params(**params))
        self.live = {}

    def submit(self, img, mask, iters: int, out=None) -> int:
        import torch
        if out is None:
            out = torch.empty(img.shape, dtype=torch.float32, pin_memory=img.is_pinned())
        for t in (img, mask, out):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("server requests take contiguous host tensors")
        if img.dtype != torch.float32 or mask.dtype != torch.uint8 or out.dtype != torch.float32:
            raise ValueError("img/out float32, mask uint8")
        H, W = img.shape
        t = fsr_server_submit(self.ptr, img.data_ptr(), mask.data_ptr(), H, W, iters, out.data_ptr(),
                              self.handle.ptr)
        self.live[t] = (img, mask, out)
        return t

    def poll(self, wait_ms: int = 0):
        """[(ticket, latency_ms, output tensor)] of the requests completed since the last poll."""
        res = []
        for t, lat in fsr_server_poll(self.ptr, 1024, wait_ms):
            img, mask, out = self.live.pop(t)
            res.append((t, lat, out))
        return res

    def stats(self) -> dict:
        return fsr_server_stats(self.ptr)

    def close(self):
        if self.ptr:
            fsr_server_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
