"""The C-ABI library loads and exports every declared entry point (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2202_13926_gb300 import build as B
from paper_2202_13926_gb300 import fsr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fsr_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return fsr.load_library()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert declared, "no declarations found in include/"
    assert declared == set(fsr.EXPORTED)
    so = ctypes.CDLL(B.LIB)
    for name in declared:
        assert hasattr(so, name), name


def test_num_blocks(lib):
    assert fsr.fsr_num_blocks(1080, 1920, 4) == 270 * 480
    assert fsr.fsr_num_blocks(128, 128, 4) == 1024
    assert fsr.fsr_num_blocks(37, 53, 4) == 10 * 14
    assert fsr.fsr_num_blocks(0, 5, 4) == 0
    assert fsr.fsr_num_blocks(5, 5, 0) == 0


def test_null_handle_is_rejected_on_host(lib):
    p = fsr.make_params()
    r = lib.fsr_reconstruct(None, 1, 1, 8, 8, 8, ctypes.byref(p), 1, None)
    assert r == fsr.FSR_ERR_INVALID_ARG
    assert "handle" in lib.fsr_last_error(None).decode()


def test_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.fsr_create(None, ctypes.byref(h)) == fsr.FSR_ERR_INVALID_ARG
    assert h.value is None
    assert lib.fsr_create(ctypes.byref(fsr.fsr_config(0, 0)), None) == fsr.FSR_ERR_INVALID_ARG


def test_destroy_null_is_noop(lib):
    assert lib.fsr_destroy(None) == fsr.FSR_OK


def test_status_entry_points_reject_null_handle(lib):
    assert lib.fsr_check_status(None, None) == fsr.FSR_ERR_INVALID_ARG
    assert lib.fsr_inject_tile_wait_fault(None) == fsr.FSR_ERR_INVALID_ARG
    c = ctypes.c_longlong()
    assert lib.fsr_empty_blocks(None, None, ctypes.byref(c)) == fsr.FSR_ERR_INVALID_ARG


def test_static_batch_rejects_bad_parameters_before_any_device_work(lib):
    """The allocation-free batch entry point validates its parameters on the
    host first: these calls return their codes without touching a GPU."""
    d = (fsr.fsr_image_desc * 1)(fsr.fsr_image_desc(1, 1, 1, 8, 8, 8, 10, None))
    buf = ctypes.create_string_buffer(256)
    cases = [(fsr.make_params(update="conj_pair"), fsr.FSR_ERR_UNSUPPORTED),
             (fsr.make_params(block=4, border=6), fsr.FSR_ERR_UNSUPPORTED),
             (fsr.make_params(precision="tc_bf16x3"), fsr.FSR_ERR_UNSUPPORTED),
             (fsr.make_params(rho=0.0), fsr.FSR_ERR_INVALID_ARG)]
    for p, code in cases:
        got = lib.fsr_reconstruct_batch_static(1, d, ctypes.byref(p), None, buf, len(buf))
        assert got == code, (got, buf.value)
        assert buf.value
    assert lib.fsr_reconstruct_batch_static(0, d, ctypes.byref(fsr.make_params()), None, buf,
                                            len(buf)) == fsr.FSR_ERR_INVALID_ARG


def test_binding_geometry_ignores_strides_of_size_one_dimensions():
    """The row pitch the binding passes is the image's; a dimension of size
    1 has an arbitrary stride in torch and must not be compared."""
    torch = pytest.importorskip("torch")
    from paper_2202_13926_gb300 import fsr
    one = torch.zeros((1, 1), dtype=torch.float32)
    odd = torch.zeros((2, 2), dtype=torch.float32)[:1, :1]   # stride (2, 1)
    m = torch.zeros((1, 1), dtype=torch.uint8)
    assert fsr._geometry(one, m, odd) == (1, 1, 1)
    row = torch.zeros((1, 7), dtype=torch.float32)
    assert fsr._geometry(row, torch.zeros((1, 7), dtype=torch.uint8), torch.zeros((3, 7))[:1]) == (1, 7, 7)
    img = torch.zeros((4, 5), dtype=torch.float32)
    with pytest.raises(ValueError):
        fsr._geometry(img, torch.zeros((4, 5), dtype=torch.uint8), torch.zeros((4, 6))[:, :5])
