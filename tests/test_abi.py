"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/gks.h declares.  No compute calls."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gks.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gks_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2309_10534_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gks_create", "gks_destroy", "gks_set_gas", "gks_set_scheme", "gks_set_stream",
                 "gks_set_state", "gks_get_state", "gks_compute_dt", "gks_stage", "gks_step",
                 "gks_advance_to", "gks_get_diagnostics", "gks_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gks_status_string.restype = ctypes.c_char_p
    assert lib.gks_status_string(0) == b"ok"
    assert lib.gks_status_string(4) == b"non-physical state"


def test_create_rejects_bad_descriptors_before_touching_the_device(libpath):
    from paper_2309_10534_gb300 import gks
    L = gks.lib()
    d = gks.GridDesc()
    d.dim, d.nx, d.ny = 3, 10, 10  # bad dim
    d.x0, d.x1, d.y0, d.y1 = 0, 1, 0, 1
    h = ctypes.c_void_p()
    assert L.gks_create(ctypes.byref(d), ctypes.byref(h)) == gks.GKS_EINVAL
    d.dim, d.nx = 2, 2  # too few cells
    assert L.gks_create(ctypes.byref(d), ctypes.byref(h)) == gks.GKS_EINVAL
    d.nx = 10
    d.bc[0], d.bc[1] = 0, 1  # periodic on one side only
    assert L.gks_create(ctypes.byref(d), ctypes.byref(h)) == gks.GKS_EINVAL
    assert L.gks_create(None, ctypes.byref(h)) == gks.GKS_EINVAL
    d.bc[0], d.bc[1] = 1, 1
    d.nx, d.ny = 65536, 32769  # above the 2^31-cell limit of 32-bit plane offsets
    assert L.gks_create(ctypes.byref(d), ctypes.byref(h)) == gks.GKS_EINVAL
    d.nx, d.ny = 10, 10
    d.bc[0] = 6  # the wall-after-x0 rule belongs to the y sides
    assert L.gks_create(ctypes.byref(d), ctypes.byref(h)) == gks.GKS_EINVAL


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2309_10534_gb300 import gks
    monkeypatch.setattr(gks, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gks, "_lib", None)
    with pytest.raises(ImportError):
        gks.lib()


def test_noalloc_wrapper_refuses_bad_tensors_before_any_call():
    """step1d_noalloc hands raw device pointers to the library, so every
    tensor that is not a contiguous float64 CUDA tensor of 3 * nx values is
    refused on the host, before the library is called."""
    torch = pytest.importorskip("torch")
    import numpy as np

    from paper_2309_10534_gb300 import gks

    good_shape = (3, 32)
    cases = [
        (torch.ones(good_shape, dtype=torch.float64), torch.ones(good_shape, dtype=torch.float64)),  # CPU
        (np.ones(good_shape), np.ones(good_shape)),                                                   # numpy
        (torch.ones(good_shape, dtype=torch.float32), torch.ones(good_shape, dtype=torch.float32)),  # float32
        (torch.ones((32, 3), dtype=torch.float64).t(), torch.ones(good_shape, dtype=torch.float64)),  # strided
    ]
    for a, b in cases:
        with pytest.raises(gks.GKSError) as e:
            gks.step1d_noalloc(a, b, 1.0 / 32, 1e-4)
        assert e.value.status == gks.GKS_EINVAL
