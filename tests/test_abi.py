"""The C-ABI library loads, exports every symbol include/hsr.h declares, and
rejects bad arguments before touching a device (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hsr():
    from paper_1904_01201_b300 import build
    build.build()
    from paper_1904_01201_b300 import hsr as mod
    return mod


def declared_symbols():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if path.endswith(".h"):
            text = open(os.path.join(ROOT, "include", path)).read()
            names += re.findall(r"^HSR_API\s+[\w\s\*]*?\b(hsr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_api():
    names = declared_symbols()
    for n in ("hsr_scene_load", "hsr_scene_free", "hsr_render", "hsr_render_batch", "hsr_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(hsr):
    lib = ctypes.CDLL(hsr.LIB_PATH)
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_status_strings(hsr):
    assert hsr.hsr_status_string(0) == "ok"
    assert "invalid" in hsr.hsr_status_string(1)
    assert hsr.hsr_status_string(99) == "unknown status"
    assert re.match(r"^\d+\.\d+\.\d+$", hsr.hsr_version())


def test_invalid_arguments_rejected_on_host(hsr):
    lib = hsr.library()
    out = ctypes.c_void_p()
    assert lib.hsr_scene_load(None, 0, None, 0, None, None, None, 0, 0, None, ctypes.byref(out)) == 1
    xyz = np.zeros((3, 3), np.float32)
    bad_idx = np.array([[0, 1, 3]], np.uint32)
    st = lib.hsr_scene_load(xyz.ctypes.data, 3, bad_idx.ctypes.data, 1, None, None, None, 0, 0, None, ctypes.byref(out))
    assert st == hsr.HSR_ERR_INVALID_ARG
    nan_xyz = xyz.copy()
    nan_xyz[1, 1] = np.nan
    idx = np.array([[0, 1, 2]], np.uint32)
    st = lib.hsr_scene_load(nan_xyz.ctypes.data, 3, idx.ctypes.data, 1, None, None, None, 0, 0, None, ctypes.byref(out))
    assert st == hsr.HSR_ERR_INVALID_ARG
    sem = np.array([0xFFFFFFFF], np.uint32)
    st = lib.hsr_scene_load(xyz.ctypes.data, 3, idx.ctypes.data, 1, None, None, None, 0, 0, sem.ctypes.data,
                            ctypes.byref(out))
    assert st == hsr.HSR_ERR_INVALID_ARG
    intr = hsr.hsr_intrinsics(32, 32, 32, 32, 0.01, 10)
    poses = np.array([[0, 0, 0, 1, 0, 0, 0]], np.float32)
    assert lib.hsr_render(None, poses.ctypes.data, 1, ctypes.byref(intr), 64, 64, None, None, None, None) == 1
    assert lib.hsr_scene_free(None) == 0


def test_scene_load_without_device_reports_no_device(hsr):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    xyz = np.array([[0, 0, -1], [1, 0, -1], [0, 1, -1]], np.float32)
    idx = np.array([[0, 1, 2]], np.uint32)
    with pytest.raises(hsr.HsrError) as e:
        hsr.hsr_scene_load(xyz, idx)
    assert e.value.status == hsr.HSR_ERR_NO_DEVICE
