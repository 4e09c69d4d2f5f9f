"""CPU oracle for the sensor-rendering path (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package; the product path never does.  The rasteriser itself
is plain C in ``hsr_oracle.c`` (rules stated in its header); this module only
compiles it with gcc on first use and marshals numpy arrays.

Floating point: every value that decides an integer result (snapped vertex,
coverage, the depth test) is computed in float32 with a fixed operation order,
the precision the CUDA kernels use, so triangle ids and coverage are exact.
Shading (perspective-correct weights, bilinear filtering) is done in float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

OK, ERR_ARG, ERR_OOM, ERR_RANGE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle (no fast-math, no FMA contraction: it must stay exact)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.oracle_camera.argtypes = [P, P]
        _lib.oracle_camera.restype = ctypes.c_int
        _lib.oracle_render.argtypes = [P, ctypes.c_uint32, P, ctypes.c_uint32, P, P, P, ctypes.c_uint32,
                                       ctypes.c_uint32, P, P, ctypes.c_uint32, P, ctypes.c_uint32,
                                       ctypes.c_uint32, P, P, P, P, ctypes.c_int]
        _lib.oracle_render.restype = ctypes.c_int
        _lib.oracle_render_noisy.argtypes = _lib.oracle_render.argtypes + [ctypes.c_float, ctypes.c_uint64, P]
        _lib.oracle_render_noisy.restype = ctypes.c_int
        _lib.oracle_render_full.argtypes = _lib.oracle_render_noisy.argtypes + [ctypes.c_int, P]
        _lib.oracle_render_full.restype = ctypes.c_int
        _lib.oracle_philox4x32_10.argtypes = [P, P, P]
        _lib.oracle_philox4x32_10.restype = None
        _lib.oracle_actuate.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_float,
                                        ctypes.c_float, ctypes.c_float, ctypes.c_uint32, ctypes.c_uint32, P, P]
        _lib.oracle_actuate.restype = ctypes.c_int
        _lib.oracle_guard_clip.argtypes = [P, ctypes.c_int, ctypes.c_float, ctypes.c_float, P]
        _lib.oracle_guard_clip.restype = ctypes.c_int
    return _lib


def guard_clip(poly, gx: float, gy: float) -> np.ndarray:
    """The rasteriser's guard-band clip of one polygon ([n <= 4, 3] rows of
    (x_e, y_e, d)) against |x_e| <= gx d, |y_e| <= gy d; returns [m, 3]."""
    v = np.ascontiguousarray(poly, dtype=np.float32).reshape(-1, 3)
    out = np.zeros((8, 3), dtype=np.float32)
    m = lib().oracle_guard_clip(_ptr(v), v.shape[0], float(gx), float(gy), _ptr(out))
    if m < 0:
        raise ValueError("a polygon of at most 4 vertices")
    return out[:m].copy()


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox-4x32-10 block (Salmon et al. 2011) of a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(2)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


STOP, MOVE_FORWARD, TURN_LEFT, TURN_RIGHT = 0, 1, 2, 3


def actuate(pose, action: int, navmap, step: float = 0.25, turn_deg: float = 10.0):
    """Pose after one action (Sec. 4 action space) on a navigability grid.

    navmap: (x0, z0, cell, grid [nz, nx] uint8).  Returns (new pose [7]
    float32, moved: bool)."""
    p = np.ascontiguousarray(pose, dtype=np.float32).reshape(7)
    x0, z0, cell, grid = navmap
    g = np.ascontiguousarray(grid, dtype=np.uint8)
    out = np.zeros(7, dtype=np.float32)
    st = lib().oracle_actuate(_ptr(p), int(action), float(step), float(turn_deg), float(x0), float(z0),
                              float(cell), g.shape[1], g.shape[0], _ptr(g), _ptr(out))
    if st < 0 or st > 1:
        raise ValueError("unknown action")
    return out, bool(st)


def camera(pose) -> np.ndarray:
    """World-to-eye 3x4 float32 matrix of a pose (x, y, z, qw, qx, qy, qz)."""
    p = np.ascontiguousarray(pose, dtype=np.float32).reshape(7)
    M = np.zeros(12, dtype=np.float32)
    st = lib().oracle_camera(_ptr(p), _ptr(M))
    if st != OK:
        raise ValueError("pose quaternion is not unit length")
    return M.reshape(3, 4)


def render(scene, poses, intr, width: int, height: int, nthreads: int = 0,
           ids: bool = True, coverage: bool = False, noise_sigma: float = 0.0, noise_seed: int = 0,
           agent_ids=None, trilinear: bool = False, lod: bool = False) -> dict:
    """Render every pose of `poses` ([N,7]) and return numpy outputs.

    `scene` has attributes xyz, idx, uv, vrgb, atlas, sem (see workloads.Scene);
    `intr` is (fx, fy, cx, cy, znear, zfar).  Returns rgb [N,H,W,3] u8,
    depth [N,H,W] f32, ids [N,H,W] u32 and, if asked, cover [N,H,W] u32, the
    number of fragments that passed the coverage test at each pixel, and lod
    [N,H,W] f32, the mip level-of-detail lambda of each textured pixel (NaN
    elsewhere; trilinear sampling only).
    """
    xyz = np.ascontiguousarray(scene.xyz, dtype=np.float32)
    idx = np.ascontiguousarray(scene.idx, dtype=np.uint32)
    uv = None if scene.uv is None else np.ascontiguousarray(scene.uv, dtype=np.float32)
    vrgb = None if scene.vrgb is None else np.ascontiguousarray(scene.vrgb, dtype=np.uint8)
    atlas = None if scene.atlas is None else np.ascontiguousarray(scene.atlas, dtype=np.uint8)
    sem = None if scene.sem is None else np.ascontiguousarray(scene.sem, dtype=np.uint32)
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    intr = np.ascontiguousarray(getattr(intr, "as_array", lambda: intr)(), dtype=np.float32).reshape(6)
    n = poses.shape[0]
    rgb = np.zeros((n, height, width, 3), dtype=np.uint8)
    depth = np.zeros((n, height, width), dtype=np.float32)
    out_ids = np.zeros((n, height, width), dtype=np.uint32) if ids else None
    cover = np.zeros((n, height, width), dtype=np.uint32) if coverage else None
    aw = ah = 0
    if atlas is not None:
        ah, aw = atlas.shape[0], atlas.shape[1]
    agents = None if agent_ids is None else np.ascontiguousarray(agent_ids, dtype=np.uint32).reshape(n)
    out_lod = np.full((n, height, width), np.nan, dtype=np.float32) if lod else None
    st = lib().oracle_render_full(_ptr(xyz), xyz.shape[0], _ptr(idx), idx.shape[0], _ptr(uv), _ptr(vrgb),
                                  _ptr(atlas), aw, ah, _ptr(sem), _ptr(poses), n, _ptr(intr), width, height,
                                  _ptr(rgb), _ptr(depth), _ptr(out_ids), _ptr(cover), int(nthreads),
                                  float(noise_sigma), int(noise_seed) & ((1 << 64) - 1), _ptr(agents),
                                  1 if trilinear else 0, _ptr(out_lod))
    if st != OK:
        raise ValueError(f"oracle_render failed with status {st}")
    out = {"rgb": rgb, "depth": depth}
    if ids:
        out["ids"] = out_ids
    if coverage:
        out["cover"] = cover
    if lod:
        out["lod"] = out_lod
    return out
