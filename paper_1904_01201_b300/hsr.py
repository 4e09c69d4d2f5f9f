"""Python binding of the hsr C-ABI (include/hsr.h): argument marshalling only.

Every step of rendering runs in the CUDA library ``_lib/libhsr.so``; this
module only converts numpy / torch arguments to pointers. There is no
fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhsr.so")

HSR_OK = 0
HSR_ERR_INVALID_ARG = 1
HSR_ERR_OOM = 2
HSR_ERR_CUDA = 3
HSR_ERR_TIMEOUT = 4
HSR_ERR_OVERFLOW = 5
HSR_ERR_NO_DEVICE = 6
BACKGROUND_ID = 0xFFFFFFFF


class hsr_pose(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_float * 3), ("quat", ctypes.c_float * 4)]


class hsr_intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("zfar", ctypes.c_float)]


class hsr_scene_info(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_uint32), ("n_verts", ctypes.c_uint32), ("n_meshlets", ctypes.c_uint32),
                ("n_groups", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64),
                ("aabb_min", ctypes.c_float * 3), ("aabb_max", ctypes.c_float * 3)]


class hsr_config(ctypes.Structure):
    _fields_ = [("small_px", ctypes.c_uint32), ("bin_px", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("n_phases", ctypes.c_uint32), ("phase_r", ctypes.c_float * 2)]

    def as_dict(self):
        return {"small_px": self.small_px, "bin_px": self.bin_px, "chunk": self.chunk,
                "ctas_per_sm": self.ctas_per_sm, "n_phases": self.n_phases, "phase_r": list(self.phase_r)}

    @classmethod
    def from_dict(cls, d):
        return cls(d["small_px"], d["bin_px"], d["chunk"], d["ctas_per_sm"], d["n_phases"],
                   (ctypes.c_float * 2)(*d["phase_r"]))


class hsr_depth_noise(ctypes.Structure):
    _fields_ = [("depth_sigma", ctypes.c_float), ("reserved", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("agent_ids", ctypes.c_void_p)]


class hsr_view(ctypes.Structure):
    _fields_ = [("pose", hsr_pose), ("scene", ctypes.c_uint32), ("frame", ctypes.c_uint32),
                ("outputs", ctypes.c_uint32)]


HSR_OUT_RGB, HSR_OUT_DEPTH, HSR_OUT_IDS = 1, 2, 4
HSR_SAMPLE_BILINEAR, HSR_SAMPLE_TRILINEAR = 0, 1
VIEW_DTYPE = np.dtype([("pose", np.float32, 7), ("scene", np.uint32), ("frame", np.uint32), ("outputs", np.uint32)])


class hsr_navmap(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_float), ("z0", ctypes.c_float), ("cell", ctypes.c_float), ("nx", ctypes.c_uint32),
                ("nz", ctypes.c_uint32), ("grid", ctypes.c_void_p)]


class hsr_actuation(ctypes.Structure):
    _fields_ = [("forward_m", ctypes.c_float), ("turn_deg", ctypes.c_float)]


HSR_ACTION_STOP, HSR_ACTION_MOVE_FORWARD, HSR_ACTION_TURN_LEFT, HSR_ACTION_TURN_RIGHT = 0, 1, 2, 3


class hsr_server_config(ctypes.Structure):
    _fields_ = [("n_res", ctypes.c_uint32), ("res", ctypes.c_uint32 * 8), ("res_weight", ctypes.c_float * 8),
                ("fb_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32), ("n_streams", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("max_wait_us", ctypes.c_uint32), ("znear", ctypes.c_float),
                ("zfar", ctypes.c_float), ("with_ids", ctypes.c_int)]


class hsr_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("res", ctypes.c_uint32),
                ("slot", ctypes.c_uint32), ("rgb", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("ids", ctypes.c_void_p), ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class hsr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("queued", ctypes.c_uint32), ("in_flight", ctypes.c_uint32),
                ("fb_bytes_used", ctypes.c_uint64), ("fb_bytes_total", ctypes.c_uint64)]


# hsr_request as a numpy record (tag, scene, res, pose[7]), 48 bytes
REQUEST_DTYPE = np.dtype([("tag", np.uint64), ("scene", np.uint32), ("res", np.uint32), ("pose", np.float32, 7),
                          ("agent", np.int32), ("action", np.uint32)], align=True)
assert REQUEST_DTYPE.itemsize == 56


class HsrError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {hsr_status_string(status)} ({status})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"hsr CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P, U32 = ctypes.c_void_p, ctypes.c_uint32
    sig = {
        "hsr_scene_load": ([P, U32, P, U32, P, P, P, U32, U32, P, ctypes.POINTER(P)], ctypes.c_int),
        "hsr_scene_free": ([P], ctypes.c_int),
        "hsr_scene_get_info": ([P, ctypes.POINTER(hsr_scene_info)], ctypes.c_int),
        "hsr_render": ([P, P, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P, P], ctypes.c_int),
        "hsr_render_batch": ([P, U32, P, P, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P, P],
                             ctypes.c_int),
        "hsr_render_noalloc": ([P, P, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P, P], ctypes.c_int),
        "hsr_set_stage_timing": ([ctypes.c_int], ctypes.c_int),
        "hsr_get_stage_timing": ([P], ctypes.c_int),
        "hsr_set_stage_stats": ([ctypes.c_int], ctypes.c_int),
        "hsr_get_stage_stats": ([P], ctypes.c_int),
        "hsr_config_default": ([ctypes.POINTER(hsr_config)], ctypes.c_int),
        "hsr_autotune": ([P, U32, P, P, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P, P, U32,
                          ctypes.POINTER(hsr_config), ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "hsr_set_tuned_config": ([P, U32, U32, U32, U32, ctypes.c_int, ctypes.POINTER(hsr_config)], ctypes.c_int),
        "hsr_batch_create": ([P, U32, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P,
                              ctypes.POINTER(hsr_config), ctypes.POINTER(P)], ctypes.c_int),
        "hsr_batch_render": ([P, P, P, U32, P, P], ctypes.c_int),
        "hsr_batch_destroy": ([P], ctypes.c_int),
        "hsr_scene_set_sampling": ([P, ctypes.c_int], ctypes.c_int),
        "hsr_device_status": ([ctypes.c_int], ctypes.c_int),
        "hsr_debug_inject_wait_fault": ([U32], ctypes.c_int),
        "hsr_render_views": ([P, U32, P, U32, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P,
                              ctypes.POINTER(hsr_depth_noise), P], ctypes.c_int),
        "hsr_batch_render_views": ([P, P, U32, ctypes.POINTER(hsr_depth_noise), P], ctypes.c_int),
        "hsr_agents_create": ([P, U32, P, U32, P, P, ctypes.POINTER(hsr_actuation), ctypes.POINTER(P)],
                              ctypes.c_int),
        "hsr_agents_get_poses": ([P, P, P], ctypes.c_int),
        "hsr_agents_set_poses": ([P, P, P, U32, P], ctypes.c_int),
        "hsr_agents_destroy": ([P], ctypes.c_int),
        "hsr_batch_step": ([P, P, P, P, U32, P, ctypes.POINTER(hsr_depth_noise), P], ctypes.c_int),
        "hsr_render_noisy": ([P, U32, P, P, U32, ctypes.POINTER(hsr_intrinsics), U32, U32, P, P, P,
                              ctypes.POINTER(hsr_depth_noise), P], ctypes.c_int),
        "hsr_batch_render_noisy": ([P, P, P, U32, P, ctypes.POINTER(hsr_depth_noise), P], ctypes.c_int),
        "hsr_batch_render_host": ([P, P, P, U32, P, P, P, P, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "hsr_server_create": ([P, U32, ctypes.POINTER(hsr_server_config), ctypes.POINTER(P)], ctypes.c_int),
        "hsr_server_submit": ([P, P, U32], ctypes.c_int),
        "hsr_server_attach_agents": ([P, P], ctypes.c_int),
        "hsr_server_poll": ([P, P, U32, ctypes.POINTER(U32), U32], ctypes.c_int),
        "hsr_server_release": ([P, P, U32], ctypes.c_int),
        "hsr_server_get_stats": ([P, ctypes.POINTER(hsr_server_stats)], ctypes.c_int),
        "hsr_server_now": ([], ctypes.c_double),
        "hsr_server_destroy": ([P], ctypes.c_int),
        "hsr_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "hsr_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def library():
    return _lib


# -------------------------------------------------------------- raw C-ABI names
def hsr_status_string(status: int) -> str:
    return _lib.hsr_status_string(int(status)).decode()


def hsr_set_stage_timing(enable: bool) -> None:
    st = _lib.hsr_set_stage_timing(1 if enable else 0)
    if st != HSR_OK:
        raise HsrError(st, "hsr_set_stage_timing")


def hsr_get_stage_timing():
    """Stage durations (ms) of the last timed render call: cull, raster, shade, total."""
    ms = np.zeros(4, dtype=np.float32)
    st = _lib.hsr_get_stage_timing(_np_ptr(ms))
    if st != HSR_OK:
        raise HsrError(st, "hsr_get_stage_timing")
    return {"cull": float(ms[0]), "raster": float(ms[1]), "shade": float(ms[2]), "total": float(ms[3])}


def hsr_set_stage_stats(enable: bool) -> None:
    st = _lib.hsr_set_stage_stats(1 if enable else 0)
    if st != HSR_OK:
        raise HsrError(st, "hsr_set_stage_stats")


def hsr_get_stage_stats():
    """Work counters of the last render call: pairs and skipped meshlets per occlusion phase."""
    c = np.zeros(9, dtype=np.uint32)
    st = _lib.hsr_get_stage_stats(_np_ptr(c))
    if st != HSR_OK:
        raise HsrError(st, "hsr_get_stage_stats")
    return {"pairs": [int(v) for v in c[:3]], "skipped": [int(v) for v in c[3:6]],
            "frustum_meshlets": int(c[6]), "backfacing_kept": int(c[7]), "backfacing_culled": int(c[8])}


def hsr_device_status(clear: bool = True) -> int:
    """HSR_ERR_TIMEOUT if a kernel's bounded wait expired since the last clear, else HSR_OK."""
    return _lib.hsr_device_status(1 if clear else 0)


def hsr_debug_inject_wait_fault(extra_bytes: int) -> None:
    """Test hook: later renders wait for bytes that never arrive (0 restores normal operation)."""
    _lib.hsr_debug_inject_wait_fault(int(extra_bytes))


def hsr_version() -> str:
    return _lib.hsr_version().decode()


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def as_intrinsics(intr) -> hsr_intrinsics:
    if isinstance(intr, hsr_intrinsics):
        return intr
    a = np.asarray(getattr(intr, "as_array", lambda: intr)(), dtype=np.float32).reshape(6)
    return hsr_intrinsics(*[float(v) for v in a])


def hsr_scene_load(xyz, idx, uv=None, vert_rgb=None, atlas=None, tri_semantic=None):
    """Load a scene from host arrays; returns an opaque handle (int)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    idx = np.ascontiguousarray(idx, dtype=np.uint32).reshape(-1, 3)
    uv = None if uv is None else np.ascontiguousarray(uv, dtype=np.float32).reshape(-1, 2)
    vert_rgb = None if vert_rgb is None else np.ascontiguousarray(vert_rgb, dtype=np.uint8).reshape(-1, 3)
    aw = ah = 0
    if atlas is not None:
        atlas = np.ascontiguousarray(atlas, dtype=np.uint8)
        ah, aw = atlas.shape[0], atlas.shape[1]
    sem = None if tri_semantic is None else np.ascontiguousarray(tri_semantic, dtype=np.uint32).reshape(-1)
    out = ctypes.c_void_p()
    st = _lib.hsr_scene_load(_np_ptr(xyz), xyz.shape[0], _np_ptr(idx), idx.shape[0], _np_ptr(uv), _np_ptr(vert_rgb),
                             _np_ptr(atlas), aw, ah, _np_ptr(sem), ctypes.byref(out))
    if st != HSR_OK:
        raise HsrError(st, "hsr_scene_load")
    return out.value


def hsr_scene_free(handle) -> None:
    _lib.hsr_scene_free(ctypes.c_void_p(handle))


def hsr_scene_get_info(handle) -> hsr_scene_info:
    info = hsr_scene_info()
    st = _lib.hsr_scene_get_info(ctypes.c_void_p(handle), ctypes.byref(info))
    if st != HSR_OK:
        raise HsrError(st, "hsr_scene_get_info")
    return info


def hsr_render(handle, poses, intr, width, height, rgb, depth, ids=None, stream=None) -> int:
    """Raw render call; outputs are device tensors (or device pointers). Returns the status."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    ci = as_intrinsics(intr)
    return _lib.hsr_render(ctypes.c_void_p(handle), _np_ptr(poses), poses.shape[0], ctypes.byref(ci), int(width),
                           int(height), _dev_ptr(rgb), _dev_ptr(depth), _dev_ptr(ids), _stream_ptr(stream))


def hsr_render_noalloc(handle, poses, intr, width, height, rgb, depth, ids=None, stream=None) -> int:
    """Allocation-free variant of hsr_render (fixed device scratch; see include/hsr.h). Returns the status."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    ci = as_intrinsics(intr)
    return _lib.hsr_render_noalloc(ctypes.c_void_p(handle), _np_ptr(poses), poses.shape[0], ctypes.byref(ci),
                                   int(width), int(height), _dev_ptr(rgb), _dev_ptr(depth), _dev_ptr(ids),
                                   _stream_ptr(stream))


def hsr_render_batch(handles: Sequence[int], scene_of_agent, poses, intr, width, height, rgb, depth, ids=None,
                     stream=None) -> int:
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    arr = (ctypes.c_void_p * len(handles))(*handles)
    soa = np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
    ci = as_intrinsics(intr)
    return _lib.hsr_render_batch(arr, len(handles), _np_ptr(soa), _np_ptr(poses), poses.shape[0], ctypes.byref(ci),
                                 int(width), int(height), _dev_ptr(rgb), _dev_ptr(depth), _dev_ptr(ids),
                                 _stream_ptr(stream))


def _noise(sigma, seed, agent_ids):
    """(hsr_depth_noise or None, keep-alive array) for the noisy entry points."""
    if sigma is None:
        return None, None
    aid = None if agent_ids is None else np.ascontiguousarray(agent_ids, dtype=np.uint32).reshape(-1)
    nz = hsr_depth_noise(float(sigma), 0, int(seed) & 0xFFFFFFFFFFFFFFFF,
                         None if aid is None else aid.ctypes.data)
    return nz, aid


def hsr_render_noisy(handles: Sequence[int], scene_of_agent, poses, intr, width, height, rgb, depth, ids=None,
                     noise_sigma=None, noise_seed=0, agent_ids=None, stream=None) -> int:
    """hsr_render_batch with inverse-depth Gaussian noise (Appendix C). Returns the status."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    arr = (ctypes.c_void_p * len(handles))(*handles)
    soa = None if scene_of_agent is None else np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
    nz, keep = _noise(noise_sigma, noise_seed, agent_ids)
    st = _lib.hsr_render_noisy(arr, len(handles), _np_ptr(soa), _np_ptr(poses), poses.shape[0],
                               ctypes.byref(as_intrinsics(intr)), int(width), int(height), _dev_ptr(rgb),
                               _dev_ptr(depth), _dev_ptr(ids), None if nz is None else ctypes.byref(nz),
                               _stream_ptr(stream))
    del keep
    return st


def make_views(poses, scene, frames, outputs=0) -> np.ndarray:
    """A view list (VIEW_DTYPE) from poses [N,7] and per-view (or scalar) scene,
    frame and output mask."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    v = np.zeros(poses.shape[0], dtype=VIEW_DTYPE)
    v["pose"] = poses
    v["scene"] = scene
    v["frame"] = frames
    v["outputs"] = outputs
    return v


def hsr_render_views(handles: Sequence[int], views, n_frames, intr, width, height, rgb, depth, ids=None,
                     noise_sigma=None, noise_seed=0, agent_ids=None, stream=None) -> int:
    views = np.ascontiguousarray(views, dtype=VIEW_DTYPE)
    arr = (ctypes.c_void_p * len(handles))(*handles)
    nz, keep = _noise(noise_sigma, noise_seed, agent_ids)
    st = _lib.hsr_render_views(arr, len(handles), _np_ptr(views), len(views), int(n_frames),
                               ctypes.byref(as_intrinsics(intr)), int(width), int(height), _dev_ptr(rgb),
                               _dev_ptr(depth), _dev_ptr(ids), None if nz is None else ctypes.byref(nz),
                               _stream_ptr(stream))
    del keep
    return st


def hsr_batch_render_views(batch, views, noise_sigma=None, noise_seed=0, agent_ids=None, stream=None) -> int:
    views = np.ascontiguousarray(views, dtype=VIEW_DTYPE)
    nz, keep = _noise(noise_sigma, noise_seed, agent_ids)
    st = _lib.hsr_batch_render_views(ctypes.c_void_p(batch), _np_ptr(views), len(views),
                                     None if nz is None else ctypes.byref(nz), _stream_ptr(stream))
    del keep
    return st


def hsr_config_default() -> hsr_config:
    c = hsr_config()
    _lib.hsr_config_default(ctypes.byref(c))
    return c


def hsr_autotune(handles: Sequence[int], scene_of_agent, poses, intr, width, height, rgb, depth, ids=None,
                 stream=None, reps: int = 3):
    """Tune the launch configuration for this workload; returns (hsr_config, ms)."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    arr = (ctypes.c_void_p * len(handles))(*handles)
    soa = None if scene_of_agent is None else np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
    best = hsr_config()
    ms = ctypes.c_float()
    st = _lib.hsr_autotune(arr, len(handles), _np_ptr(soa), _np_ptr(poses), poses.shape[0],
                           ctypes.byref(as_intrinsics(intr)), int(width), int(height), _dev_ptr(rgb), _dev_ptr(depth),
                           _dev_ptr(ids), _stream_ptr(stream), int(reps), ctypes.byref(best), ctypes.byref(ms))
    if st != HSR_OK:
        raise HsrError(st, "hsr_autotune")
    return best, float(ms.value)


def hsr_set_tuned_config(handles: Sequence[int], n, width, height, with_ids, cfg) -> None:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    st = _lib.hsr_set_tuned_config(arr, len(handles), int(n), int(width), int(height), 1 if with_ids else 0,
                                   None if cfg is None else ctypes.byref(cfg))
    if st != HSR_OK:
        raise HsrError(st, "hsr_set_tuned_config")


def hsr_batch_create(handles: Sequence[int], n_cap, intr, width, height, rgb, depth, ids=None, cfg=None) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    out = ctypes.c_void_p()
    st = _lib.hsr_batch_create(arr, len(handles), int(n_cap), ctypes.byref(as_intrinsics(intr)), int(width),
                               int(height), _dev_ptr(rgb), _dev_ptr(depth), _dev_ptr(ids),
                               None if cfg is None else ctypes.byref(cfg), ctypes.byref(out))
    if st != HSR_OK:
        raise HsrError(st, "hsr_batch_create")
    return out.value


def hsr_batch_render(batch, scene_of_agent, poses, frames=None, stream=None) -> int:
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    soa = None if scene_of_agent is None else np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
    fr = None if frames is None else np.ascontiguousarray(frames, dtype=np.uint32).reshape(-1)
    return _lib.hsr_batch_render(ctypes.c_void_p(batch), _np_ptr(soa), _np_ptr(poses), poses.shape[0], _np_ptr(fr),
                                 _stream_ptr(stream))


def hsr_batch_render_noisy(batch, scene_of_agent, poses, frames=None, noise_sigma=None, noise_seed=0,
                           agent_ids=None, stream=None) -> int:
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    soa = None if scene_of_agent is None else np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
    fr = None if frames is None else np.ascontiguousarray(frames, dtype=np.uint32).reshape(-1)
    nz, keep = _noise(noise_sigma, noise_seed, agent_ids)
    st = _lib.hsr_batch_render_noisy(ctypes.c_void_p(batch), _np_ptr(soa), _np_ptr(poses), poses.shape[0],
                                     _np_ptr(fr), None if nz is None else ctypes.byref(nz), _stream_ptr(stream))
    del keep
    return st


def _host_ptr(a, nbytes: int, what: str):
    """Address of a host buffer (numpy array or CPU torch tensor, contiguous)
    of at least nbytes, or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.nbytes < nbytes:
            raise ValueError(f"{what}: needs a contiguous host array of {nbytes} bytes")
        return ctypes.c_void_p(a.ctypes.data)
    if a.is_cuda or not a.is_contiguous() or a.numel() * a.element_size() < nbytes:
        raise ValueError(f"{what}: needs a contiguous host tensor of {nbytes} bytes")
    return ctypes.c_void_p(a.data_ptr())


def hsr_batch_render_host(batch, scene_of_agent, poses, width, height, host_rgb=None, host_depth=None,
                          host_ids=None, stream=None):
    """Render into frames 0..n-1 and copy them to the given host buffers on
    `stream` (asynchronous). Returns (status, bytes uploaded)."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    n = poses.shape[0]
    soa = None if scene_of_agent is None else np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
    px = n * width * height
    h2d = ctypes.c_uint64(0)
    st = _lib.hsr_batch_render_host(ctypes.c_void_p(batch), _np_ptr(soa), _np_ptr(poses), n,
                                    _host_ptr(host_rgb, 3 * px, "host_rgb"), _host_ptr(host_depth, 4 * px, "host_depth"),
                                    _host_ptr(host_ids, 4 * px, "host_ids"), _stream_ptr(stream), ctypes.byref(h2d))
    return st, int(h2d.value)


def hsr_batch_destroy(batch) -> None:
    _lib.hsr_batch_destroy(ctypes.c_void_p(batch))


class Agents:
    """Device-resident agent poses on navigability grids (see hsr_agents_create).

    navmaps: per scene (x0, z0, cell, grid [nz, nx] u8)."""

    def __init__(self, scenes, navmaps, poses, scene_of_agent=None, forward_m=0.25, turn_deg=10.0):
        self.scenes = list(scenes)
        poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
        self.n = poses.shape[0]
        grids = [np.ascontiguousarray(g, dtype=np.uint8) for (_, _, _, g) in navmaps]
        maps = (hsr_navmap * len(grids))(*[hsr_navmap(float(x0), float(z0), float(c), g.shape[1], g.shape[0],
                                                      g.ctypes.data)
                                           for (x0, z0, c, _), g in zip(navmaps, grids)])
        arr = (ctypes.c_void_p * len(self.scenes))(*[sc.handle for sc in self.scenes])
        soa = None if scene_of_agent is None else np.ascontiguousarray(scene_of_agent, dtype=np.uint32).reshape(-1)
        act = hsr_actuation(float(forward_m), float(turn_deg))
        out = ctypes.c_void_p()
        st = _lib.hsr_agents_create(arr, len(self.scenes), maps, self.n, _np_ptr(soa), _np_ptr(poses),
                                    ctypes.byref(act), ctypes.byref(out))
        if st != HSR_OK:
            raise HsrError(st, "hsr_agents_create")
        self.handle = out.value

    def poses(self, stream=None) -> np.ndarray:
        out = np.zeros((self.n, 7), dtype=np.float32)
        st = _lib.hsr_agents_get_poses(ctypes.c_void_p(self.handle), _np_ptr(out), _stream_ptr(stream))
        if st != HSR_OK:
            raise HsrError(st, "hsr_agents_get_poses")
        return out

    def set_poses(self, idx, poses, stream=None):
        idx = np.ascontiguousarray(idx, dtype=np.uint32).reshape(-1)
        poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
        st = _lib.hsr_agents_set_poses(ctypes.c_void_p(self.handle), _np_ptr(idx), _np_ptr(poses), idx.shape[0],
                                       _stream_ptr(stream))
        if st != HSR_OK:
            raise HsrError(st, "hsr_agents_set_poses")

    def close(self):
        if getattr(self, "handle", None):
            _lib.hsr_agents_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hsr_batch_step(batch, agents, agent_idx, actions, frames=None, noise_sigma=None, noise_seed=0, agent_ids=None,
                   stream=None) -> int:
    idx = np.ascontiguousarray(agent_idx, dtype=np.uint32).reshape(-1)
    act = np.ascontiguousarray(actions, dtype=np.uint8).reshape(-1)
    if act.shape != idx.shape:
        return HSR_ERR_INVALID_ARG
    fr = None if frames is None else np.ascontiguousarray(frames, dtype=np.uint32).reshape(-1)
    nz, keep = _noise(noise_sigma, noise_seed, agent_ids)
    st = _lib.hsr_batch_step(ctypes.c_void_p(batch), ctypes.c_void_p(agents), _np_ptr(idx), _np_ptr(act),
                             idx.shape[0], _np_ptr(fr), None if nz is None else ctypes.byref(nz),
                             _stream_ptr(stream))
    del keep
    return st


class Batch:
    """A persistent graph-captured render batch bound to output tensors."""

    def __init__(self, scenes, n_cap, intr, width, height, ids=True, cfg=None, device="cuda", depth=True):
        self.scenes = list(scenes)
        self.out = alloc_outputs(n_cap, width, height, ids, device, depth)
        self.handle = hsr_batch_create([s.handle for s in self.scenes], n_cap, intr, width, height,
                                       self.out["rgb"], self.out["depth"], self.out.get("ids"), cfg)

    def render(self, poses, scene_of_agent=None, frames=None, stream=None, noise_sigma=None, noise_seed=0,
               agent_ids=None):
        if noise_sigma is None:
            st = hsr_batch_render(self.handle, scene_of_agent, poses, frames, stream)
        else:
            st = hsr_batch_render_noisy(self.handle, scene_of_agent, poses, frames, noise_sigma, noise_seed,
                                        agent_ids, stream)
        if st != HSR_OK:
            raise HsrError(st, "hsr_batch_render")
        return self.out

    def render_host(self, poses, host, scene_of_agent=None, stream=None) -> int:
        """Render into frames 0..n-1 and copy their outputs to host buffers
        (dict with any of "rgb", "depth", "ids": page-locked CPU tensors) on
        `stream`; the host buffers are complete once the stream has passed the
        copies. Returns the bytes uploaded (view descriptors)."""
        W, H = self.out["rgb"].shape[2], self.out["rgb"].shape[1]
        st, h2d = hsr_batch_render_host(self.handle, scene_of_agent, poses, W, H, host.get("rgb"),
                                        host.get("depth"), host.get("ids"), stream)
        if st != HSR_OK:
            raise HsrError(st, "hsr_batch_render_host")
        return h2d

    def step(self, agents: "Agents", agent_idx, actions, frames=None, stream=None, noise_sigma=None, noise_seed=0,
             agent_ids=None):
        """Apply one action per listed agent on the device, then render them."""
        st = hsr_batch_step(self.handle, agents.handle, agent_idx, actions, frames, noise_sigma, noise_seed,
                            agent_ids, stream)
        if st != HSR_OK:
            raise HsrError(st, "hsr_batch_step")
        return self.out

    def close(self):
        if self.handle:
            hsr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------- conveniences
class SceneHandle:
    """Owns a loaded scene; frees it on close() or garbage collection."""

    def __init__(self, scene):
        self.handle = hsr_scene_load(scene.xyz, scene.idx, scene.uv, scene.vrgb, scene.atlas, scene.sem)
        self.info = hsr_scene_get_info(self.handle)

    def set_sampling(self, mode: int) -> None:
        """HSR_SAMPLE_BILINEAR or HSR_SAMPLE_TRILINEAR (mip chain built on first use)."""
        st = _lib.hsr_scene_set_sampling(ctypes.c_void_p(self.handle), int(mode))
        if st != HSR_OK:
            raise HsrError(st, "hsr_scene_set_sampling")

    def close(self):
        if self.handle:
            hsr_scene_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alloc_outputs(n: int, width: int, height: int, ids: bool = True, device="cuda", depth: bool = True):
    import torch
    rgb = torch.empty((n, height, width, 3), dtype=torch.uint8, device=device)
    out = {"rgb": rgb, "depth": None}
    if depth:
        out["depth"] = torch.empty((n, height, width), dtype=torch.float32, device=device)
    if ids:
        out["ids"] = torch.empty((n, height, width), dtype=torch.int32, device=device)
    return out


def render(scene: SceneHandle, poses, intr, width: int, height: int, ids: bool = True, out=None, stream=None,
           noise_sigma=None, noise_seed=0, agent_ids=None):
    """Render poses [N,7] of one scene into (new or given) device tensors;
    noise_sigma adds inverse-depth Gaussian noise to the depth (Appendix C)."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    out = out or alloc_outputs(poses.shape[0], width, height, ids)
    if noise_sigma is None:
        st = hsr_render(scene.handle, poses, intr, width, height, out["rgb"], out["depth"], out.get("ids"), stream)
    else:
        st = hsr_render_noisy([scene.handle], None, poses, intr, width, height, out["rgb"], out["depth"],
                              out.get("ids"), noise_sigma, noise_seed, agent_ids, stream)
    if st != HSR_OK:
        raise HsrError(st, "hsr_render_noisy" if noise_sigma is not None else "hsr_render")
    return out


def render_batch(scenes: Sequence[SceneHandle], scene_of_agent, poses, intr, width: int, height: int,
                 ids: bool = True, out=None, stream=None):
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    out = out or alloc_outputs(poses.shape[0], width, height, ids)
    st = hsr_render_batch([s.handle for s in scenes], scene_of_agent, poses, intr, width, height, out["rgb"],
                          out["depth"], out.get("ids"), stream)
    if st != HSR_OK:
        raise HsrError(st, "hsr_render_batch")
    return out


def render_semantic(scene: SceneHandle, sem_scene: SceneHandle, poses, intr, width: int, height: int, out=None,
                    stream=None):
    """Colour and depth from `scene`, ids from a separate semantic mesh
    `sem_scene`, at the same poses, in one call (two views per frame)."""
    poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 7)
    n = poses.shape[0]
    out = out or alloc_outputs(n, width, height, True)
    f = np.arange(n, dtype=np.uint32)
    views = np.concatenate([make_views(poses, 0, f, HSR_OUT_RGB | HSR_OUT_DEPTH), make_views(poses, 1, f, HSR_OUT_IDS)])
    st = hsr_render_views([scene.handle, sem_scene.handle], views, n, intr, width, height, out["rgb"], out["depth"],
                          out["ids"], stream=stream)
    if st != HSR_OK:
        raise HsrError(st, "hsr_render_views")
    return out


def ids_u32(t):
    """View an int32 id tensor as uint32 numpy."""
    return t.cpu().numpy().view(np.uint32)
