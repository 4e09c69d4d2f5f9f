"""Autotuning cache: launch configurations per GPU and workload signature.

The tuning itself runs in the library (hsr_autotune: candidate configurations
timed with CUDA events, coordinate descent). This module only stores and
reloads its results as JSON files under ``$HSR_TUNING_DIR`` (default: the
package's ``tuning/`` directory), one per (GPU name, workload signature), so
that a second process skips the search.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Optional, Sequence

from . import hsr


def cache_dir() -> str:
    return os.environ.get("HSR_TUNING_DIR", os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning"))


def signature(scenes: Sequence, n: int, width: int, height: int, with_ids: bool) -> str:
    parts = [f"{s.n_tris}:{s.n_verts}:{0 if s.atlas is None else s.atlas.shape[0]}" for s in scenes]
    key = "|".join(parts) + f"|n{n}|{width}x{height}|ids{int(bool(with_ids))}"
    return hashlib.sha1(key.encode()).hexdigest()[:16]


def _path(gpu: str, sig: str) -> str:
    safe = "".join(ch if ch.isalnum() else "_" for ch in gpu)
    return os.path.join(cache_dir(), safe, sig + ".json")


def ensure_tuned(scenes: Sequence, handles: Sequence, scene_of_agent, poses, intr, width: int, height: int,
                 out: dict, stream=None, gpu: Optional[str] = None, use_cache: bool = True, reps: int = 3):
    """Load the tuned configuration of this workload, or tune and store it.

    `scenes` are workloads.Scene objects (for the signature), `handles` the
    loaded hsr.SceneHandle objects. Returns (config dict, source) where source
    is "cache" or "tuned"."""
    import torch
    gpu = gpu or torch.cuda.get_device_name()
    n = len(poses)
    with_ids = out.get("ids") is not None
    sig = signature(scenes, n, width, height, with_ids)
    path = _path(gpu, sig)
    hs = [h.handle for h in handles]
    if use_cache and os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        hsr.hsr_set_tuned_config(hs, n, width, height, with_ids, hsr.hsr_config.from_dict(d["config"]))
        return d["config"], "cache"
    cfg, ms = hsr.hsr_autotune(hs, scene_of_agent if len(hs) > 1 else None, poses, intr, width, height,
                               out["rgb"], out["depth"], out.get("ids"), stream, reps)
    d = {"gpu": gpu, "signature": sig, "config": cfg.as_dict(), "ms": ms}
    if use_cache:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1)
        os.replace(tmp, path)
    return d["config"], "tuned"
