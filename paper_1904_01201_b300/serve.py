"""Serving front end: a thin wrapper of the hsr_server_* C-ABI and a Poisson
load generator (the core — admission, micro-batching, streams, completion —
is C++ in csrc/serve.cpp).

Workload (the serving configuration): agents step by random walks (Sec. 4
"Agent embodiment and action space": move_forward 0.25 m, turn 10 degrees),
each step submits one render request at a resolution drawn from the mix, and
requests arrive as a Poisson process at a given rate.
"""
from __future__ import annotations

import ctypes
import math
import threading
import time
from typing import Dict, List, Sequence

import numpy as np

from . import hsr
from . import workloads as wl


class Server:
    def __init__(self, scenes: Sequence, res=(64, 128, 256, 512), weights=(0.2, 0.4, 0.3, 0.1),
                 fb_bytes: int = 2 << 30, max_batch: int = 64, n_streams: int = 2, max_queue: int = 1 << 20,
                 max_wait_us: int = 200, znear: float = 0.01, zfar: float = 10.0, with_ids: bool = False):
        self.scenes = list(scenes)
        c = hsr.hsr_server_config()
        c.n_res = len(res)
        for k, (r, w) in enumerate(zip(res, weights)):
            c.res[k] = int(r)
            c.res_weight[k] = float(w)
        c.fb_bytes = int(fb_bytes)
        c.max_batch = int(max_batch)
        c.n_streams = int(n_streams)
        c.max_queue = int(max_queue)
        c.max_wait_us = int(max_wait_us)
        c.znear, c.zfar = float(znear), float(zfar)
        c.with_ids = 1 if with_ids else 0
        self.config = c
        arr = (ctypes.c_void_p * len(self.scenes))(*[s.handle for s in self.scenes])
        out = ctypes.c_void_p()
        st = hsr.library().hsr_server_create(arr, len(self.scenes), ctypes.byref(c), ctypes.byref(out))
        if st != hsr.HSR_OK:
            raise hsr.HsrError(st, "hsr_server_create")
        self.handle = out.value
        self._buf = (hsr.hsr_result * 4096)()

    def attach_agents(self, agents) -> None:
        """Bind the hsr.Agents set that action requests step (None detaches)."""
        st = hsr.library().hsr_server_attach_agents(ctypes.c_void_p(self.handle),
                                                    None if agents is None else ctypes.c_void_p(agents.handle))
        if st != hsr.HSR_OK:
            raise hsr.HsrError(st, "hsr_server_attach_agents")
        self.agents = agents

    def submit(self, requests: np.ndarray) -> None:
        requests = np.ascontiguousarray(requests, dtype=hsr.REQUEST_DTYPE)
        st = hsr.library().hsr_server_submit(ctypes.c_void_p(self.handle), requests.ctypes.data_as(ctypes.c_void_p),
                                             len(requests))
        if st != hsr.HSR_OK:
            raise hsr.HsrError(st, "hsr_server_submit")

    def poll(self, wait_us: int = 1000) -> List[hsr.hsr_result]:
        n = ctypes.c_uint32()
        st = hsr.library().hsr_server_poll(ctypes.c_void_p(self.handle), self._buf, len(self._buf), ctypes.byref(n),
                                           int(wait_us))
        if st != hsr.HSR_OK:
            raise hsr.HsrError(st, "hsr_server_poll")
        return [hsr.hsr_result.from_buffer_copy(self._buf[i]) for i in range(n.value)]

    def release(self, results: Sequence[hsr.hsr_result]) -> None:
        if not results:
            return
        arr = (hsr.hsr_result * len(results))(*results)
        hsr.library().hsr_server_release(ctypes.c_void_p(self.handle), arr, len(results))

    def stats(self) -> Dict[str, int]:
        s = hsr.hsr_server_stats()
        hsr.library().hsr_server_get_stats(ctypes.c_void_p(self.handle), ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in s._fields_}

    @staticmethod
    def now() -> float:
        return hsr.library().hsr_server_now()

    def close(self):
        if self.handle:
            hsr.library().hsr_server_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevArray:
    """A device buffer seen through the CUDA array interface (zero-copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def frame_tensors(r: hsr.hsr_result, with_ids: bool = False):
    """Copies of a result's device frame as torch tensors (take them before release)."""
    import torch
    out = {"rgb": torch.as_tensor(_DevArray(r.rgb, (r.res, r.res, 3), "|u1"), device="cuda").clone(),
           "depth": torch.as_tensor(_DevArray(r.depth, (r.res, r.res), "<f4"), device="cuda").clone()}
    if with_ids and r.ids:
        out["ids"] = torch.as_tensor(_DevArray(r.ids, (r.res, r.res), "<i4"), device="cuda").clone()
    return out


def make_requests(scenes_np: Sequence, n_requests: int, n_agents: int = 1024, res=(64, 128, 256, 512),
                  weights=(0.2, 0.4, 0.3, 0.1), seed: int = 0) -> np.ndarray:
    """Requests of agents stepping random walks over the scenes (agents split
    Dirichlet(0.5) across scenes), resolutions drawn from the mix."""
    split = wl.dirichlet_split(n_agents, len(scenes_np), 0.5, seed)
    walks, owner = [], []
    for si, (sc, k) in enumerate(zip(scenes_np, split)):
        walks.append(wl.RandomWalk(sc, int(k), seed + si))
        owner += [(si, j) for j in range(int(k))]
    rs = wl.Stream(seed, "serving")
    agent = rs.integers(n_requests, 0, n_agents)
    cw = np.cumsum(np.asarray(weights, dtype=np.float64) / sum(weights))
    ri = np.minimum(np.searchsorted(cw, rs.uniform(n_requests), side="right"), len(res) - 1)
    req = np.zeros(n_requests, dtype=hsr.REQUEST_DTYPE)
    req["agent"] = -1
    for i in range(n_requests):
        si, j = owner[int(agent[i])]
        req[i]["tag"] = i
        req[i]["scene"] = si
        req[i]["res"] = res[int(ri[i])]
        req[i]["pose"] = walks[si].step(j)
    return req


def make_agents(scenes_np: Sequence, handles: Sequence, n_agents: int = 1024, seed: int = 0, cell: float = 0.05):
    """Device-resident agents split Dirichlet(0.5) over the scenes, placed on
    navigable cells of each scene's grid; returns (hsr.Agents, scene_of_agent)."""
    split = wl.dirichlet_split(n_agents, len(scenes_np), 0.5, seed)
    navs = [wl.navmap(sc, cell) for sc in scenes_np]
    poses = np.concatenate([wl.navigable_poses(sc, nav, int(k), seed + si)
                            for si, (sc, nav, k) in enumerate(zip(scenes_np, navs, split))])
    soa = np.repeat(np.arange(len(scenes_np), dtype=np.uint32), split)
    return hsr.Agents(handles, navs, poses, scene_of_agent=soa), soa


def make_action_requests(n_requests: int, n_agents: int = 1024, res=(64, 128, 256, 512),
                         weights=(0.2, 0.4, 0.3, 0.1), seed: int = 0) -> np.ndarray:
    """Action requests: each advances one agent (uniform) by move_forward,
    turn_left or turn_right (uniform), at a resolution drawn from the mix."""
    rs = wl.Stream(seed, "serving-actions")
    agent = rs.integers(n_requests, 0, n_agents)
    action = rs.integers(n_requests, hsr.HSR_ACTION_MOVE_FORWARD, hsr.HSR_ACTION_TURN_RIGHT + 1)
    cw = np.cumsum(np.asarray(weights, dtype=np.float64) / sum(weights))
    ri = np.minimum(np.searchsorted(cw, rs.uniform(n_requests), side="right"), len(res) - 1)
    req = np.zeros(n_requests, dtype=hsr.REQUEST_DTYPE)
    req["tag"] = np.arange(n_requests)
    req["res"] = np.asarray(res, dtype=np.uint32)[ri]
    req["agent"] = agent
    req["action"] = action
    return req


def run_load(server: Server, requests: np.ndarray, rate: float, warmup: int = 0, seed: int = 0) -> dict:
    """Submit `requests` as a Poisson process of `rate` requests/s, consume and
    release every result as it completes; latency statistics exclude the
    first `warmup` requests."""
    n = len(requests)
    gaps = -np.log1p(-wl.Stream(seed, "arrivals").uniform(n)) / rate
    arrival = np.cumsum(gaps)
    lat = np.full(n, np.nan)
    status = np.zeros(n, dtype=np.int64)
    done_count = [0]
    finished = threading.Event()

    def consumer():
        while done_count[0] < n:
            res = server.poll(2000)
            for r in res:
                lat[r.tag] = r.t_done - r.t_submit
                status[r.tag] = r.status
            server.release(res)
            done_count[0] += len(res)
        finished.set()

    th = threading.Thread(target=consumer, daemon=True)
    t0 = server.now()
    th.start()
    i = 0
    while i < n:
        now = server.now() - t0
        j = int(np.searchsorted(arrival, now, side="right"))
        if j > i:
            server.submit(requests[i:j])
            i = j
        else:
            time.sleep(min(2e-4, max(0.0, arrival[i] - now)))
    finished.wait(timeout=120)
    t1 = server.now()
    ok = status == 0
    meas = np.arange(n) >= warmup
    l_ok = lat[ok & meas]
    span_first = arrival[warmup] if warmup < n else 0.0
    return {"rate_rps": rate, "requests": n, "completed": int(np.isfinite(lat).sum()), "errors": int((~ok).sum()),
            "frames_per_s": float((ok & meas).sum() / max(1e-9, (t1 - t0) - span_first)),
            "p50_ms": float(np.percentile(l_ok, 50) * 1e3) if len(l_ok) else None,
            "p99_ms": float(np.percentile(l_ok, 99) * 1e3) if len(l_ok) else None,
            "mean_ms": float(np.mean(l_ok) * 1e3) if len(l_ok) else None,
            "stats": server.stats()}
