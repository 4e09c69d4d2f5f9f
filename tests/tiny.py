"""Hand-built tiny scenes for tests (inputs only; no rendering arithmetic)."""
from __future__ import annotations

import numpy as np

from paper_1904_01201_b300.workloads import Scene, Intrinsics


def identity_pose(x=0.0, y=0.0, z=0.0):
    return np.array([x, y, z, 1, 0, 0, 0], dtype=np.float32)


def screen_intr(W, H, near=0.01, far=10.0):
    """90 degree HFOV pinhole: fx = W/2, cx = W/2 (Sec. 4 "Sensory input")."""
    return Intrinsics(W / 2.0, W / 2.0, W / 2.0, H / 2.0, near, far)


def screen_to_world(sx, sy, W, H, d=1.0):
    """World point (identity camera at the origin) that projects to (sx, sy) at depth d."""
    f = W / 2.0
    x = (np.asarray(sx, dtype=np.float64) - W / 2.0) / f * d
    y = (H / 2.0 - np.asarray(sy, dtype=np.float64)) / f * d
    return np.stack([x, y, -np.full_like(x, d)], -1)


def front_facing(tri_xyz):
    """Reorder a triangle so that it is counter-clockwise seen from the origin camera."""
    a, b, c = tri_xyz
    n = np.cross(b - a, c - a)
    if np.dot(n, -a) < 0:
        return [a, c, b]
    return [a, b, c]


def scene_from_tris(tris, front=True, **kw):
    """Scene from a list of 3x3 world triangles (no vertex sharing)."""
    xyz, idx = [], []
    for t in tris:
        t = [np.asarray(v, dtype=np.float64) for v in t]
        if front:
            t = front_facing(t)
        base = len(xyz)
        xyz += t
        idx.append([base, base + 1, base + 2])
    return Scene(xyz=np.array(xyz, dtype=np.float32), idx=np.array(idx, dtype=np.uint32), **kw)


def grid_scene(corners, n, m, jitter=0.0, rng=None):
    """Planar n x m grid between 4 world corners (shared vertices), optional in-plane jitter."""
    p00, p10, p01 = (np.asarray(c, dtype=np.float64) for c in corners)
    i, j = np.meshgrid(np.arange(n + 1), np.arange(m + 1), indexing="xy")
    fi = (i / n).astype(np.float64)
    fj = (j / m).astype(np.float64)
    if jitter and rng is not None:
        inner = (i > 0) & (i < n) & (j > 0) & (j < m)
        fi = fi + inner * rng.uniform(-jitter, jitter, fi.shape) / n
        fj = fj + inner * rng.uniform(-jitter, jitter, fj.shape) / m
    xyz = p00 + fi.reshape(-1, 1) * (p10 - p00) + fj.reshape(-1, 1) * (p01 - p00)
    ci, cj = np.meshgrid(np.arange(n), np.arange(m), indexing="xy")
    v00 = (cj * (n + 1) + ci).reshape(-1)
    v10, v01 = v00 + 1, v00 + n + 1
    v11 = v01 + 1
    idx = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    # orient towards the camera at the origin
    a, b, c = xyz[idx[:, 0]], xyz[idx[:, 1]], xyz[idx[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, -a) < 0
    idx[flip, 1], idx[flip, 2] = idx[flip, 2].copy(), idx[flip, 1].copy()
    return Scene(xyz=xyz.astype(np.float32), idx=idx.astype(np.uint32))


def random_tiny_scene(rng, T):
    """T random triangles around the origin camera (centres in a box reaching
    behind it, sizes from 5 cm to 1.5 m), unoriented."""
    tris = []
    for _ in range(T):
        c = rng.uniform([-2, -2, -5], [2, 2, 0.3])
        tri = c + rng.normal(scale=rng.uniform(0.05, 1.5), size=(3, 3))
        tris.append(tri)
    return scene_from_tris(tris, front=False)
