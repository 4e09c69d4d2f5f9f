"""The whole-meshlet back-face cull changes no pixel. Planar grids (one plane
per meshlet) are seen from just behind their plane (0.1 mm to 0.5 m) at
grazing angles, where snapping can turn the orientation of thin projected
triangles either way: the cull must keep every meshlet whose triangles it
cannot prove culled, so ids and depth equal the oracle's bit for bit and RGB
within 1/255. The counters show both outcomes occur (meshlets skipped, and
meshlets kept by the margin)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1904_01201_b300 import build as _build  # noqa: E402

_build.build()
from paper_1904_01201_b300 import hsr  # noqa: E402
from paper_1904_01201_b300.workloads import Intrinsics, Scene  # noqa: E402
from tests.test_gpu_parity import assert_parity, gpu_render  # noqa: E402


def _walls(rng):
    """Several planar grid patches at random orientations; each grid is wound
    so its front faces +n."""
    xyz, idx = [], []
    for _ in range(6):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        u = np.cross(n, [0.0, 1.0, 0.0] if abs(n[1]) < 0.9 else [1.0, 0.0, 0.0])
        u /= np.linalg.norm(u)
        v = np.cross(n, u)
        origin = rng.uniform(-1.0, 1.0, 3)
        k, size = 24, rng.uniform(0.5, 3.0)
        base = len(xyz)
        for j in range(k + 1):
            for i in range(k + 1):
                xyz.append(origin + (i / k - 0.5) * size * u + (j / k - 0.5) * size * v)
        for j in range(k):
            for i in range(k):
                a = base + j * (k + 1) + i
                b, c, d = a + 1, a + k + 1, a + k + 2
                idx += [[a, b, d], [a, d, c]]      # counter-clockwise about +n (u x v = n)
    xyz = np.asarray(xyz, dtype=np.float32)
    idx = np.asarray(idx, dtype=np.uint32)
    return Scene(xyz=xyz, idx=idx, vrgb=rng.integers(0, 256, (len(xyz), 3), dtype=np.uint8))


def _look_pose(pos, fwd):
    """Pose at pos looking along fwd (camera -Z), +Y up where possible."""
    f = np.asarray(fwd, dtype=np.float64)
    f /= np.linalg.norm(f)
    up = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.95 else np.array([1.0, 0.0, 0.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(x, f)
    R = np.stack([x, y, -f], 1)                  # world-from-camera columns
    w = math.sqrt(max(1e-12, 1.0 + R[0, 0] + R[1, 1] + R[2, 2])) / 2.0
    q = np.array([w, (R[2, 1] - R[1, 2]) / (4 * w), (R[0, 2] - R[2, 0]) / (4 * w), (R[1, 0] - R[0, 1]) / (4 * w)])
    return np.r_[pos, q / np.linalg.norm(q)].astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cull_keeps_every_pixel(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    sc = _walls(rng)
    # cameras just behind a patch's plane, looking along it (grazing) or into it
    poses = []
    tri = sc.xyz[sc.idx[::97]]
    for t in tri[:24]:
        n = np.cross(t[1] - t[0], t[2] - t[0])
        n /= np.linalg.norm(n)
        h = 10.0 ** rng.uniform(-4, math.log10(0.5))
        pos = t.mean(0) - h * n
        tangent = np.cross(n, rng.normal(size=3))
        fwd = tangent / np.linalg.norm(tangent) + rng.uniform(-0.2, 0.2) * n
        poses.append(_look_pose(pos, fwd))
    poses = np.stack(poses)
    W, H = 96, 64
    intr = Intrinsics(48.0, 48.0, 48.0, 32.0, 0.01, 10.0)
    hsr.hsr_set_stage_stats(True)
    g = gpu_render(sc, poses, intr, W, H)
    stats = hsr.hsr_get_stage_stats()
    hsr.hsr_set_stage_stats(False)
    o = oracle_mod.render(sc, poses, intr, W, H)
    assert_parity(g, o, f"walls seed {seed}")
    assert stats["backfacing_culled"] > 0 and stats["backfacing_kept"] > 0, stats
