"""Large-triangle paths (the warp's row-span raster: queued per warp or
binned for the separate pass; int32 edges for bounding boxes under 2^15
sub-pixels, int64 otherwise) against the oracle, under launch
configurations that send every triangle above a few pixels down one path or
the other. Ids bit-exact, depth bit-exact, RGB within 1/255."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1904_01201_b300 import build as _build  # noqa: E402

_build.build()
from paper_1904_01201_b300 import hsr  # noqa: E402
from paper_1904_01201_b300.workloads import Scene  # noqa: E402
from tests.tiny import identity_pose, screen_intr, screen_to_world  # noqa: E402

BG = 0xFFFFFFFF

# (small_px, bin_px): bins for everything above 8 / 32 candidates, or the
# per-warp queue for everything above 32 candidates
CONFIGS = [(8, 8), (32, 32), (32, 1 << 20)]


def _render(sc, W, H, small, bin_, near):
    h = hsr.SceneHandle(sc)
    poses = identity_pose()[None]
    intr = screen_intr(W, H, near, 100.0)
    cfg = hsr.hsr_config(small, bin_, 4, 3, 1, (4.0, 10.0))
    hsr.hsr_set_tuned_config([h.handle], 1, W, H, True, cfg)
    out = hsr.render(h, poses, intr, W, H, ids=True)
    torch.cuda.synchronize()
    hsr.hsr_set_tuned_config([h.handle], 1, W, H, True, None)
    res = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}
    h.close()
    return res, poses, intr


def _check(sc, W, H, oracle_mod, what, near=0.01):
    o = None
    for small, bin_ in CONFIGS:
        g, poses, intr = _render(sc, W, H, small, bin_, near)
        if o is None:
            o = oracle_mod.render(sc, poses, intr, W, H)
        bad = g["ids"] != o["ids"]
        assert not bad.any(), f"{what} {small}/{bin_}: {int(bad.sum())} id mismatches (first {np.argwhere(bad)[:3]})"
        assert np.array_equal(g["depth"].view(np.uint32), o["depth"].view(np.uint32)), f"{what}: depth"
        d = np.abs(g["rgb"].astype(np.int16) - o["rgb"].astype(np.int16))
        assert d.max() <= 1, f"{what}: rgb {d.max()}"
    return o


def _mesh(sx, sy, d, idx, rng):
    """Screen-space vertices (sx, sy) at depths d, faces idx, vertex colours."""
    xyz = screen_to_world(sx, sy, W_, H_, 1.0) * np.asarray(d)[:, None]
    sc = Scene(xyz=xyz.astype(np.float32), idx=np.asarray(idx, np.uint32))
    sc.vrgb = rng.integers(0, 256, (sc.n_verts, 3), dtype=np.uint8)
    return sc


W_, H_ = 256, 192


def _grid(n, m, x0, x1, y0, y1, rng, jitter, on_centres):
    gx, gy = np.meshgrid(np.linspace(x0, x1, n + 1), np.linspace(y0, y1, m + 1), indexing="xy")
    inner = np.zeros_like(gx, bool)
    inner[1:-1, 1:-1] = True
    gx = gx + inner * rng.uniform(-jitter, jitter, gx.shape)
    gy = gy + inner * rng.uniform(-jitter, jitter, gy.shape)
    if on_centres:          # vertices on sample positions: the top-left rule decides shared-edge samples
        gx, gy = np.floor(gx) + 0.5, np.floor(gy) + 0.5
    v = (np.arange(m)[:, None] * (n + 1) + np.arange(n)[None, :]).reshape(-1)
    idx = np.concatenate([np.stack([v, v + n + 2, v + 1], 1), np.stack([v, v + n + 1, v + n + 2], 1)])
    d = rng.uniform(1.0, 3.0, gx.size)
    return gx.reshape(-1), gy.reshape(-1), d, idx


@pytest.mark.parametrize("seed,n,m,on_centres", [(0, 5, 4, False), (1, 3, 2, True), (2, 8, 6, True), (3, 2, 1, False)])
def test_screen_grids_no_holes(oracle_mod, seed, n, m, on_centres):
    """Shared-edge grids of 20-250 pixel triangles (perspective depths): parity
    on every path, and every sample inside the grid's outline is covered."""
    rng = np.random.default_rng(seed)
    sx, sy, d, idx = _grid(n, m, 3.3, W_ - 4.1, 2.7, H_ - 3.2, rng, 0.3 * W_ / n, on_centres)
    o = _check(_mesh(sx, sy, d, idx, rng), W_, H_, oracle_mod, f"grid {n}x{m}")
    inner = o["ids"][0, 4:H_ - 4, 5:W_ - 5]
    assert (inner != BG).all()


def test_slivers_and_near_axis_edges(oracle_mod):
    """Long thin triangles with edges a fraction of a pixel off horizontal or
    vertical (row bounds far outside the image on one side), the third vertex
    on either side (so the near-axis edge is a top, bottom, left or right
    edge), all wound to face the camera."""
    rng = np.random.default_rng(7)
    sx, sy, idx = [], [], []
    for k in range(48):
        a = rng.uniform(-20, W_ + 20, 2)
        L = rng.uniform(40, 400)
        side = 1.0 if (k // 2) % 2 else -1.0
        if k % 2:
            b, c = a + [L, rng.uniform(-0.3, 0.3)], a + [rng.uniform(0, L), side * rng.uniform(1, 30)]
        else:
            b, c = a + [rng.uniform(-0.3, 0.3), L], a + [side * rng.uniform(1, 30), rng.uniform(0, L)]
        if (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]) > 0:
            b, c = c, b                                  # screen-space area < 0: faces the camera
        sx += [a[0], b[0], c[0]]
        sy += [a[1], b[1], c[1]]
        idx.append([3 * k, 3 * k + 1, 3 * k + 2])
    d = rng.uniform(1.0, 4.0, len(sx))
    o = _check(_mesh(np.array(sx), np.array(sy), d, idx, rng), W_, H_, oracle_mod, "slivers")
    assert len(np.unique(o["ids"])) > 20


def test_wide_triangles_int64_rows(oracle_mod):
    """Bounding boxes beyond 2^15 sub-pixels (vertices up to thousands of
    pixels off screen): the int64 row bounds. The near plane at 0.5 keeps
    every snapped coordinate of the scene within the renderer's 2^30 range."""
    rng = np.random.default_rng(11)
    sx, sy, idx = [], [], []
    for k in range(12):
        p = rng.uniform([-3000, -3000], [W_ + 3000, H_ + 3000], (3, 2))
        p[k % 3] = rng.uniform([0, 0], [W_, H_])         # one vertex on screen
        sx += list(p[:, 0])
        sy += list(p[:, 1])
        idx.append([3 * k, 3 * k + 1, 3 * k + 2])
    d = rng.uniform(1.0, 50.0, len(sx))
    o = _check(_mesh(np.array(sx), np.array(sy), d, idx, rng), W_, H_, oracle_mod, "wide", near=0.5)
    assert (o["ids"] != BG).mean() > 0.2
