"""Guard-band clipping on the device against the oracle, through the C-ABI.

Triangles whose snapped vertices would reach +-2^30 sub-pixels (near the
camera at high resolution, or with tiny near planes) are clipped to a guard
band 2^21 pixels either side of the principal point instead of being
refused. Ids and depth must equal the oracle bit for bit, RGB within 1/255,
on every path such a triangle can take: the one-shot render, the
graph-captured batch, the large-triangle bins or the per-warp queue, and the
allocation-free entry point.
"""
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
from paper_1904_01201_b300 import workloads as wl  # noqa: E402
from paper_1904_01201_b300.workloads import Scene, Intrinsics  # noqa: E402
from tests.tiny import identity_pose, random_tiny_scene, scene_from_tris  # noqa: E402

BG = 0xFFFFFFFF


def _np(out):
    torch.cuda.synchronize()
    r = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy()}
    if out.get("ids") is not None:
        r["ids"] = hsr.ids_u32(out["ids"])
    return r


def _parity(g, o, what):
    bad = g["ids"] != o["ids"]
    assert not bad.any(), f"{what}: {int(bad.sum())} id mismatches (first {np.argwhere(bad)[:3]})"
    assert np.array_equal(g["depth"].view(np.uint32), o["depth"].view(np.uint32)), f"{what}: depth"
    d = np.abs(g["rgb"].astype(np.int16) - o["rgb"].astype(np.int16))
    assert d.max() <= 1, f"{what}: rgb {d.max()}"


def _max_snap(scene, poses, intr, oracle_mod):
    """Largest |256 s| over every view's vertices in front of the near plane
    and near-plane crossing points (float64), i.e. how far the unclipped
    projection would reach."""
    fx, fy, cx, cy, near, _ = [float(v) for v in intr.as_array()]
    best = 0.0
    for pose in poses:
        M = oracle_mod.camera(pose).astype(np.float64)
        e = scene.xyz.astype(np.float64) @ M[:, :3].T + M[:, 3]
        t3 = e[scene.idx.astype(np.int64)]                    # [T, 3, 3]
        for a in range(3):
            p, r = t3[:, a], t3[:, (a + 1) % 3]
            dp, dr = -p[:, 2], -r[:, 2]
            pts = [p[dp >= near]]
            cross = (dp >= near) != (dr >= near)
            t = (near - dp[cross]) / (dr[cross] - dp[cross])
            pts.append(p[cross] + t[:, None] * (r[cross] - p[cross]))
            for c in pts:
                if len(c):
                    d = np.maximum(-c[:, 2], near)
                    best = max(best, np.abs(256 * (fx * c[:, 0] / d + cx)).max(),
                               np.abs(256 * (-fy * c[:, 1] / d + cy)).max())
    return best


def _wide_room(seed, half=25.0):
    """A 50 x 3 x 50 m room (floor 1.5 m below the origin camera), each face
    two triangles, 12 boxes, uv from a planar map, a 64x64 noise atlas."""
    rng = np.random.default_rng(seed)
    lo, hi = np.array([-half, -1.5, -half]), np.array([half, 1.5, half])
    tris = []

    def box(a, b):
        c = [np.array([a[0] if i & 1 == 0 else b[0], a[1] if i & 2 == 0 else b[1], a[2] if i & 4 == 0 else b[2]])
             for i in range(8)]
        for f in ((0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)):
            tris.append([c[f[0]], c[f[1]], c[f[2]]])
            tris.append([c[f[0]], c[f[2]], c[f[3]]])

    box(lo, hi)
    for _ in range(12):
        ctr = rng.uniform([-8, -1.5, -8], [8, 0.5, 8])
        if np.abs(ctr[[0, 2]]).max() < 0.8:
            ctr[0] += 2.0
        s = rng.uniform(0.3, 2.5, 3)
        box(ctr - s / 2, ctr + s / 2)
    sc = scene_from_tris(tris)
    x, y, z = sc.xyz[:, 0], sc.xyz[:, 1], sc.xyz[:, 2]
    sc.uv = np.stack([(x + 0.3 * y) / (2 * half) + 0.5, (z + 0.7 * y) / (2 * half) + 0.5], 1).astype(np.float32)
    sc.atlas = rng.integers(0, 256, (64, 64, 4), dtype=np.uint8)
    sc.sem = (np.arange(sc.n_tris, dtype=np.uint32) // 2) * 3 + 1
    return sc


def _room_poses():
    poses = [[0, 0, 0, *wl.yaw_quat(np.array(th))] for th in (0.3, 2.0)]
    # pitched 40 degrees down, towards the floor at the camera's feet
    a = math.radians(-40)
    poses.append([0, 0, 0, math.cos(a / 2), math.sin(a / 2), 0, 0])
    return np.array(poses, np.float32)


def test_wide_room_4096_at_near_1cm(oracle_mod):
    """A 4096^2 view of a 50 m room at near 0.01 m: the floor's and walls'
    near-clip points project up to ~10^7 pixels off screen, beyond the
    fixed-point range (the case the renderer used to refuse)."""
    sc = _wide_room(0)
    poses = _room_poses()
    W = H = 4096
    intr = wl.pinhole_90(W, H, 0.01, 60.0)
    assert _max_snap(sc, poses, intr, oracle_mod) > 2.0 ** 30
    h = hsr.SceneHandle(sc)
    g = _np(hsr.render(h, poses, intr, W, H, ids=True))
    assert hsr.hsr_device_status(1) == hsr.HSR_OK
    o = oracle_mod.render(sc, poses, intr, W, H)
    _parity(g, o, "wide room 4096")
    assert (g["ids"] != BG).mean() > 0.999
    h.close()


@pytest.mark.parametrize("small,bin_", [(8, 8), (32, 1 << 20)])
def test_wide_room_tiny_near_every_path(oracle_mod, small, bin_):
    """1024^2 at near 2e-6 m: through the one-shot render, the graph batch
    (with large triangles binned, or all kept in the per-warp queue), and
    the allocation-free entry point."""
    sc = _wide_room(1)
    poses = _room_poses()
    W = H = 1024
    intr = Intrinsics(W / 2, W / 2 * 1.2, W / 2, H / 2, 2e-6, 60.0)
    assert _max_snap(sc, poses, intr, oracle_mod) > 2.0 ** 36
    o = oracle_mod.render(sc, poses, intr, W, H)
    h = hsr.SceneHandle(sc)
    cfg = hsr.hsr_config(small, bin_, 4, 3, 2, (4.0, 10.0))
    hsr.hsr_set_tuned_config([h.handle], len(poses), W, H, True, cfg)
    _parity(_np(hsr.render(h, poses, intr, W, H, ids=True)), o, f"one-shot {small}/{bin_}")
    b = hsr.Batch([h], len(poses), intr, W, H, ids=True)
    b.render(poses)
    _parity(_np(b.out), o, f"batch {small}/{bin_}")
    b.close()
    hsr.hsr_set_tuned_config([h.handle], len(poses), W, H, True, None)
    out = hsr.alloc_outputs(1, W, H)
    for i in range(len(poses)):
        st = hsr.hsr_render_noalloc(h.handle, poses[i:i + 1], intr, W, H, out["rgb"], out["depth"], out["ids"])
        assert st == hsr.HSR_OK, hsr.hsr_status_string(st)
        gi = _np(out)
        _parity(gi, {k: v[i:i + 1] for k, v in o.items()}, f"noalloc view {i}")
    assert hsr.hsr_device_status(1) == hsr.HSR_OK
    h.close()


def _floor_fan(n=32, half=3.0, y=-1.5, zb=0.5, za=-4.0, spread=2.0):
    """n floor triangles sharing one base edge behind the camera (x = -half
    .. half at z = zb) with apexes spread ahead (z = za): n + 2 vertices, so
    the scene is one meshlet. Every triangle crosses the near plane, and its
    clip points project far outside the fixed-point range on three sides."""
    base = [np.array([-half, y, zb]), np.array([half, y, zb])]
    apex = [np.array([-spread + 2 * spread * i / max(n - 1, 1), y, za]) for i in range(n)]
    xyz = np.array(base + apex, np.float32)
    idx = []
    for i in range(n):
        t = [0, 1, 2 + i]
        a, b, c = (xyz[k].astype(np.float64) for k in t)
        if np.dot(np.cross(b - a, c - a), -a) < 0:         # counter-clockwise seen from the camera
            t = [0, 2 + i, 1]
        idx.append(t)
    sc = Scene(xyz=xyz, idx=np.array(idx, np.uint32))
    sc.vrgb = (np.arange(3 * (n + 2)) * 37 % 256).astype(np.uint8).reshape(-1, 3)
    return sc


def _guard_subtriangles(sc, intr, oracle_mod):
    """Sub-triangles the guard band cuts the identity view's triangles into
    (near clip in float64, then the oracle's guard clip)."""
    fx, fy, cx, cy, near, _ = [float(v) for v in intr.as_array()]
    total = 0
    for t in sc.xyz[sc.idx].astype(np.float64):
        P = [(v[0], v[1], -v[2]) for v in t]
        poly = []
        for k in range(3):
            a, b = P[k], P[(k + 1) % 3]
            if a[2] >= near:
                poly.append(a)
            if (a[2] >= near) != (b[2] >= near):
                s = (near - a[2]) / (b[2] - a[2])
                poly.append(tuple(a[j] + s * (b[j] - a[j]) for j in range(3)))
        if len(poly) < 3:
            continue
        snap = max(max(abs(256 * (fx * x / d + cx)), abs(256 * (-fy * y / d + cy))) for x, y, d in poly)
        if snap >= 2.0 ** 30:
            total += max(len(oracle_mod.guard_clip(np.array(poly, np.float32), 2.0 ** 21 / fx, 2.0 ** 21 / fy)) - 2, 0)
    return total


def test_guard_fans_beyond_one_warp_queue(oracle_mod):
    """One meshlet whose 32 triangles are all cut by the guard band into
    three sub-triangles each, 96 large ones for one warp: more than the
    warp's queue holds at once, so they go through it in rounds. Through the
    per-warp queue (no bins), the bins, and the allocation-free entry point."""
    sc = _floor_fan()
    W = H = 1024
    intr = Intrinsics(512.0, 512.0, 512.0, 512.0, 2e-6, 60.0)
    assert _guard_subtriangles(sc, intr, oracle_mod) > 64
    poses = identity_pose()[None]
    o = oracle_mod.render(sc, poses, intr, W, H)
    assert (o["ids"] != BG).mean() > 0.25 and len(np.unique(o["ids"])) == 33
    h = hsr.SceneHandle(sc)
    for small, bin_ in ((8, 1 << 20), (8, 8)):
        cfg = hsr.hsr_config(small, bin_, 4, 3, 1, (4.0, 10.0))
        hsr.hsr_set_tuned_config([h.handle], 1, W, H, True, cfg)
        _parity(_np(hsr.render(h, poses, intr, W, H, ids=True)), o, f"one-shot {small}/{bin_}")
        b = hsr.Batch([h], 1, intr, W, H, ids=True)
        b.render(poses)
        _parity(_np(b.out), o, f"batch {small}/{bin_}")
        b.close()
    hsr.hsr_set_tuned_config([h.handle], 1, W, H, True, None)
    out = hsr.alloc_outputs(1, W, H)
    st = hsr.hsr_render_noalloc(h.handle, poses, intr, W, H, out["rgb"], out["depth"], out["ids"])
    assert st == hsr.HSR_OK, hsr.hsr_status_string(st)
    _parity(_np(out), o, "noalloc")
    assert hsr.hsr_device_status(1) == hsr.HSR_OK
    h.close()


def test_huge_fronto_parallel_quad(oracle_mod):
    """A quad at depth D reaching 10^6 m to every side: every pixel covered,
    depth exactly D, as the oracle."""
    W, H = 160, 96
    intr = Intrinsics(80.0, 80.0, 80.0, 48.0, 0.01, 10.0)
    for D in (1.0, 4.0):
        c = np.array([[-1e6, -1e6, -D], [1e6, -1e6, -D], [-1e6, 1e6, -D], [1e6, 1e6, -D]])
        sc = scene_from_tris([[c[0], c[1], c[3]], [c[0], c[3], c[2]]])
        sc.vrgb = np.array([[255, 0, 0], [0, 255, 0], [0, 0, 255]] * 2, np.uint8)
        h = hsr.SceneHandle(sc)
        g = _np(hsr.render(h, identity_pose()[None], intr, W, H, ids=True))
        h.close()
        o = oracle_mod.render(sc, identity_pose()[None], intr, W, H)
        _parity(g, o, f"quad D={D}")
        assert np.all(g["ids"] != BG) and np.all(g["depth"] == np.float32(D))


@pytest.mark.parametrize("block", range(2))
def test_random_scenes_tiny_near(oracle_mod, block):
    """Random scenes around the camera, near planes of 1e-6 .. 1e-5 m, fx !=
    fy, several poses: near-clipped triangles whose clip points project far
    outside the fixed-point range."""
    rng = np.random.default_rng(2000 + block)
    for trial in range(40):
        W, H = int(rng.integers(8, 160)), int(rng.integers(8, 160))
        T = int(rng.integers(4, 60))
        sc = random_tiny_scene(rng, T)
        if rng.uniform() < 0.5:
            sc.uv = rng.uniform(-0.2, 1.2, (sc.n_verts, 2)).astype(np.float32)
            sc.atlas = rng.integers(0, 256, (int(rng.integers(1, 40)), int(rng.integers(1, 40)), 4), dtype=np.uint8)
        else:
            sc.vrgb = rng.integers(0, 256, (sc.n_verts, 3), dtype=np.uint8)
        n = int(rng.integers(1, 4))
        q = rng.normal(size=(n, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        poses = np.concatenate([rng.uniform(-0.3, 0.3, (n, 3)), q], 1).astype(np.float32)
        f = float(rng.uniform(0.4, 1.2)) * W
        intr = Intrinsics(f, f * float(rng.uniform(0.7, 1.4)), W / 2 + float(rng.uniform(-2, 2)),
                          H / 2 + float(rng.uniform(-2, 2)), float(10 ** rng.uniform(-6, -5)), 6.0)
        h = hsr.SceneHandle(sc)
        g = _np(hsr.render(h, poses, intr, W, H, ids=True))
        h.close()
        _parity(g, oracle_mod.render(sc, poses, intr, W, H), f"trial {trial} {W}x{H} T={T}")
    assert hsr.hsr_device_status(1) == hsr.HSR_OK


def test_intrinsics_limits():
    sc = wl.make_room(0, 2000)
    h = hsr.SceneHandle(sc)
    out = hsr.alloc_outputs(1, 16, 16)
    pose = wl.random_poses(sc, 1, 0)
    ok = [Intrinsics(4000, 4000, 8, 8, 1e-6, 10.0), Intrinsics(8, 8, 65536, -65536, 2.0 ** -20, 10.0)]
    bad = [Intrinsics(8, 8, 65537, 8, 0.01, 10.0), Intrinsics(8, 8, 8, -70000, 0.01, 10.0),
           Intrinsics(8, 8, 8, 8, 2.0 ** -21, 10.0)]
    for intr in ok:
        assert hsr.hsr_render(h.handle, pose, intr, 16, 16, out["rgb"], out["depth"], out["ids"]) == hsr.HSR_OK
    for intr in bad:
        assert hsr.hsr_render(h.handle, pose, intr, 16, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert hsr.hsr_device_status(1) == hsr.HSR_OK
    h.close()


def test_wide_room_guard_band_with_noisy_depth(oracle_mod):
    """The shading variant with both the guard-band path and depth noise
    (Appendix C): the wide room at 1024^2 and near 2e-6 m with sigma 0.4.
    Ids and RGB equal the noise-free guard-band render, and depth meets the
    noise tests' derived fp32/fp64 bound against the oracle."""
    from tests.test_gpu_noise import assert_noisy_parity
    sc = _wide_room(1)
    poses = _room_poses()
    W = H = 1024
    intr = Intrinsics(W / 2, W / 2 * 1.2, W / 2, H / 2, 2e-6, 60.0)
    assert _max_snap(sc, poses, intr, oracle_mod) > 2.0 ** 36
    h = hsr.SceneHandle(sc)
    sigma, seed = 0.4, 0x5EED
    g = _np(hsr.render(h, poses, intr, W, H, ids=True, noise_sigma=sigma, noise_seed=seed))
    assert hsr.hsr_device_status(1) == hsr.HSR_OK
    o = oracle_mod.render(sc, poses, intr, W, H, noise_sigma=sigma, noise_seed=seed)
    n_both, _ = assert_noisy_parity(g, o, intr, sigma, "guard band + noise")
    assert n_both > 0.3 * g["depth"].size
    clean = _np(hsr.render(h, poses, intr, W, H, ids=True))
    assert np.array_equal(clean["ids"], g["ids"]) and np.array_equal(clean["rgb"], g["rgb"])
    h.close()


def test_wide_room_guard_band_trilinear(oracle_mod):
    """Trilinear sampling on guard-clipped triangles (the level of detail
    comes from each guard sub-triangle's own derivatives): the wide room with
    a 2048^2 atlas at 1024^2 and near 2e-6 m, so that its floor is magnified
    near the camera and minified by several levels far away."""
    sc = _wide_room(1)
    sc.atlas = np.random.default_rng(9).integers(0, 256, (2048, 2048, 4), dtype=np.uint8)
    poses = _room_poses()
    W = H = 1024
    intr = Intrinsics(W / 2, W / 2 * 1.2, W / 2, H / 2, 2e-6, 60.0)
    assert _max_snap(sc, poses, intr, oracle_mod) > 2.0 ** 36
    h = hsr.SceneHandle(sc)
    h.set_sampling(hsr.HSR_SAMPLE_TRILINEAR)
    g = _np(hsr.render(h, poses, intr, W, H, ids=True))
    assert hsr.hsr_device_status(1) == hsr.HSR_OK
    o = oracle_mod.render(sc, poses, intr, W, H, trilinear=True, lod=True)
    hit = np.isfinite(o["lod"])
    assert (o["lod"][hit] > 1).mean() > 0.02 and (o["lod"][hit] <= 0).mean() > 0.02
    _parity(g, o, "guard band, trilinear")
    h.close()
