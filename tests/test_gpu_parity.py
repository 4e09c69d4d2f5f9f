"""CUDA path vs the CPU oracle, element by element, through the C-ABI.

Bar (stated rules, both sides): triangle ids and coverage bit-exact; depth
within 1e-5 relative where ids match (the shared fp32 recipe makes it
bit-exact in practice, which is also checked); RGB within 1/255 (the oracle
shades in fp64, the kernels in fp32).
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
from tests.tiny import identity_pose, scene_from_tris, screen_intr, screen_to_world  # noqa: E402

BG = 0xFFFFFFFF
DEPTH_RTOL = 1e-5
RGB_TOL = 1


def gpu_render(scene, poses, intr, W, H, ids=True):
    h = hsr.SceneHandle(scene)
    out = hsr.render(h, poses, intr, W, H, ids=ids)
    torch.cuda.synchronize()
    res = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy()}
    if ids:
        res["ids"] = hsr.ids_u32(out["ids"])
    h.close()
    return res


def assert_parity(g, o, what=""):
    assert g["ids"].shape == o["ids"].shape
    bad = g["ids"] != o["ids"]
    assert not bad.any(), f"{what}: {int(bad.sum())} id mismatches of {bad.size} (first at {np.argwhere(bad)[:3]})"
    dg, do = g["depth"], o["depth"]
    rel = np.abs(dg.astype(np.float64) - do) <= DEPTH_RTOL * np.abs(do.astype(np.float64))
    assert rel.all(), f"{what}: depth beyond 1e-5 relative at {int((~rel).sum())} pixels"
    assert np.array_equal(dg.view(np.uint32), do.view(np.uint32)), f"{what}: depth not bit-exact"
    diff = np.abs(g["rgb"].astype(np.int16) - o["rgb"].astype(np.int16))
    assert diff.max() <= RGB_TOL, f"{what}: rgb diff {diff.max()} at {int((diff > RGB_TOL).sum())} channels"


# ------------------------------------------------------------------ small room
def test_small_room_full_config(oracle_mod):
    """Small room: ~10k triangles, vertex colours, 16 poses, 128x128."""
    sc = wl.make_room(0)
    poses = wl.random_poses(sc, 16, 0)
    intr = wl.pinhole_90(128, 128)
    g = gpu_render(sc, poses, intr, 128, 128)
    o = oracle_mod.render(sc, poses, intr, 128, 128)
    assert_parity(g, o, "room")
    assert (g["ids"] != BG).mean() > 0.99


@pytest.mark.parametrize("W,H", [(100, 37), (65, 129), (1, 64), (64, 1), (1, 1), (17, 200)])
def test_room_ragged_sizes(oracle_mod, W, H):
    sc = wl.make_room(3, 4000)
    poses = wl.random_poses(sc, 3, 3)
    intr = Intrinsics(W / 2, W / 2, W / 2, H / 2, 0.01, 10.0)
    assert_parity(gpu_render(sc, poses, intr, W, H), oracle_mod.render(sc, poses, intr, W, H), f"{W}x{H}")


# ------------------------------------------------------------------ random tiny scenes
def _random_scene(rng, T, textured):
    tris = []
    for _ in range(T):
        c = rng.uniform([-2, -2, -5], [2, 2, 0.3])
        tris.append(c + rng.normal(scale=rng.uniform(0.02, 2.0), size=(3, 3)))
    sc = scene_from_tris(tris, front=False)
    V = sc.n_verts
    if textured:
        sc.uv = rng.uniform(-0.2, 1.2, (V, 2)).astype(np.float32)
        aw, ah = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        sc.atlas = rng.integers(0, 256, (ah, aw, 4), dtype=np.uint8)
    else:
        sc.vrgb = rng.integers(0, 256, (V, 3), dtype=np.uint8)
    if rng.uniform() < 0.5:
        sc.sem = rng.integers(0, 1000, T).astype(np.uint32)
    return sc


@pytest.mark.parametrize("block", range(3))
def test_random_tiny_scenes(oracle_mod, block):
    rng = np.random.default_rng(1000 + block)
    for trial in range(60):
        W, H = int(rng.integers(1, 140)), int(rng.integers(1, 140))
        sc = _random_scene(rng, int(rng.integers(1, 60)), bool(rng.integers(0, 2)))
        n = int(rng.integers(1, 4))
        q = rng.normal(size=(n, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        poses = np.concatenate([rng.uniform(-0.3, 0.3, (n, 3)), q], 1).astype(np.float32)
        f = float(rng.uniform(0.3, 1.5)) * max(W, 1)
        intr = Intrinsics(f, f * float(rng.uniform(0.8, 1.25)), W / 2 + float(rng.uniform(-3, 3)),
                          H / 2 + float(rng.uniform(-3, 3)), float(rng.uniform(0.01, 0.3)), float(rng.uniform(2, 8)))
        assert_parity(gpu_render(sc, poses, intr, W, H), oracle_mod.render(sc, poses, intr, W, H),
                      f"trial {trial} {W}x{H} T={sc.n_tris}")


# ------------------------------------------------------------------ edge cases
def test_huge_and_subpixel_triangles(oracle_mod):
    W = H = 256
    intr = screen_intr(W, H, 0.01, 100.0)
    rng = np.random.default_rng(5)
    tris = [screen_to_world(np.array([-5000.0, 9000.0, 200.0]), np.array([-3000.0, 100.0, 8000.0]), W, H, 3.0)]
    for _ in range(300):   # sub-pixel triangles in front of it
        c = rng.uniform(0, 256, 2)
        o = rng.normal(scale=0.4, size=(3, 2))
        tris.append(screen_to_world(c[0] + o[:, 0], c[1] + o[:, 1], W, H, float(rng.uniform(1, 2.9))))
    sc = scene_from_tris(tris)
    sc.vrgb = rng.integers(0, 256, (sc.n_verts, 3), dtype=np.uint8)
    assert_parity(gpu_render(sc, identity_pose()[None], intr, W, H),
                  oracle_mod.render(sc, identity_pose()[None], intr, W, H), "huge+subpixel")


def test_camera_inside_box_clips_everywhere(oracle_mod):
    sc = wl.make_room(4, 3000)
    # camera at a box corner region, looking through walls at grazing angles
    poses = []
    for th in np.linspace(0, 2 * math.pi, 7, endpoint=False):
        for y in (0.02, 1.5, 2.98):
            poses.append([0.004, y, 0.004, *wl.yaw_quat(np.array(th))])
    poses = np.array(poses, np.float32)
    intr = wl.pinhole_90(96, 80, 0.01, 10.0)
    assert_parity(gpu_render(sc, poses, intr, 96, 80), oracle_mod.render(sc, poses, intr, 96, 80), "inside")


def test_nothing_visible():
    sc = Scene(xyz=np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], np.float32), idx=np.array([[0, 1, 2]], np.uint32))
    g = gpu_render(sc, identity_pose()[None], screen_intr(33, 17), 33, 17)
    assert np.all(g["ids"] == BG) and np.all(g["depth"] == 0) and np.all(g["rgb"] == 0)


def test_invalid_arguments_on_device():
    sc = wl.make_room(0, 2000)
    h = hsr.SceneHandle(sc)
    out = hsr.alloc_outputs(1, 16, 16)
    intr = wl.pinhole_90(16, 16)
    good = wl.random_poses(sc, 1, 0)
    bad_q = good.copy()
    bad_q[0, 3:] *= 1.01
    nan_p = good.copy()
    nan_p[0, 0] = np.nan
    assert hsr.hsr_render(h.handle, good, intr, 16, 16, out["rgb"], out["depth"], out["ids"]) == hsr.HSR_OK
    assert hsr.hsr_render(h.handle, bad_q, intr, 16, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render(h.handle, nan_p, intr, 16, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render(h.handle, good, intr, 0, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render(h.handle, good, intr, 4097, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    bad_i = Intrinsics(8, 8, 8, 8, 0.0, 10.0)
    assert hsr.hsr_render(h.handle, good, bad_i, 16, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    # principal point beyond 2^16 pixels, near plane below 2^-20 m
    assert hsr.hsr_render(h.handle, good, Intrinsics(8, 8, 70000, 8, 0.01, 10.0), 16, 16, out["rgb"],
                          out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render(h.handle, good, Intrinsics(8, 8, 8, 8, 1e-7, 10.0), 16, 16, out["rgb"],
                          out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    # zero views, no output buffer, null handle
    assert hsr.hsr_render(h.handle, good[:0], intr, 16, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render(h.handle, good, intr, 16, 16, None, None, None) == hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render_noalloc(h.handle, good[:0], intr, 16, 16, out["rgb"], out["depth"]) == \
        hsr.HSR_ERR_INVALID_ARG
    assert hsr.hsr_render(0, good, intr, 16, 16, out["rgb"], out["depth"]) == hsr.HSR_ERR_INVALID_ARG
    # a later call still works
    assert hsr.hsr_render(h.handle, good, intr, 16, 16, out["rgb"], out["depth"], out["ids"]) == hsr.HSR_OK
    torch.cuda.synchronize()
    h.close()


def test_empty_and_invalid_scenes_refused():
    """A scene with no triangles or no vertices, an index beyond the vertex
    count, or a non-finite position is refused at load (zero counts and bad
    indices are invalid arguments by the ABI's contract)."""
    xyz = np.array([[0, 0, -5], [1, 0, -5], [0, 1, -5]], np.float32)
    idx = np.array([[0, 1, 2]], np.uint32)
    for x, i in ((xyz, idx[:0]), (xyz[:0], idx), (xyz, np.array([[0, 1, 3]], np.uint32)),
                 (np.array([[0, 0, -5], [np.nan, 0, -5], [0, 1, -5]], np.float32), idx)):
        with pytest.raises(hsr.HsrError) as e:
            hsr.hsr_scene_load(x, i)
        assert e.value.status == hsr.HSR_ERR_INVALID_ARG
    h = hsr.hsr_scene_load(xyz, idx)          # the valid one loads, renders and frees
    out = hsr.alloc_outputs(1, 8, 8)
    assert hsr.hsr_render(h, identity_pose()[None], screen_intr(8, 8), 8, 8, out["rgb"], out["depth"]) == hsr.HSR_OK
    torch.cuda.synchronize()
    hsr.hsr_scene_free(h)


def test_determinism_and_order_independence():
    sc = wl.make_room(6, 6000)
    poses = wl.random_poses(sc, 8, 6)
    intr = wl.pinhole_90(128, 128)
    a = gpu_render(sc, poses, intr, 128, 128)
    for _ in range(3):
        b = gpu_render(sc, poses, intr, 128, 128)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    perm = np.random.default_rng(0).permutation(sc.n_tris)
    sp = Scene(xyz=sc.xyz, idx=sc.idx[perm].copy(), vrgb=sc.vrgb)
    c = gpu_render(sp, poses, intr, 128, 128)
    ids = np.where(c["ids"] == BG, BG, perm[np.minimum(c["ids"], sc.n_tris - 1)])
    assert np.array_equal(ids, a["ids"])
    assert np.array_equal(c["depth"], a["depth"]) and np.array_equal(c["rgb"], a["rgb"])


# ------------------------------------------------------------------ full-size configs, sampled
@pytest.fixture(scope="module")
def house():
    return wl.make_house(0, 1_000_000, 4096)


def test_house_full_size_sampled(oracle_mod, house):
    """1M-triangle house, 4096^2 atlas, 64 agents at 256^2: all 64 rendered in
    one launch; 3 sampled agents checked against the oracle element by element."""
    poses = wl.random_poses(house, 64, 0)
    intr = wl.pinhole_90(256, 256)
    g = gpu_render(house, poses, intr, 256, 256)
    for i in (0, 31, 63):
        o = oracle_mod.render(house, poses[i:i + 1], intr, 256, 256)
        assert_parity({k: v[i:i + 1] for k, v in g.items()}, o, f"house agent {i}")
    assert (g["ids"] != BG).mean() > 0.9


def test_batch_equals_plain_and_oracle(oracle_mod):
    """Batching: several resident scenes of uneven size in one launch; each
    agent's output equals its single-scene render bit for bit, and sampled
    agents match the oracle."""
    scenes = [wl.make_house(11, 60_000, 512), wl.make_house(12, 250_000, 1024), wl.make_room(13)]
    split = np.array([5, 20, 7])
    soa = np.repeat(np.arange(3), split).astype(np.uint32)
    rng = np.random.default_rng(3)
    rng.shuffle(soa)
    poses = np.zeros((len(soa), 7), np.float32)
    for s in range(3):
        poses[soa == s] = wl.random_poses(scenes[s], int((soa == s).sum()), 20 + s)
    intr = wl.pinhole_90(128, 128)
    hs = [hsr.SceneHandle(s) for s in scenes]
    out = hsr.render_batch(hs, soa, poses, intr, 128, 128)
    torch.cuda.synchronize()
    gb = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}
    for s in range(3):
        sel = np.nonzero(soa == s)[0]
        plain = hsr.render(hs[s], poses[sel], intr, 128, 128)
        torch.cuda.synchronize()
        for k, v in (("rgb", plain["rgb"].cpu().numpy()), ("depth", plain["depth"].cpu().numpy()),
                     ("ids", hsr.ids_u32(plain["ids"]))):
            assert np.array_equal(gb[k][sel], v), (s, k)
        i = int(sel[0])
        o = oracle_mod.render(scenes[s], poses[i:i + 1], intr, 128, 128)
        assert_parity({k: v[i:i + 1] for k, v in gb.items()}, o, f"batch scene {s}")
    for h in hs:
        h.close()
