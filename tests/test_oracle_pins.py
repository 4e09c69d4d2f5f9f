"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed-form depth, hand-derived fill-rule and filtering cases, invariants of a
watertight rasteriser, and brute-force ray casting in double precision.

The paper (Sec. 3 "Rendering engine", Sec. 4 "Sensory input") defines the
sensors (pinhole RGB, idealised depth at the same pose, semantic ids) but no
rasterisation rules or pixel values; the rules pinned here are the stated
readings in the oracle's header.
"""
import math
import os

import numpy as np
import pytest

from paper_1904_01201_b300.workloads import Scene, Intrinsics, make_room, random_poses, pinhole_90
from tests.tiny import identity_pose, screen_intr, screen_to_world, scene_from_tris, grid_scene, random_tiny_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BG = 0xFFFFFFFF


# ---------------------------------------------------------------- camera
def test_camera_identity_is_translation(oracle_mod):
    M = oracle_mod.camera([1.0, 2.0, -3.0, 1, 0, 0, 0])
    assert np.array_equal(M[:, :3], np.eye(3, dtype=np.float32))
    assert np.array_equal(M[:, 3], np.array([-1.0, -2.0, 3.0], dtype=np.float32))


def test_camera_yaw_looks_along_rotated_axis(oracle_mod):
    # +90 degrees about +Y turns the viewing direction -Z into -X.
    th = math.pi / 2
    pos = np.array([0.5, 1.5, -2.0])
    M = oracle_mod.camera([*pos, math.cos(th / 2), 0, math.sin(th / 2), 0]).astype(np.float64)
    p = pos + np.array([-3.0, 0.0, 0.0])
    e = M[:, :3] @ p + M[:, 3]
    assert np.allclose(e, [0, 0, -3], atol=1e-6)
    # the camera right axis (+X eye) now points along world -Z
    r = pos + np.array([0.0, 0.0, -1.0])
    er = M[:, :3] @ r + M[:, 3]
    assert np.allclose(er, [1, 0, 0], atol=1e-6)


def test_camera_rotation_properties(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(200):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        pos = rng.uniform(-10, 10, 3)
        M = oracle_mod.camera([*pos, *q]).astype(np.float64)
        R = M[:, :3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        assert np.linalg.det(R) > 0.999
        assert np.allclose(R @ pos + M[:, 3], 0, atol=2e-5 * (1 + np.abs(pos).max()))
        # independent route: rotate the eye -Z axis by the quaternion (Hamilton product)
        w, v = q[0], q[1:]
        fwd = np.array([0, 0, -1.0])
        rot = fwd + 2 * w * np.cross(v, fwd) + 2 * np.cross(v, np.cross(v, fwd))
        assert np.allclose(R.T @ np.array([0, 0, -1.0]), rot, atol=1e-6)


def test_camera_rejects_non_unit_quaternion(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.camera([0, 0, 0, 1.01, 0, 0, 0])
    M = oracle_mod.camera([0, 0, 0, 1.0005, 0, 0, 0])
    assert np.array_equal(M[:, :3], np.eye(3, dtype=np.float32))


# ---------------------------------------------------------------- fill rule
def _read_golden_masks(name):
    cases, cur = [], None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("triangle"):
            parts = line.split()
            cur = (parts[1], [float(v) for v in parts[2:]], [])
            cases.append(cur)
        else:
            cur[2].append([int(c) for c in line])
    return cases


def test_top_left_rule_hand_cases(oracle_mod):
    W = H = 4
    intr = screen_intr(W, H)
    union = np.zeros((H, W), dtype=int)
    for name, v, mask in _read_golden_masks("topleft_4x4.txt"):
        pts = screen_to_world(np.array(v[0::2]), np.array(v[1::2]), W, H, 1.0)
        sc = scene_from_tris([pts])
        out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, coverage=True)
        got = (out["ids"][0] != BG).astype(int)
        assert np.array_equal(got, np.array(mask)), name
        assert np.array_equal(out["cover"][0], np.array(mask)), name
        union += got
    assert union.max() == 1


def test_fan_around_pixel_centre_has_one_owner(oracle_mod):
    W = H = 8
    intr = screen_intr(W, H)
    c = (3.5, 4.5)                     # a pixel centre
    k = 7
    tris = []
    for i in range(k):
        a0, a1 = 2 * math.pi * i / k + 0.1, 2 * math.pi * (i + 1) / k + 0.1
        p = [c, (c[0] + 3 * math.cos(a0), c[1] + 3 * math.sin(a0)), (c[0] + 3 * math.cos(a1), c[1] + 3 * math.sin(a1))]
        pts = screen_to_world(np.array([q[0] for q in p]), np.array([q[1] for q in p]), W, H, 1.0)
        tris.append(pts)
    # shared centre vertex: build with an explicit shared index
    sc = scene_from_tris(tris)
    out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, coverage=True)
    assert out["cover"][0][4, 3] == 1
    assert out["cover"][0].max() == 1


@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_grid_on_pixel_centres_covers_each_pixel_once(oracle_mod, jitter):
    W, H = 16, 12
    intr = screen_intr(W, H)
    rng = np.random.default_rng(7)
    # grid lines at pixel centres (x = 0.5 + 2k), extending beyond the screen
    x0, x1, y0, y1 = -1.5, 17.5, -1.5, 13.5
    corners = screen_to_world(np.array([x0, x1, x0]), np.array([y0, y0, y1]), W, H, 1.0)
    sc = grid_scene(corners, 10, 8, jitter=jitter, rng=rng)
    out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, coverage=True)
    assert np.all(out["cover"][0] == 1)


def test_slanted_subdivided_plane_is_watertight(oracle_mod):
    W, H = 48, 40
    intr = Intrinsics(24.0, 24.0, 24.0, 20.0, 0.05, 50.0)
    rng = np.random.default_rng(3)
    # a tilted plane much larger than the frustum at depths 1..30
    corners = np.array([[-40.0, -20.0, -1.0], [40.0, -20.0, -1.0], [-40.0, 25.0, -30.0]])
    sc = grid_scene(corners, 37, 29, jitter=0.1, rng=rng)   # <= 0.1 cell: no fold-overs
    out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, coverage=True)
    cov = out["cover"][0]
    assert cov.max() == 1
    assert np.all(cov == (out["ids"][0] != BG))
    assert cov.sum() > 0.8 * W * H


# ---------------------------------------------------------------- depth
def test_fronto_parallel_quad_depth_is_exact(oracle_mod):
    W, H = 32, 24
    intr = screen_intr(W, H)
    for D in (0.5, 2.0, 3.0, 7.25):
        c = screen_to_world(np.array([-3.0, 40.0, -3.0, 40.0]), np.array([-3.0, -3.0, 30.0, 30.0]), W, H, D)
        sc = scene_from_tris([[c[0], c[1], c[3]], [c[0], c[3], c[2]]])
        out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, coverage=True)
        assert np.all(out["cover"][0] == 1)
        assert np.all(out["depth"][0] == np.float32(D))
        assert set(np.unique(out["ids"][0])) <= {0, 1}


def test_floor_plane_depth_closed_form(oracle_mod):
    # camera 1.5 m above a floor, pitch 0 (Sec. 4 "Sensory input"); floor
    # trapezoid from d = 2 to d = 8 spanning the 90-degree frustum exactly.
    W = H = 128
    intr = pinhole_90(W, H, 0.01, 10.0)
    v = np.array([[-2, 0, -2], [2, 0, -2], [8, 0, -8], [-8, 0, -8]], dtype=np.float64)
    sc = Scene(xyz=v.astype(np.float32), idx=np.array([[0, 1, 2], [0, 2, 3]], dtype=np.uint32))
    # floor faces up: counter-clockwise seen from above
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if n[1] < 0:
        sc.idx = sc.idx[:, [0, 2, 1]].copy()
    out = oracle_mod.render(sc, identity_pose(0, 1.5, 0)[None], intr, W, H)
    d = out["depth"][0]
    rows = np.arange(H)
    inside = (rows + 0.5 > 76) & (rows + 0.5 < 112)
    assert np.all(out["ids"][0][~inside] == BG)
    assert np.all(out["ids"][0][inside] != BG)
    expect = 1.5 * 64.0 / (rows[inside] + 0.5 - 64.0)
    rel = np.abs(d[inside] / expect[:, None] - 1.0)
    assert rel.max() < 1e-5


def test_near_clipped_wall(oracle_mod):
    # a wall receding from behind the camera to d = 5 crosses the near plane
    W = H = 64
    intr = pinhole_90(W, H, 0.2, 10.0)
    v = np.array([[-1.0, -3, 1.0], [-1.0, -3, -5.0], [-1.0, 3, -5.0], [-1.0, 3, 1.0]])
    idx = np.array([[0, 1, 2], [0, 2, 3]])
    # visible side faces +X (towards the camera at x = 0)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if n[0] < 0:
        idx = idx[:, [0, 2, 1]]
    sc = Scene(xyz=v.astype(np.float32), idx=idx.astype(np.uint32))
    out = oracle_mod.render(sc, identity_pose()[None], intr, W, H)
    d = out["depth"][0]
    hit = out["ids"][0] != BG
    assert hit.sum() > 100
    assert d[hit].min() >= np.float32(0.2) * (1 - 1e-6)
    bf = brute_force(sc, identity_pose(), intr, W, H)
    ok = ~bf["ambiguous"]
    assert np.array_equal(hit[ok], bf["ids"][ok] != BG)
    assert bf["ambiguous"].mean() < 0.05


# ---------------------------------------------------------------- colour
def _fullscreen_quad(W, H, D=1.0, uv=True):
    c = screen_to_world(np.array([0.0, W, 0.0, W]), np.array([0.0, 0.0, H, H]), W, H, D)
    sc = scene_from_tris([[c[0], c[1], c[3]], [c[0], c[3], c[2]]])
    if uv:
        # recover the screen position of each (reordered) vertex for its uv
        f = W / 2.0
        sx = sc.xyz[:, 0] / -sc.xyz[:, 2] * f + W / 2.0
        sy = H / 2.0 - sc.xyz[:, 1] / -sc.xyz[:, 2] * f
        sc.uv = np.stack([sx / W, sy / H], 1).astype(np.float32)
    return sc


def test_bilinear_2x2_hand_values(oracle_mod):
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "bilinear_2x2.txt")) if l.strip() and not l.startswith("#")]
    tex = [int(v) for v in lines[0].split()[1:]]
    expect = np.array([[int(v) for v in l.split()] for l in lines[2:6]])
    W = H = 4
    sc = _fullscreen_quad(W, H)
    atlas = np.zeros((2, 2, 4), dtype=np.uint8)
    atlas[0, 0, 0], atlas[0, 1, 0], atlas[1, 0, 0], atlas[1, 1, 0] = tex
    atlas[..., 3] = 255
    sc.atlas = atlas
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H)
    assert np.array_equal(out["rgb"][0][..., 0], expect)
    assert np.all(out["rgb"][0][..., 1:] == 0)


def test_constant_atlas_and_vertex_colours(oracle_mod):
    W = H = 16
    sc = _fullscreen_quad(W, H)
    sc.atlas = np.zeros((8, 8, 4), dtype=np.uint8)
    sc.atlas[...] = (17, 140, 251, 255)
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H)
    assert np.all(out["rgb"][0] == np.array([17, 140, 251], dtype=np.uint8))
    sc2 = _fullscreen_quad(W, H, uv=False)
    sc2.vrgb = np.tile(np.array([[9, 99, 199]], dtype=np.uint8), (sc2.n_verts, 1))
    out = oracle_mod.render(sc2, identity_pose()[None], screen_intr(W, H), W, H)
    assert np.all(out["rgb"][0] == np.array([9, 99, 199], dtype=np.uint8))
    sc3 = _fullscreen_quad(W, H, uv=False)
    out = oracle_mod.render(sc3, identity_pose()[None], screen_intr(W, H), W, H)
    assert np.all(out["rgb"][0] == 255)


def test_gradient_texture_ramp(oracle_mod):
    W = H = 64
    sc = _fullscreen_quad(W, H)
    atlas = np.zeros((1, 256, 4), dtype=np.uint8)
    atlas[0, :, 0] = np.arange(256)
    sc.atlas = atlas
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H)
    # u = (x + 0.5) / W; texel coordinate s = 256 u - 0.5 -> value s (linear ramp)
    s = 256 * (np.arange(W) + 0.5) / W - 0.5
    assert np.all(np.abs(out["rgb"][0][:, :, 0].astype(float) - np.round(s)[None, :]) <= 1)


def test_perspective_correct_texture_on_floor(oracle_mod):
    W = H = 128
    intr = pinhole_90(W, H, 0.01, 10.0)
    v = np.array([[-2, 0, -2], [2, 0, -2], [8, 0, -8], [-8, 0, -8]], dtype=np.float64)
    uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    idx = np.array([[0, 1, 2], [0, 2, 3]])
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if n[1] < 0:
        idx = idx[:, [0, 2, 1]]
    atlas = np.zeros((256, 1, 4), dtype=np.uint8)
    atlas[:, 0, 0] = np.arange(256)
    sc = Scene(xyz=v.astype(np.float32), idx=idx.astype(np.uint32), uv=uv, atlas=atlas)
    out = oracle_mod.render(sc, identity_pose(0, 1.5, 0)[None], intr, W, H)
    rows = np.arange(76, 112)
    d = 96.0 / (rows + 0.5 - 64.0)
    vv = (d - 2.0) / 6.0                      # v is linear along the floor in the world
    expect = np.clip(np.round(256 * vv - 0.5), 0, 255)
    got = out["rgb"][0][rows][:, :, 0].astype(float)
    assert np.all(np.abs(got - expect[:, None]) <= 1)


def _round_half_up(c):
    return np.clip(np.floor(np.asarray(c, dtype=np.float64) + 0.5), 0, 255)


def test_vertex_colours_linear_on_fronto_parallel_quad(oracle_mod):
    # Distinct vertex colours that are a linear function of the screen
    # position of a fronto-parallel quad (constant depth): every interpolated
    # pixel must equal that function at its centre. Pairing a weight with the
    # wrong vertex moves the ramps by up to their whole range.
    W, H = 16, 12
    sc = _fullscreen_quad(W, H, uv=False)
    f = W / 2.0
    sx = sc.xyz[:, 0].astype(np.float64) / -sc.xyz[:, 2] * f + W / 2.0
    sy = H / 2.0 - sc.xyz[:, 1].astype(np.float64) / -sc.xyz[:, 2] * f
    # corners sit at sx in {0, W}, sy in {0, H}: integer channel values there
    col = np.stack([255 * sx / W, 255 * sy / H, 40 + 120 * sx / W + 60 * sy / H], 1)
    assert np.allclose(col, np.round(col), atol=1e-9)
    sc.vrgb = np.round(col).astype(np.uint8)
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H)
    px = np.arange(W) + 0.5
    py = np.arange(H) + 0.5
    X, Y = np.meshgrid(px, py)
    expect = np.stack([255 * X / W, 255 * Y / H, 40 + 120 * X / W + 60 * Y / H], -1)
    got = out["rgb"][0].astype(np.float64)
    assert np.all(np.abs(got - _round_half_up(expect)) <= 1)
    assert np.mean(got != _round_half_up(expect)) < 0.02


def test_vertex_colours_perspective_correct_on_floor(oracle_mod):
    # Camera 1.5 m above a floor trapezoid from d = 2 to d = 8 (pitch 0, the
    # 90-degree pinhole of Sec. 4). Vertex colours are linear in world x and
    # depth d, so at every pixel the colour is that linear function at the
    # floor point its centre ray hits: d = h fy / (y + 1/2 - cy),
    # x = (x_px + 1/2 - cx) d / fx. Affine (screen-linear) weights get the
    # red ramp wrong by tens of units in the middle rows.
    W = H = 128
    intr = pinhole_90(W, H, 0.01, 10.0)
    v = np.array([[-2, 0, -2], [2, 0, -2], [8, 0, -8], [-8, 0, -8]], dtype=np.float64)
    idx = np.array([[0, 1, 2], [0, 2, 3]])
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if n[1] < 0:
        idx = idx[:, [0, 2, 1]]
    d_v, x_v = -v[:, 2], v[:, 0]

    def colour(x, d):
        return np.stack([40 * (d - 2), 15 * (x + 8), 10 + 20 * (d - 2) + 5 * (x + 8)], -1)

    cv = colour(x_v, d_v)
    assert np.allclose(cv, np.round(cv)) and cv.min() >= 0 and cv.max() <= 255
    sc = Scene(xyz=v.astype(np.float32), idx=idx.astype(np.uint32), vrgb=np.round(cv).astype(np.uint8))
    out = oracle_mod.render(sc, identity_pose(0, 1.5, 0)[None], intr, W, H)
    hit = out["ids"][0] != BG
    rows = np.arange(76, 112)
    assert np.all(hit[rows].sum(1) > 0)
    d = 1.5 * 64.0 / (rows + 0.5 - 64.0)
    X = (np.arange(W)[None, :] + 0.5 - 64.0) * d[:, None] / 64.0
    expect = _round_half_up(colour(X, np.repeat(d[:, None], W, 1)))
    got = out["rgb"][0][rows].astype(np.float64)
    m = hit[rows]
    # one snapped vertex moves the floor by under 2^-9 px: within one unit
    assert np.all(np.abs(got[m] - expect[m]) <= 1)


def test_near_clipped_floor_interpolates_uv_at_the_clip_points(oracle_mod):
    # A textured floor from behind the camera (d = -2) to d = 8 crosses the
    # near plane, so the visible part of its triangles comes from the
    # clipped polygons, whose new vertices carry uv interpolated along the
    # clipped edges. With u linear in world x, v linear in world depth and a
    # texture holding (R, G) = (row, column), each pixel's colour is fixed by
    # the floor point its centre ray hits; a clip point with the wrong uv
    # (swapped endpoints, t measured from the other end) bends the ramps.
    W = H = 64
    near = 0.25
    intr = pinhole_90(W, H, near, 10.0)
    h = 0.3
    v = np.array([[-10, 0, 2], [10, 0, 2], [10, 0, -8], [-10, 0, -8]], dtype=np.float64)
    idx = np.array([[0, 1, 2], [0, 2, 3]])
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if n[1] < 0:
        idx = idx[:, [0, 2, 1]]
    uv = np.stack([(v[:, 0] + 10) / 20, (-v[:, 2] + 2) / 10], 1).astype(np.float32)
    atlas = np.zeros((256, 256, 4), dtype=np.uint8)
    atlas[..., 0] = np.arange(256)[:, None]
    atlas[..., 1] = np.arange(256)[None, :]
    sc = Scene(xyz=v.astype(np.float32), idx=idx.astype(np.uint32), uv=uv, atlas=atlas)
    pose = identity_pose(0, h, 0)
    out = oracle_mod.render(sc, pose[None], intr, W, H)
    hit = out["ids"][0] != BG
    rows = np.arange(H // 2 + 1, H)          # below the horizon
    assert hit[rows].all()
    d = h * 32.0 / (rows + 0.5 - 32.0)
    assert d.min() > near and d.max() < 8
    X = (np.arange(W)[None, :] + 0.5 - 32.0) * d[:, None] / 32.0
    u = (X + 10) / 20
    vv = (np.repeat(d[:, None], W, 1) + 2) / 10
    # texel row t = 256 v - 1/2 holds the value t (a ramp): bilinear returns t
    expect_r = _round_half_up(256 * vv - 0.5)
    expect_g = _round_half_up(256 * u - 0.5)
    got = out["rgb"][0][rows].astype(np.float64)
    assert np.all(np.abs(got[..., 0] - expect_r) <= 1)
    assert np.all(np.abs(got[..., 1] - expect_g) <= 1)
    # both floor triangles reach behind the camera: every hit pixel is shaded
    # from a clipped polygon
    d_tri = -v[idx][:, :, 2]
    assert np.all((d_tri < near).any(1))


# ---------------------------------------------------------------- invariants
def test_order_and_rotation_independence(oracle_mod):
    sc = make_room(2, 4000)
    poses = random_poses(sc, 3, 5)
    intr = pinhole_90(64, 64)
    base = oracle_mod.render(sc, poses, intr, 64, 64)
    rng = np.random.default_rng(0)
    perm = rng.permutation(sc.n_tris)
    sp = Scene(xyz=sc.xyz, idx=sc.idx[perm].copy(), vrgb=sc.vrgb)
    o = oracle_mod.render(sp, poses, intr, 64, 64)
    ids = np.where(o["ids"] == BG, BG, perm[np.minimum(o["ids"], sc.n_tris - 1)])
    assert np.array_equal(ids, base["ids"])
    assert np.array_equal(o["depth"], base["depth"])
    assert np.array_equal(o["rgb"], base["rgb"])
    sr = Scene(xyz=sc.xyz, idx=sc.idx[:, [1, 2, 0]].copy(), vrgb=sc.vrgb)
    o = oracle_mod.render(sr, poses, intr, 64, 64)
    for k in ("ids", "depth", "rgb"):
        assert np.array_equal(o[k], base[k]), k


def test_semantic_table_and_background(oracle_mod):
    sc = make_room(1, 2000)
    sc.sem = (np.arange(sc.n_tris, dtype=np.uint32) * 7 + 3)
    poses = random_poses(sc, 2, 1)
    intr = pinhole_90(32, 32)
    a = oracle_mod.render(Scene(xyz=sc.xyz, idx=sc.idx, vrgb=sc.vrgb), poses, intr, 32, 32)
    b = oracle_mod.render(sc, poses, intr, 32, 32)
    hit = a["ids"] != BG
    assert np.array_equal(b["ids"][hit], a["ids"][hit] * 7 + 3)
    # a pose looking at nothing: everything is background
    empty = Scene(xyz=np.array([[0, 0, 5], [1, 0, 5], [0, 1, 5]], dtype=np.float32),
                  idx=np.array([[0, 1, 2]], dtype=np.uint32))
    o = oracle_mod.render(empty, identity_pose()[None], intr, 32, 32)
    assert np.all(o["ids"] == BG) and np.all(o["depth"] == 0) and np.all(o["rgb"] == 0)


def test_far_plane_discards_per_fragment(oracle_mod):
    W = H = 32
    intr = screen_intr(W, H, 0.01, 4.0)
    # fronto-parallel quads at 3.9 (kept) and 4.1 (discarded)
    for D, kept in ((3.9, True), (4.1, False)):
        c = screen_to_world(np.array([0.0, W, 0.0, W]), np.array([0.0, 0.0, H, H]), W, H, D)
        sc = scene_from_tris([[c[0], c[1], c[3]], [c[0], c[3], c[2]]])
        o = oracle_mod.render(sc, identity_pose()[None], intr, W, H)
        assert np.all((o["ids"][0] != BG) == kept)


def test_invalid_inputs(oracle_mod):
    sc = Scene(xyz=np.zeros((3, 3), np.float32), idx=np.array([[0, 1, 3]], np.uint32))
    with pytest.raises(ValueError):
        oracle_mod.render(sc, identity_pose()[None], screen_intr(8, 8), 8, 8)
    sc = Scene(xyz=np.zeros((3, 3), np.float32), idx=np.array([[0, 1, 2]], np.uint32))
    with pytest.raises(ValueError):
        oracle_mod.render(sc, np.array([[0, 0, 0, 2, 0, 0, 0]], np.float32), screen_intr(8, 8), 8, 8)


# ---------------------------------------------------------------- brute force
def _rodrigues(axis, ang):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def brute_force(scene, pose, intr, W, H, R=None, delta=2.0 ** -7):
    """Nearest front-facing ray-triangle hit per pixel centre (Moller-Trumbore, float64).

    R is the world-from-camera rotation; if None it is taken as identity
    (only valid for identity-quaternion poses)."""
    fx, fy, cx, cy, near, far = [float(v) for v in getattr(intr, "as_array", lambda: intr)()]
    pos = np.asarray(pose[:3], dtype=np.float64)
    R = np.eye(3) if R is None else R
    tri = scene.xyz.astype(np.float64)[scene.idx.astype(np.int64)]          # [T,3,3]
    e1 = tri[:, 1] - tri[:, 0]
    e2 = tri[:, 2] - tri[:, 0]
    nrm = np.cross(e1, e2)
    results = []
    offs = [(0, 0), (delta, delta), (-delta, delta), (delta, -delta), (-delta, -delta)]
    second = None
    grazing = None
    for ox, oy in offs:
        xs = (np.arange(W) + 0.5 + ox - cx) / fx
        ys = -(np.arange(H) + 0.5 + oy - cy) / fy
        X, Y = np.meshgrid(xs, ys)
        de = np.stack([X, Y, -np.ones_like(X)], -1).reshape(-1, 3)            # eye dirs, d-component 1
        dw = de @ R.T                                                       # world dirs
        p = np.cross(dw[:, None, :], e2[None])                               # [P,T,3]
        det = np.einsum("ptk,tk->pt", p, e1)
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / det
            s = pos[None, None, :] - tri[None, :, 0]
            u = np.einsum("ptk,ptk->pt", s, p) * inv
            qv = np.cross(s, e1[None])
            v = np.einsum("pk,ptk->pt", dw, qv) * inv
            t = np.einsum("tk,ptk->pt", e2, qv) * inv
        front = np.einsum("pk,tk->pt", dw, nrm) < 0
        ok = (u >= 0) & (v >= 0) & (u + v <= 1) & (t >= near) & (t <= far) & front & np.isfinite(t)
        tt = np.where(ok, t, np.inf)
        best = np.argmin(tt, axis=1)
        bt = tt[np.arange(len(best)), best]
        ids = np.where(np.isfinite(bt), best, BG).astype(np.int64)
        results.append((ids, bt))
        if second is None:
            srt = np.sort(tt, axis=1)
            second = srt[:, 1] if tt.shape[1] > 1 else np.full(len(best), np.inf)
            cosang = np.abs(np.einsum("pk,tk->pt", dw, nrm)) / (
                np.linalg.norm(dw, axis=1)[:, None] * np.linalg.norm(nrm, axis=1)[None] + 1e-300)
            grazing = np.any((cosang < 1e-3) & np.isfinite(np.where((u >= -1e-3) & (v >= -1e-3) & (u + v <= 1 + 1e-3), t, np.inf)), axis=1)
    ids0, t0 = results[0]
    amb = np.zeros(len(ids0), dtype=bool)
    spread = np.zeros(len(ids0))
    fin = np.isfinite(t0)
    for ids, tj in results[1:]:
        amb |= ids != ids0
        spread = np.maximum(spread, np.where(fin & np.isfinite(tj), np.abs(tj - t0), 0.0))
    with np.errstate(invalid="ignore"):
        amb |= fin & (np.abs(np.where(fin, second, 0) - np.where(fin, t0, 0)) <= 1e-6 * np.abs(np.where(fin, t0, 1)))
    amb |= fin & ((np.abs(t0 - near) < 1e-4 * near) | (np.abs(t0 - far) < 1e-4 * far))
    amb |= grazing
    return {"ids": np.where(ids0 == BG, BG, ids0).reshape(H, W).astype(np.uint32),
            "depth": np.where(fin, t0, 0).reshape(H, W), "ambiguous": amb.reshape(H, W),
            "spread": spread.reshape(H, W)}


@pytest.mark.parametrize("block", range(4))
def test_brute_force_ray_casting(oracle_mod, block):
    rng = np.random.default_rng(100 + block)
    n_trials, amb_total, px_total = 400, 0, 0
    for trial in range(n_trials):
        W, H = int(rng.integers(8, 40)), int(rng.integers(8, 40))
        T = int(rng.integers(1, 51))
        sc = random_tiny_scene(rng, T)
        axis = rng.normal(size=3)
        ang = float(rng.uniform(-0.6, 0.6))
        R = _rodrigues(axis, ang)
        ax = axis / np.linalg.norm(axis)
        quat = np.array([math.cos(ang / 2), *(math.sin(ang / 2) * ax)])
        pos = rng.uniform(-0.3, 0.3, 3)
        pose = np.array([*pos, *quat], dtype=np.float32)
        f = float(rng.uniform(0.3, 1.2)) * W
        intr = Intrinsics(f, f * float(rng.uniform(0.8, 1.25)), W / 2 + float(rng.uniform(-2, 2)),
                          H / 2 + float(rng.uniform(-2, 2)), 0.05, 6.0)
        o = oracle_mod.render(sc, pose[None], intr, W, H)
        # the pose is stored in float32: cast the exact rotation through the same path
        bf = brute_force(sc, pose.astype(np.float64), intr, W, H, R=_rot_from_float_quat(pose))
        ok = ~bf["ambiguous"]
        assert np.array_equal(o["ids"][0][ok], bf["ids"][ok]), (trial, W, H, T)
        hit = ok & (bf["ids"] != BG)
        if hit.any():
            # snapping moves vertices by <= 2^-9 px; the ray's own depth change
            # over +-2^-7 px bounds the effect on the interpolated depth
            err = np.abs(o["depth"][0][hit].astype(np.float64) - bf["depth"][hit])
            assert np.all(err <= bf["spread"][hit] + 2e-6 * bf["depth"][hit]), (trial, err.max())
        amb_total += int(bf["ambiguous"].sum())
        px_total += W * H
    assert amb_total / px_total < 0.01


def _rot_from_float_quat(pose):
    """Rotation of the float32 quaternion by Rodrigues' formula (axis-angle route)."""
    q = pose[3:].astype(np.float64)
    q = q / np.linalg.norm(q)
    w = np.clip(q[0], -1, 1)
    ang = 2 * math.acos(w)
    s = math.sqrt(max(0.0, 1 - w * w))
    if s < 1e-12:
        return np.eye(3)
    return _rodrigues(q[1:] / s, ang)


# ---------------------------------------------------------------- guard band
def _max_snap(scene, pose, intr):
    """Largest |256 s| over the scene's vertices in front of the near plane
    and its near-plane crossing points (double precision, identity rotation)."""
    fx, fy, cx, cy, near, far = [float(v) for v in intr.as_array()]
    e = scene.xyz.astype(np.float64) - np.asarray(pose[:3], dtype=np.float64)
    best = 0.0
    for tri in scene.idx.astype(np.int64):
        pts = [e[i] for i in tri]
        for a in range(3):
            p, r = pts[a], pts[(a + 1) % 3]
            dp, dr = -p[2], -r[2]
            cand = [p] if dp >= near else []
            if (dp >= near) != (dr >= near):
                t = (near - dp) / (dr - dp)
                cand.append(p + t * (r - p))
            for c in cand:
                d = max(-c[2], near)
                best = max(best, abs(256 * (fx * c[0] / d + cx)), abs(256 * (-fy * c[1] / d + cy)))
    return best


def _clip64(poly, gx, gy):
    """Sutherland-Hodgman in float64 against x >= -gx d, x <= gx d,
    y >= -gy d, y <= gy d (the exact clip the float32 one approximates)."""
    pts = [np.asarray(p, dtype=np.float64) for p in poly]
    for k in range(4):
        g, comp, sgn = (gx, 0, 1.0) if k == 0 else (gx, 0, -1.0) if k == 1 else (gy, 1, 1.0) if k == 2 else (gy, 1, -1.0)
        dist = [g * p[2] + sgn * p[comp] for p in pts]
        out = []
        for i in range(len(pts)):
            j = (i + 1) % len(pts)
            if dist[i] >= 0:
                out.append(pts[i])
            if (dist[i] >= 0) != (dist[j] >= 0):
                t = dist[i] / (dist[i] - dist[j])
                out.append(pts[i] + t * (pts[j] - pts[i]))
        pts = out
        if not pts:
            break
    return np.array(pts).reshape(-1, 3)


def test_guard_clip_points_lie_on_the_cut_edges(oracle_mod):
    # Polygons with vertices from 1e-6 m to 10 m deep and up to 10 m to the
    # side, so that cuts fall close to one endpoint of edges whose other
    # endpoint is 10^6 times farther: each cut point must agree with the
    # float64 clip to float precision of its own size (a cut computed from
    # the far endpoint is off by that endpoint's rounding, up to ~10 %).
    rng = np.random.default_rng(9)
    gx, gy = np.float32(2.0 ** 21) / np.float32(24.0), np.float32(2.0 ** 21) / np.float32(30.0)
    checked = 0
    for trial in range(3000):
        n = int(rng.integers(3, 5))
        d = 10.0 ** rng.uniform(-6, 1, n)
        poly = np.stack([rng.uniform(-10, 10, n), rng.uniform(-10, 10, n), d], 1).astype(np.float32)
        got = oracle_mod.guard_clip(poly, gx, gy)
        ref = _clip64(poly.astype(np.float64), float(gx), float(gy))
        if len(got) != len(ref):
            continue                    # a vertex within rounding of a plane
        checked += 1
        assert np.all(np.abs(got[:, 2] - ref[:, 2]) <= 1e-5 * ref[:, 2]), trial
        scale = np.abs(ref[:, :2]) + np.array([gx, gy]) * ref[:, 2:3]
        assert np.all(np.abs(got[:, :2] - ref[:, :2]) <= 1e-5 * scale), trial
    assert checked > 2900


def test_guard_band_huge_fronto_parallel_quad(oracle_mod):
    # A quad at depth D reaching 10^6 m to every side: all four vertices snap
    # far beyond +-2^30 sub-pixels, so both triangles are clipped to the
    # guard band. The clipped polygons keep the quad's plane (d = D at every
    # clip point), so every pixel is covered exactly once at depth D exactly,
    # and the shared diagonal, which crosses the screen, leaves no crack.
    W, H = 40, 24
    for D in (1.0, 0.5, 4.0):
        c = np.array([[-1e6, -1e6, -D], [1e6, -1e6, -D], [-1e6, 1e6, -D], [1e6, 1e6, -D]])
        for diag in (0, 1):
            tris = [[c[0], c[1], c[3]], [c[0], c[3], c[2]]] if diag == 0 else [[c[0], c[1], c[2]], [c[1], c[3], c[2]]]
            sc = scene_from_tris(tris)
            intr = screen_intr(W, H)
            assert _max_snap(sc, identity_pose(), intr) > 2.0 ** 30
            out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, coverage=True)
            assert np.all(out["cover"][0] == 1)
            assert np.all(out["depth"][0] == np.float32(D))


def test_guard_band_floor_interpolates_uv_at_guard_points(oracle_mod):
    # The near-clipped floor of the near-clip pin with a near plane of 2e-6 m:
    # its clip points project ~10^9 pixels below the image, so the polygons
    # are clipped again at the guard planes (bottom, left and right), and
    # every visible pixel is shaded through guard-clip vertices. u is linear
    # in world x, v in depth; the colour must follow the closed form.
    W = H = 64
    near = 2e-6
    intr = Intrinsics(32.0, 32.0, 32.0, 32.0, near, 10.0)
    h = 0.3
    v = np.array([[-10, 0, 2], [10, 0, 2], [10, 0, -8], [-10, 0, -8]], dtype=np.float64)
    idx = np.array([[0, 1, 2], [0, 2, 3]])
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if n[1] < 0:
        idx = idx[:, [0, 2, 1]]
    uv = np.stack([(v[:, 0] + 10) / 20, (-v[:, 2] + 2) / 10], 1).astype(np.float32)
    atlas = np.zeros((256, 256, 4), dtype=np.uint8)
    atlas[..., 0] = np.arange(256)[:, None]
    atlas[..., 1] = np.arange(256)[None, :]
    sc = Scene(xyz=v.astype(np.float32), idx=idx.astype(np.uint32), uv=uv, atlas=atlas)
    pose = identity_pose(0, h, 0)
    assert _max_snap(sc, pose, intr) > 2.0 ** 33
    out = oracle_mod.render(sc, pose[None], intr, W, H)
    rows = np.arange(H // 2 + 1, H)
    assert (out["ids"][0][rows] != BG).all()
    d = h * 32.0 / (rows + 0.5 - 32.0)
    X = (np.arange(W)[None, :] + 0.5 - 32.0) * d[:, None] / 32.0
    expect_r = _round_half_up(256 * (np.repeat(d[:, None], W, 1) + 2) / 10 - 0.5)
    expect_g = _round_half_up(256 * (X + 10) / 20 - 0.5)
    got = out["rgb"][0][rows].astype(np.float64)
    assert np.all(np.abs(got[..., 0] - expect_r) <= 1)
    assert np.all(np.abs(got[..., 1] - expect_g) <= 1)
    # and the floor's depth follows d = h fy / (y + 1/2 - cy), i.e. q is
    # (y + 1/2 - cy) / (h fy): snapping moves each vertex by at most 2^-9 px,
    # which moves q by at most 2^-9 / (h fy) per unit of slope (doubled here)
    q_true = (rows + 0.5 - 32.0) / (h * 32.0)
    q_got = 1.0 / out["depth"][0][rows].astype(np.float64)
    assert np.all(np.abs(q_got - q_true[:, None]) <= 2.0 ** -8 / (h * 32.0) + 1e-6 * q_true[:, None])


@pytest.mark.parametrize("block", range(2))
def test_guard_band_random_scenes_vs_ray_casting(oracle_mod, block):
    # Random scenes around the camera with near planes of 1e-6 .. 1e-5 m and
    # fx != fy: triangles reaching behind the camera are near-clipped at
    # points that project far outside the fixed-point range, then clipped to
    # the guard band. Ids must equal the float64 ray cast on every
    # unambiguous pixel.
    rng = np.random.default_rng(500 + block)
    n_guard = 0
    amb_total = px_total = 0
    for trial in range(60):
        W, H = int(rng.integers(8, 40)), int(rng.integers(8, 40))
        T = int(rng.integers(4, 40))
        sc = random_tiny_scene(rng, T)
        f = float(rng.uniform(0.4, 1.2)) * W
        intr = Intrinsics(f, f * float(rng.uniform(0.7, 1.4)), W / 2 + float(rng.uniform(-2, 2)),
                          H / 2 + float(rng.uniform(-2, 2)), float(10 ** rng.uniform(-6, -5)), 6.0)
        pose = identity_pose()
        n_guard += _max_snap(sc, pose, intr) >= 2.0 ** 30
        o = oracle_mod.render(sc, pose[None], intr, W, H)
        bf = brute_force(sc, pose.astype(np.float64), intr, W, H)
        ok = ~bf["ambiguous"]
        assert np.array_equal(o["ids"][0][ok], bf["ids"][ok]), (trial, W, H, T)
        amb_total += int(bf["ambiguous"].sum())
        px_total += W * H
    assert n_guard >= 30
    assert amb_total / px_total < 0.02


def test_equal_depth_ties_go_to_lower_index(oracle_mod):
    # coincident coplanar triangles give equal keys' depth parts: the lower
    # triangle index must win every tie, whatever the submission order
    W = H = 16
    c = screen_to_world(np.array([1.0, 14.0, 2.0]), np.array([1.0, 3.0, 15.0]), W, H, 2.0)
    sc = scene_from_tris([c, c, c])
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H, coverage=True)
    hit = out["ids"][0] != BG
    assert hit.sum() > 20
    assert np.all(out["ids"][0][hit] == 0)
    assert np.all(out["cover"][0][hit] == 3)


def test_depth_within_winning_triangle_vertex_range(oracle_mod):
    # Every point of a triangle lies between its vertices' depths; long thin
    # slivers with strong depth variation are where rounding of the plane
    # evaluation would otherwise step outside that range.
    rng = np.random.default_rng(1)
    W, H = 512, 320
    intr = Intrinsics(256.0, 256.0, 256.0, 160.0, 0.05, 100.0)
    violations = 0
    for trial in range(12):
        tris = []
        for _ in range(200):
            a = rng.uniform([-3, -2, -1.0], [3, 2, -0.3])
            b = rng.uniform([-3, -2, -60.0], [3, 2, -20.0])
            c = a + (b - a) * rng.uniform(0.2, 0.8) + rng.normal(scale=1e-4, size=3)
            tris.append(np.array([a, b, c]))
        sc = scene_from_tris(tris)
        o = oracle_mod.render(sc, identity_pose()[None], intr, W, H)
        ids, dep = o["ids"][0], o["depth"][0]
        hit = ids != BG
        d = -sc.xyz[sc.idx.astype(np.int64)][:, :, 2].astype(np.float64)     # vertex depths (identity camera)
        lo, hi = d.min(1)[ids[hit]], d.max(1)[ids[hit]]
        dd = dep[hit].astype(np.float64)
        violations += int(((dd < lo * (1 - 1e-6)) | (dd > hi * (1 + 1e-6))).sum())
    assert violations == 0
