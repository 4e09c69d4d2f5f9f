"""Pins of the oracle's trilinear (mipmapped) texture sampling, the reading
for minified textures: the mip chain against a hand-derived chain, level of
detail against closed forms (exact texel-to-pixel ratios; a textured floor
seen in perspective), and the blend weight against the extreme colours of a
stripe pattern whose two blended levels are known."""
import math
import os

import numpy as np
import pytest

from tests.tiny import identity_pose, scene_from_tris, screen_intr, screen_to_world

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    blocks, cur = {}, None
    for line in open(os.path.join(GOLDEN, "mip_4x4.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            cur = tuple(line.split())
            blocks[cur] = []
        else:
            blocks[cur].append([int(v) for v in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def _quad(W, H, su=1.0, sv=1.0):
    """Screen-filling quad at depth 1, uv = (su * sx / W, sv * sy / H)."""
    c = screen_to_world(np.array([0.0, W, 0.0, W]), np.array([0.0, 0.0, H, H]), W, H, 1.0)
    sc = scene_from_tris([[c[0], c[1], c[3]], [c[0], c[3], c[2]]])
    f = W / 2.0
    sx = sc.xyz[:, 0] / -sc.xyz[:, 2] * f + W / 2.0
    sy = H / 2.0 - sc.xyz[:, 1] / -sc.xyz[:, 2] * f
    sc.uv = np.stack([su * sx / W, sv * sy / H], 1).astype(np.float32)
    return sc


def test_mip_chain_read_back_at_integer_lod(oracle_mod):
    """A 4x4 texture seen at 1, 2 and 4 texels per pixel, pixel centres on
    texel centres of level 0, 1 and 2: the image is that level, texel for
    texel, and lambda is that level."""
    g = _golden()
    atlas = np.zeros((4, 4, 4), dtype=np.uint8)
    atlas[..., 0] = g[("level0", "red")]
    atlas[..., 1] = 255 - g[("level0", "red")]
    atlas[..., 2] = g[("level0", "blue")]
    atlas[..., 3] = 255
    for level, W in ((0, 4), (1, 2), (2, 1)):
        sc = _quad(W, W)
        sc.atlas = atlas
        out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, W), W, W, trilinear=True, lod=True)
        img = out["rgb"][0].astype(np.int64)
        if level == 0:
            want = [atlas[..., 0], atlas[..., 1], atlas[..., 2]]
        else:
            want = [g[(f"level{level}", c)] for c in ("red", "green", "blue")]
        for c in range(3):
            assert np.array_equal(img[..., c], want[c]), (level, c)
        assert np.allclose(out["lod"][0], level, atol=1e-9)


def test_odd_sized_chain(oracle_mod):
    """A 6x2 texture: level 1 is 3x1 (read back at 2 texels per pixel),
    level 2 is 1x1 (a single pixel sees the whole texture, lambda =
    log2 6 beyond the last level)."""
    g = _golden()
    atlas = np.zeros((2, 6, 4), dtype=np.uint8)
    atlas[..., 0] = g[("odd6x2", "level0", "red")]
    atlas[..., 3] = 255
    sc = _quad(3, 1)
    sc.atlas = atlas
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(3, 1), 3, 1, trilinear=True, lod=True)
    assert np.allclose(out["lod"][0], 1.0, atol=1e-9)
    assert np.array_equal(out["rgb"][0][..., 0], g[("odd6x2", "level1", "red")])
    sc = _quad(1, 1)
    sc.atlas = atlas
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(1, 1), 1, 1, trilinear=True, lod=True)
    assert np.allclose(out["lod"][0], math.log2(6.0), atol=1e-9)
    assert np.array_equal(out["rgb"][0][..., 0], g[("odd6x2", "level2", "red")])


def test_magnified_texture_equals_plain_bilinear(oracle_mod):
    """Below one texel per pixel (lambda <= 0) trilinear sampling is the plain
    bilinear rule, bit for bit."""
    W = H = 16
    sc = _quad(W, H, 0.5, 0.75)
    rs = np.random.default_rng(3)
    sc.atlas = rs.integers(0, 256, (8, 8, 4), dtype=np.uint8)
    a = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H, trilinear=True, lod=True)
    b = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H)
    assert np.array_equal(a["rgb"], b["rgb"])
    assert np.all(a["lod"] <= 0)


@pytest.mark.parametrize("level", [0, 1])
def test_fractional_lod_blend_weight(oracle_mod, level):
    """Stripes of period 2^(l+1) texels in x (half 0, half 255): level l
    alternates 0 / 255 texel by texel, level l+1 is 128 everywhere. At
    2^(l + 0.25) texels per pixel, lambda = l + 0.25, so colours are
    0.75 * (level-l sample) + 0.25 * 128: over a wide row they reach from 32
    up to 223."""
    W, H = 256, 4
    r = 2.0 ** (level + 0.25)
    W0, H0 = 1024, 16
    sc = _quad(W, H, r * W / W0, r * H / H0)
    atlas = np.zeros((H0, W0, 4), dtype=np.uint8)
    period = 2 ** (level + 1)
    atlas[:, (np.arange(W0) % period) >= period // 2, :3] = 255
    sc.atlas = atlas
    out = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H), W, H, trilinear=True, lod=True)
    assert np.allclose(out["lod"][0], level + 0.25, atol=1e-9)
    red = out["rgb"][0][..., 0].astype(np.int64)
    assert 32 <= red.min() <= 34 and 221 <= red.max() <= 223, (red.min(), red.max())


def test_floor_lod_closed_form(oracle_mod):
    """A textured floor 1.5 m below a level camera, uv = world (x, z) * s:
    at a pixel centre (sx, sy) below the horizon the hit lies at depth
    d = h fy / (sy - cy), so du/dx = s d / fx, dv/dx = 0, du/dy =
    -s (sx - cx) d^2 / (fx h fy), dv/dy = s d^2 / (h fy); lambda =
    log2 max(W0 |du/dx|, |(W0 du/dy, H0 dv/dy)|)."""
    W = H = 64
    h, s, W0, H0 = 1.5, 0.02, 512, 256
    intr = screen_intr(W, H, 0.01, 100.0)
    fx = fy = W / 2.0
    cx, cy = W / 2.0, H / 2.0
    L = 40.0
    p = np.array([[-L, -h, -L], [L, -h, -L], [L, -h, 0.5], [-L, -h, 0.5]])
    sc = scene_from_tris([[p[0], p[2], p[1]], [p[0], p[3], p[2]]])
    sc.uv = (np.stack([sc.xyz[:, 0], sc.xyz[:, 2]], 1) * s).astype(np.float32)
    sc.atlas = np.full((H0, W0, 4), 200, dtype=np.uint8)
    out = oracle_mod.render(sc, identity_pose()[None], intr, W, H, trilinear=True, lod=True)
    lod = out["lod"][0]
    ys, xs = np.nonzero(np.isfinite(lod))
    assert len(ys) > 500
    sxc, syc = xs + 0.5, ys + 0.5
    d = h * fy / (syc - cy)
    dudx = s * d / fx
    dudy = -s * (sxc - cx) * d * d / (fx * h * fy)
    dvdy = s * d * d / (h * fy)
    rho = np.maximum(W0 * dudx, np.hypot(W0 * dudy, H0 * dvdy))
    want = np.log2(rho)
    err = np.abs(lod[ys, xs] - want)
    assert err.max() < 2e-3, err.max()
    # the floor is minified far away and magnified up close
    assert lod[ys, xs].max() > 3 and lod[ys, xs].min() < 0
