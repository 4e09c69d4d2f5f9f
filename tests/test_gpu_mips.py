"""Trilinear (mipmapped) texture sampling on the CUDA path vs the oracle:
ids and depth bit-exact (sampling changes colour only), RGB within 1/255
(the oracle computes lambda and the blend in fp64, the kernel in fp32; the
colour is continuous in lambda, including across level boundaries, so the
difference stays below one step after rounding)."""
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
from paper_1904_01201_b300.workloads import Intrinsics  # noqa: E402
from tests.test_gpu_parity import assert_parity, gpu_render  # noqa: E402
from tests.test_oracle_mips import _golden, _quad  # noqa: E402
from tests.tiny import identity_pose, screen_intr  # noqa: E402


def _render(sc, poses, intr, W, H, mode):
    h = hsr.SceneHandle(sc)
    h.set_sampling(mode)
    out = hsr.render(h, poses, intr, W, H, ids=True)
    torch.cuda.synchronize()
    res = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}
    h.close()
    return res


@pytest.mark.parametrize("W,H,atlas", [(64, 64, 4096), (97, 41, 1024)])
def test_house_trilinear_matches_oracle(oracle_mod, W, H, atlas):
    """A textured house seen at low resolution: most surfaces are minified by
    several levels; near walls are magnified or near-clipped."""
    sc = wl.make_house(51, 60_000, atlas)
    poses = wl.random_poses(sc, 6, 3)
    intr = Intrinsics(W / 2, W / 2, W / 2, H / 2, 0.01, 10.0)
    g = _render(sc, poses, intr, W, H, hsr.HSR_SAMPLE_TRILINEAR)
    o = oracle_mod.render(sc, poses, intr, W, H, trilinear=True, lod=True)
    hit = np.isfinite(o["lod"])
    # both regimes occur: minified by more than a level, and magnified
    assert (o["lod"][hit] > 1).mean() > 0.05 and (o["lod"][hit] <= 0).mean() > 0.01
    diff = np.abs(g["rgb"].astype(np.int16) - o["rgb"].astype(np.int16))
    assert diff.max() <= 1, f"rgb off by {diff.max()} at {int((diff > 1).sum())} channels"
    assert np.array_equal(g["ids"], o["ids"]) and np.array_equal(g["depth"].view(np.uint32), o["depth"].view(np.uint32))
    # sampling mode switches back: bilinear is the plain rule again
    b = _render(sc, poses, intr, W, H, hsr.HSR_SAMPLE_BILINEAR)
    assert_parity(b, oracle_mod.render(sc, poses, intr, W, H), "bilinear")


def test_mip_chain_read_back_on_gpu():
    """The hand-derived chain: a 4x4 texture read at 1, 2 and 4 texels per
    pixel returns level 0, 1 and 2 texel for texel."""
    g = _golden()
    atlas = np.zeros((4, 4, 4), dtype=np.uint8)
    atlas[..., 0] = g[("level0", "red")]
    atlas[..., 1] = 255 - g[("level0", "red")]
    atlas[..., 2] = g[("level0", "blue")]
    atlas[..., 3] = 255
    for level, W in ((0, 4), (1, 2), (2, 1)):
        sc = _quad(W, W)
        sc.atlas = atlas
        out = _render(sc, identity_pose()[None], screen_intr(W, W), W, W, hsr.HSR_SAMPLE_TRILINEAR)
        img = out["rgb"][0].astype(np.int64)
        want = [atlas[..., c] for c in range(3)] if level == 0 else \
            [g[(f"level{level}", c)] for c in ("red", "green", "blue")]
        for c in range(3):
            assert np.array_equal(img[..., c], want[c]), (level, c)


def test_untextured_scene_refuses_trilinear():
    sc = wl.make_room(1, 2000)
    h = hsr.SceneHandle(sc)
    with pytest.raises(hsr.HsrError):
        h.set_sampling(hsr.HSR_SAMPLE_TRILINEAR)
    with pytest.raises(hsr.HsrError):
        h.set_sampling(7)
    h.close()
