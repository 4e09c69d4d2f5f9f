"""View lists (hsr_render_views, hsr_batch_render_views): several sensors per
agent in one call, e.g. colour and depth from a textured mesh and semantic
ids from a separate, denser semantic mesh (Table 2 footnote). Each output
equals the oracle's render of the mesh that view names (ids and depth
bit-exact, RGB within 1/255); the batch path equals the one-shot path; bad
lists are refused."""
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
from tests.test_gpu_parity import assert_parity  # noqa: E402


@pytest.fixture(scope="module")
def meshes():
    col = wl.make_house(41, 40_000, 512)
    sem = wl.make_semantic_mesh(41, 90_000)
    hs = [hsr.SceneHandle(col), hsr.SceneHandle(sem)]
    yield col, sem, hs
    for h in hs:
        h.close()


def _np(out):
    torch.cuda.synchronize()
    return {k: (hsr.ids_u32(v) if k == "ids" else v.cpu().numpy()) for k, v in out.items() if v is not None}


def test_semantic_mesh_sensor_matches_oracle(meshes, oracle_mod):
    col, sem, hs = meshes
    poses = wl.random_poses(col, 5, 8)
    W, H = 72, 56
    intr = Intrinsics(36.0, 36.0, 36.0, 28.0, 0.01, 10.0)
    g = _np(hsr.render_semantic(hs[0], hs[1], poses, intr, W, H))
    oc = oracle_mod.render(col, poses, intr, W, H)
    osem = oracle_mod.render(sem, poses, intr, W, H)
    assert_parity({"rgb": g["rgb"], "depth": g["depth"], "ids": oc["ids"]}, oc, "colour mesh")
    assert np.array_equal(g["ids"], osem["ids"]), "semantic ids differ from the semantic mesh's"
    # the semantic mesh's own ids, not the colour mesh's triangle indices
    assert (g["ids"] != 0xFFFFFFFF).mean() > 0.5
    assert set(np.unique(g["ids"])) <= set(np.unique(sem.sem)) | {0xFFFFFFFF}


def test_batch_views_equal_one_shot(meshes):
    col, sem, hs = meshes
    n = 6
    poses = wl.random_poses(col, n, 9)
    W, H = 64, 64
    intr = wl.pinhole_90(W, H)
    frames = np.array([3, 5, 0, 1, 4, 2], dtype=np.uint32)
    views = np.concatenate([hsr.make_views(poses, 0, frames, hsr.HSR_OUT_RGB | hsr.HSR_OUT_DEPTH),
                            hsr.make_views(poses, 1, frames, hsr.HSR_OUT_IDS)])
    one = hsr.alloc_outputs(n, W, H, True)
    assert hsr.hsr_render_views([h.handle for h in hs], views, n, intr, W, H, one["rgb"], one["depth"],
                                one["ids"]) == hsr.HSR_OK
    b = hsr.Batch(hs, 2 * n, intr, W, H)
    assert hsr.hsr_batch_render_views(b.handle, views) == hsr.HSR_OK
    a, c = _np(one), _np(b.out)
    for k in ("rgb", "depth", "ids"):
        assert np.array_equal(a[k], c[k][:n]), k
    # the same as rendering each mesh on its own into unpermuted frames
    ref = _np(hsr.render(hs[0], poses, intr, W, H, ids=False))
    inv = np.argsort(frames)
    assert np.array_equal(a["rgb"], ref["rgb"][inv]) and np.array_equal(a["depth"], ref["depth"][inv])
    b.close()


def test_ids_only_and_depth_only_views(meshes):
    col, sem, hs = meshes
    poses = wl.random_poses(col, 3, 10)
    W, H = 40, 24
    intr = Intrinsics(20.0, 20.0, 20.0, 12.0, 0.01, 10.0)
    out = hsr.alloc_outputs(3, W, H, True)
    views = hsr.make_views(poses, 1, np.arange(3), hsr.HSR_OUT_IDS)
    assert hsr.hsr_render_views([h.handle for h in hs], views, 3, intr, W, H, None, None, out["ids"]) == hsr.HSR_OK
    ref = _np(hsr.render(hs[1], poses, intr, W, H, ids=True))
    assert np.array_equal(_np({"ids": out["ids"]})["ids"], ref["ids"])
    views = hsr.make_views(poses, 0, np.arange(3), hsr.HSR_OUT_DEPTH)
    assert hsr.hsr_render_views([h.handle for h in hs], views, 3, intr, W, H, None, out["depth"], None) == hsr.HSR_OK
    ref0 = _np(hsr.render(hs[0], poses, intr, W, H, ids=False))
    assert np.array_equal(_np({"depth": out["depth"]})["depth"], ref0["depth"])


def test_bad_view_lists_refused(meshes):
    col, sem, hs = meshes
    poses = wl.random_poses(col, 2, 11)
    W, H = 16, 16
    intr = Intrinsics(8.0, 8.0, 8.0, 8.0, 0.01, 10.0)
    out = hsr.alloc_outputs(2, W, H, True)
    handles = [h.handle for h in hs]

    def call(views, rgb=out["rgb"], depth=out["depth"], ids=out["ids"], n_frames=2):
        return hsr.hsr_render_views(handles, views, n_frames, intr, W, H, rgb, depth, ids)

    both = hsr.make_views(poses[[0, 1]], 0, [0, 0], [hsr.HSR_OUT_RGB, hsr.HSR_OUT_RGB])
    assert call(both) == hsr.HSR_ERR_INVALID_ARG                       # frame 0's colour written twice
    assert call(hsr.make_views(poses[:1], 0, [2])) == hsr.HSR_ERR_INVALID_ARG          # frame out of range
    assert call(hsr.make_views(poses[:1], 2, [0])) == hsr.HSR_ERR_INVALID_ARG          # no such scene
    assert call(hsr.make_views(poses[:1], 0, [0], hsr.HSR_OUT_IDS), ids=None) == hsr.HSR_ERR_INVALID_ARG
    assert call(hsr.make_views(poses[:1], 0, [0], 8)) == hsr.HSR_ERR_INVALID_ARG       # unknown output bit
    ok = hsr.make_views(poses[[0, 0]], [0, 1], [1, 1], [hsr.HSR_OUT_RGB | hsr.HSR_OUT_DEPTH, hsr.HSR_OUT_IDS])
    assert call(ok) == hsr.HSR_OK
