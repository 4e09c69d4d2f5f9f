"""Sensor sets: a colour-only render (depth NULL) writes the same colour and
ids as the colour + depth render of the same views, on the one-shot and the
graph-replayed batch paths."""
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


@pytest.mark.parametrize("W,H", [(64, 64), (50, 37)])
def test_colour_only_matches_rgbd(W, H):
    sc = wl.make_house(21, 50_000, 256, semantic=True)
    poses = wl.random_poses(sc, 8, 4)
    intr = Intrinsics(W / 2, W / 2, W / 2, H / 2, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    full = hsr.render(h, poses, intr, W, H, ids=True)
    col = hsr.alloc_outputs(8, W, H, ids=True, depth=False)
    assert hsr.hsr_render(h.handle, poses, intr, W, H, col["rgb"], None, col["ids"]) == hsr.HSR_OK
    b = hsr.Batch([h], 8, intr, W, H, ids=True, depth=False)
    bo = b.render(poses)
    torch.cuda.synchronize()
    for out in (col, bo):
        assert out["depth"] is None
        assert torch.equal(out["rgb"], full["rgb"]) and torch.equal(out["ids"], full["ids"])
    b.close()
    h.close()
