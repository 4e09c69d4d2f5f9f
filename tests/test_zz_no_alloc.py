"""The allocation-free entry point, hsr_render_noalloc, against hsr_render.

It exists for callers that cannot let a library allocate device memory (a
framework that already owns the memory in its own pool, a loop that cannot
afford an allocator call, a host that routes all allocations through its own
allocator). Its scratch is one fixed array shared by all calls, so two calls
in a row must each start from a clean state: the second call here renders
different poses of a different scene, and both must match hsr_render within
the parity tolerance (ids exact, depth 1e-5 relative, RGB 1/255). The file is
named so that pytest collects it last.
"""
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


def _to_np(out):
    torch.cuda.synchronize()
    return {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}


def _check(a, b):
    assert np.array_equal(a["ids"], b["ids"])
    d = np.abs(a["depth"].astype(np.float64) - b["depth"])
    assert np.all(d <= 1e-5 * np.abs(b["depth"].astype(np.float64)))
    assert np.abs(a["rgb"].astype(int) - b["rgb"].astype(int)).max() <= 1


def test_noalloc_matches_render_on_two_calls_in_a_row():
    cases = [(wl.make_room(0), 8, 128, 128, 0), (wl.make_house(3, 60_000, 512), 5, 96, 80, 7)]
    for scene, n, W, H, seed in cases:
        h = hsr.SceneHandle(scene)
        poses = wl.random_poses(scene, n, seed)
        intr = wl.pinhole_90(W, H)
        ref = _to_np(hsr.render(h, poses, intr, W, H))
        out = hsr.alloc_outputs(n, W, H)
        st = hsr.hsr_render_noalloc(h.handle, poses, intr, W, H, out["rgb"], out["depth"], out["ids"])
        assert st == hsr.HSR_OK, hsr.hsr_status_string(st)
        got = _to_np(out)
        _check(got, ref)
        assert (got["ids"] != hsr.BACKGROUND_ID).mean() > 0.5
        h.close()


def test_noalloc_rejects_calls_beyond_its_scratch():
    scene = wl.make_room(1, 2000)
    h = hsr.SceneHandle(scene)
    poses = wl.random_poses(scene, 8, 1)
    out = hsr.alloc_outputs(1, 4, 4)
    # 8 views of 1024 x 1024 need 64 MiB of z-buffer alone (limit 32 MiB)
    st = hsr.hsr_render_noalloc(h.handle, poses, wl.pinhole_90(1024, 1024), 1024, 1024, out["rgb"], out["depth"])
    assert st == hsr.HSR_ERR_OVERFLOW
    torch.cuda.synchronize()
    h.close()
