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
    out = hsr.alloc_outputs(8, 1024, 1024, ids=False)
    # 8 views of 1024 x 1024 need 64 MiB of z-buffer alone (limit 32 MiB)
    st = hsr.hsr_render_noalloc(h.handle, poses, wl.pinhole_90(1024, 1024), 1024, 1024, out["rgb"], out["depth"])
    assert st == hsr.HSR_ERR_OVERFLOW
    torch.cuda.synchronize()
    h.close()


def _overflows(h, poses, W, H, out):
    """Whether a 1-view W x H call is refused; `out` holds 1 x H x 4096
    outputs, enough for any W <= 4096 (a call that fits renders into it)."""
    assert W <= 4096 and out["depth"].numel() >= W * H
    st = hsr.hsr_render_noalloc(h.handle, poses, wl.pinhole_90(W, H), W, H, out["rgb"], out["depth"])
    assert st in (hsr.HSR_OK, hsr.HSR_ERR_OVERFLOW), hsr.hsr_status_string(st)
    torch.cuda.synchronize()
    return st == hsr.HSR_ERR_OVERFLOW


def test_noalloc_at_the_scratch_limit():
    """The largest width (at height 1024) whose scratch fits the 32 MiB
    array renders like hsr_render; one pixel column more is refused."""
    scene = wl.make_room(2, 3000)
    h = hsr.SceneHandle(scene)
    poses = wl.random_poses(scene, 1, 2)
    H = 1024
    big = hsr.alloc_outputs(1, 4096, H, ids=False)
    lo, hi = 1, 4096                         # lo fits, hi does not (8 B/pixel alone: 32 MiB at 4096 x 1024)
    assert not _overflows(h, poses, lo, H, big) and _overflows(h, poses, hi, H, big)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if _overflows(h, poses, mid, H, big):
            hi = mid
        else:
            lo = mid
    W = lo
    assert W > 3000
    intr = wl.pinhole_90(W, H)
    ref = _to_np(hsr.render(h, poses, intr, W, H))
    out = hsr.alloc_outputs(1, W, H)
    st = hsr.hsr_render_noalloc(h.handle, poses, intr, W, H, out["rgb"], out["depth"], out["ids"])
    assert st == hsr.HSR_OK
    _check(_to_np(out), ref)
    out2 = hsr.alloc_outputs(1, W + 1, H)
    assert hsr.hsr_render_noalloc(h.handle, poses, wl.pinhole_90(W + 1, H), W + 1, H, out2["rgb"], out2["depth"],
                                  out2["ids"]) == hsr.HSR_ERR_OVERFLOW
    torch.cuda.synchronize()
    h.close()


def test_noalloc_host_descriptor_limit():
    """5,457 views fill the 1 MiB host staging buffer exactly; one more is refused."""
    scene = wl.make_room(3, 500)
    h = hsr.SceneHandle(scene)
    poses = wl.random_poses(scene, 5458, 3)
    out = hsr.alloc_outputs(5458, 2, 2)
    intr = wl.pinhole_90(2, 2)
    assert hsr.hsr_render_noalloc(h.handle, poses, intr, 2, 2, out["rgb"], out["depth"], out["ids"]) == \
        hsr.HSR_ERR_OVERFLOW
    st = hsr.hsr_render_noalloc(h.handle, poses[:5457], intr, 2, 2, out["rgb"], out["depth"], out["ids"])
    assert st == hsr.HSR_OK
    got = _to_np({k: v[:5457] for k, v in out.items()})
    ref = _to_np(hsr.render(h, poses[:5457], intr, 2, 2))
    _check(got, ref)
    h.close()


def test_noalloc_side_stream_without_ids():
    """On a non-default stream, with no id buffer (colour + depth only)."""
    scene = wl.make_house(4, 40_000, 256)
    h = hsr.SceneHandle(scene)
    poses = wl.random_poses(scene, 4, 4)
    W, H = 120, 72
    intr = wl.pinhole_90(W, H)
    ref = _to_np(hsr.render(h, poses, intr, W, H))
    out = hsr.alloc_outputs(4, W, H, ids=False)
    s = torch.cuda.Stream()
    for _ in range(2):
        with torch.cuda.stream(s):
            out["rgb"].zero_()
            out["depth"].zero_()
            st = hsr.hsr_render_noalloc(h.handle, poses, intr, W, H, out["rgb"], out["depth"], None, stream=s)
        assert st == hsr.HSR_OK
        s.synchronize()
        assert np.array_equal(out["depth"].cpu().numpy().view(np.uint32), ref["depth"].view(np.uint32))
        assert np.abs(out["rgb"].cpu().numpy().astype(int) - ref["rgb"].astype(int)).max() <= 1
    h.close()
