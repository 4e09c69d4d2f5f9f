"""Graph-captured persistent batch: every replay equals the one-shot render
of the same views bit for bit (poses change between replays, fewer views than
the capacity, mixed scenes, permuted output frames)."""
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


def _np(out, sel=None):
    torch.cuda.synchronize()
    r = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}
    return {k: (v if sel is None else v[sel]) for k, v in r.items()}


def test_batch_replays_match_one_shot():
    scenes = [wl.make_house(21, 80_000, 512), wl.make_room(22, 8000)]
    hs = [hsr.SceneHandle(s) for s in scenes]
    W, H, cap = 96, 80, 12
    intr = wl.pinhole_90(W, H)
    b = hsr.Batch(hs, cap, intr, W, H)
    rng = np.random.default_rng(0)
    for rep in range(4):
        n = [cap, 7, cap, 3][rep]
        soa = rng.integers(0, 2, n).astype(np.uint32)
        poses = np.zeros((n, 7), np.float32)
        for s in range(2):
            k = int((soa == s).sum())
            if k:
                poses[soa == s] = wl.random_poses(scenes[s], k, 100 * rep + s)
        frames = rng.permutation(cap)[:n].astype(np.uint32) if rep % 2 else None
        out = b.render(poses, soa, frames)
        got = _np(out, frames if frames is not None else np.arange(n))
        ref = _np(hsr.render_batch(hs, soa, poses, intr, W, H))
        for key in ref:
            assert np.array_equal(got[key], ref[key]), (rep, key)
    b.close()
    for h in hs:
        h.close()


def test_batch_rejects_too_many_views():
    sc = wl.make_room(3, 2000)
    h = hsr.SceneHandle(sc)
    b = hsr.Batch([h], 2, wl.pinhole_90(32, 32), 32, 32)
    assert hsr.hsr_batch_render(b.handle, None, wl.random_poses(sc, 3, 0)) == hsr.HSR_ERR_OVERFLOW
    assert hsr.hsr_batch_render(b.handle, None, wl.random_poses(sc, 2, 0), np.array([0, 5], np.uint32)) == \
        hsr.HSR_ERR_INVALID_ARG
    b.close()
    h.close()


def test_render_host_matches_device_outputs():
    """hsr_batch_render_host: the host copies equal the device frames of the
    same replay, two batches alternating on two streams (the overlapped form);
    outputs the batch lacks are rejected."""
    sc = wl.make_house(23, 60_000, 256)
    h = hsr.SceneHandle(sc)
    W, H, n = 80, 64, 9
    intr = wl.pinhole_90(W, H)
    bs = [hsr.Batch([h], n, intr, W, H), hsr.Batch([h], n, intr, W, H)]
    ss = [torch.cuda.Stream(), torch.cuda.Stream()]
    hosts = [{k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in b.out.items()} for b in bs]
    for rep in range(4):
        k = rep % 2
        ss[k].synchronize()
        poses = wl.random_poses(sc, n, 300 + rep)
        up = bs[k].render_host(poses, hosts[k], stream=ss[k])
        assert up > 0
        ss[k].synchronize()
        ref = _np(hsr.render(h, poses, intr, W, H))
        got = {"rgb": hosts[k]["rgb"].numpy(), "depth": hosts[k]["depth"].numpy(),
               "ids": hosts[k]["ids"].numpy().view(np.uint32)}
        for key in ref:
            assert np.array_equal(got[key], ref[key]), (rep, key)
    nod = hsr.Batch([h], 2, intr, W, H, ids=False)
    st, _ = hsr.hsr_batch_render_host(nod.handle, None, wl.random_poses(sc, 2, 0), W, H,
                                      host_ids=torch.empty((2, H, W), dtype=torch.int32, pin_memory=True))
    assert st == hsr.HSR_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        hsr.hsr_batch_render_host(nod.handle, None, wl.random_poses(sc, 2, 0), W, H,
                                  host_rgb=torch.empty((1, H, W, 3), dtype=torch.uint8))
    for b in bs + [nod]:
        b.close()
    h.close()


@pytest.mark.parametrize("depth,ids", [(False, False), (True, False), (True, True)])
def test_transfer_strategies_deliver_the_same_frames(oracle_mod, depth, ids):
    """The frame hand-offs of the transfer experiment (Table 2): frames left in
    device memory (GPU->GPU), copied to page-locked host memory (GPU->CPU),
    and copied on to a separate device buffer (GPU->CPU->GPU), for the colour,
    colour + depth and colour + depth + semantic sensor sets, queued on a side
    stream after the render as the benchmark does. Every leg equals the
    device frames bit for bit; two views against the oracle."""
    sc = wl.make_house(24, 60_000, 256, semantic=True)
    h = hsr.SceneHandle(sc)
    W = H = 96
    n = 6
    intr = wl.pinhole_90(W, H)
    poses = wl.random_poses(sc, n, 41)
    b = hsr.Batch([h], n, intr, W, H, ids=ids, depth=depth)
    s = torch.cuda.Stream()
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in b.out.items() if v is not None}
    back = {k: torch.empty_like(v) for k, v in b.out.items() if v is not None}
    b.render(poses, stream=s)
    with torch.cuda.stream(s):
        for k, dst in host.items():
            dst.copy_(b.out[k], non_blocking=True)
        for k, dst in back.items():
            dst.copy_(host[k], non_blocking=True)
    s.synchronize()
    for k in host:
        dev = b.out[k].cpu()
        assert torch.equal(host[k], dev), ("gpu-cpu", k)
        assert torch.equal(back[k].cpu(), dev), ("gpu-cpu-gpu", k)
    for i in (0, n - 1):
        o = oracle_mod.render(sc, poses[i:i + 1], intr, W, H, ids=True)
        assert np.abs(back["rgb"][i].cpu().numpy().astype(int) - o["rgb"][0].astype(int)).max() <= 1
        if depth:
            assert np.array_equal(back["depth"][i].cpu().numpy().view(np.uint32), o["depth"][0].view(np.uint32))
        if ids:
            assert np.array_equal(back["ids"][i].cpu().numpy().view(np.uint32), o["ids"][0])
    b.close()
    h.close()
