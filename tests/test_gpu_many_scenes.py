"""Calls over more than 32 resident scenes. The culling kernel then decodes
each warp item's scene slot from the call's slot table rather than from a
per-CTA copy, and tests one view per item. Both the multi-scene one-shot
call and the graph-captured batch must equal per-scene renders (which take
the other culling kernel) bit for bit, with scenes that no view of the call
looks at and views in shuffled scene order. Sampled views must equal the
oracle."""
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

N_SCENES = 40          # above the 32 scene slots the per-CTA slot table holds


def _np(out):
    torch.cuda.synchronize()
    return {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}


def test_calls_over_many_scenes_match_per_scene_renders(oracle_mod):
    scenes = [wl.make_room(300 + s, 1500) for s in range(N_SCENES)]
    hs = [hsr.SceneHandle(s) for s in scenes]
    W, H = 64, 48
    intr = wl.pinhole_90(W, H)
    rng = np.random.default_rng(5)
    seen = rng.permutation(N_SCENES)[:30]
    soa = np.concatenate([np.full(int(rng.integers(1, 4)), s, np.uint32) for s in seen])
    rng.shuffle(soa)
    n = soa.size
    poses = np.zeros((n, 7), np.float32)
    for s in np.unique(soa):
        k = int((soa == s).sum())
        poses[soa == s] = wl.random_poses(scenes[s], k, 1000 + int(s))

    ref = {"rgb": np.zeros((n, H, W, 3), np.uint8), "depth": np.zeros((n, H, W), np.float32),
           "ids": np.zeros((n, H, W), np.uint32)}
    for s in np.unique(soa):
        idx = np.flatnonzero(soa == s)
        r = _np(hsr.render(hs[s], poses[idx], intr, W, H))
        for key in ref:
            ref[key][idx] = r[key]

    one = _np(hsr.render_batch(hs, soa, poses, intr, W, H))
    b = hsr.Batch(hs, n, intr, W, H)
    bat = _np(b.render(poses, soa))
    for key in ref:
        assert np.array_equal(one[key], ref[key]), ("one-shot", key)
        assert np.array_equal(bat[key], ref[key]), ("batch", key)
    assert (ref["ids"] != 0xFFFFFFFF).any()

    for i in (0, n // 2, n - 1):
        o = oracle_mod.render(scenes[int(soa[i])], poses[i:i + 1], intr, W, H, ids=True)
        assert np.array_equal(bat["ids"][i], o["ids"][0]), i
        assert np.array_equal(bat["depth"][i].view(np.uint32), o["depth"][0].view(np.uint32)), i
        assert np.abs(bat["rgb"][i].astype(int) - o["rgb"][0].astype(int)).max() <= 1, i
    b.close()
    for h in hs:
        h.close()
