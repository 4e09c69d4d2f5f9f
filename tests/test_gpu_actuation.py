"""On-device actuation (Sec. 4 action space) through the C-ABI
(hsr_agents_*, hsr_batch_step): agent poses after each step are bit-exact
with the oracle's actuation, and the rendered frames match the oracle's
render of those poses (ids and depth bit-exact, RGB within 1/255), and
equal bit for bit a pose-driven render of the same poses."""
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


def _np(out, frames=None):
    torch.cuda.synchronize()
    r = {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}
    if frames is not None:
        r = {k: v[frames] for k, v in r.items()}
    return r


def _oracle_step(oracle_mod, poses, idx, actions, navs, scene_of):
    new = poses.copy()
    for a, act in zip(idx, actions):
        new[a], _ = oracle_mod.actuate(poses[a], int(act), navs[scene_of[a]])
    return new


def test_random_walk_steps_match_oracle(oracle_mod):
    """Room, 12 agents, ragged 72x40 frames, 8 steps of random actions on a
    random subset of agents written to permuted frames."""
    sc = wl.make_room(0)
    nav = wl.navmap(sc, 0.05)
    n = 12
    poses = wl.navigable_poses(sc, nav, n, 1)
    W, H = 72, 40
    intr = Intrinsics(36.0, 36.0, 36.0, 20.0, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    ag = hsr.Agents([h], [nav], poses)
    b = hsr.Batch([h], n, intr, W, H)
    assert np.array_equal(ag.poses().view(np.uint32), poses.view(np.uint32))
    rs = np.random.default_rng(7)
    cur = poses.copy()
    moved_fwd = refused = 0
    for step in range(8):
        k = int(rs.integers(3, n + 1))
        idx = rs.permutation(n)[:k].astype(np.uint32)
        # mostly forward moves, so that walls refuse some
        actions = rs.choice([0, 1, 1, 1, 2, 3], size=k).astype(np.uint8)
        frames = rs.permutation(n)[:k].astype(np.uint32)
        out = b.step(ag, idx, actions, frames=frames)
        want = _oracle_step(oracle_mod, cur, idx, actions, [nav], np.zeros(n, np.int64))
        got = ag.poses()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), f"step {step}: poses differ"
        for a, act in zip(idx, actions):
            if act == 1:
                if np.array_equal(want[a], cur[a]):
                    refused += 1
                else:
                    moved_fwd += 1
        cur = want
        g = _np(out, frames)
        o = oracle_mod.render(sc, cur[idx], intr, W, H)
        assert_parity(g, o, f"step {step}")
    assert moved_fwd > 0


def test_step_equals_pose_render_two_scenes():
    """Two scenes, agents split between them: the frames of a step equal, bit
    for bit, a pose-driven batch render of the poses the agents reached (the
    device builds the same cameras as the host)."""
    scenes = [wl.make_house(11, 120_000, 512), wl.make_room(2, 8000)]
    navs = [wl.navmap(s, 0.05) for s in scenes]
    n0, n1 = 20, 12
    poses = np.concatenate([wl.navigable_poses(scenes[0], navs[0], n0, 3),
                            wl.navigable_poses(scenes[1], navs[1], n1, 4)])
    soa = np.r_[np.zeros(n0), np.ones(n1)].astype(np.uint32)
    n = n0 + n1
    W, H = 96, 96
    intr = wl.pinhole_90(W, H)
    hs = [hsr.SceneHandle(s) for s in scenes]
    ag = hsr.Agents(hs, navs, poses, scene_of_agent=soa)
    b = hsr.Batch(hs, n, intr, W, H)
    rs = np.random.default_rng(3)
    for step in range(4):
        idx = rs.permutation(n).astype(np.uint32)
        actions = rs.integers(0, 4, n).astype(np.uint8)
        g = _np(b.step(ag, idx, actions))
        reached = ag.poses()
        ref = _np(hsr.render_batch(hs, soa[idx], reached[idx], intr, W, H))
        for key in ("rgb", "depth", "ids"):
            assert np.array_equal(g[key], ref[key]), (step, key)


def test_step_with_noise_and_stop():
    """Stop re-renders the same pose: ids and colour repeat, while the depth
    noise follows the per-call seed."""
    sc = wl.make_room(5, 6000)
    nav = wl.navmap(sc, 0.05)
    poses = wl.navigable_poses(sc, nav, 4, 2)
    W, H = 48, 32
    intr = Intrinsics(24.0, 24.0, 24.0, 16.0, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    ag = hsr.Agents([h], [nav], poses)
    b = hsr.Batch([h], 4, intr, W, H)
    idx = np.arange(4, dtype=np.uint32)
    stop = np.zeros(4, np.uint8)
    a = _np(b.step(ag, idx, stop, noise_sigma=0.4, noise_seed=1))
    c = _np(b.step(ag, idx, stop, noise_sigma=0.4, noise_seed=2))
    d = _np(b.step(ag, idx, stop, noise_sigma=0.4, noise_seed=1))
    assert np.array_equal(a["ids"], c["ids"]) and np.array_equal(a["rgb"], c["rgb"])
    assert not np.array_equal(a["depth"], c["depth"])
    assert np.array_equal(a["depth"], d["depth"])
    assert np.array_equal(ag.poses().view(np.uint32), poses.view(np.uint32))


def test_step_validation():
    sc = wl.make_room(6, 4000)
    nav = wl.navmap(sc, 0.05)
    poses = wl.navigable_poses(sc, nav, 3, 0)
    intr = Intrinsics(16.0, 16.0, 16.0, 16.0, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    ag = hsr.Agents([h], [nav], poses)
    b = hsr.Batch([h], 3, intr, 32, 32)
    bad = [
        (np.array([0, 0], np.uint32), np.array([1, 1], np.uint8)),    # the same agent twice
        (np.array([3], np.uint32), np.array([1], np.uint8)),          # no such agent
        (np.array([1], np.uint32), np.array([4], np.uint8)),          # no such action
    ]
    for idx, act in bad:
        assert hsr.hsr_batch_step(b.handle, ag.handle, idx, act) == hsr.HSR_ERR_INVALID_ARG
    # a pose off the navigable grid is refused at creation and by set_poses
    off = poses[:1].copy()
    off[0, 0] = 1000.0
    with pytest.raises(hsr.HsrError):
        hsr.Agents([h], [nav], off)
    with pytest.raises(hsr.HsrError):
        ag.set_poses([0], off)
    ag.set_poses([2], poses[:1])
    assert np.array_equal(ag.poses()[2], poses[0])
    # agents of another scene list cannot step this batch
    h2 = hsr.SceneHandle(sc)
    ag2 = hsr.Agents([h2], [nav], poses)
    assert hsr.hsr_batch_step(b.handle, ag2.handle, [0], [0]) == hsr.HSR_ERR_INVALID_ARG
