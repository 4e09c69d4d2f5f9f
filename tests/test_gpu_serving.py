"""Serving: every request's result equals its one-shot render bit for bit,
alone and in the mix; admission waits for framebuffers; queue overflow and bad
requests are reported per request."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1904_01201_b300 import build as _build  # noqa: E402

_build.build()
from paper_1904_01201_b300 import hsr, serve  # noqa: E402
from paper_1904_01201_b300 import workloads as wl  # noqa: E402

RES = (32, 64, 96)


@pytest.fixture(scope="module")
def scenes():
    sc = [wl.make_house(31, 60_000, 512), wl.make_room(32, 6000)]
    hs = [hsr.SceneHandle(s) for s in sc]
    yield sc, hs
    for h in hs:
        h.close()


def _requests(sc, n, seed):
    rng = np.random.default_rng(seed)
    req = np.zeros(n, dtype=hsr.REQUEST_DTYPE)
    req["agent"] = -1                          # pose requests
    for i in range(n):
        s = int(rng.integers(0, len(sc)))
        req[i]["tag"] = i
        req[i]["scene"] = s
        req[i]["res"] = RES[int(rng.integers(0, len(RES)))]
        req[i]["pose"] = wl.random_poses(sc[s], 1, seed * 1000 + i)[0]
    return req


def _collect(srv, n, with_ids, release=True):
    got = {}
    while len(got) < n:
        res = srv.poll(100000)
        assert res, "server stalled"
        for r in res:
            got[r.tag] = (r.status, serve.frame_tensors(r, with_ids) if r.status == 0 else None)
        if release:
            srv.release(res)
    return got


def _check_alone(sc, hs, req, got, with_ids):
    for i, rq in enumerate(req):
        st, fr = got[int(rq["tag"])]
        assert st == 0
        r = int(rq["res"])
        ref = hsr.render(hs[int(rq["scene"])], rq["pose"][None], wl.pinhole_90(r, r), r, r, ids=with_ids)
        torch.cuda.synchronize()
        assert torch.equal(fr["rgb"], ref["rgb"][0]), i
        assert torch.equal(fr["depth"], ref["depth"][0]), i
        if with_ids:
            assert torch.equal(fr["ids"], ref["ids"][0]), i


def test_served_results_equal_one_shot_renders(scenes):
    sc, hs = scenes
    srv = serve.Server(hs, res=RES, weights=(1, 1, 1), fb_bytes=64 << 20, max_batch=8, n_streams=2,
                       max_wait_us=100, with_ids=True)
    req = _requests(sc, 90, 1)
    for k in range(0, 90, 15):                 # bursts: later requests arrive while earlier ones render
        srv.submit(req[k:k + 15])
    got = _collect(srv, 90, True)
    _check_alone(sc, hs, req, got, True)
    st = srv.stats()
    assert st["completed"] == 90 and st["rejected"] == 0 and st["fb_bytes_used"] == 0
    assert st["batches"] >= 90 // 8
    srv.close()


def test_admission_waits_for_framebuffers(scenes):
    sc, hs = scenes
    # room for about two frames per resolution: requests wait for releases
    srv = serve.Server(hs, res=RES, weights=(1, 1, 1), fb_bytes=3 * 2 * 96 * 96 * 7, max_batch=8, n_streams=2,
                       max_wait_us=0, with_ids=False)
    req = _requests(sc, 40, 2)
    srv.submit(req)
    got = _collect(srv, 40, False)
    _check_alone(sc, hs, req, got, False)
    srv.close()


def test_queue_overflow_and_bad_requests(scenes):
    sc, hs = scenes
    srv = serve.Server(hs, res=RES, weights=(1, 1, 1), fb_bytes=8 << 20, max_batch=4, n_streams=1, max_queue=5,
                       with_ids=False)
    req = _requests(sc, 30, 3)
    req[0]["res"] = 33                          # not served
    srv.submit(req)
    got = _collect(srv, 30, False)
    statuses = [got[i][0] for i in range(30)]
    assert statuses[0] == hsr.HSR_ERR_INVALID_ARG
    assert statuses.count(hsr.HSR_ERR_OVERFLOW) >= 1
    assert all(s in (0, hsr.HSR_ERR_OVERFLOW, hsr.HSR_ERR_INVALID_ARG) for s in statuses)
    st = srv.stats()
    assert st["rejected"] == statuses.count(hsr.HSR_ERR_OVERFLOW)
    srv.close()


def test_action_requests_step_agents_in_order(scenes, oracle_mod):
    """Action requests of a few agents, mixed with pose requests: every
    agent's actions apply in submission order (its poses follow the oracle's
    actuation), each result is the render of the pose its action reached, and
    a second action of a busy agent waits for the first."""
    sc, hs = scenes
    navs = [wl.navmap(s, 0.05) for s in sc]
    n_agents = 5
    soa = np.array([0, 1, 0, 1, 0], dtype=np.uint32)
    poses0 = np.stack([wl.navigable_poses(sc[int(s)], navs[int(s)], 1, 40 + a)[0] for a, s in enumerate(soa)])
    ag = hsr.Agents(hs, navs, poses0, scene_of_agent=soa)
    srv = serve.Server(hs, res=RES, weights=(1, 1, 1), fb_bytes=64 << 20, max_batch=8, n_streams=3,
                       max_wait_us=50, with_ids=True)
    srv.attach_agents(ag)
    rng = np.random.default_rng(11)
    n_act = 60
    act = np.zeros(n_act, dtype=hsr.REQUEST_DTYPE)
    act["tag"] = np.arange(n_act)
    act["agent"] = rng.integers(0, n_agents, n_act)
    act["action"] = rng.choice([0, 1, 1, 2, 3], n_act)
    act["res"] = np.asarray(RES)[rng.integers(0, len(RES), n_act)]
    pose_req = _requests(sc, 20, 5)
    pose_req["tag"] += 1000
    for k in range(0, n_act, 12):
        srv.submit(act[k:k + 12])
        srv.submit(pose_req[k // 3:k // 3 + 4])
    got = _collect(srv, n_act + 20, True)
    # expected pose after each action, by submission order per agent
    cur = poses0.copy()
    for i, rq in enumerate(act):
        a = int(rq["agent"])
        cur[a], _ = oracle_mod.actuate(cur[a], int(rq["action"]), navs[int(soa[a])])
        st, fr = got[i]
        assert st == 0
        r = int(rq["res"])
        ref = hsr.render(hs[int(soa[a])], cur[a][None], wl.pinhole_90(r, r), r, r, ids=True)
        torch.cuda.synchronize()
        for key in ("rgb", "depth", "ids"):
            assert torch.equal(fr[key], ref[key][0]), (i, key)
    assert np.array_equal(ag.poses().view(np.uint32), cur.view(np.uint32))
    for i, rq in enumerate(pose_req):
        assert got[int(rq["tag"])][0] == 0
    srv.close()
    ag.close()


def test_action_requests_need_attached_agents(scenes):
    sc, hs = scenes
    srv = serve.Server(hs, res=RES, weights=(1, 1, 1), fb_bytes=8 << 20, max_batch=4, n_streams=1)
    req = np.zeros(2, dtype=hsr.REQUEST_DTYPE)
    req["tag"] = [0, 1]
    req["res"] = RES[0]
    req["agent"] = [0, 0]
    req["action"] = [1, 7]
    srv.submit(req)
    got = _collect(srv, 2, False)
    assert got[0][0] == hsr.HSR_ERR_INVALID_ARG and got[1][0] == hsr.HSR_ERR_INVALID_ARG
    # agents over another scene list cannot be attached
    navs = [wl.navmap(sc[1], 0.05)]
    ag = hsr.Agents([hs[1]], navs, wl.navigable_poses(sc[1], navs[0], 2, 0))
    with pytest.raises(hsr.HsrError):
        srv.attach_agents(ag)
    srv.close()
    ag.close()


def test_serving_workload_settings(oracle_mod):
    """The serving configuration as bench.py runs it: the 8 batching scenes
    resident (0.2M-2M triangles), 1,024 device-resident agents, action
    requests at 64/128/256/512 (weights 0.2/0.4/0.3/0.1) in bursts, micro-
    batches of up to 64 views on 4 streams, 50 us wait, 4 GiB of
    framebuffers. Every result equals the one-shot render of the pose its
    action reached (the oracle's actuation in submission order), bit for bit;
    two results per resolution against the oracle."""
    res = (64, 128, 256, 512)
    sc = wl.batching_scenes(0)
    hs = [hsr.SceneHandle(s) for s in sc]
    agents, soa = serve.make_agents(sc, hs, 1024, seed=0)
    navs = [wl.navmap(s, 0.05) for s in sc]
    poses0 = agents.poses()
    srv = serve.Server(hs, res=res, weights=(0.2, 0.4, 0.3, 0.1), fb_bytes=4 << 30, max_batch=64, n_streams=4,
                       max_wait_us=50)
    srv.attach_agents(agents)
    n = 800
    req = serve.make_action_requests(n, 1024, res=res, seed=3)
    for k in range(0, n, 100):                 # bursts: later ones arrive while earlier ones render
        srv.submit(req[k:k + 100])
    got = _collect(srv, n, False)
    cur = poses0.copy()
    reached = []
    for i, rq in enumerate(req):
        a = int(rq["agent"])
        cur[a], _ = oracle_mod.actuate(cur[a], int(rq["action"]), navs[int(soa[a])])
        reached.append(cur[a].copy())
        st, fr = got[i]
        assert st == 0, i
        r = int(rq["res"])
        ref = hsr.render(hs[int(soa[a])], cur[a][None], wl.pinhole_90(r, r), r, r, ids=False)
        torch.cuda.synchronize()
        assert torch.equal(fr["rgb"], ref["rgb"][0]), i
        assert torch.equal(fr["depth"], ref["depth"][0]), i
    assert np.array_equal(agents.poses().view(np.uint32), cur.view(np.uint32))
    for r in res:
        for i in [j for j, rq in enumerate(req) if int(rq["res"]) == r][:2]:
            a = int(req[i]["agent"])
            o = oracle_mod.render(sc[int(soa[a])], reached[i][None], wl.pinhole_90(r, r), r, r, ids=False)
            assert np.array_equal(got[i][1]["depth"].cpu().numpy().view(np.uint32), o["depth"][0].view(np.uint32))
            assert np.abs(got[i][1]["rgb"].cpu().numpy().astype(int) - o["rgb"][0].astype(int)).max() <= 1
    st = srv.stats()
    assert st["completed"] == n and st["rejected"] == 0
    srv.close()
    agents.close()
    for h in hs:
        h.close()
