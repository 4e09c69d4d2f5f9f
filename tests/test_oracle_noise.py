"""Pins of the oracle's noisy depth sensor (Appendix C: iid Gaussian noise,
mean 0, std sigma = 0.4, added to inverse depth at each pixel): the counter
based generator against its published known answers, and the sample moments
of the noisy inverse depth on a fronto-parallel plane against the stated
distribution."""
import os

import numpy as np
import pytest

from tests.tiny import identity_pose, scene_from_tris, screen_intr, screen_to_world

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle_mod):
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = oracle_mod.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def _plane(D, W, H):
    c = screen_to_world(np.array([-2.0, W + 2.0, -2.0, W + 2.0]), np.array([-2.0, -2.0, H + 2.0, H + 2.0]), W, H, D)
    return scene_from_tris([[c[0], c[1], c[3]], [c[0], c[3], c[2]]])


@pytest.mark.parametrize("D,sigma", [(0.5, 0.4), (2.0, 0.05)])
def test_inverse_depth_noise_moments(oracle_mod, D, sigma):
    W = H = 64
    n = 6
    sc = _plane(D, W, H)
    poses = np.repeat(identity_pose()[None], n, 0)
    o = oracle_mod.render(sc, poses, screen_intr(W, H, 0.01, 100.0), W, H, noise_sigma=sigma, noise_seed=1234)
    d = o["depth"].astype(np.float64)
    assert np.all(d > 0)
    q = 1.0 / d                      # noisy inverse depth
    N = q.size
    assert abs(q.mean() - 1.0 / D) < 5 * sigma / np.sqrt(N)
    var = q.var()
    assert abs(var / sigma ** 2 - 1) < 5 * np.sqrt(2.0 / N)
    # no correlation between horizontally adjacent pixels
    e = q - q.mean()
    r = (e[:, :, 1:] * e[:, :, :-1]).mean() / var
    assert abs(r) < 5 / np.sqrt(N)


def test_noise_is_keyed_by_seed_agent_and_pixel(oracle_mod):
    W = H = 32
    sc = _plane(1.0, W, H)
    intr = screen_intr(W, H, 0.01, 100.0)
    poses = np.repeat(identity_pose()[None], 3, 0)
    a = oracle_mod.render(sc, poses, intr, W, H, noise_sigma=0.2, noise_seed=7)["depth"]
    assert not np.array_equal(a[0], a[1])                    # agents differ
    b = oracle_mod.render(sc, poses[:1], intr, W, H, noise_sigma=0.2, noise_seed=7, agent_ids=[2])["depth"]
    assert np.array_equal(b[0], a[2])                        # same agent id, same noise, any batch position
    c = oracle_mod.render(sc, poses[:1], intr, W, H, noise_sigma=0.2, noise_seed=8)["depth"]
    assert not np.array_equal(c[0], a[0])                    # seed changes it
    z = oracle_mod.render(sc, poses[:1], intr, W, H, noise_sigma=0.0)["depth"]
    assert np.all(z == np.float32(1.0))


def test_noise_beyond_far_gives_no_return(oracle_mod):
    # inverse depth pushed below 1/far reports 0, like a missing return
    W = H = 64
    sc = _plane(5.0, W, H)
    o = oracle_mod.render(sc, identity_pose()[None], screen_intr(W, H, 0.01, 10.0), W, H, noise_sigma=0.4,
                          noise_seed=3)
    d = o["depth"][0]
    assert (d == 0).mean() > 0.1 and (d > 0).mean() > 0.1
    assert d.max() <= 10.0
