"""Noisy depth sensor (Appendix C: iid Gaussian noise of std sigma added to
inverse depth at each pixel) on the CUDA path vs the oracle, through the
C-ABI (hsr_render_noisy, hsr_batch_render_noisy).

Both sides draw the same Philox-4x32-10 words, so the integer part of the
sensor (which pixels are hit, the counter and key of each draw) is exact;
the Box-Muller transform is fp64 in the oracle and fp32 (logf, cospif,
sqrtf) in the kernel, the cosine as cospi(2 u2), whose argument is exact in
fp32. Bound on the noisy inverse depth q' = q + sigma z:
  |dz| <= s |d cos| + |z| (|d log|/|log| + |d sqrt| + |d mul|)
       <= 5.77 * 1.2e-7 + 5.77 * 2.4e-7  < 2.1e-6,
with s = sqrt(-2 ln u1) <= sqrt(-2 ln 2^-24) = 5.77, cospif within 2 ulp,
logf within 1 ulp and each fp32 rounding 2^-24 relative; the fma adds
2^-24 |q'| and each reciprocal (depth = 1/q', then q' = 1/depth in the test)
2^-24 more. Hence |q'_gpu - q'_oracle| <= sigma * 2.1e-6 + 2.5e-7 |q'|.
Every returned pixel has q' > 1/far, so the relative depth error is at most
sigma * 2.1e-6 * far + 2.5e-7: 8.7e-6 for the paper's sigma 0.4 at far 10 m,
inside the 1e-5 depth tolerance. Pixels whose noisy inverse depth lies
within the bound of the 1/far cutoff may report 0 on one side only.
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
from paper_1904_01201_b300.workloads import Intrinsics  # noqa: E402

SIGMA = 0.4
SEED = 0x0123456789ABCDEF


def _np(out):
    torch.cuda.synchronize()
    return {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}


def assert_noisy_parity(g, o, intr, sigma, what=""):
    bad = g["ids"] != o["ids"]
    assert not bad.any(), f"{what}: {int(bad.sum())} id mismatches"
    diff = np.abs(g["rgb"].astype(np.int16) - o["rgb"].astype(np.int16))
    assert diff.max() <= 1, f"{what}: rgb diff {diff.max()}"
    dg = g["depth"].astype(np.float64)
    do = o["depth"].astype(np.float64)
    bg = g["ids"] == 0xFFFFFFFF
    assert np.all(dg[bg] == 0) and np.all(do[bg] == 0), f"{what}: background depth not 0"
    inv_far = 1.0 / intr.zfar
    both = (dg > 0) & (do > 0)
    qg, qo = 1.0 / dg[both], 1.0 / do[both]
    tol = sigma * 2.1e-6 + 2.5e-7 * np.abs(qo)
    err = np.abs(qg - qo)
    assert np.all(err <= tol), f"{what}: noisy inverse depth off by {err.max():.3g} (bound {tol[np.argmax(err)]:.3g})"
    rel = np.abs(dg[both] - do[both]) / do[both]
    assert np.all(rel <= sigma * 2.1e-6 * intr.zfar + 3e-7), f"{what}: relative depth error {rel.max():.3g}"
    if sigma * 2.1e-6 * intr.zfar + 3e-7 <= 1e-5:
        assert rel.max() <= 1e-5, f"{what}: relative depth error {rel.max():.3g} beyond 1e-5"
    only_g = (dg > 0) & (do == 0) & ~bg
    only_o = (do > 0) & (dg == 0) & ~bg
    tol_cut = sigma * 2.1e-6 + 2.5e-7 * inv_far
    assert np.all(1.0 / dg[only_g] <= inv_far + tol_cut), f"{what}: GPU returns where the oracle has none"
    assert np.all(1.0 / do[only_o] <= inv_far + tol_cut), f"{what}: GPU drops a return the oracle keeps"
    return int(both.sum()), int(((dg == 0) & (do == 0) & ~bg).sum())


def test_noisy_depth_room_oneshot(oracle_mod):
    """Room, 12 agents, ragged 100x61 frames, sigma 0.4: a sizeable share of
    pixels is pushed past the far cutoff and must report 0 on both sides."""
    sc = wl.make_room(1)
    poses = wl.random_poses(sc, 12, 5)
    W, H = 100, 61
    intr = Intrinsics(W / 2, W / 2, W / 2, H / 2, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    g = _np(hsr.render(h, poses, intr, W, H, noise_sigma=SIGMA, noise_seed=SEED))
    o = oracle_mod.render(sc, poses, intr, W, H, noise_sigma=SIGMA, noise_seed=SEED)
    n_both, n_cut = assert_noisy_parity(g, o, intr, SIGMA, "room")
    assert n_both > 0.5 * g["depth"].size and n_cut > 0
    # colour and ids are those of the noise-free render
    clean = _np(hsr.render(h, poses, intr, W, H))
    assert np.array_equal(clean["ids"], g["ids"]) and np.array_equal(clean["rgb"], g["rgb"])
    h.close()


def test_noisy_depth_agent_keys_and_batch(oracle_mod):
    """Explicit agent keys on the one-shot path, and a graph-replayed batch
    writing permuted frames (keys default to the output frame)."""
    sc = wl.make_room(2, 6000)
    poses = wl.random_poses(sc, 6, 9)
    W, H = 64, 48
    intr = Intrinsics(32.0, 32.0, 32.0, 24.0, 0.01, 8.0)
    h = hsr.SceneHandle(sc)
    keys = np.array([7, 7, 1000, 3, 0xFFFFFFFF, 42], dtype=np.uint32)
    g = _np(hsr.render(h, poses, intr, W, H, noise_sigma=0.1, noise_seed=99, agent_ids=keys))
    o = oracle_mod.render(sc, poses, intr, W, H, noise_sigma=0.1, noise_seed=99, agent_ids=keys)
    assert_noisy_parity(g, o, intr, 0.1, "agent keys")

    frames = np.array([5, 0, 3, 1, 4, 2], dtype=np.uint32)
    b = hsr.Batch([h], 6, intr, W, H)
    out = b.render(poses, frames=frames, noise_sigma=0.1, noise_seed=99)
    gb = _np(out)
    inv = np.argsort(frames)
    ob = oracle_mod.render(sc, poses[inv], intr, W, H, noise_sigma=0.1, noise_seed=99)
    assert_noisy_parity(gb, ob, intr, 0.1, "batch")
    # the next replay of the same graph without noise is the clean render
    gc = _np(b.render(poses[inv]))
    clean = _np(hsr.render(h, poses[inv], intr, W, H))
    for k in ("rgb", "ids", "depth"):
        assert np.array_equal(gc[k], clean[k]), k
    b.close()
    h.close()


def test_zero_sigma_is_noise_free_and_bad_sigma_rejected():
    sc = wl.make_room(4, 3000)
    poses = wl.random_poses(sc, 3, 1)
    W, H = 40, 30
    intr = Intrinsics(20.0, 20.0, 20.0, 15.0, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    a = _np(hsr.render(h, poses, intr, W, H, noise_sigma=0.0, noise_seed=5))
    c = _np(hsr.render(h, poses, intr, W, H))
    for k in ("rgb", "ids", "depth"):
        assert np.array_equal(a[k], c[k]), k
    out = hsr.alloc_outputs(3, W, H)
    for bad in (float("nan"), -0.1, float("inf")):
        st = hsr.hsr_render_noisy([h.handle], None, poses, intr, W, H, out["rgb"], out["depth"], out["ids"],
                                  noise_sigma=bad, noise_seed=1)
        assert st == hsr.HSR_ERR_INVALID_ARG
    h.close()
