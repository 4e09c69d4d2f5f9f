"""Autotuner: every launch configuration gives identical outputs, and a tuned
configuration is picked up by later calls with the same workload signature."""
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


def _np(out):
    torch.cuda.synchronize()
    return {"rgb": out["rgb"].cpu().numpy(), "depth": out["depth"].cpu().numpy(), "ids": hsr.ids_u32(out["ids"])}


def test_autotune_keeps_outputs_identical(tmp_path, monkeypatch):
    monkeypatch.setenv("HSR_TUNING_DIR", str(tmp_path))
    from paper_1904_01201_b300 import tuning
    sc = wl.make_house(2, 120_000, 512)
    h = hsr.SceneHandle(sc)
    poses = wl.random_poses(sc, 12, 2)
    intr = wl.pinhole_90(96, 96)
    ref = _np(hsr.render(h, poses, intr, 96, 96))
    out = hsr.alloc_outputs(12, 96, 96)
    cfg, src = tuning.ensure_tuned([sc], [h], None, poses, intr, 96, 96, out)
    assert src == "tuned" and 1 <= cfg["small_px"] <= 32 and 1 <= cfg["n_phases"] <= 3
    got = _np(hsr.render(h, poses, intr, 96, 96))          # uses the registered tuned config
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    # second process-equivalent: the cache is read back
    cfg2, src2 = tuning.ensure_tuned([sc], [h], None, poses, intr, 96, 96, out)
    assert src2 == "cache" and cfg2 == cfg
    h.close()


@pytest.mark.parametrize("small,bin_,chunk,phases,r0,r1,ctas", [
    (1, 1, 1, 1, 3.0, 7.0, 1), (32, 4096, 32, 3, 0.5, 1.0, 3), (8, 16, 2, 2, 2.0, 2.0, 2), (16, 64, 8, 3, 0.0, 30.0, 3)])
def test_every_config_gives_identical_images(small, bin_, chunk, phases, r0, r1, ctas):
    sc = wl.make_room(5, 6000)
    h = hsr.SceneHandle(sc)
    poses = wl.random_poses(sc, 6, 5)
    intr = wl.pinhole_90(80, 72)
    ref = _np(hsr.render(h, poses, intr, 80, 72))
    cfg = hsr.hsr_config(small, bin_, chunk, ctas, phases, (r0, r1))
    hsr.hsr_set_tuned_config([h.handle], 6, 80, 72, True, cfg)
    got = _np(hsr.render(h, poses, intr, 80, 72))
    hsr.hsr_set_tuned_config([h.handle], 6, 80, 72, True, None)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    h.close()
