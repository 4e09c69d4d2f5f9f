"""Failure detection of the raster's bounded waits, without a GPU fault: a
test hook arms every geometry staging for bytes that never arrive, each wait
gives up after its time limit, the kernel records the failure and returns;
the host reads HSR_ERR_TIMEOUT, and the next render on the same context is
correct again."""
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


def test_expired_wait_is_reported_and_context_survives():
    sc = wl.make_room(7, 3000)
    poses = wl.random_poses(sc, 2, 1)
    W = H = 32
    intr = Intrinsics(16.0, 16.0, 16.0, 16.0, 0.01, 10.0)
    h = hsr.SceneHandle(sc)
    cfg = hsr.hsr_config_default()
    cfg.n_phases = 1                          # one raster launch: about two seconds of expiring waits
    hsr.hsr_set_tuned_config([h.handle], 2, W, H, True, cfg)
    assert hsr.hsr_device_status(True) == hsr.HSR_OK
    ref = hsr.render(h, poses, intr, W, H)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in ref.items()}
    try:
        hsr.hsr_debug_inject_wait_fault(16)
        hsr.render(h, poses, intr, W, H)
        assert hsr.hsr_device_status(True) == hsr.HSR_ERR_TIMEOUT
    finally:
        hsr.hsr_debug_inject_wait_fault(0)
    again = hsr.render(h, poses, intr, W, H)
    torch.cuda.synchronize()
    assert hsr.hsr_device_status(True) == hsr.HSR_OK
    for k in ("rgb", "depth", "ids"):
        assert torch.equal(again[k], ref[k]), k
    hsr.hsr_set_tuned_config([h.handle], 2, W, H, True, None)
    h.close()
