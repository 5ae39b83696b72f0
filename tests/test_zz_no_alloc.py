"""The allocation-free cost entry point against the existing mba_evaluate cost.

mba_cost_noalloc serves callers that cannot allocate device memory; it keeps
its scratch in a fixed device array inside the library.  This test calls it
through the C ABI twice in a row (different inputs each time, so stale scratch
from the first call would show) and compares each cost with mba_evaluate on the
same data, at the FP64 cost tolerance the other GPU tests use (1e-12 relative).
It sorts last so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from scenes import make_scene

pytestmark = pytest.mark.gpu


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def test_cost_noalloc_matches_evaluate_on_two_calls():
    import torch

    from paper_2112_01349_gb300 import _build, mba

    _build.build()
    mba.load()
    sc = make_scene(20, 3000, track=("geom", 0.25), sigma=1.0, outlier_frac=0.02, seed=31)
    pts2 = sc.points + 0.01
    stream = torch.cuda.current_stream()
    d_cams = _dev(torch, sc.cameras, np.float64)
    d_obs = _dev(torch, sc.observations, np.float64)
    d_ci = _dev(torch, sc.cam_idx, np.int32)
    d_pi = _dev(torch, sc.pt_idx, np.int32)
    d_cost = torch.zeros(1, dtype=torch.float64, device="cuda")
    for loss, delta in (("none", 0.0), ("huber", 2.0)):
        for pts in (sc.points, pts2):  # two calls in a row with different points
            d_pts = _dev(torch, pts, np.float64)
            mba.mba_cost_noalloc(d_cams.data_ptr(), sc.nc, d_pts.data_ptr(), sc.np_, d_obs.data_ptr(),
                                 d_ci.data_ptr(), d_pi.data_ptr(), sc.n, loss, delta, d_cost.data_ptr(), stream)
            torch.cuda.synchronize()
            got = float(d_cost.item())
            with mba.Problem(sc.cameras, pts, sc.observations, sc.cam_idx, sc.pt_idx, loss=loss,
                             huber_delta=delta) as pr:
                ref = pr.evaluate(residuals=False, jacobians=False)[0]
            assert got == pytest.approx(ref, rel=1e-12), (loss, got, ref)


def test_cost_noalloc_rejects_too_many_cameras():
    import torch

    from paper_2112_01349_gb300 import mba

    mba.load()
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(mba.MbaError) as ei:
        mba.mba_cost_noalloc(d.data_ptr(), 8193, d.data_ptr(), 1, d.data_ptr(), d.data_ptr(), d.data_ptr(), 1,
                             "none", 0.0, d.data_ptr(), None)
    assert ei.value.status == mba.MBA_ERR_INVALID_ARG
