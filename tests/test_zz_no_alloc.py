"""The allocation-free cost entry point against the oracle's FP64 cost and the
existing mba_evaluate cost.

mba_cost_noalloc serves callers that cannot allocate device memory; it keeps
its scratch in a fixed device array inside the library.  This test calls it
through the C ABI on two different scenes in a row, the second with fewer
cameras and far fewer observations than the first, so that it uses fewer
camera-table rows and fewer partial sums than the call before it: stale
scratch from the first call would show in the second cost.  Each cost is
compared with the oracle's cost and with mba_evaluate on the same data, at the
FP64 cost tolerance the other GPU tests use (1e-12 relative).  An observation
index out of range gives a NaN cost.  It sorts last so a failure here comes
after every other test has run.
"""
import math

import numpy as np
import pytest

import oracle
from scenes import make_scene

pytestmark = pytest.mark.gpu


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _cost_noalloc(torch, mba, cams, pts, obs, ci, pi, loss, delta):
    stream = torch.cuda.current_stream()
    d = [_dev(torch, cams, np.float64), _dev(torch, pts, np.float64), _dev(torch, obs, np.float64),
         _dev(torch, ci, np.int32), _dev(torch, pi, np.int32)]
    d_cost = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    mba.mba_cost_noalloc(d[0].data_ptr(), cams.shape[0], d[1].data_ptr(), pts.shape[0], d[2].data_ptr(),
                         d[3].data_ptr(), d[4].data_ptr(), obs.shape[0], loss, delta, d_cost.data_ptr(), stream)
    torch.cuda.synchronize()
    return float(d_cost.item())


def test_cost_noalloc_matches_oracle_on_two_calls():
    import torch

    from paper_2112_01349_gb300 import _build, mba

    _build.build()
    mba.load()
    big = make_scene(20, 3000, track=("geom", 0.25), sigma=1.0, outlier_frac=0.02, seed=31)
    small = make_scene(5, 150, track=("geom", 0.25), sigma=1.0, outlier_frac=0.02, seed=32)
    assert small.nc < big.nc and small.n < big.n // 10
    for loss, delta in (("none", 0.0), ("huber", 2.0)):
        for sc in (big, small):  # two calls in a row; the second needs less scratch than the first
            args = (sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
            got = _cost_noalloc(torch, mba, *args, loss, delta)
            ref = oracle.evaluate(*args, loss, delta, jacobians=False)[0]
            assert got == pytest.approx(ref, rel=1e-12), (loss, sc.nc, got, ref)
            with mba.Problem(*args, loss=loss, huber_delta=delta) as pr:
                ev = pr.evaluate(residuals=False, jacobians=False)[0]
            assert got == pytest.approx(ev, rel=1e-12), (loss, sc.nc, got, ev)


def test_cost_noalloc_out_of_range_index_gives_nan():
    import torch

    from paper_2112_01349_gb300 import _build, mba

    _build.build()
    mba.load()
    sc = make_scene(5, 150, sigma=1.0, seed=33)
    ci = sc.cam_idx.copy()
    ci[17] = sc.nc  # one camera index past the end
    got = _cost_noalloc(torch, mba, sc.cameras, sc.points, sc.observations, ci, sc.pt_idx, "none", 0.0)
    assert math.isnan(got)
    # the next call with valid indices is unaffected
    args = (sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    got = _cost_noalloc(torch, mba, *args, "none", 0.0)
    assert got == pytest.approx(oracle.evaluate(*args, jacobians=False)[0], rel=1e-12)


def test_cost_noalloc_rejects_too_many_cameras():
    import torch

    from paper_2112_01349_gb300 import _build, mba

    _build.build()
    mba.load()
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(mba.MbaError) as ei:
        mba.mba_cost_noalloc(d.data_ptr(), 8193, d.data_ptr(), 1, d.data_ptr(), d.data_ptr(), d.data_ptr(), 1,
                             "none", 0.0, d.data_ptr(), None)
    assert ei.value.status == mba.MBA_ERR_INVALID_ARG
