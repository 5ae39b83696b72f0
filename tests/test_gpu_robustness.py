"""Error paths through the C ABI on the GPU: the device-memory cap of
mba_set_device_memory_limit for problems and batches, and invalid solver
options.  None of these faults or hangs a GPU: the cap is checked on the host
before any allocation, and option checks come before any launch."""
import numpy as np
import pytest

import oracle
from scenes import make_scene, make_windows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mba():
    from paper_2112_01349_gb300 import _build, mba as m

    _build.build()
    m.load()
    return m


def test_memory_cap_gives_oom_for_problems_and_batches(mba):
    sc = make_scene(8, 300, sigma=0.5, seed=51)
    args = (sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    ws = make_windows(3, seed=9, cams=(5, 8), pts=(40, 80))
    tup = [(w.cameras, w.points, w.observations, w.cam_idx, w.pt_idx) for w in ws]
    with mba.Problem(*args) as before:  # created before the cap: unaffected by it
        mba.mba_set_device_memory_limit(64 * 1024)
        try:
            with pytest.raises(mba.MbaError) as e1:
                mba.Problem(*args)
            assert e1.value.status == mba.MBA_ERR_OOM
            with pytest.raises(mba.MbaError) as e2:
                mba.Batch(tup, precision="fp64")
            assert e2.value.status == mba.MBA_ERR_OOM
            s = before.solve(max_iter=3, pcg_max_iter=20)
            assert s["status"] == 0
        finally:
            mba.mba_set_device_memory_limit(0)
    # with the cap lifted, creation and a solve work and match the oracle
    ref = oracle.lm_solve(*args, max_iter=3, pcg_max=20)
    with mba.Problem(*args) as pr:
        s = pr.solve(max_iter=3, pcg_max_iter=20)
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=1e-6)
    with mba.Batch(tup, precision="fp64") as b:
        r = b.solve(max_iter=3, pcg_max_iter=20)
    assert all(sm["status"] == 0 for sm in r["summaries"])


def test_a_generous_cap_does_not_get_in_the_way(mba):
    sc = make_scene(8, 300, sigma=0.5, seed=52)
    mba.mba_set_device_memory_limit(1 << 30)
    try:
        with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision="fp32") as pr:
            s = pr.solve(max_iter=3, pcg_max_iter=20)
            assert s["status"] == 0 and pr.info["device_bytes"] < (1 << 30)
    finally:
        mba.mba_set_device_memory_limit(0)


@pytest.mark.parametrize("bad", [dict(cost_arithmetic=7), dict(preconditioner=5), dict(forcing=3), dict(max_iter=-1)])
def test_invalid_solver_options_are_rejected(mba, bad):
    sc = make_scene(4, 40, sigma=0.5, seed=53)
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision="fp32") as pr:
        o = mba.solver_options(max_iter=2)
        for k, v in bad.items():
            setattr(o, k, v)
        import ctypes

        s = mba.Summary()
        st = mba.load().mba_solve(pr.handle, ctypes.byref(o), ctypes.byref(s))
        assert st == mba.MBA_ERR_INVALID_ARG
        # the handle is still usable afterwards
        assert pr.solve(max_iter=2, pcg_max_iter=10)["status"] == 0
    assert np.isfinite(sc.cameras).all()
