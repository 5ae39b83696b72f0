"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances: index work bit-exact; FP64 residuals/Jacobians 1e-9 relative;
FP64 blocks and Schur products 1e-9 per parameter column; final cost after a
fixed number of LM iterations 1e-6 (FP64) and 1e-4 (FP32-mixed) relative.
"""
import numpy as np
import pytest

import oracle
from scenes import config_scene, make_scene
from tests.gpu_util import rel_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mba():
    from paper_2112_01349_gb300 import _build, mba as m

    _build.build()
    m.load()
    return m


def _scene(kind):
    if kind == "small":
        return make_scene(6, 400, sigma=0.5, seed=21)
    if kind == "ragged":  # many point chunks, geometric tracks, ragged tail
        return make_scene(40, 9001, track=("geom", 0.25), sigma=1.0, seed=22)
    if kind == "huber":
        return make_scene(12, 3001, track=("geom", 0.25), sigma=1.0, outlier_frac=0.05, seed=23)
    if kind == "cfg1":
        return config_scene(1)
    if kind == "longtrack":  # heavy-tailed tracks up to 300 observations
        return make_scene(320, 3000, track=("lognormal", 6.5, 300), sigma=1.0, seed=24)
    if kind == "manycams":  # camera rows too large for shared memory: the staged FP32 point pass
        return make_scene(5000, 20000, track=("lognormal", 6.5, 300), sigma=1.0, seed=25)
    raise KeyError(kind)


def _problem(m, sc, precision="fp64", loss="none", delta=0.0):
    return m.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision, loss=loss,
                     huber_delta=delta)


def _colwise(got, ref, rtol, what):
    got, ref = np.asarray(got).reshape(-1, got.shape[-1]), np.asarray(ref).reshape(-1, ref.shape[-1])
    for a in range(ref.shape[1]):
        rel_close(got[:, a], ref[:, a], rtol, f"{what}[:, {a}]")


@pytest.mark.parametrize("kind", ["small", "ragged", "longtrack"])
def test_ordering_is_bit_exact(mba, kind):
    sc = _scene(kind)
    with _problem(mba, sc) as pr:
        pt_perm, pt_ptr, cam_perm, cam_ptr = pr.ordering()
    rp, rpp = oracle.stable_sort(sc.pt_idx, sc.np_)
    rc, rcp = oracle.stable_sort(sc.cam_idx, sc.nc)
    np.testing.assert_array_equal(pt_perm, rp)
    np.testing.assert_array_equal(pt_ptr, rpp)
    np.testing.assert_array_equal(cam_perm, rc)
    np.testing.assert_array_equal(cam_ptr, rcp)


@pytest.mark.parametrize("kind", ["small", "ragged"])
def test_evaluate_fp64(mba, kind):
    sc = _scene(kind)
    with _problem(mba, sc) as pr:
        cost, e, jc, jp = pr.evaluate()
    rcost, re, rjc, rjp, _ = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    assert cost == pytest.approx(rcost, rel=1e-12)
    rel_close(e, re, 1e-9, "residual")
    _colwise(jc.reshape(-1, 9), rjc.reshape(-1, 9), 1e-9, "Jc")
    _colwise(jp.reshape(-1, 3), rjp.reshape(-1, 3), 1e-9, "Jp")


def test_evaluate_fp32_mixed(mba):
    sc = _scene("ragged")
    with _problem(mba, sc, "fp32") as pr:
        cost, e, jc, jp = pr.evaluate()
    rcost, re, rjc, rjp, _ = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    assert cost == pytest.approx(rcost, rel=1e-12)  # the cost is FP64 in both forms
    rel_close(e, re, 1e-4, "residual")
    _colwise(jc.reshape(-1, 9), rjc.reshape(-1, 9), 1e-4, "Jc")
    _colwise(jp.reshape(-1, 3), rjp.reshape(-1, 3), 1e-4, "Jp")


@pytest.mark.parametrize("kind,loss", [("small", "none"), ("ragged", "none"), ("huber", "huber")])
def test_linear_system_fp64(mba, kind, loss):
    sc = _scene(kind)
    mu = 1e-3
    with _problem(mba, sc, loss=loss, delta=2.0) as pr:
        ls = pr.linear_system(mu)
    Hpp, v, Hll, w = oracle.blocks(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0)
    rhs = oracle.schur(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, loss=loss,
                       delta=2.0)["rhs"].reshape(-1, 9)
    _colwise(ls["Hpp"].reshape(-1, 9), Hpp.reshape(-1, 9), 1e-9, "Hpp")
    _colwise(ls["v"], v, 1e-9, "v")
    _colwise(ls["Hll"].reshape(-1, 3), Hll.reshape(-1, 3), 1e-9, "Hll")
    _colwise(ls["w"], w, 1e-9, "w")
    _colwise(ls["rhs"], rhs, 1e-8, "rhs")


@pytest.mark.parametrize("kind,damping", [("small", "diag"), ("ragged", "diag"), ("ragged", "identity"),
                                          ("longtrack", "diag")])
def test_schur_matvec_fp64(mba, kind, damping):
    sc = _scene(kind)
    mu = 1e-2
    x = np.random.default_rng(5).normal(size=(sc.nc, 9))
    with _problem(mba, sc) as pr:
        y = pr.schur_matvec(mu, x, damping)
    ref = oracle.schur(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, x=x.reshape(-1),
                       damping=damping)["y"].reshape(-1, 9)
    _colwise(y, ref, 1e-9, "Sx")


@pytest.mark.parametrize("kind", ["ragged", "manycams"])
def test_schur_matvec_fp32_mixed(mba, kind):
    sc = _scene(kind)
    mu = 1e-2
    x = np.random.default_rng(6).normal(size=(sc.nc, 9))
    with _problem(mba, sc, "fp32") as pr:
        y = pr.schur_matvec(mu, x)
    ref = oracle.schur(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu,
                       x=x.reshape(-1))["y"].reshape(-1, 9)
    rel_close(y, ref, 1e-4, "Sx fp32")


@pytest.mark.parametrize("kind", ["small", "ragged"])
def test_step_fp64(mba, kind):
    sc = _scene(kind)
    mu = 1e-3
    # a fixed number of PCG steps on both sides (tolerance 0), so the comparison
    # does not hinge on which side crosses a stopping threshold first
    with _problem(mba, sc) as pr:
        st = pr.step(mu, pcg_max_iter=30, pcg_rel_tol=0.0)
    ref = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, pcg_max=30, pcg_tol=0.0)
    assert st["pcg_iters"] == ref["pcg_iters"] == 30
    _colwise(st["dc"], ref["dc"], 1e-6, "dc")
    _colwise(st["dp"], ref["dp"], 1e-6, "dp")
    assert st["model_dec"] == pytest.approx(ref["model_dec"], rel=1e-6)


@pytest.mark.parametrize("arith,rtol", [("fp64", 1e-12), ("float-float", 1e-11)])
@pytest.mark.parametrize("kind,loss", [("ragged", "none"), ("huber", "huber"), ("cfg1", "none")])
def test_fp32_mixed_solve_cost_matches_fp64(mba, kind, loss, arith, rtol):
    """The FP32-mixed solve evaluates the cost for accept/reject in FP64 (the
    default) or, as an option, in float-float arithmetic: its initial and final
    costs equal the oracle's FP64 costs at the same parameters to 1e-12 (FP64)
    or 1e-11 (float-float) relative."""
    sc = _scene(kind)
    rc0 = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0,
                          jacobians=False)[0]
    with _problem(mba, sc, "fp32", loss=loss, delta=2.0) as pr:
        s = pr.solve(max_iter=3, pcg_max_iter=20, cost_arithmetic=arith)
        cams, pts = pr.parameters()
    rc1 = oracle.evaluate(cams, pts, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0, jacobians=False)[0]
    assert s["initial_cost"] == pytest.approx(rc0, rel=rtol)
    assert s["final_cost"] == pytest.approx(rc1, rel=rtol)


@pytest.mark.parametrize("kind,loss", [("ragged", "none"), ("huber", "huber"), ("manycams", "none")])
def test_step_fp32_mixed(mba, kind, loss):
    """One damped step in FP32-mixed (the factored Schur product and
    back-substitution) against the FP64 oracle: camera and point steps and the
    model decrease at 1e-4, with 10 fixed PCG iterations on both sides."""
    sc = _scene(kind)
    mu = 1e-2
    with _problem(mba, sc, "fp32", loss=loss, delta=2.0) as pr:
        st = pr.step(mu, pcg_max_iter=10, pcg_rel_tol=0.0)
    ref = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, pcg_max=10, pcg_tol=0.0,
                      loss=loss, delta=2.0)
    assert st["pcg_iters"] == ref["pcg_iters"] == 10
    rel_close(st["dc"], ref["dc"], 1e-4, "dc")
    rel_close(st["dp"], ref["dp"], 1e-4, "dp")
    assert st["model_dec"] == pytest.approx(ref["model_dec"], rel=1e-4)


@pytest.mark.parametrize("kind,loss,iters,pcg", [("cfg1", "none", 10, 50), ("ragged", "none", 6, 40),
                                                 ("huber", "huber", 6, 40), ("longtrack", "none", 5, 30)])
def test_solve_fp64_final_cost(mba, kind, loss, iters, pcg):
    sc = _scene(kind)
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=iters, pcg_max=pcg,
                          loss=loss, delta=2.0)
    with _problem(mba, sc, loss=loss, delta=2.0) as pr:
        s = pr.solve(trace_capacity=iters, max_iter=iters, pcg_max_iter=pcg)
        cams, pts = pr.parameters()
    assert s["iterations"] == iters
    assert s["initial_cost"] == pytest.approx(ref["trace"][0]["cost"], rel=1e-12)
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=1e-6)
    # the early, decisive iterations follow the same trajectory
    for t, r in list(zip(s["trace"], ref["trace"]))[:3]:
        assert t["accepted"] == r["accepted"]
        assert t["cost_new"] == pytest.approx(r["cost_new"], rel=1e-6)
    # the returned parameters carry the reported cost
    rc = oracle.evaluate(cams, pts, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0, jacobians=False)[0]
    assert rc == pytest.approx(s["final_cost"], rel=1e-12)


@pytest.mark.parametrize("kind,loss,iters", [("cfg1", "none", 10), ("huber", "huber", 10), ("manycams", "none", 5)])
def test_solve_fp32_mixed_final_cost(mba, kind, loss, iters):
    sc = _scene(kind)
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=iters, pcg_max=50,
                          loss=loss, delta=2.0)
    with _problem(mba, sc, "fp32", loss=loss, delta=2.0) as pr:
        s = pr.solve(max_iter=iters, pcg_max_iter=50)
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=1e-4)


def test_staged_point_pass_repeats_bit_for_bit(mba):
    """The staged FP32 point pass (camera rows too large for shared memory, so
    tiles are copied into shared-memory stages while warps drift across them)
    gives the same bits on every run: each chunk's sums do not depend on which
    warp or stage took it."""
    sc = _scene("manycams")
    mu = 1e-2
    with _problem(mba, sc, "fp32") as pr:
        a = pr.step(mu, pcg_max_iter=15, pcg_rel_tol=0.0)
        b = pr.step(mu, pcg_max_iter=15, pcg_rel_tol=0.0)
    np.testing.assert_array_equal(a["dc"], b["dc"])
    np.testing.assert_array_equal(a["dp"], b["dp"])


def test_degenerate_minimal_problem(mba):
    # two cameras, one point each seen once or twice: singular undamped blocks, damping makes them definite
    cams = np.array([[0.1, -0.2, 0.05, 0.0, 0.0, -5.0, 800.0, 0.0, 0.0],
                     [-0.05, 0.1, 0.0, 0.2, 0.0, -6.0, 900.0, 0.01, 0.0]])
    pts = np.array([[0.1, 0.2, -0.1], [0.0, -0.1, 0.3], [0.2, 0.0, 0.0]])
    cam_idx = np.array([0, 1, 0, 1], np.int32)
    pt_idx = np.array([0, 0, 1, 2], np.int32)
    obs = np.array([oracle.project(cams[c], pts[p]) for c, p in zip(cam_idx, pt_idx)]) + 0.5
    ref = oracle.lm_solve(cams, pts, obs, cam_idx, pt_idx, max_iter=4, pcg_max=20)
    with mba.Problem(cams, pts, obs, cam_idx, pt_idx) as pr:
        s = pr.solve(max_iter=4, pcg_max_iter=20)
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=1e-6, abs=1e-12)


def test_invalid_inputs_are_rejected(mba):
    sc = _scene("small")
    bad = sc.cam_idx.copy()
    bad[3] = sc.nc
    with pytest.raises(mba.MbaError) as ei:
        mba.Problem(sc.cameras, sc.points, sc.observations, bad, sc.pt_idx)
    assert ei.value.status == mba.MBA_ERR_INVALID_ARG
    obs = sc.observations.copy()
    obs[7, 1] = np.nan
    with pytest.raises(mba.MbaError) as ei:
        mba.Problem(sc.cameras, sc.points, obs, sc.cam_idx, sc.pt_idx)
    assert ei.value.status == mba.MBA_ERR_NONFINITE
    # an extra camera nobody observes
    cams = np.concatenate([sc.cameras, sc.cameras[:1]])
    with pytest.raises(mba.MbaError) as ei:
        mba.Problem(cams, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    assert ei.value.status == mba.MBA_ERR_INVALID_ARG


def test_track_longer_than_supported_is_rejected(mba):
    sc = make_scene(1100, 2, track=("fixed", 1100), sigma=1.0, seed=3)
    with pytest.raises(mba.MbaError) as ei:
        mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    assert ei.value.status == mba.MBA_ERR_INVALID_ARG


def test_barrier_timeout_returns_status_and_context_survives(mba):
    sc = _scene("ragged")
    with _problem(mba, sc) as pr:
        with pytest.raises(mba.MbaError) as ei:
            pr.solve(max_iter=2, pcg_max_iter=10, barrier_spin_limit=1)
        assert ei.value.status == mba.MBA_ERR_TIMEOUT
        pr.reset()
        s = pr.solve(max_iter=2, pcg_max_iter=10)
        assert s["status"] == 0 and s["iterations"] == 2


def test_non_positive_definite_block_is_a_rejected_iteration(mba):
    """The oracle pin's scene (a point seen by one camera, identity damping at
    mu = 1e-16): the solve completes, and every iteration without a step (no PCG
    iterations) is rejected with no candidate cost; the final cost is not above
    the initial one."""
    from tests.test_oracle_pins import _one_view_point_scene

    cams, pts, obs, ci, pi = _one_view_point_scene()
    with mba.Problem(cams, pts, obs, ci, pi) as pr:
        s = pr.solve(trace_capacity=6, max_iter=6, pcg_max_iter=20, damping="identity", initial_radius=1e16)
    assert s["status"] == 0 and s["iterations"] == 6
    for t in s["trace"]:
        if t["pcg_iters"] == 0:
            assert not t["accepted"] and not np.isfinite(t["cost_new"])
    assert s["final_cost"] <= s["initial_cost"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resume_from_a_checkpoint_continues_the_trajectory(mba, precision):
    """Checkpoint / resume through host memory: a solve stopped after an
    accepted step, checkpointed (parameters read back, final radius kept) and
    resumed in a fresh handle created from those parameters with that radius,
    continues the uninterrupted solve bit for bit (after any accepted step the
    trust region's decrease factor is 2, as at a start).  Tiny workload, split
    after the third iteration, both forms."""
    sc = _scene("cfg1")
    kw = dict(pcg_max_iter=50, pcg_rel_tol=1e-10)
    with _problem(mba, sc, precision) as pr:
        full = pr.solve(trace_capacity=10, max_iter=10, **kw)
        cams_full, pts_full = pr.parameters()
        pr.reset()
        first = pr.solve(trace_capacity=3, max_iter=3, **kw)
        cams_ck, pts_ck = pr.parameters()
    assert first["trace"][-1]["accepted"] == 1
    with mba.Problem(cams_ck, pts_ck, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision) as pr2:
        rest = pr2.solve(trace_capacity=7, max_iter=7, initial_radius=first["final_radius"], **kw)
        cams, pts = pr2.parameters()
    assert rest["final_cost"] == full["final_cost"]
    assert [t["cost_new"] for t in rest["trace"]] == [t["cost_new"] for t in full["trace"][3:]]
    assert [t["accepted"] for t in rest["trace"]] == [t["accepted"] for t in full["trace"][3:]]
    np.testing.assert_array_equal(cams, cams_full)
    np.testing.assert_array_equal(pts, pts_full)
