"""Solver variants beside Alg. 2 (Schur-Jacobi preconditioner, inexact-Newton
forcing sequence): the CUDA path against the oracle's implementation of the
same variant."""
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
    if kind == "ragged":
        return make_scene(40, 9001, track=("geom", 0.25), sigma=1.0, seed=22)
    if kind == "huber":
        return make_scene(12, 3001, track=("geom", 0.25), sigma=1.0, outlier_frac=0.05, seed=23)
    raise KeyError(kind)


def _colwise(got, ref, rtol, what):
    got, ref = np.asarray(got), np.asarray(ref)
    for a in range(ref.shape[1]):
        rel_close(got[:, a], ref[:, a], rtol, f"{what}[:, {a}]")


@pytest.mark.parametrize("kind", ["small", "ragged"])
def test_schur_jacobi_step_fp64_matches_oracle(mba, kind):
    sc = _scene(kind)
    mu = 1e-3
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx) as pr:
        st = pr.step(mu, pcg_max_iter=30, pcg_rel_tol=0.0, preconditioner="schur_jacobi")
    ref = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, pcg_max=30, pcg_tol=0.0,
                      precond="schur_jacobi")
    assert st["pcg_iters"] == ref["pcg_iters"] == 30
    _colwise(st["dc"], ref["dc"], 1e-6, "dc")
    _colwise(st["dp"], ref["dp"], 1e-6, "dp")
    assert st["model_dec"] == pytest.approx(ref["model_dec"], rel=1e-6)


def test_schur_jacobi_exact_for_one_camera(mba):
    """One camera: the preconditioner is S^-1, PCG stops after one step."""
    sc = make_scene(3, 80, track=("fixed", 2), sigma=1.0, seed=72)
    keep = sc.cam_idx == 1
    used = np.unique(sc.pt_idx[keep])
    remap = -np.ones(sc.np_, dtype=np.int64)
    remap[used] = np.arange(len(used))
    args = (sc.cameras[1:2], sc.points[used], sc.observations[keep], np.zeros(int(keep.sum()), np.int32),
            remap[sc.pt_idx[keep]].astype(np.int32))
    with mba.Problem(*args) as pr:
        st = pr.step(1e-3, pcg_max_iter=50, pcg_rel_tol=1e-10, preconditioner="schur_jacobi")
        bj = pr.step(1e-3, pcg_max_iter=50, pcg_rel_tol=1e-10)
    assert st["pcg_iters"] == 1 and bj["pcg_iters"] > 1


@pytest.mark.parametrize("kind,loss,precision,tol", [("ragged", "none", "fp64", 1e-6), ("huber", "huber", "fp64", 1e-6),
                                                     ("ragged", "none", "fp32", 1e-4)])
def test_schur_jacobi_solve_matches_oracle(mba, kind, loss, precision, tol):
    sc = _scene(kind)
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=6, pcg_max=40,
                          loss=loss, delta=2.0, precond="schur_jacobi")
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision, loss=loss,
                     huber_delta=2.0) as pr:
        s = pr.solve(trace_capacity=6, max_iter=6, pcg_max_iter=40, preconditioner="schur_jacobi")
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=tol)
    if precision == "fp64":
        for t, r in list(zip(s["trace"], ref["trace"]))[:3]:
            assert t["accepted"] == r["accepted"]
            assert abs(t["pcg_iters"] - r["pcg_iters"]) <= 1


@pytest.mark.parametrize("precond", ["block_jacobi", "schur_jacobi"])
def test_forcing_solve_matches_oracle(mba, precond):
    sc = _scene("ragged")
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=8, pcg_max=100,
                          precond=precond, forcing=True)
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx) as pr:
        s = pr.solve(trace_capacity=8, max_iter=8, pcg_max_iter=100, preconditioner=precond, forcing=1)
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=1e-6)
    assert s["trace"][0]["pcg_rel_residual"] <= 0.1
    assert abs(s["pcg_iters_total"] - sum(t["pcg_iters"] for t in ref["trace"])) <= 8


def test_variants_on_the_venice_shaped_problem(mba):
    """Full size, FP32-mixed, the bench's solve: each variant (and both together,
    whose inexact steps drive mu to about 1e-7, where FP32 rounding in the Schur
    product matters most) ends with status 0 at the paper's solver's final cost
    within 1e-3; the forcing sequence needs fewer PCG iterations in total, and on
    one damped system the Schur-Jacobi preconditioner needs fewer than the block
    Jacobi one (totals over a solve follow different LM trajectories)."""
    sc = config_scene(2)
    opts = dict(max_iter=20, pcg_max_iter=100, pcg_rel_tol=1e-10)
    out = {}
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision="fp32") as pr:
        for name, kw in (("bj", {}), ("sj", dict(preconditioner="schur_jacobi")), ("forcing", dict(forcing=1)),
                         ("both", dict(preconditioner="schur_jacobi", forcing=1))):
            pr.reset()
            out[name] = pr.solve(**opts, **kw)
        pr.reset()
        bj = pr.step(1e-3, pcg_max_iter=200, pcg_rel_tol=1e-8)
        sj = pr.step(1e-3, pcg_max_iter=200, pcg_rel_tol=1e-8, preconditioner="schur_jacobi")
    base = out["bj"]
    for name in ("sj", "forcing", "both"):
        assert out[name]["status"] == 0
        assert abs(out[name]["final_cost"] - base["final_cost"]) <= 1e-3 * base["final_cost"]
    assert out["forcing"]["pcg_iters_total"] < base["pcg_iters_total"]
    assert out["both"]["pcg_iters_total"] < base["pcg_iters_total"]
    assert sj["pcg_iters"] < bj["pcg_iters"]
