"""Fixed (constant) nodes on the GPU against the oracle's fixed-node masks.

A node held constant has zero Jacobian columns (the g2o / Ceres convention of
the paper's graph API, Sec. 5.3).  The oracle takes the same masks and is
pinned on the CPU against a dense solve with the fixed rows and columns
deleted; here the CUDA path is compared with it through the C ABI: one damped
step (fixed PCG iteration count on both sides), whole LM solves, both forms,
Huber, the Schur-Jacobi preconditioner, and the graph API.
"""
import numpy as np
import pytest

import oracle
from scenes import make_scene
from tests.gpu_util import rel_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mba():
    from paper_2112_01349_gb300 import _build, mba as m

    _build.build()
    m.load()
    return m


def _masks(sc):
    cf = np.zeros(sc.nc, np.uint8)
    cf[[0, 3]] = 1
    pf = np.zeros(sc.np_, np.uint8)
    pf[::7] = 1
    return cf, pf


def _scene(kind):
    if kind == "ragged":
        return make_scene(40, 9001, track=("geom", 0.25), sigma=1.0, seed=22)
    if kind == "huber":
        return make_scene(12, 3001, track=("geom", 0.25), sigma=1.0, outlier_frac=0.05, seed=23)
    raise KeyError(kind)


@pytest.mark.parametrize("precision,pcg,tol", [("fp64", 30, 1e-6), ("fp32", 10, 1e-4)])
@pytest.mark.parametrize("kind", ["ragged", "huber"])
def test_fixed_step_matches_oracle(mba, kind, precision, pcg, tol):
    sc = _scene(kind)
    loss = "huber" if kind == "huber" else "none"
    cf, pf = _masks(sc)
    mu = 1e-2
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision, loss=loss,
                     huber_delta=2.0) as pr:
        pr.set_fixed(cf, pf)
        st = pr.step(mu, pcg_max_iter=pcg, pcg_rel_tol=0.0)
    ref = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, loss=loss, delta=2.0,
                      pcg_max=pcg, pcg_tol=0.0, cam_fixed=cf, pt_fixed=pf)
    assert st["pcg_iters"] == ref["pcg_iters"] == pcg
    assert np.all(st["dc"][cf == 1] == 0.0) and np.all(st["dp"][pf == 1] == 0.0)
    rel_close(st["dc"], ref["dc"], tol, "dc")
    rel_close(st["dp"], ref["dp"], tol, "dp")
    assert st["model_dec"] == pytest.approx(ref["model_dec"], rel=tol)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
@pytest.mark.parametrize("precond", ["block_jacobi", "schur_jacobi"])
def test_fixed_solve_matches_oracle(mba, precision, tol, precond):
    """Eight LM iterations with fixed nodes: final cost against the oracle's,
    the fixed nodes bit-identical to their initial values, the free ones moved."""
    sc = make_scene(16, 2000, sigma=0.5, seed=34)
    cf, pf = _masks(sc)
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=8, pcg_max=40,
                          precond=precond, cam_fixed=cf, pt_fixed=pf)
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision) as pr:
        pr.set_fixed(cf, pf)
        s = pr.solve(trace_capacity=8, max_iter=8, pcg_max_iter=40, preconditioner=precond)
        cams, pts = pr.parameters()
    assert s["iterations"] == 8 and s["accepted"] > 0
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=tol)
    np.testing.assert_array_equal(cams[cf == 1], sc.cameras[cf == 1])
    np.testing.assert_array_equal(pts[pf == 1], sc.points[pf == 1])
    assert np.any(cams[cf == 0] != sc.cameras[cf == 0]) and np.any(pts[pf == 0] != sc.points[pf == 0])
    assert [t["accepted"] for t in s["trace"]][:3] == [t["accepted"] for t in ref["trace"]][:3]


def test_all_nodes_fixed_gives_no_step(mba):
    sc = make_scene(6, 300, sigma=0.5, seed=35)
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx) as pr:
        pr.set_fixed(np.ones(sc.nc), np.ones(sc.np_))
        st = pr.step(1e-3, pcg_max_iter=20)
        s = pr.solve(trace_capacity=3, max_iter=3, pcg_max_iter=20)
        cams, pts = pr.parameters()
    assert np.all(st["dc"] == 0.0) and np.all(st["dp"] == 0.0) and st["model_dec"] == 0.0
    assert s["accepted"] == 0
    np.testing.assert_array_equal(cams, sc.cameras)
    np.testing.assert_array_equal(pts, sc.points)


def test_clearing_the_marks_restores_the_free_problem(mba):
    sc = _scene("ragged")
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx) as pr:
        free = pr.step(1e-2, pcg_max_iter=10, pcg_rel_tol=0.0)
        pr.set_fixed(*_masks(sc))
        pr.set_fixed(None, None)
        again = pr.step(1e-2, pcg_max_iter=10, pcg_rel_tol=0.0)
    np.testing.assert_array_equal(free["dc"], again["dc"])
    np.testing.assert_array_equal(free["dp"], again["dp"])


def test_graph_fixed_nodes_equal_the_array_masks(mba):
    sc = make_scene(8, 400, sigma=0.5, seed=36)
    cf, pf = _masks(sc)
    g = mba.Graph()
    for i in range(sc.nc):
        g.add_camera(sc.cameras[i], fixed=bool(cf[i]))
    for j in range(sc.np_):
        g.add_point(sc.points[j], fixed=bool(pf[j]))
    for k in range(sc.n):
        g.add_edge(int(sc.cam_idx[k]), int(sc.pt_idx[k]), sc.observations[k])
    with g.problem() as pr:
        s1 = pr.solve(max_iter=5, pcg_max_iter=30)
        c1, p1 = pr.parameters()
    with mba.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx) as pr:
        pr.set_fixed(cf, pf)
        s2 = pr.solve(max_iter=5, pcg_max_iter=30)
        c2, p2 = pr.parameters()
    assert s1["final_cost"] == s2["final_cost"]
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(p1, p2)
