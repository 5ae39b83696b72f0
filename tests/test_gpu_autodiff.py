"""Dual-number (forward-mode) Jacobians on the GPU (Sec. 3.2's automatic-
differentiation path) against the oracle's analytic Jacobian and the oracle's
solver, through the C ABI with jacobian="autodiff".

Tolerances as for the analytic path: residuals and Jacobians 1e-9 (FP64) and
1e-4 (FP32-mixed) relative; final cost after a fixed number of LM iterations
1e-6 (FP64) and 1e-4 (FP32-mixed); adjoint 1e-7 (FP64)."""
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
    if kind == "cfg1":
        return config_scene(1)
    if kind == "zero_rotation":  # first-order rotation branch: |w|^2 = 0 and |w|^2 below eps
        sc = make_scene(8, 600, sigma=0.5, seed=25)
        sc.cameras[0, :3] = 0.0
        sc.cameras[1, :3] = 1e-9
        return sc
    raise KeyError(kind)


def _problem(m, sc, precision="fp64", loss="none", jacobian="autodiff"):
    return m.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision, loss=loss,
                     huber_delta=2.0, jacobian=jacobian)


def _colwise(got, ref, rtol, what):
    got, ref = np.asarray(got).reshape(-1, got.shape[-1]), np.asarray(ref).reshape(-1, ref.shape[-1])
    for a in range(ref.shape[1]):
        rel_close(got[:, a], ref[:, a], rtol, f"{what}[:, {a}]")


@pytest.mark.parametrize("kind", ["small", "ragged", "zero_rotation"])
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_autodiff_evaluate_matches_oracle(mba, kind, precision, rtol):
    sc = _scene(kind)
    with _problem(mba, sc, precision) as pr:
        cost, e, jc, jp = pr.evaluate()
    rcost, re, rjc, rjp, _ = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    assert cost == pytest.approx(rcost, rel=1e-12)
    rel_close(e, re, rtol, "residual")
    _colwise(jc.reshape(-1, 9), rjc.reshape(-1, 9), rtol, "Jc")
    _colwise(jp.reshape(-1, 3), rjp.reshape(-1, 3), rtol, "Jp")


def test_autodiff_equals_analytic_fp64(mba):
    """Two derivations of the same Jacobian: equal to rounding (1e-12)."""
    sc = _scene("ragged")
    out = {}
    for jac in ("analytic", "autodiff"):
        with _problem(mba, sc, jacobian=jac) as pr:
            out[jac] = pr.evaluate()
    for i, what in ((1, "residual"), (2, "Jc"), (3, "Jp")):
        rel_close(out["autodiff"][i], out["analytic"][i], 1e-12, what)


@pytest.mark.parametrize("kind,loss,precision,tol", [("cfg1", "none", "fp64", 1e-6), ("huber", "huber", "fp64", 1e-6),
                                                     ("cfg1", "none", "fp32", 1e-4), ("huber", "huber", "fp32", 1e-4)])
def test_autodiff_solve_matches_oracle(mba, kind, loss, precision, tol):
    sc = _scene(kind)
    iters, pcg = 8, 50
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=iters, pcg_max=pcg,
                          loss=loss, delta=2.0)
    with _problem(mba, sc, precision, loss) as pr:
        s = pr.solve(trace_capacity=iters, max_iter=iters, pcg_max_iter=pcg)
        cams, pts = pr.parameters()
    assert s["status"] == 0 and s["iterations"] == iters
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=tol)
    if precision == "fp64":
        for t, r in list(zip(s["trace"], ref["trace"]))[:3]:
            assert t["accepted"] == r["accepted"]
            assert t["cost_new"] == pytest.approx(r["cost_new"], rel=1e-6)
        rc = oracle.evaluate(cams, pts, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0, jacobians=False)[0]
        assert rc == pytest.approx(s["final_cost"], rel=1e-12)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_autodiff_schur_jacobi_solve_matches_oracle(mba, precision, tol):
    sc = _scene("ragged")
    ref = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=6, pcg_max=40,
                          precond="schur_jacobi")
    with _problem(mba, sc, precision) as pr:
        s = pr.solve(max_iter=6, pcg_max_iter=40, preconditioner="schur_jacobi")
    assert s["final_cost"] == pytest.approx(ref["final_cost"], rel=tol)


def test_autodiff_adjoint_matches_oracle(mba):
    sc = _scene("huber")
    mu = 1e-2
    rng = np.random.default_rng(7)
    gc, gp = rng.normal(size=(sc.nc, 9)), rng.normal(size=(sc.np_, 3))
    ref = oracle.adjoint(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, gc, gp, loss="huber",
                         delta=2.0, pcg_max=1000, pcg_tol=1e-14)
    with _problem(mba, sc, "fp64", "huber") as pr:
        r = pr.adjoint(gc, gp, mu=mu, pcg_max_iter=1000, pcg_rel_tol=1e-14)
    rel_close(r["grad_obs"], ref["grad_obs"], 1e-7, "grad_obs")
    rel_close(r["grad_init_cam"], ref["grad_c0"], 1e-7, "grad_init_cam")
    rel_close(r["grad_init_pt"], ref["grad_p0"], 1e-7, "grad_init_pt")


def test_autodiff_fp32_schur_product_matches_oracle(mba):
    """FP32-mixed with dual numbers: the PCG camera pass streams the stored
    camera-major Jacobian; one S~p product against the oracle's."""
    sc = _scene("ragged")
    mu = 1e-2
    x = np.random.default_rng(6).normal(size=(sc.nc, 9))
    ref = oracle.schur(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu,
                       x=x.reshape(-1))["y"].reshape(-1, 9)
    with _problem(mba, sc, "fp32") as pr:
        got = pr.schur_matvec(mu, x)
    rel_close(got, ref, 1e-4, "S p")


def test_batch_rejects_autodiff(mba):
    ws = [make_scene(5, 60, sigma=1.0, seed=70 + i) for i in range(2)]
    arrays = mba.concat_windows([(s.cameras, s.points, s.observations, s.cam_idx, s.pt_idx) for s in ws])
    with pytest.raises(mba.MbaError, match="INVALID_ARG"):
        mba.mba_batch_create(*arrays, jacobian="autodiff")
