"""Parity at the benchmark's full sizes, in the launch configuration the bench
times (one persistent PCG CTA per SM): the Venice-shaped problem (1,700
cameras, 1M points, 5.0M observations) and the Final-shaped problem (13,000
cameras, 4.5M points, 29M observations, Huber).  Outputs the oracle can compute
one by one are compared on samples; the rest through properties that hold at
any size.  The Final-shaped problem has too many cameras for the search
direction to fit in shared memory, so its PCG runs the four-barrier form."""
import numpy as np
import pytest

import oracle
from scenes import config_scene
from tests.gpu_util import rel_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mba():
    from paper_2112_01349_gb300 import _build, mba as m

    _build.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def venice():
    return config_scene(2)


@pytest.fixture(scope="module")
def final():
    return config_scene(3)


def _problem(m, sc, precision, loss="none"):
    return m.Problem(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, precision=precision, loss=loss,
                     huber_delta=2.0)


def _colwise(got, ref, rtol, what):
    got, ref = np.asarray(got).reshape(-1, got.shape[-1]), np.asarray(ref).reshape(-1, ref.shape[-1])
    for a in range(ref.shape[1]):
        rel_close(got[:, a], ref[:, a], rtol, f"{what}[:, {a}]")


def _sub(sc, keep):
    return sc.observations[keep], sc.cam_idx[keep], sc.pt_idx[keep]


def _check_ordering(pr, sc):
    pt_perm, pt_ptr, cam_perm, cam_ptr = pr.ordering()
    rp, rpp = oracle.stable_sort(sc.pt_idx, sc.np_)
    np.testing.assert_array_equal(pt_perm, rp)
    np.testing.assert_array_equal(pt_ptr, rpp)
    rc, rcp = oracle.stable_sort(sc.cam_idx, sc.nc)
    np.testing.assert_array_equal(cam_perm, rc)
    np.testing.assert_array_equal(cam_ptr, rcp)


def _check_sampled_evaluate(pr, sc, loss, rtol_e, rtol_j, jacobians, seed):
    cost, e_all, jc_all, jp_all = pr.evaluate(residuals=True, jacobians=jacobians)
    k = np.random.default_rng(seed).choice(sc.n, size=2000, replace=False)
    e_ref, jc_ref, jp_ref = [], [], []
    for i in k:
        e, jc, jp = oracle.residual_jacobian(sc.cameras[sc.cam_idx[i]], sc.points[sc.pt_idx[i]], sc.observations[i])
        e_ref.append(e)
        jc_ref.append(jc)
        jp_ref.append(jp)
    _colwise(e_all[k], np.array(e_ref), rtol_e, "e")
    if jacobians:
        _colwise(jc_all[k].reshape(-1, 9), np.array(jc_ref).reshape(-1, 9), rtol_j, "Jc")
        _colwise(jp_all[k].reshape(-1, 3), np.array(jp_ref).reshape(-1, 3), rtol_j, "Jp")
    cost_ref = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0,
                               jacobians=False)[0]
    assert cost == pytest.approx(cost_ref, rel=1e-12)


def _check_schur_symmetric_spd(pr, sc, mu, tol):
    rng = np.random.default_rng(11)
    x, y = rng.normal(size=(sc.nc, 9)), rng.normal(size=(sc.nc, 9))
    sx, sy = pr.schur_matvec(mu, x), pr.schur_matvec(mu, y)
    a, b = float(np.sum(y * sx)), float(np.sum(x * sy))
    assert abs(a - b) <= tol * max(abs(a), abs(b))
    assert float(np.sum(x * sx)) > 0.0 and float(np.sum(y * sy)) > 0.0


# ---------------------------------------------------------------- Venice-shaped
def test_venice_ordering_bit_exact(mba, venice):
    with _problem(mba, venice, "fp32") as pr:
        _check_ordering(pr, venice)


@pytest.mark.parametrize("precision,rtol_e,rtol_j", [("fp64", 1e-9, 1e-9), ("fp32", 1e-4, 1e-4)])
def test_venice_evaluate_sampled(mba, venice, precision, rtol_e, rtol_j):
    with _problem(mba, venice, precision) as pr:
        _check_sampled_evaluate(pr, venice, "none", rtol_e, rtol_j, True, seed=1)


def test_venice_blocks_sampled(mba, venice):
    """B, v of sampled cameras and C, w of sampled points against the oracle's
    blocks over exactly the observations that feed them."""
    sc = venice
    with _problem(mba, sc, "fp64") as pr:
        ls = pr.linear_system(1e-2)
    rng = np.random.default_rng(2)
    cams = rng.choice(sc.nc, size=4, replace=False)
    obs, ci, pi = _sub(sc, np.isin(sc.cam_idx, cams))
    Hpp, v, _, _ = oracle.blocks(sc.cameras, sc.points, obs, ci, pi)
    _colwise(ls["Hpp"][cams].reshape(-1, 81), Hpp[cams].reshape(-1, 81), 1e-9, "B")
    _colwise(ls["v"][cams], v[cams], 1e-9, "v")
    pts = rng.choice(sc.np_, size=200, replace=False)
    obs, ci, pi = _sub(sc, np.isin(sc.pt_idx, pts))
    _, _, Hll, w = oracle.blocks(sc.cameras, sc.points, obs, ci, pi)
    _colwise(ls["Hll"][pts].reshape(-1, 9), Hll[pts].reshape(-1, 9), 1e-9, "C")
    _colwise(ls["w"][pts], w[pts], 1e-9, "w")


def test_venice_schur_product_symmetric_definite(mba, venice):
    with _problem(mba, venice, "fp64") as pr:
        _check_schur_symmetric_spd(pr, venice, 1e-3, 1e-10)


def test_venice_step_fp64_matches_oracle(mba, venice):
    """One damped step at full size: linearise, 20 PCG iterations (tolerance 0 on
    both sides), back-substitution and model decrease, against the oracle."""
    sc = venice
    mu = 1e-3
    with _problem(mba, sc, "fp64") as pr:
        st = pr.step(mu, pcg_max_iter=20, pcg_rel_tol=0.0)
    ref = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, pcg_max=20, pcg_tol=0.0)
    assert st["pcg_iters"] == ref["pcg_iters"] == 20
    _colwise(st["dc"], ref["dc"], 1e-6, "dc")
    _colwise(st["dp"], ref["dp"], 1e-6, "dp")
    assert st["model_dec"] == pytest.approx(ref["model_dec"], rel=1e-6)


def _compare_trajectory(s, ref, rtol, what):
    """Accept decisions of a GPU solve against the oracle's, iteration by
    iteration, and the new cost of every accepted step (within rtol), up to the first
    iteration whose decision sits at the rounding floor: a candidate cost
    within 1e-10 relative of the current cost, or a gain ratio within 1e-3 of
    the acceptance threshold.  There both decisions are correct and the
    trajectories may part.  A rejected candidate's cost is not compared: at the
    small damping where LM rejects, the step is dominated by the least
    determined directions of the system, so its cost says nothing about
    parity."""
    compared = 0
    for i, (t, r) in enumerate(zip(s["trace"], ref["trace"])):
        if abs(r["cost"] - r["cost_new"]) <= 1e-10 * r["cost"] or abs(r["gain"] - 1e-3) < 1e-3:
            break
        assert t["accepted"] == r["accepted"], f"{what}: iteration {i} accept {t['accepted']} vs {r['accepted']}"
        if r["accepted"]:
            assert t["cost_new"] == pytest.approx(r["cost_new"], rel=rtol), f"{what}: iteration {i}"
        compared += 1
    return compared


@pytest.fixture(scope="module")
def venice_oracle(venice):
    """The oracle's 20-iteration LM solve of the Venice-shaped problem (PCG <= 100)."""
    sc = venice
    return oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=20, pcg_max=100,
                           pcg_tol=1e-10)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_venice_trajectory_matches_oracle(mba, venice, venice_oracle, precision, rtol):
    """The bench's solve (20 LM iterations, PCG <= 100) against the oracle's on
    the same scene: final cost within 1e-6 (FP64) / 1e-4 (FP32-mixed), the
    same accept decisions wherever they are above the rounding floor, monotone
    accepted cost, and the returned parameters carrying the reported cost.  The
    parameter error against the oracle is printed raw and after the Umeyama
    similarity alignment."""
    from oracle.align import parameter_error

    sc, ref = venice, venice_oracle
    with _problem(mba, sc, precision) as pr:
        s = pr.solve(trace_capacity=20, max_iter=20, pcg_max_iter=100, pcg_rel_tol=1e-10)
        cams, pts = pr.parameters()
    assert s["status"] == 0 and s["iterations"] == 20
    assert s["initial_cost"] == pytest.approx(ref["trace"][0]["cost"], rel=1e-12)
    assert abs(s["final_cost"] - ref["final_cost"]) <= rtol * ref["final_cost"]
    acc = [t["cost_new"] for t in s["trace"] if t["accepted"]]
    assert all(b < a for a, b in zip(acc, acc[1:]))
    # intermediate FP32-mixed iterates of a capped PCG are less converged than
    # FP64's (measured: 2.2e-4 relative in the accepted cost at iteration 7);
    # the final cost is held to 1e-4 above
    n_cmp = _compare_trajectory(s, ref, rtol if precision == "fp64" else 1e-3, precision)
    assert n_cmp >= 2
    rc = oracle.evaluate(cams, pts, sc.observations, sc.cam_idx, sc.pt_idx, jacobians=False)[0]
    assert rc == pytest.approx(s["final_cost"], rel=1e-12)
    err = parameter_error(cams, pts, ref["cameras"], ref["points"])
    print(f"\nvenice {precision}: final cost {s['final_cost']!r} oracle {ref['final_cost']!r} rel "
          f"{(s['final_cost'] - ref['final_cost']) / ref['final_cost']:.3e}; decisions compared {n_cmp}; "
          f"accepted {s['accepted']} (oracle {sum(t['accepted'] for t in ref['trace'])}); parameter error {err}")
    assert np.isfinite(list(err.values())).all()
    assert err["aligned_point_rms"] <= err["raw_point_rms"] * (1 + 1e-9) + 1e-15


def test_venice_fp32_mixed_equals_fp64_final_cost(mba, venice):
    """FP32-mixed against FP64 on the bench's solve: equal final cost within
    1e-4 relative and the same initial cost (both evaluate it in FP64)."""
    opts = dict(max_iter=20, pcg_max_iter=100, pcg_rel_tol=1e-10)
    out = {}
    for prec in ("fp64", "fp32"):
        with _problem(mba, venice, prec) as pr:
            s = pr.solve(**opts)
        assert s["status"] == 0 and s["iterations"] == 20
        out[prec] = s["final_cost"]
        out[prec + "_initial"] = s["initial_cost"]
    assert abs(out["fp32"] - out["fp64"]) <= 1e-4 * out["fp64"]
    assert out["fp32_initial"] == pytest.approx(out["fp64_initial"], rel=1e-12)


# ---------------------------------------------------------------- Final-shaped
def test_final_ordering_bit_exact(mba, final):
    with _problem(mba, final, "fp32", "huber") as pr:
        _check_ordering(pr, final)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_final_residuals_sampled(mba, final, precision, rtol):
    with _problem(mba, final, precision, "huber") as pr:
        _check_sampled_evaluate(pr, final, "huber", rtol, rtol, False, seed=3)


def test_final_schur_product_symmetric_definite(mba, final):
    with _problem(mba, final, "fp64", "huber") as pr:
        _check_schur_symmetric_spd(pr, final, 1e-3, 1e-10)


@pytest.fixture(scope="module")
def final_oracle(final):
    """The oracle's first three LM iterations of the Final-shaped problem
    (Huber, delta 2 px, PCG <= 100)."""
    sc = final
    return oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=3, pcg_max=100,
                           pcg_tol=1e-10, loss="huber", delta=2.0)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_final_three_iterations_match_oracle(mba, final, final_oracle, precision, rtol):
    """Three LM iterations of the Final-shaped Huber problem (four-barrier PCG)
    against the oracle's: initial cost 1e-12, final cost within 1e-6 (FP64) /
    1e-4 (FP32-mixed), the same accept decisions above the rounding floor.  The
    parameter error against the oracle is printed raw and aligned."""
    from oracle.align import parameter_error

    sc, ref = final, final_oracle
    with _problem(mba, sc, precision, "huber") as pr:
        s = pr.solve(trace_capacity=3, max_iter=3, pcg_max_iter=100, pcg_rel_tol=1e-10)
        cams, pts = pr.parameters()
    assert s["status"] == 0 and s["iterations"] == 3
    assert s["initial_cost"] == pytest.approx(ref["trace"][0]["cost"], rel=1e-12)
    assert abs(s["final_cost"] - ref["final_cost"]) <= rtol * ref["final_cost"]
    n_cmp = _compare_trajectory(s, ref, rtol if precision == "fp64" else 1e-3, precision)
    assert n_cmp >= 1
    err = parameter_error(cams, pts, ref["cameras"], ref["points"])
    print(f"\nfinal {precision}: final cost {s['final_cost']!r} oracle {ref['final_cost']!r} rel "
          f"{(s['final_cost'] - ref['final_cost']) / ref['final_cost']:.3e}; decisions compared {n_cmp}; "
          f"parameter error {err}")
    assert np.isfinite(list(err.values())).all()


def test_final_fp32_mixed_equals_fp64_three_iterations(mba, final):
    """Three LM iterations of the Huber problem (four-barrier PCG) in both
    forms: the same accept/reject decisions, decreasing cost over the accepted
    steps, at least one accepted step, equal final cost within 1e-4."""
    opts = dict(max_iter=3, pcg_max_iter=100, pcg_rel_tol=1e-10)
    out = {}
    for prec in ("fp64", "fp32"):
        with _problem(mba, final, prec, "huber") as pr:
            s = pr.solve(trace_capacity=3, **opts)
        assert s["status"] == 0 and s["iterations"] == 3
        acc = [t["cost_new"] for t in s["trace"] if t["accepted"]]
        assert acc and acc[0] < s["initial_cost"]
        assert all(b < a for a, b in zip(acc, acc[1:]))
        out[prec] = s
    assert [t["accepted"] for t in out["fp32"]["trace"]] == [t["accepted"] for t in out["fp64"]["trace"]]
    f32, f64 = out["fp32"]["final_cost"], out["fp64"]["final_cost"]
    assert abs(f32 - f64) <= 1e-4 * f64
