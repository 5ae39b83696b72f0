"""Batched local-BA windows: every window of one launch against the CPU
oracle solving that window alone (same LM rule, PCG and adjoint)."""
import numpy as np
import pytest

import oracle
from scenes import make_scene, make_windows
from tests.gpu_util import rel_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mba():
    from paper_2112_01349_gb300 import _build, mba as m

    _build.build()
    m.load()
    return m


def _tuples(ws):
    return [(s.cameras, s.points, s.observations, s.cam_idx, s.pt_idx) for s in ws]


def _small(count=12, seed=11, cams=(5, 12), pts=(40, 300)):
    return make_windows(count, seed=seed, cams=cams, pts=pts)


OPTS = dict(max_iter=8, pcg_max_iter=100, pcg_rel_tol=1e-10)


def _oracle_solve(s, loss="none", delta=0.0, **kw):
    o = dict(max_iter=OPTS["max_iter"], pcg_max=OPTS["pcg_max_iter"], pcg_tol=OPTS["pcg_rel_tol"])
    o.update(kw)
    return oracle.lm_solve(s.cameras, s.points, s.observations, s.cam_idx, s.pt_idx, loss=loss, delta=delta, **o)


@pytest.mark.parametrize("schur", ["implicit", "explicit"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_windows_match_oracle(mba, precision, tol, schur):
    ws = _small()
    with mba.Batch(_tuples(ws), precision=precision) as b:
        b.set_schedule(schur=schur)
        assert b.schedule()["schur"] == schur
        r = b.solve(**OPTS)
        for w, s in enumerate(ws):
            ref = _oracle_solve(s)
            sm = r["summaries"][w]
            assert sm["status"] == 0
            assert sm["iterations"] == ref["iterations"]
            rel_close(sm["final_cost"], ref["final_cost"], tol, f"window {w} final cost")
            if precision == "fp64":
                assert sm["accepted"] == sum(t["accepted"] for t in ref["trace"])
                cams, pts = b.window_parameters(w)
                rel_close(cams, ref["cameras"], 1e-5, f"window {w} cameras")
                rel_close(pts, ref["points"], 1e-5, f"window {w} points")
            assert sm["final_cost"] < sm["initial_cost"]


@pytest.mark.parametrize("schur", ["implicit", "explicit"])
def test_windows_huber_match_oracle(mba, schur):
    ws = [make_scene(int(nc), int(npt), track=("geom", 1.0 / 3.0), sigma=1.0, outlier_frac=0.05, seed=100 + i)
          for i, (nc, npt) in enumerate([(6, 120), (9, 250), (14, 400), (5, 60)])]
    with mba.Batch(_tuples(ws), precision="fp64", loss="huber", huber_delta=2.0) as b:
        b.set_schedule(schur=schur)
        r = b.solve(**OPTS)
    for w, s in enumerate(ws):
        ref = _oracle_solve(s, loss="huber", delta=2.0)
        rel_close(r["summaries"][w]["final_cost"], ref["final_cost"], 1e-6, f"huber window {w}")


@pytest.mark.parametrize("schur", ["implicit", "explicit"])
def test_window_long_tracks(mba, schur):
    """Points seen by more than 32 cameras take the long-track path of the point
    passes; 48 cameras give 1176 Schur blocks per window."""
    ws = [make_scene(48, 150, track=("fixed", 40), sigma=1.0, seed=61), make_scene(40, 80, track=("fixed", 36),
                                                                                   sigma=1.0, seed=62),
          make_scene(7, 90, sigma=1.0, seed=63)]
    with mba.Batch(_tuples(ws), precision="fp64") as b:
        b.set_schedule(schur=schur)
        r = b.solve(**OPTS)
    for w, s in enumerate(ws):
        ref = _oracle_solve(s)
        rel_close(r["summaries"][w]["final_cost"], ref["final_cost"], 1e-6, f"long-track window {w}")


def test_batch_matches_single_problem_solver(mba):
    """The same window through mba_solve (grid-wide kernels) and through the batch."""
    s = make_windows(3, seed=5)[1]
    with mba.Problem(s.cameras, s.points, s.observations, s.cam_idx, s.pt_idx) as pr:
        single = pr.solve(**OPTS)
        cs, ps = pr.parameters()
    with mba.Batch(_tuples([s]), precision="fp64") as b:
        r = b.solve(**OPTS)
        cb, pb = b.parameters()
    rel_close(r["summaries"][0]["final_cost"], single["final_cost"], 1e-9, "final cost")
    rel_close(cb, cs, 1e-7, "cameras")
    rel_close(pb, ps, 1e-7, "points")


@pytest.mark.parametrize("schur", ["implicit", "explicit"])
@pytest.mark.parametrize("precision,mu,tol,init", [("fp64", -1.0, 1e-6, True), ("fp64", 1e-2, 1e-6, True),
                                                   ("fp32", -1.0, 3e-3, False), ("fp32", 1e-2, 3e-3, True)])
def test_batch_adjoint_matches_oracle(mba, precision, mu, tol, init, schur):
    """mu < 0: each window's last accepted mu (tiny after 8 good steps, so the
    damped system is nearly singular along the 7-DoF gauge).  The observation
    gradient W J v does not see the gauge and matches in both precisions; the
    initial-estimate gradient mu D v is mostly gauge there and is compared in
    FP32 only at a well-conditioned mu."""
    ws = _small(count=6, seed=31)
    rng = np.random.default_rng(9)
    with mba.Batch(_tuples(ws), precision=precision) as b:
        b.set_schedule(schur=schur)
        gc = rng.normal(size=(b.info["nc"], 9))
        gp = rng.normal(size=(b.info["np"], 3))
        r = b.solve(gc, gp, adjoint_pcg_max_iter=1000, adjoint_pcg_rel_tol=1e-14, adjoint_mu=mu, **OPTS)
        g = b.gradients()
        cams, pts = b.parameters()
    co, po, oo = b.offsets
    for w, s in enumerate(ws):
        sm = r["summaries"][w]
        assert sm["accepted"] > 0 and sm["mu_accepted"] > 0 and sm["adjoint_pcg_iters"] > 0
        c, p = cams[co[w]:co[w + 1]], pts[po[w]:po[w + 1]]
        ref = oracle.adjoint(c, p, s.observations, s.cam_idx, s.pt_idx, sm["mu_accepted"] if mu < 0 else mu,
                             gc[co[w]:co[w + 1]], gp[po[w]:po[w + 1]], pcg_max=1000, pcg_tol=1e-14)
        rel_close(g["grad_obs"][oo[w]:oo[w + 1]], ref["grad_obs"], tol, f"window {w} grad_obs")
        if init:
            rel_close(g["grad_init_cam"][co[w]:co[w + 1]], ref["grad_c0"], tol, f"window {w} grad_init_cam")
            rel_close(g["grad_init_pt"][po[w]:po[w + 1]], ref["grad_p0"], tol, f"window {w} grad_init_pt")


def test_adjoint_without_accepted_step_is_identity(mba):
    ws = _small(count=3, seed=41)
    rng = np.random.default_rng(2)
    with mba.Batch(_tuples(ws), precision="fp64") as b:
        gc, gp = rng.normal(size=(b.info["nc"], 9)), rng.normal(size=(b.info["np"], 3))
        r = b.solve(gc, gp, max_iter=0)
        g = b.gradients()
    assert all(s["accepted"] == 0 and s["mu_accepted"] == -1.0 for s in r["summaries"])
    assert np.all(g["grad_obs"] == 0.0)
    assert np.array_equal(g["grad_init_cam"], gc) and np.array_equal(g["grad_init_pt"], gp)


def test_schedules_agree_and_repeat_bit_exactly(mba):
    ws = _small(count=10, seed=51)
    out = {}
    with mba.Batch(_tuples(ws), precision="fp32") as b:
        for nt, schur in ((256, "implicit"), (512, "implicit"), (256, "explicit"), (512, "explicit")):
            b.set_schedule(nt, 1, schur)
            res = []
            for _ in range(2):
                b.reset()
                res.append((b.solve(**OPTS), b.parameters()))
            (r1, (c1, p1)), (r2, (c2, p2)) = res
            assert np.array_equal(c1, c2) and np.array_equal(p1, p2), f"schedule {nt} is not deterministic"
            assert [s["final_cost"] for s in r1["summaries"]] == [s["final_cost"] for s in r2["summaries"]]
            out[(nt, schur)] = np.array([s["final_cost"] for s in r1["summaries"]])
        best = b.autotune(**OPTS)
        assert best["threads_per_cta"] in (256, 512) and best["ctas_per_sm"] >= 1 and best["ms"] > 0
        assert best["schur"] in ("implicit", "explicit")
        assert b.schedule()["threads_per_cta"] == best["threads_per_cta"]
    for k in out:
        rel_close(out[k], out[(256, "implicit")], 1e-4, f"final costs, schedule {k}")


def test_invalid_batches(mba):
    s = make_scene(6, 50, sigma=1.0, seed=3)
    t = (s.cameras, s.points, s.observations, s.cam_idx, s.pt_idx)
    bad_idx = (s.cameras, s.points, s.observations, s.cam_idx + 6, s.pt_idx)
    with pytest.raises(mba.MbaError) as e:
        mba.Batch([t, bad_idx])
    assert e.value.status == mba.MBA_ERR_INVALID_ARG
    big = make_scene(65, 200, track=("fixed", 5), sigma=1.0, seed=4)
    with pytest.raises(mba.MbaError) as e:
        mba.Batch(_tuples([big]))
    assert e.value.status == mba.MBA_ERR_INVALID_ARG
    keep = s.cam_idx != 2
    with pytest.raises(mba.MbaError) as e:  # camera 2 loses all of its observations
        mba.Batch([(s.cameras, s.points, s.observations[keep], s.cam_idx[keep], s.pt_idx[keep])])
    assert e.value.status == mba.MBA_ERR_INVALID_ARG
    nan_obs = s.observations.copy()
    nan_obs[3, 0] = np.nan
    with pytest.raises(mba.MbaError) as e:
        mba.Batch([(s.cameras, s.points, nan_obs, s.cam_idx, s.pt_idx)])
    assert e.value.status == mba.MBA_ERR_NONFINITE
    nan_cam = s.cameras.copy()
    nan_cam[1, 4] = np.inf
    with pytest.raises(mba.MbaError) as e:
        mba.Batch([t, (nan_cam, s.points, s.observations, s.cam_idx, s.pt_idx)])
    assert e.value.status == mba.MBA_ERR_NONFINITE
    bad_pt = s.pt_idx.copy()
    bad_pt[7] = -1
    with pytest.raises(mba.MbaError) as e:
        mba.Batch([t, (s.cameras, s.points, s.observations, s.cam_idx, bad_pt)])
    assert e.value.status == mba.MBA_ERR_INVALID_ARG
    keep_pt = s.pt_idx != 5
    with pytest.raises(mba.MbaError) as e:  # point 5 loses all of its observations
        mba.Batch([(s.cameras, s.points, s.observations[keep_pt], s.cam_idx[keep_pt], s.pt_idx[keep_pt]), t])
    assert e.value.status == mba.MBA_ERR_INVALID_ARG
    # a valid batch after the failures
    with mba.Batch([t, t]) as b:
        r = b.solve(max_iter=2, pcg_max_iter=20)
    assert r["summaries"][0]["final_cost"] == r["summaries"][1]["final_cost"]


def test_device_layout_repeats_bit_for_bit(mba):
    """The batch's layout (orders, warp chunks, Schur pair lists) is built on the
    device with stable sorts: two creations of the same batch give the same
    bits, and a window's result does not depend on the windows around it."""
    ws = _small(count=10, seed=81)
    runs = []
    for _ in range(2):
        with mba.Batch(_tuples(ws), precision="fp32") as b:
            b.set_schedule(256, 2, "explicit")
            r = b.solve(**OPTS)
            runs.append(([x["final_cost"] for x in r["summaries"]], b.parameters()))
    assert runs[0][0] == runs[1][0]
    np.testing.assert_array_equal(runs[0][1][0], runs[1][1][0])
    np.testing.assert_array_equal(runs[0][1][1], runs[1][1][1])
    with mba.Batch(_tuples(ws[3:6]), precision="fp32") as b:
        b.set_schedule(256, 2, "explicit")
        r = b.solve(**OPTS)
    assert [x["final_cost"] for x in r["summaries"]] == runs[0][0][3:6]


def test_full_batch_sampled_windows(mba):
    """The 512-window workload in the bench's launch configuration: every window
    finishes, lowers its cost, and sampled windows match the oracle (FP32-mixed)."""
    ws = make_windows(512)
    rng = np.random.default_rng(17)
    with mba.Batch(_tuples(ws), precision="fp32") as b:
        gc, gp = rng.normal(size=(b.info["nc"], 9)), rng.normal(size=(b.info["np"], 3))
        r = b.solve(gc, gp, **OPTS)
        g = b.gradients()
    sm = r["summaries"]
    assert all(s["status"] == 0 for s in sm)
    assert all(s["iterations"] == 8 and s["final_cost"] < s["initial_cost"] for s in sm)
    assert np.isfinite(g["grad_obs"]).all() and np.isfinite(g["grad_init_cam"]).all()
    order = np.argsort([s.n for s in ws])
    for w in [int(order[0]), int(order[255]), int(order[-1]), 7]:
        ref = _oracle_solve(ws[w])
        rel_close(sm[w]["final_cost"], ref["final_cost"], 1e-4, f"window {w}")


@pytest.mark.parametrize("schur", ["implicit", "explicit"])
def test_batch_schur_jacobi_matches_oracle(mba, schur):
    """Schur-Jacobi preconditioner (solver variant) per window; it runs the
    explicit form whatever the schedule."""
    ws = _small(count=6, seed=61)
    with mba.Batch(_tuples(ws), precision="fp64") as b:
        b.set_schedule(schur=schur)
        r = b.solve(preconditioner="schur_jacobi", **OPTS)
    for w, s in enumerate(ws):
        ref = _oracle_solve(s, precond="schur_jacobi")
        rel_close(r["summaries"][w]["final_cost"], ref["final_cost"], 1e-6, f"window {w} final cost")
        assert r["summaries"][w]["accepted"] == sum(t["accepted"] for t in ref["trace"])


def test_batch_forcing_matches_oracle(mba):
    ws = _small(count=6, seed=62)
    with mba.Batch(_tuples(ws), precision="fp64") as b:
        r = b.solve(forcing=1, **OPTS)
    for w, s in enumerate(ws):
        ref = _oracle_solve(s, forcing=True)
        rel_close(r["summaries"][w]["final_cost"], ref["final_cost"], 1e-6, f"window {w} final cost")
        assert abs(r["summaries"][w]["pcg_iters_total"] - sum(t["pcg_iters"] for t in ref["trace"])) <= 4


@pytest.mark.parametrize("schur", ["implicit", "explicit"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_batch_single_reduction_pcg_matches_oracle(mba, precision, tol, schur):
    """The single-reduction PCG (Chronopoulos-Gear form) per window against the
    oracle's twin of it: iterations, PCG steps, accept decisions (FP64) and
    final cost; then the adjoint through the same recurrence."""
    ws = _small(count=8, seed=71)
    rng = np.random.default_rng(3)
    with mba.Batch(_tuples(ws), precision=precision) as b:
        b.set_schedule(schur=schur)
        r = b.solve(pcg_variant="single_reduction", **OPTS)
        b.reset()
        gc = rng.normal(size=(b.info["nc"], 9))
        gp = rng.normal(size=(b.info["np"], 3))
        ra = b.solve(gc, gp, adjoint_pcg_max_iter=1000, adjoint_pcg_rel_tol=1e-14, adjoint_mu=1e-2,
                     pcg_variant="single_reduction", **OPTS)
        g = b.gradients()
        cams, pts = b.parameters()
    co, po, oo = b.offsets
    for w, s in enumerate(ws):
        ref = _oracle_solve(s, pcg_variant="single_reduction")
        sm = r["summaries"][w]
        assert sm["status"] == 0 and sm["iterations"] == ref["iterations"]
        rel_close(sm["final_cost"], ref["final_cost"], tol, f"window {w} final cost")
        if precision == "fp64":
            assert sm["accepted"] == sum(t["accepted"] for t in ref["trace"])
            assert abs(sm["pcg_iters_total"] - sum(t["pcg_iters"] for t in ref["trace"])) <= 8
        c, p = cams[co[w]:co[w + 1]], pts[po[w]:po[w + 1]]
        adj = oracle.adjoint(c, p, s.observations, s.cam_idx, s.pt_idx, 1e-2, gc[co[w]:co[w + 1]],
                             gp[po[w]:po[w + 1]], pcg_max=1000, pcg_tol=1e-14, pcg_variant="single_reduction")
        rel_close(g["grad_obs"][oo[w]:oo[w + 1]], adj["grad_obs"], 1e-6 if precision == "fp64" else 3e-3,
                  f"window {w} observation gradient")


def test_measured_order_changes_no_result(mba):
    """After a solve the next launch claims windows longest-first by their
    measured times; the results repeat bit for bit in the new order."""
    ws = _small(count=12, seed=83)
    with mba.Batch(_tuples(ws), precision="fp32") as b:
        with pytest.raises(mba.MbaError):
            b.window_times()
        r1 = b.solve(**OPTS)
        p1 = b.parameters()
        t1 = b.window_times()
        b.reset()
        r2 = b.solve(**OPTS)
        p2 = b.parameters()
    assert t1.shape == (12,) and np.all(t1 > 0)
    assert [x["final_cost"] for x in r1["summaries"]] == [x["final_cost"] for x in r2["summaries"]]
    np.testing.assert_array_equal(p1[0], p2[0])
    np.testing.assert_array_equal(p1[1], p2[1])
