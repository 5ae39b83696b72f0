"""Pins for the CPU oracle against things other than itself.

Each test checks the oracle against a library routine, a closed form, an
invariant stated by the paper, or a brute-force dense computation, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from scenes import make_scene


def _rand_cam(rng, big_rotation=True):
    w = rng.normal(0, 1.0 if big_rotation else 1e-3, 3)
    t = rng.normal(0, 0.3, 3) + np.array([0.0, 0.0, -6.0])
    return np.concatenate([w, t, [rng.uniform(500, 1500), rng.normal(0, 0.05), rng.normal(0, 0.05)]])


def _rand_point_in_front(rng, cam):
    # pick a camera-frame point with negative depth and map it back to the world
    R = Rotation.from_rotvec(cam[:3]).as_matrix()
    Pc = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-8, -4)])
    return R.T @ (Pc - cam[3:6])


def _bal_pixel_scipy(cam, X):
    """BAL projection with the rotation from scipy (library routine)."""
    P = Rotation.from_rotvec(cam[:3]).apply(X) + cam[3:6]
    p = -P[:2] / P[2]
    r2 = p @ p
    return cam[6] * (1 + cam[7] * r2 + cam[8] * r2 * r2) * p


def _bal_pixel_torch(theta, X):
    """Differentiable BAL projection through torch.linalg.matrix_exp (no Rodrigues)."""
    w, t, f, k1, k2 = theta[0:3], theta[3:6], theta[6], theta[7], theta[8]
    zero = torch.zeros((), dtype=theta.dtype)
    K = torch.stack([torch.stack([zero, -w[2], w[1]]), torch.stack([w[2], zero, -w[0]]),
                     torch.stack([-w[1], w[0], zero])])
    R = torch.linalg.matrix_exp(K)
    P = R @ X + t
    p = -P[:2] / P[2]
    r2 = (p * p).sum()
    return f * (1 + k1 * r2 + k2 * r2 * r2) * p


@pytest.mark.parametrize("big", [True, False])
def test_projection_matches_library_rotation(big):
    rng = np.random.default_rng(10 + big)
    for _ in range(50):
        cam = _rand_cam(rng, big)
        X = _rand_point_in_front(rng, cam)
        np.testing.assert_allclose(oracle.project(cam, X), _bal_pixel_scipy(cam, X), rtol=1e-12, atol=1e-9)


def test_first_order_branch_and_pinhole_special_case():
    rng = np.random.default_rng(3)
    # w = 0 exactly takes the first-order branch; with k1 = k2 = 0 it is the
    # textbook pinhole -f P_xy / P_z with P = X + t.
    cam = np.array([0, 0, 0, 0.1, -0.2, -5.0, 800.0, 0.0, 0.0])
    X = rng.normal(0, 0.5, 3)
    P = X + cam[3:6]
    np.testing.assert_allclose(oracle.project(cam, X), -800.0 * P[:2] / P[2], rtol=1e-14)
    # tiny rotation (theta^2 < DBL_EPSILON) agrees with the library rotation to first order
    cam2 = cam.copy()
    cam2[:3] = [1e-9, -2e-9, 5e-10]
    np.testing.assert_allclose(oracle.project(cam2, X), _bal_pixel_scipy(cam2, X), rtol=1e-12)


def test_jacobian_central_differences():
    rng = np.random.default_rng(4)
    for _ in range(20):
        cam = _rand_cam(rng)
        X = _rand_point_in_front(rng, cam)
        u = oracle.project(cam, X) + rng.normal(0, 1, 2)
        e, Jc, Jp = oracle.residual_jacobian(cam, X, u)
        np.testing.assert_allclose(e, oracle.project(cam, X) - u, rtol=1e-13, atol=1e-10)
        theta = np.concatenate([cam, X])
        J = np.concatenate([Jc, Jp], axis=1)
        for a in range(12):
            h = 1e-6 * max(1.0, abs(theta[a]))
            tp, tm = theta.copy(), theta.copy()
            tp[a] += h
            tm[a] -= h
            fd = (_bal_pixel_scipy(tp[:9], tp[9:]) - _bal_pixel_scipy(tm[:9], tm[9:])) / (2 * h)
            scale = max(1.0, np.abs(J[:, a]).max())
            np.testing.assert_allclose(J[:, a], fd, atol=2e-6 * scale, rtol=1e-6)


@pytest.mark.parametrize("big", [True, False])
def test_jacobian_matches_autodiff_of_matrix_exponential(big):
    rng = np.random.default_rng(5 + big)
    for _ in range(20):
        cam = _rand_cam(rng, big)
        X = _rand_point_in_front(rng, cam)
        u = rng.normal(0, 100, 2)
        _, Jc, Jp = oracle.residual_jacobian(cam, X, u)
        tc = torch.tensor(cam, dtype=torch.float64)
        tX = torch.tensor(X, dtype=torch.float64)
        Jc_ad = torch.func.jacfwd(lambda th: _bal_pixel_torch(th, tX))(tc).numpy()
        Jp_ad = torch.func.jacfwd(lambda x: _bal_pixel_torch(tc, x))(tX).numpy()
        np.testing.assert_allclose(Jc, Jc_ad, rtol=1e-9, atol=1e-9 * np.abs(Jc_ad).max())
        np.testing.assert_allclose(Jp, Jp_ad, rtol=1e-9, atol=1e-9 * np.abs(Jp_ad).max())


def test_huber_loss_properties():
    delta = 2.0
    for s in [0.0, 0.5, 3.99, 4.0, 4.01, 100.0]:
        rho, w = oracle.loss("huber", delta, s)
        r_plain, w_plain = oracle.loss("none", delta, s)
        assert (r_plain, w_plain) == (s, 1.0)
        if s <= delta ** 2:
            assert (rho, w) == (s, 1.0)
        else:
            # closed form and derivative rho'(s) = delta / sqrt(s) by central difference
            assert rho == pytest.approx(2 * delta * math.sqrt(s) - delta ** 2, rel=1e-15)
            h = 1e-6 * s
            d = (oracle.loss("huber", delta, s + h)[0] - oracle.loss("huber", delta, s - h)[0]) / (2 * h)
            assert w == pytest.approx(d, rel=1e-7)
    # continuity at s = delta^2
    assert oracle.loss("huber", delta, 4.0 + 1e-12)[0] == pytest.approx(4.0, abs=1e-11)
    # a huge delta reduces Huber to the plain loss on a whole scene
    sc = make_scene(4, 30, sigma=1.0, seed=7)
    c1 = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, "huber", 1e9)[0]
    c0 = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, "none")[0]
    assert c1 == c0


def test_stable_sort_matches_numpy():
    rng = np.random.default_rng(6)
    keys = rng.integers(0, 37, size=2000).astype(np.int32)
    perm, ptr = oracle.stable_sort(keys, 40)
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable"))
    np.testing.assert_array_equal(ptr, np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=40))]))


def _dense_system(sc, loss="none", delta=0.0):
    """Dense J (2n x (9nc+3np)), W per residual row and e, from per-observation oracle terms."""
    cost, e, Jc, Jp, W = oracle.evaluate(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, loss, delta)
    n, nc, np_ = sc.n, sc.nc, sc.np_
    J = np.zeros((2 * n, 9 * nc + 3 * np_))
    for k in range(n):
        i, j = sc.cam_idx[k], sc.pt_idx[k]
        J[2 * k:2 * k + 2, 9 * i:9 * i + 9] = Jc[k]
        J[2 * k:2 * k + 2, 9 * nc + 3 * j:9 * nc + 3 * j + 3] = Jp[k]
    Wr = np.repeat(W, 2)
    return J, Wr, e.reshape(-1), cost


@pytest.mark.parametrize("loss", ["none", "huber"])
def test_blocks_equal_dense_normal_equations(loss):
    sc = make_scene(3, 10, sigma=3.0, seed=8, outlier_frac=0.2)
    J, Wr, e, _ = _dense_system(sc, loss, 2.0)
    H = J.T @ (Wr[:, None] * J)
    g = -J.T @ (Wr * e)
    Hpp, v, Hll, w, E = oracle.blocks(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, loss, 2.0,
                                      with_E=True)
    nc = sc.nc
    sc_ = 1e-13 * np.abs(H).max()
    for i in range(nc):
        np.testing.assert_allclose(Hpp[i], H[9 * i:9 * i + 9, 9 * i:9 * i + 9], atol=sc_)
        np.testing.assert_allclose(v[i], g[9 * i:9 * i + 9], atol=1e-13 * np.abs(g).max())
    for j in range(sc.np_):
        o = 9 * nc + 3 * j
        np.testing.assert_allclose(Hll[j], H[o:o + 3, o:o + 3], atol=sc_)
        np.testing.assert_allclose(w[j], g[o:o + 3], atol=1e-13 * np.abs(g).max())
    # off-diagonal camera-point blocks: sum of per-edge E_k
    Eb = np.zeros((9 * nc, 3 * sc.np_))
    for k in range(sc.n):
        i, j = sc.cam_idx[k], sc.pt_idx[k]
        Eb[9 * i:9 * i + 9, 3 * j:3 * j + 3] += E[k]
    np.testing.assert_allclose(Eb, H[:9 * nc, 9 * nc:], atol=sc_)
    # camera-camera and point-point off-diagonal blocks of H are zero (B, C block diagonal)
    for i in range(nc):
        for i2 in range(nc):
            if i2 != i:
                assert np.all(H[9 * i:9 * i + 9, 9 * i2:9 * i2 + 9] == 0)


def _damped_dense(sc, mu, damping="diag", loss="none", delta=0.0):
    J, Wr, e, _ = _dense_system(sc, loss, delta)
    H = J.T @ (Wr[:, None] * J)
    g = -J.T @ (Wr * e)
    d = np.clip(np.diag(H), 1e-6, 1e32) if damping == "diag" else np.ones(H.shape[0])
    return H + mu * np.diag(d), g, J, Wr, e


@pytest.mark.parametrize("damping", ["diag", "identity"])
def test_schur_step_equals_direct_solve(damping):
    sc = make_scene(4, 25, sigma=1.0, seed=9)
    mu = 1e-3
    Hd, g, *_ = _damped_dense(sc, mu, damping)
    dx = np.linalg.solve(Hd, g)
    nc = sc.nc
    for mode, tol in [("dense", 1e-9), ("explicit_pcg", 1e-7), ("implicit_pcg", 1e-7)]:
        r = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, damping=damping,
                        schur=mode, pcg_max=500, pcg_tol=1e-15)
        got = np.concatenate([r["dc"].reshape(-1), r["dp"].reshape(-1)])
        np.testing.assert_allclose(got, dx, atol=tol * np.abs(dx).max(), err_msg=mode)
        assert r["dc"].shape == (nc, 9)


def test_implicit_schur_product_equals_dense_complement():
    sc = make_scene(4, 25, sigma=1.0, seed=11)
    mu = 0.1
    Hd, g, *_ = _damped_dense(sc, mu)
    m = 9 * sc.nc
    B, E, Cm = Hd[:m, :m], Hd[:m, m:], Hd[m:, m:]
    S = B - E @ np.linalg.solve(Cm, E.T)
    rhs = g[:m] - E @ np.linalg.solve(Cm, g[m:])
    x = np.random.default_rng(1).normal(size=m)
    r = oracle.schur(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, x=x, dense=True)
    np.testing.assert_allclose(r["y"], S @ x, atol=1e-10 * np.abs(S @ x).max())
    np.testing.assert_allclose(r["rhs"], rhs, atol=1e-10 * np.abs(rhs).max())
    np.testing.assert_allclose(r["S"], S, atol=1e-10 * np.abs(S).max())
    # symmetric positive definite
    np.testing.assert_allclose(S, S.T, atol=1e-9 * np.abs(S).max())
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0


def test_model_decrease_matches_quadratic_model():
    sc = make_scene(4, 25, sigma=2.0, seed=12, outlier_frac=0.1)
    mu = 1e-2
    r = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, loss="huber", delta=2.0,
                    schur="dense")
    _, _, J, Wr, e = _damped_dense(sc, mu, loss="huber", delta=2.0)
    dx = np.concatenate([r["dc"].reshape(-1), r["dp"].reshape(-1)])
    f = e + J @ dx
    ref = 0.5 * np.sum(Wr * (e * e - f * f))
    assert r["model_dec"] == pytest.approx(ref, rel=1e-10)


def test_split_sum_invariant():
    """H = sum_k H_k over any edge partition (Sec. 4.1)."""
    sc = make_scene(5, 40, sigma=1.0, seed=13)
    full = oracle.blocks(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    K = 3
    parts = np.array_split(np.arange(sc.n), K)
    acc = [np.zeros_like(a) for a in full]
    for p in parts:
        sub = oracle.blocks(sc.cameras, sc.points, sc.observations[p], sc.cam_idx[p], sc.pt_idx[p])
        for a, b in zip(acc, sub):
            a += b
    for a, b in zip(acc, full):
        np.testing.assert_allclose(a, b, atol=1e-12 * max(1.0, np.abs(b).max()))


def test_noise_free_scene_reaches_zero_cost():
    sc = make_scene(6, 200, sigma=0.0, seed=14)
    # the generator's ideal pixels are exactly the oracle's projections at the truth
    c_true = oracle.evaluate(sc.cameras_true, sc.points_true, sc.observations, sc.cam_idx, sc.pt_idx)[0]
    assert c_true < 1e-18 * sc.n
    r = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=30, pcg_max=200,
                        pcg_tol=1e-14)
    assert r["trace"][0]["cost"] > 1.0
    assert r["final_cost"] < 1e-16 * sc.n


def test_accepted_cost_is_monotone_and_reaches_noise_floor():
    sc = make_scene(16, 2000, sigma=0.5, seed=0)
    r = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=10, pcg_max=50)
    costs = [t["cost"] for t in r["trace"]] + [r["final_cost"]]
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    for t in r["trace"]:
        if t["accepted"]:
            assert t["cost_new"] < t["cost"]
    # least-squares noise floor: E[sum |e|^2] = sigma^2 (2n - dof)
    dof = 9 * sc.nc + 3 * sc.np_
    expected = 0.5 * 0.25 * (2 * sc.n - dof)
    assert r["final_cost"] == pytest.approx(expected, rel=0.05)


@pytest.mark.parametrize("loss", ["none", "huber"])
def test_adjoint_matches_dense_implicit_function_gradient(loss):
    """dL/du_k = W_k J_k M^-1 gbar and dL/dx0 = mu D M^-1 gbar with a dense solve."""
    sc = make_scene(4, 25, sigma=2.0, seed=15, outlier_frac=0.1)
    mu = 1e-2
    rng = np.random.default_rng(2)
    gc, gp = rng.normal(size=(sc.nc, 9)), rng.normal(size=(sc.np_, 3))
    r = oracle.adjoint(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, gc, gp, loss=loss,
                       delta=2.0)
    J, Wr, e, _ = _dense_system(sc, loss, 2.0)
    H = J.T @ (Wr[:, None] * J)
    d = np.clip(np.diag(H), 1e-6, 1e32)
    v = np.linalg.solve(H + mu * np.diag(d), np.concatenate([gc.reshape(-1), gp.reshape(-1)]))
    g_obs = (Wr * (J @ v)).reshape(-1, 2)
    np.testing.assert_allclose(r["grad_obs"], g_obs, atol=1e-8 * np.abs(g_obs).max())
    g0 = mu * d * v
    np.testing.assert_allclose(np.concatenate([r["grad_c0"].reshape(-1), r["grad_p0"].reshape(-1)]), g0,
                               atol=1e-8 * np.abs(g0).max())


# ---------------------------------------------------------------------------
# Schur-Jacobi preconditioner and forcing sequence (solver variants beside
# Alg. 2's block-Jacobi preconditioner and fixed tolerance)
# ---------------------------------------------------------------------------
def test_schur_jacobi_blocks_are_the_diagonal_blocks_of_the_dense_complement():
    """With every (camera, point) pair observed once, the Schur-Jacobi camera
    blocks are the 9x9 diagonal blocks of S = B~ - E C~^-1 E^T formed densely."""
    sc = make_scene(5, 60, track=("fixed", 3), sigma=1.0, seed=71)
    mu = 1e-2
    blocks = oracle.schur_jacobi_blocks(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu)
    S = oracle.schur(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, dense=True)["S"]
    for i in range(sc.nc):
        np.testing.assert_allclose(blocks[i], S[9 * i:9 * i + 9, 9 * i:9 * i + 9], rtol=1e-12,
                                   atol=1e-12 * np.abs(S).max())


def _single_camera(sc, cam):
    keep = sc.cam_idx == cam
    pts_used = np.unique(sc.pt_idx[keep])
    remap = -np.ones(sc.np_, dtype=np.int64)
    remap[pts_used] = np.arange(len(pts_used))
    return (sc.cameras[cam:cam + 1], sc.points[pts_used], sc.observations[keep],
            np.zeros(int(keep.sum()), dtype=np.int32), remap[sc.pt_idx[keep]].astype(np.int32))


def test_schur_jacobi_is_exact_for_one_camera():
    """With one camera S has a single block, so the Schur-Jacobi preconditioner
    is S^-1 and PCG stops after one step; block-Jacobi on B~ needs more."""
    sc = make_scene(3, 80, track=("fixed", 2), sigma=1.0, seed=72)
    prob = _single_camera(sc, 1)
    sj = oracle.step(*prob, mu=1e-3, pcg_max=50, pcg_tol=1e-10, precond="schur_jacobi")
    bj = oracle.step(*prob, mu=1e-3, pcg_max=50, pcg_tol=1e-10, precond="block_jacobi")
    assert sj["pcg_iters"] == 1 and sj["rel_res"] < 1e-10
    assert bj["pcg_iters"] > 1
    np.testing.assert_allclose(sj["dc"], bj["dc"], rtol=1e-6, atol=1e-9 * np.abs(bj["dc"]).max())


def test_schur_jacobi_step_equals_direct_solve():
    sc = make_scene(6, 120, track=("geom", 0.25), sigma=1.0, seed=73)
    mu = 1e-3
    ref = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, schur="dense")
    got = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, pcg_max=500, pcg_tol=1e-14,
                      precond="schur_jacobi")
    np.testing.assert_allclose(got["dc"], ref["dc"], rtol=1e-7, atol=1e-9 * np.abs(ref["dc"]).max())
    np.testing.assert_allclose(got["dp"], ref["dp"], rtol=1e-7, atol=1e-9 * np.abs(ref["dp"]).max())


def test_forcing_sequence_loosens_early_solves():
    """Forcing tolerance max(tol, min(0.1, sqrt(|g_k| / |g_0|))): the first solve
    stops at relative residual 0.1, the LM still lowers the cost monotonically."""
    sc = make_scene(8, 300, track=("geom", 0.25), sigma=1.0, seed=74)
    fixed = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=6, pcg_max=200)
    forced = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=6, pcg_max=200,
                             forcing=True)
    t0 = forced["trace"][0]
    assert t0["pcg_rel_res"] <= 0.1 and t0["pcg_rel_res"] > 1e-3
    assert t0["pcg_iters"] < fixed["trace"][0]["pcg_iters"]
    costs = [t["cost_new"] for t in forced["trace"] if t["accepted"]]
    assert costs and all(b < a for a, b in zip(costs, costs[1:]))
    assert forced["final_cost"] < forced["trace"][0]["cost"]


def _one_view_point_scene():
    """A small scene plus one point seen by a single camera: its block J^T J has
    rank 2, so with identity damping at mu = 1e-16 (radius 1e16) the damped 3x3
    block is singular to FP64 rounding."""
    sc = make_scene(3, 20, sigma=0.5, seed=0)
    X = np.random.default_rng(0).normal(0, 0.3, 3)
    pts = np.vstack([sc.points, X])
    pix = oracle.residual_jacobian(sc.cameras[0], X, np.zeros(2))[0]
    obs = np.vstack([sc.observations, pix + 0.3])
    ci = np.concatenate([sc.cam_idx, [0]]).astype(np.int32)
    pi = np.concatenate([sc.pt_idx, [len(pts) - 1]]).astype(np.int32)
    return sc.cameras, pts, obs, ci, pi


def test_non_positive_definite_block_is_a_rejected_iteration():
    """No step exists when a damped block is not positive definite; the LM rule
    then rejects the iteration: mu follows the rejection sequence 1e-16,
    2e-16, 8e-16, 6.4e-15 (radius divided by 2, 4, 8), the trace records no
    PCG iterations and no candidate cost, and the first solvable system gives
    an accepted step that lowers the cost."""
    cams, pts, obs, ci, pi = _one_view_point_scene()
    r = oracle.lm_solve(cams, pts, obs, ci, pi, max_iter=4, pcg_max=20, damping="identity", initial_radius=1e16)
    tr = r["trace"]
    assert [t["accepted"] for t in tr] == [0, 0, 0, 1]
    for t in tr[:3]:
        assert math.isnan(t["cost_new"]) and t["pcg_iters"] == 0 and t["model_dec"] == 0.0
    assert [t["mu"] for t in tr] == pytest.approx([1e-16, 2e-16, 8e-16, 6.4e-15], rel=1e-12)
    assert tr[3]["cost_new"] < tr[3]["cost"]


def test_resume_from_a_checkpoint_continues_the_trajectory():
    """Checkpoint / resume: an LM solve that stops after an accepted step and is
    restarted from its parameters with its final trust-region radius (the
    decrease factor is 2 after any accepted step, as at a start) continues the
    uninterrupted solve bit for bit (Alg. 1 with the radius rule of the Ceres
    trust region).  Tiny workload, split after the third iteration."""
    from scenes import config_scene

    sc = config_scene(1)
    arrays = (sc.observations, sc.cam_idx, sc.pt_idx)
    kw = dict(pcg_max=50, pcg_tol=1e-10)
    full = oracle.lm_solve(sc.cameras, sc.points, *arrays, max_iter=10, **kw)
    first = oracle.lm_solve(sc.cameras, sc.points, *arrays, max_iter=3, **kw)
    assert first["trace"][-1]["accepted"] == 1
    rest = oracle.lm_solve(first["cameras"], first["points"], *arrays, max_iter=7, initial_radius=first["radius"], **kw)
    assert rest["final_cost"] == full["final_cost"]
    assert [t["cost_new"] for t in rest["trace"]] == [t["cost_new"] for t in full["trace"][3:]]
    assert [t["accepted"] for t in rest["trace"]] == [t["accepted"] for t in full["trace"][3:]]
    np.testing.assert_array_equal(rest["cameras"], full["cameras"])
    np.testing.assert_array_equal(rest["points"], full["points"])


def _fixed_masks(sc):
    cf = np.zeros(sc.nc, np.uint8)
    cf[[0, 3]] = 1
    pf = np.zeros(sc.np_, np.uint8)
    pf[::7] = 1
    return cf, pf


@pytest.mark.parametrize("damping", ["diag", "identity"])
def test_fixed_nodes_step_equals_the_reduced_dense_solve(damping):
    """Nodes held constant (the g2o / Ceres convention of Sec. 5.3): the damped
    step equals a dense solve of the damped normal equations with the fixed
    parameters' rows and columns deleted, and is exactly zero on them."""
    sc = make_scene(5, 40, sigma=1.0, seed=31)
    cf, pf = _fixed_masks(sc)
    mu = 1e-3
    Hd, g, *_ = _damped_dense(sc, mu, damping)
    nc = sc.nc
    free = np.concatenate([np.repeat(cf == 0, 9), np.repeat(pf == 0, 3)])
    dx = np.zeros(Hd.shape[0])
    dx[free] = np.linalg.solve(Hd[np.ix_(free, free)], g[free])
    for mode, tol in [("dense", 1e-9), ("explicit_pcg", 1e-7), ("implicit_pcg", 1e-7)]:
        r = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, damping=damping,
                        schur=mode, pcg_max=500, pcg_tol=1e-15, cam_fixed=cf, pt_fixed=pf)
        assert np.all(r["dc"][cf == 1] == 0.0) and np.all(r["dp"][pf == 1] == 0.0), mode
        got = np.concatenate([r["dc"].reshape(-1), r["dp"].reshape(-1)])
        np.testing.assert_allclose(got, dx, atol=tol * np.abs(dx).max(), err_msg=mode)
    # and it is not the unconstrained step
    r0 = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, damping=damping,
                     schur="dense")
    assert np.abs(np.concatenate([r0["dc"].reshape(-1), r0["dp"].reshape(-1)]) - dx).max() > 1e-3 * np.abs(dx).max()
    assert r0["dc"].shape == (nc, 9)


def test_fixed_nodes_stay_constant_through_a_solve():
    sc = make_scene(6, 300, sigma=0.5, seed=32)
    cf, pf = _fixed_masks(sc)
    r = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=8, pcg_max=50,
                        cam_fixed=cf, pt_fixed=pf)
    np.testing.assert_array_equal(r["cameras"][cf == 1], sc.cameras[cf == 1])
    np.testing.assert_array_equal(r["points"][pf == 1], sc.points[pf == 1])
    assert np.any(r["cameras"][cf == 0] != sc.cameras[cf == 0])
    acc = [t["cost_new"] for t in r["trace"] if t["accepted"]]
    assert acc and r["final_cost"] < r["trace"][0]["cost"]
    assert all(b <= a for a, b in zip(acc, acc[1:]))


def test_all_nodes_fixed_gives_no_step():
    sc = make_scene(3, 30, sigma=0.5, seed=33)
    r = oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=3, pcg_max=20,
                        cam_fixed=np.ones(sc.nc), pt_fixed=np.ones(sc.np_))
    assert all(t["model_dec"] == 0.0 and t["accepted"] == 0 for t in r["trace"])
    np.testing.assert_array_equal(r["cameras"], sc.cameras)
    np.testing.assert_array_equal(r["points"], sc.points)


# ---------------------------------------------------------------------------
# Truncated PCG iterates (Alg. 2 with a capped iteration count).  A converged
# PCG only shows that the loop reaches the solution; a capped one returns its
# k-th iterate, which every capped solve depends on.  The k-th iterate of
# preconditioned CG from x0 = 0 is, by the optimality property of CG (Saad,
# Iterative Methods for Sparse Linear Systems, 2nd ed., Sec. 6.11 and 9.2), the
# minimiser of the S-energy error |x - x*|_S over the preconditioned Krylov
# space span{M^-1 g, (M^-1 S) M^-1 g, ..., (M^-1 S)^(k-1) M^-1 g}.  That
# minimiser is computed here by a dense Galerkin projection, with S and M
# formed from the dense damped normal equations, so a wrong beta, a p/z or
# p/q mix-up in the update, or a restart at the second step changes the
# iterate and fails.
def _krylov_minimiser(S, Minv, g, k):
    V = []
    v = Minv @ g
    for _ in range(k):
        for _rep in range(2):  # Gram-Schmidt twice: the span is what matters
            for u in V:
                v = v - (u @ v) * u
        V.append(v / np.linalg.norm(v))
        v = Minv @ (S @ V[-1])
    V = np.array(V).T
    return V @ np.linalg.solve(V.T @ S @ V, V.T @ g)


def _block_inverse(A, nb):
    Ai = np.zeros_like(A)
    for i in range(nb):
        s = slice(9 * i, 9 * i + 9)
        Ai[s, s] = np.linalg.inv(A[s, s])
    return Ai


@pytest.mark.parametrize("variant", ["standard", "single_reduction"])
@pytest.mark.parametrize("precond", ["block_jacobi", "schur_jacobi"])
@pytest.mark.parametrize("schur", ["explicit_pcg", "implicit_pcg"])
def test_truncated_pcg_iterate_is_the_krylov_energy_minimiser(precond, schur, variant):
    """Both PCG forms (Alg. 2's two-reduction loop and the single-reduction
    Chronopoulos-Gear form) return, after k steps, the minimiser of the S-energy
    error over the k-dimensional preconditioned Krylov space (Saad, Iterative
    Methods for Sparse Linear Systems, Sec. 6.11 and 9.2): a wrong beta, a mixed
    p / p_prev, or a wrong alpha denominator in the single-reduction recurrence
    leaves the space or the minimum."""
    sc = make_scene(4, 25, sigma=1.0, seed=21)
    mu = 1e-3
    Hd, g, *_ = _damped_dense(sc, mu)
    m = 9 * sc.nc
    B, E, Cm = Hd[:m, :m], Hd[:m, m:], Hd[m:, m:]
    S = B - E @ np.linalg.solve(Cm, E.T)
    b = g[:m] - E @ np.linalg.solve(Cm, g[m:])
    # block-Jacobi: M = blockdiag(B~_i) (Alg. 2); Schur-Jacobi: M = the diagonal
    # 9x9 blocks of S (every (camera, point) pair is observed once here)
    Minv = _block_inverse(B if precond == "block_jacobi" else S, sc.nc)
    for k in range(1, 7):
        ref = _krylov_minimiser(S, Minv, b, k)
        r = oracle.step(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, mu, schur=schur,
                        pcg_max=k, pcg_tol=0.0, precond=precond, pcg_variant=variant)
        assert r["pcg_iters"] == k
        np.testing.assert_allclose(r["dc"].reshape(-1), ref, atol=1e-9 * np.abs(ref).max(), err_msg=f"k={k}")
    # the iterates differ from step to step, so the comparison above has teeth
    assert np.abs(_krylov_minimiser(S, Minv, b, 6) - _krylov_minimiser(S, Minv, b, 5)).max() > 1e-6 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# Trust-region radius after an ACCEPTED step (Nielsen's rule, H. B. Nielsen,
# "Damping parameter in Marquardt's method", IMM-REP-1999-05; the rule the
# Ceres trust region documents): radius /= max(1/3, 1 - (2 rho - 1)^3).  The
# gain rho is recomputed here from costs and the linear model outside the LM
# loop: F and F' by oracle.evaluate at x and x + dx, the model decrease from
# the per-observation residuals and Jacobians, dx from the dense Schur solve
# (pinned against a direct solve above).  The three scenes put rho in each
# branch of the rule: below 1/2 (radius shrinks), between 1/2 and the knee
# (grows by less than 3) and above the knee (grows by 3); max -> min, a
# squared term or a dropped "- 1" each changes the next iteration's mu.
@pytest.mark.parametrize("rot_sigma,point_sigma,seed,radius,lo,hi", [
    (0.3, 0.3, 1, 1e3, 1e-3, 0.5),
    (0.2, 0.1, 1, 1e3, 0.5, 0.9),
    (0.01, 0.02, 0, 1.0, 0.95, 1.5),
])
def test_accepted_step_radius_follows_nielsen_rule(rot_sigma, point_sigma, seed, radius, lo, hi):
    sc = make_scene(4, 25, sigma=1.0, seed=seed, rot_sigma=rot_sigma, point_sigma=point_sigma)
    args = (sc.observations, sc.cam_idx, sc.pt_idx)
    mu = 1.0 / radius
    st = oracle.step(sc.cameras, sc.points, *args, mu, schur="dense")
    F, e, Jc, Jp, W = oracle.evaluate(sc.cameras, sc.points, *args)
    Fn = oracle.evaluate(sc.cameras + st["dc"], sc.points + st["dp"], *args, jacobians=False)[0]
    f = e + np.einsum("kab,kb->ka", Jc, st["dc"][sc.cam_idx]) + np.einsum("kab,kb->ka", Jp, st["dp"][sc.pt_idx])
    L = 0.5 * np.sum(W * (np.sum(e * e, axis=1) - np.sum(f * f, axis=1)))
    rho = (F - Fn) / L
    assert lo < rho < hi and L > 0
    r = oracle.lm_solve(sc.cameras, sc.points, *args, max_iter=2, schur="dense", initial_radius=radius)
    t0, t1 = r["trace"]
    assert t0["accepted"] == 1 and t0["mu"] == pytest.approx(mu, rel=1e-15)
    assert t0["gain"] == pytest.approx(rho, rel=1e-9)
    expected_radius = radius / max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
    assert t1["mu"] == pytest.approx(1.0 / expected_radius, rel=1e-9)


# ---------------------------------------------------------------------------
# The single-reduction PCG stops where the standard one does: with a tolerance,
# both take the same number of steps and return the same solution (rounding
# apart), and an LM solve on either reaches the same accept decisions and
# final cost.
def test_single_reduction_pcg_matches_standard_with_a_tolerance():
    sc = make_scene(12, 800, track=("geom", 0.25), sigma=1.0, seed=27)
    args = (sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    a = oracle.step(*args, 1e-2, pcg_max=200, pcg_tol=1e-8)
    b = oracle.step(*args, 1e-2, pcg_max=200, pcg_tol=1e-8, pcg_variant="single_reduction")
    assert 5 < a["pcg_iters"] < 200 and a["pcg_iters"] == b["pcg_iters"]
    np.testing.assert_allclose(b["dc"], a["dc"], rtol=0, atol=1e-9 * np.abs(a["dc"]).max())
    assert b["rel_res"] == pytest.approx(a["rel_res"], rel=1e-6)
    ra = oracle.lm_solve(*args, max_iter=6, pcg_max=50)
    rb = oracle.lm_solve(*args, max_iter=6, pcg_max=50, pcg_variant="single_reduction")
    assert [t["accepted"] for t in ra["trace"]] == [t["accepted"] for t in rb["trace"]]
    assert rb["final_cost"] == pytest.approx(ra["final_cost"], rel=1e-10)
