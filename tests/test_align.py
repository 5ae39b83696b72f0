"""The parameter-error helper (oracle/align.py): Umeyama's similarity fit
recovers a known similarity exactly, and a solution moved along the 7-DoF
gauge has zero aligned error while its raw error is large."""
import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from oracle.align import camera_centres, parameter_error, umeyama
from scenes import make_scene


def _similarity(rng):
    return rng.uniform(0.5, 2.0), Rotation.from_rotvec(rng.normal(0, 1.0, 3)).as_matrix(), rng.normal(0, 1.0, 3)


def test_umeyama_recovers_a_known_similarity():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(50, 3))
    c, R, t = _similarity(rng)
    Y = c * X @ R.T + t
    c2, R2, t2 = umeyama(X, Y)
    assert abs(c2 - c) < 1e-12 * c
    np.testing.assert_allclose(R2, R, atol=1e-12)
    np.testing.assert_allclose(t2, t, atol=1e-12)
    assert np.linalg.det(R2) > 0
    # a reflection in the data is not fitted by a reflection
    c3, R3, _ = umeyama(X, X * np.array([1.0, 1.0, -1.0]))
    assert np.linalg.det(R3) > 0


def test_gauge_motion_has_zero_aligned_error():
    """Moving every point by X' = s Q X + u and every camera by R' = R Q^T,
    t' = s t - R' u leaves every projection unchanged (the gauge); the aligned
    error of the moved solution is zero, the raw error is not."""
    sc = make_scene(5, 40, sigma=0.0, seed=3)
    rng = np.random.default_rng(1)
    s, Q, u = _similarity(rng)
    pts2 = s * sc.points @ Q.T + u
    R = Rotation.from_rotvec(sc.cameras[:, :3]).as_matrix()
    R2 = np.einsum("kab,cb->kac", R, Q)
    t2 = s * sc.cameras[:, 3:6] - np.einsum("kab,b->ka", R2, u)
    cams2 = sc.cameras.copy()
    cams2[:, :3] = Rotation.from_matrix(R2).as_rotvec()
    cams2[:, 3:6] = t2
    for k in range(0, sc.n, 7):
        i, j = sc.cam_idx[k], sc.pt_idx[k]
        np.testing.assert_allclose(oracle.project(cams2[i], pts2[j]), oracle.project(sc.cameras[i], sc.points[j]),
                                   rtol=1e-10)
    np.testing.assert_allclose(camera_centres(cams2), s * camera_centres(sc.cameras) @ Q.T + u, atol=1e-10)
    e = parameter_error(cams2, pts2, sc.cameras, sc.points)
    assert e["aligned_point_rms"] < 1e-12 * e["extent"]
    assert e["aligned_centre_rms"] < 1e-10
    assert abs(e["scale"] - 1.0 / s) < 1e-12
    assert e["raw_point_rms"] > 0.1 * e["extent"] and e["raw_camera_rel"] > 1e-2
