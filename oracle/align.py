"""Parameter error between two bundle-adjustment solutions, raw and after a
similarity alignment.

TEST INFRASTRUCTURE ONLY (the tests and the benchmark's CPU-baseline leg use
it to state how far the CUDA path's parameters are from the oracle's).

Bundle adjustment fixes its solution only up to a 7-DoF similarity (the gauge:
rotation, translation, scale), so two solvers that reach the same cost can
return parameters that differ along the gauge.  The error is therefore given
twice: raw, and after the least-squares similarity that maps one point cloud
onto the other (S. Umeyama, "Least-squares estimation of transformation
parameters between two point patterns", IEEE TPAMI 13(4), 1991).  The cost is
gauge-invariant and stays the primary parity quantity.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation


def umeyama(src, dst):
    """Similarity (c, R, t) minimising sum_i |c R src_i + t - dst_i|^2 (Umeyama 1991).

    src, dst: (m, 3).  Returns scale c, rotation R (3x3, det +1), translation t.
    """
    src, dst = np.asarray(src, dtype=np.float64), np.asarray(dst, dtype=np.float64)
    mu_s, mu_d = src.mean(axis=0), dst.mean(axis=0)
    a, b = src - mu_s, dst - mu_d
    var_s = np.mean(np.sum(a * a, axis=1))
    cov = b.T @ a / src.shape[0]
    U, D, Vt = np.linalg.svd(cov)
    S = np.eye(3)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        S[2, 2] = -1.0
    R = U @ S @ Vt
    c = float(np.trace(np.diag(D) @ S) / var_s)
    t = mu_d - c * R @ mu_s
    return c, R, t


def camera_centres(cams):
    """World positions -R(w)^T t of BAL cameras (nc, 9)."""
    cams = np.asarray(cams, dtype=np.float64)
    R = Rotation.from_rotvec(cams[:, :3]).as_matrix()
    return -np.einsum("kba,kb->ka", R, cams[:, 3:6])


def parameter_error(cams, pts, cams_ref, pts_ref):
    """How far (cams, pts) are from (cams_ref, pts_ref).

    raw_camera_rel: max over the nine camera parameters of |C[:, a] - C_ref[:, a]|
    / |C_ref[:, a]| (2-norms over the cameras), so the focal length does not
    hide the rotation and translation;
    raw_point_rms: RMS of |X - X_ref| (scene units); extent: RMS distance of the
    reference points from their centroid; aligned_point_rms and
    aligned_centre_rms: RMS point and camera-centre errors after the Umeyama
    similarity fitted on the points; scale: that similarity's scale.
    """
    cams, pts = np.asarray(cams, dtype=np.float64), np.asarray(pts, dtype=np.float64)
    cams_ref, pts_ref = np.asarray(cams_ref, dtype=np.float64), np.asarray(pts_ref, dtype=np.float64)
    rms = lambda d: float(np.sqrt(np.mean(np.sum(d * d, axis=1))))  # noqa: E731
    c, R, t = umeyama(pts, pts_ref)
    pts_al = c * pts @ R.T + t
    cen_al = c * camera_centres(cams) @ R.T + t
    return {
        "raw_camera_rel": float(np.max(np.linalg.norm(cams - cams_ref, axis=0) /
                                       np.maximum(np.linalg.norm(cams_ref, axis=0), 1e-300))),
        "raw_point_rms": rms(pts - pts_ref),
        "extent": rms(pts_ref - pts_ref.mean(axis=0)),
        "aligned_point_rms": rms(pts_al - pts_ref),
        "aligned_centre_rms": rms(cen_al - camera_centres(cams_ref)),
        "scale": c,
    }
