"""Seeded synthetic scenes shaped like the paper's bundle-adjustment workloads.

Recipe (shared by every consumer; the paper's BAL and 1DSfM files are not
available, so these scenes stand in for them):

* Cameras sit evenly on a horizontal circle of radius 8 around the origin and
  look at it; the radius follows the paper's synthetic dataset (supplement,
  "Large Synthesised Dataset").  Camera parameters use the BAL layout
  (angle-axis rotation, translation, focal, k1, k2); a camera looks down its
  own -z axis, so points in front have a negative camera-frame depth.
* Focal lengths ~ U(500, 1500) px, k1 and k2 ~ N(0, 0.01^2).
* Points are uniform in the unit cube [-0.5, 0.5]^3.
* Each point is seen by L distinct cameras drawn uniformly without
  replacement.  L is fixed (5), 2 + Geometric (mean 5 or 4), or
  min(300, 2 + floor(LogNormal(mu, 1))) with mu set by bisection so that
  E[L] = 6.5.
* Observations = ideal projections + N(0, sigma^2) pixel noise; a fraction of
  them can be replaced by the ideal projection + 50 px in a uniformly random
  direction (outliers).
* Initial estimate: rotations composed with exp(eps), eps ~ N(0, 0.01^2 I);
  each translation component scaled by (1 + N(0, 0.02^2)); points moved by
  N(0, 0.02^2) per coordinate.  Intrinsics are not perturbed.
* Observations are emitted in a seeded random order, as real datasets are not
  grouped by point or by camera.

Synthesising the observations needs the forward camera model once; it is done
here with rotation matrices from ``scipy.spatial.transform.Rotation`` (a
library routine) rather than any angle-axis formula of the method, and the
result is pinned by the oracle tests (a noise-free scene has zero residual).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

CIRCLE_RADIUS = 8.0

# Workload table: the five evaluation workloads, named by what they are.
CONFIGS = {
    # tiny: 16 cameras, 2,000 points, 5 observations per point
    1: dict(name="tiny-16c-2kp-10ko", nc=16, np=2000, track=("fixed", 5), sigma=0.5,
            outlier_frac=0.0, loss="none", delta=0.0, seed=0,
            lm_iters=10, pcg_max=50, pcg_tol=1e-10),
    # Venice-1778-shaped: 1,700 cameras, 1M points, ~5M observations
    2: dict(name="venice-shaped-1700c-1mp-5mo", nc=1700, np=1_000_000, track=("geom", 0.25),
            sigma=1.0, outlier_frac=0.0, loss="none", delta=0.0, seed=1,
            lm_iters=20, pcg_max=100, pcg_tol=1e-10),
    # Final-13682-shaped: 13,000 cameras, 4.5M points, ~29M observations, Huber
    3: dict(name="final-shaped-13kc-4.5mp-29mo", nc=13000, np=4_500_000,
            track=("lognormal", 6.5, 300), sigma=1.0, outlier_frac=0.01, loss="huber",
            delta=2.0, seed=2, lm_iters=30, pcg_max=100, pcg_tol=1e-10),
    # differentiable layer: 200 cameras, 50k points, ~250k observations
    4: dict(name="layer-200c-50kp-250ko", nc=200, np=50_000, track=("geom", 0.25), sigma=1.0,
            outlier_frac=0.0, loss="none", delta=0.0, seed=3,
            lm_iters=100, pcg_max=100, pcg_tol=1e-12),
}


@dataclass
class Scene:
    cameras: np.ndarray          # (nc, 9) float64 initial estimate
    points: np.ndarray           # (np, 3) float64 initial estimate
    observations: np.ndarray     # (n, 2) float64 pixels
    cam_idx: np.ndarray          # (n,) int32
    pt_idx: np.ndarray           # (n,) int32
    cameras_true: np.ndarray     # (nc, 9) float64
    points_true: np.ndarray      # (np, 3) float64
    meta: dict = field(default_factory=dict)

    @property
    def nc(self) -> int:
        return int(self.cameras.shape[0])

    @property
    def np_(self) -> int:
        return int(self.points.shape[0])

    @property
    def n(self) -> int:
        return int(self.observations.shape[0])


def _lookat_rotations(nc: int) -> tuple[np.ndarray, np.ndarray]:
    """World-to-camera rotations and centres for cameras on the circle."""
    phi = 2.0 * np.pi * np.arange(nc) / nc
    centres = np.stack([CIRCLE_RADIUS * np.cos(phi), CIRCLE_RADIUS * np.sin(phi),
                        np.zeros(nc)], axis=1)
    z = centres / np.linalg.norm(centres, axis=1, keepdims=True)  # camera looks down -z
    up = np.array([0.0, 0.0, 1.0])
    x = np.cross(up[None, :], z)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=1)  # rows are the camera axes
    return R, centres


def lognormal_mu(mean_len: float, cap: int) -> float:
    """mu such that E[min(cap, 2 + floor(exp(N(mu, 1))))] = mean_len (bisection)."""
    ks = np.arange(1, cap - 1, dtype=np.float64)  # P(floor(Y) >= k) for k = 1 .. cap-2

    def expect(mu: float) -> float:
        z = (np.log(ks) - mu) / math.sqrt(2.0)
        tail = 0.5 * np.array([math.erfc(v) for v in z])
        return 2.0 + float(tail.sum())

    lo, hi = -10.0, 10.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if expect(mid) < mean_len:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _track_lengths(rng: np.random.Generator, npts: int, nc: int, track) -> np.ndarray:
    kind = track[0]
    if kind == "fixed":
        L = np.full(npts, int(track[1]), dtype=np.int64)
    elif kind == "geom":
        L = 1 + rng.geometric(float(track[1]), size=npts).astype(np.int64)
    elif kind == "lognormal":
        mu = lognormal_mu(float(track[1]), int(track[2]))
        L = 2 + np.floor(np.exp(rng.normal(mu, 1.0, size=npts))).astype(np.int64)
        L = np.minimum(L, int(track[2]))
    else:
        raise ValueError(f"unknown track kind {kind!r}")
    return np.minimum(L, nc)


def _choose_cameras(rng: np.random.Generator, L: np.ndarray, nc: int) -> np.ndarray:
    """For point j, L[j] distinct cameras uniformly without replacement (grouped by point)."""
    npts = L.shape[0]
    if nc <= 64:
        keys = rng.random((npts, nc))
        order = np.argsort(keys, axis=1, kind="stable")
        mask = np.arange(nc)[None, :] < L[:, None]
        return order[mask].astype(np.int64)
    pt = np.repeat(np.arange(npts, dtype=np.int64), L)
    cam = rng.integers(0, nc, size=pt.shape[0], dtype=np.int64)
    while True:
        key = pt * nc + cam
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.nonzero(ks[1:] == ks[:-1])[0] + 1
        if dup.size == 0:
            return cam
        redo = order[dup]
        cam[redo] = rng.integers(0, nc, size=redo.shape[0], dtype=np.int64)


def _synthesise_pixels(R: np.ndarray, t: np.ndarray, intr: np.ndarray, X: np.ndarray,
                       cam: np.ndarray, pt: np.ndarray, block: int = 1 << 22) -> np.ndarray:
    """Ideal pixels of points pt seen by cameras cam (rotation-matrix form)."""
    out = np.empty((cam.shape[0], 2), dtype=np.float64)
    for s in range(0, cam.shape[0], block):
        c = cam[s:s + block]
        Pc = np.einsum("kab,kb->ka", R[c], X[pt[s:s + block]]) + t[c]
        if np.any(Pc[:, 2] >= 0.0):
            raise RuntimeError("synthetic point behind a camera")
        p = -Pc[:, :2] / Pc[:, 2:3]
        r2 = np.sum(p * p, axis=1)
        f, k1, k2 = intr[c, 0], intr[c, 1], intr[c, 2]
        d = 1.0 + k1 * r2 + k2 * r2 * r2
        out[s:s + block] = (f * d)[:, None] * p
    return out


def make_scene(nc: int, npts: int, track=("fixed", 5), sigma: float = 1.0,
               outlier_frac: float = 0.0, outlier_px: float = 50.0, seed: int = 0,
               rot_sigma: float = 1e-2, trans_frac: float = 0.02, point_sigma: float = 0.02,
               shuffle: bool = True, meta: dict | None = None) -> Scene:
    """Draw one scene; every random number comes from one PCG64 stream in a fixed order."""
    if nc < 2 or npts < 1:
        raise ValueError("need at least 2 cameras and 1 point")
    rng = np.random.Generator(np.random.PCG64(seed))
    R, centres = _lookat_rotations(nc)
    t = -np.einsum("kab,kb->ka", R, centres)
    intr = np.stack([rng.uniform(500.0, 1500.0, nc), rng.normal(0.0, 1e-2, nc),
                     rng.normal(0.0, 1e-2, nc)], axis=1)
    X = rng.uniform(-0.5, 0.5, size=(npts, 3))
    L = _track_lengths(rng, npts, nc, track)
    cam = _choose_cameras(rng, L, nc)
    pt = np.repeat(np.arange(npts, dtype=np.int64), L)
    uv = _synthesise_pixels(R, t, intr, X, cam, pt)
    n = uv.shape[0]
    uv += rng.normal(0.0, sigma, size=(n, 2))
    n_out = int(round(outlier_frac * n))
    if n_out > 0:
        which = rng.choice(n, size=n_out, replace=False)
        ang = rng.uniform(0.0, 2.0 * np.pi, size=n_out)
        ideal = _synthesise_pixels(R, t, intr, X, cam[which], pt[which])
        uv[which] = ideal + outlier_px * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    if shuffle:
        order = rng.permutation(n)
        uv, cam, pt = uv[order], cam[order], pt[order]

    rot_true = Rotation.from_matrix(R)
    cams_true = np.concatenate([rot_true.as_rotvec(), t, intr], axis=1)
    eps = rng.normal(0.0, rot_sigma, size=(nc, 3))
    rot_init = Rotation.from_rotvec(eps) * rot_true
    t_init = t * (1.0 + rng.normal(0.0, trans_frac, size=(nc, 3)))
    cams_init = np.concatenate([rot_init.as_rotvec(), t_init, intr], axis=1)
    X_init = X + rng.normal(0.0, point_sigma, size=X.shape)
    m = dict(meta or {})
    m.update(nc=nc, np=npts, n=n, sigma=sigma, outlier_frac=outlier_frac, seed=seed)
    return Scene(cameras=np.ascontiguousarray(cams_init), points=np.ascontiguousarray(X_init),
                 observations=np.ascontiguousarray(uv), cam_idx=cam.astype(np.int32),
                 pt_idx=pt.astype(np.int32), cameras_true=np.ascontiguousarray(cams_true),
                 points_true=np.ascontiguousarray(X), meta=m)


def config_scene(cfg: int, scale: float = 1.0, seed: int | None = None) -> Scene:
    """Scene for one of the workloads in CONFIGS; ``scale`` shrinks cameras and points."""
    c = CONFIGS[cfg]
    nc = max(2, int(round(c["nc"] * scale)))
    npts = max(1, int(round(c["np"] * scale)))
    meta = {k: v for k, v in c.items() if k not in ("nc", "np", "track")}
    meta["config"] = cfg
    return make_scene(nc, npts, track=c["track"], sigma=c["sigma"],
                      outlier_frac=c["outlier_frac"], seed=c["seed"] if seed is None else seed,
                      meta=meta)


def make_windows(count: int = 512, seed: int = 4, cams=(5, 30), pts=(200, 3000),
                 sigma: float = 1.0) -> list[Scene]:
    """Independent local-BA windows: cameras U[5,30], points U[200,3000], track 2+Geom (mean 4)."""
    ss = np.random.SeedSequence(seed)
    rng = np.random.Generator(np.random.PCG64(ss))
    child = ss.spawn(count)
    out = []
    for w in range(count):
        nc = int(rng.integers(cams[0], cams[1] + 1))
        npts = int(rng.integers(pts[0], pts[1] + 1))
        s = int(np.random.Generator(np.random.PCG64(child[w])).integers(0, 2**62))
        out.append(make_scene(nc, npts, track=("geom", 1.0 / 3.0), sigma=sigma, seed=s,
                              meta={"window": w}))
    return out
