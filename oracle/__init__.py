"""CPU FP64 oracle for the bundle-adjustment hot path (MegBA, arXiv 2112.01349).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the product library never does.  It is
a ctypes wrapper around ``ba_oracle.c`` (plain C, FP64, fixed summation order),
built with gcc on first use.  The C file cites the paper passage behind every
function; the Python side only marshals arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ba_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

LOSS = {"none": 0, "huber": 1}
DAMPING = {"diag": 0, "identity": 1}
SCHUR = {"implicit_pcg": 0, "explicit_pcg": 1, "dense": 2}
PRECOND = {"block_jacobi": 0, "schur_jacobi": 1}
PCG_VARIANT = {"standard": 0, "single_reduction": 1}


def build(force: bool = False) -> str:
    """Compile ba_oracle.c into _build/liborc.so (gcc, OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Trace(C.Structure):
    _fields_ = [("cost", C.c_double), ("cost_new", C.c_double), ("model_dec", C.c_double),
                ("mu", C.c_double), ("gain", C.c_double), ("accepted", C.c_int),
                ("pcg_iters", C.c_int), ("pcg_rel_res", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i32, i64, dbl = C.c_int32, C.c_int64, C.c_double
            lib.orc_project.argtypes = [P, P, P]
            lib.orc_residual_jacobian.argtypes = [P, P, P, P, P, P]
            lib.orc_loss.argtypes = [C.c_int, dbl, dbl, P, P]
            lib.orc_evaluate.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, P, P, P, P, P]
            lib.orc_stable_sort.argtypes = [i64, P, i32, P, P]
            lib.orc_blocks.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, P, P, P, P, P]
            lib.orc_step.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, dbl, C.c_int, C.c_int,
                                     C.c_int, dbl, P, P, P, P, P, C.c_int, P, P, C.c_int]
            lib.orc_schur_jacobi_blocks.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, dbl, C.c_int, P]
            lib.orc_schur.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, dbl, C.c_int, P, P, P, P]
            lib.orc_lm_solve.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, C.c_int, C.c_int, dbl,
                                         C.c_int, dbl, dbl, dbl, C.c_int, P, P, P, P, C.c_int, C.c_int, P, P,
                                         C.c_int]
            lib.orc_adjoint.argtypes = [i32, i32, i64, P, P, P, P, P, C.c_int, dbl, dbl, C.c_int, C.c_int, dbl, P, P,
                                        P, P, P, P, C.c_int, C.c_int]
            lib.orc_num_threads.restype = C.c_int
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def project(cam, X):
    cam, X = _f64(cam, (9,)), _f64(X, (3,))
    out = np.zeros(2)
    _load().orc_project(_p(cam), _p(X), _p(out))
    return out


def residual_jacobian(cam, X, u):
    """(e (2,), Jc (2,9), Jp (2,3)) for one observation."""
    cam, X, u = _f64(cam, (9,)), _f64(X, (3,)), _f64(u, (2,))
    e, Jc, Jp = np.zeros(2), np.zeros((2, 9)), np.zeros((2, 3))
    _load().orc_residual_jacobian(_p(cam), _p(X), _p(u), _p(e), _p(Jc), _p(Jp))
    return e, Jc, Jp


def loss(kind: str, delta: float, s: float):
    rho, w = C.c_double(), C.c_double()
    _load().orc_loss(LOSS[kind], float(delta), float(s), C.byref(rho), C.byref(w))
    return rho.value, w.value


def _prob(cams, pts, obs, cam_idx, pt_idx):
    cams, pts, obs = _f64(cams), _f64(pts), _f64(obs)
    cam_idx, pt_idx = _i32(cam_idx), _i32(pt_idx)
    return cams, pts, obs, cam_idx, pt_idx, cams.shape[0], pts.shape[0], obs.shape[0]


def evaluate(cams, pts, obs, cam_idx, pt_idx, loss="none", delta=0.0, jacobians=True):
    """cost, e (n,2), Jc (n,2,9), Jp (n,2,3), W (n,) in input order."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    cost = C.c_double()
    e = np.zeros((n, 2))
    Jc = np.zeros((n, 2, 9)) if jacobians else None
    Jp = np.zeros((n, 2, 3)) if jacobians else None
    W = np.zeros(n)
    rc = _load().orc_evaluate(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss], float(delta),
                              C.byref(cost), _p(e), _p(Jc), _p(Jp), _p(W))
    if rc:
        raise RuntimeError(f"orc_evaluate failed: {rc}")
    return cost.value, e, Jc, Jp, W


def stable_sort(keys, nkeys):
    keys = _i32(keys)
    perm = np.zeros(keys.shape[0], dtype=np.int32)
    ptr = np.zeros(nkeys + 1, dtype=np.int32)
    rc = _load().orc_stable_sort(keys.shape[0], _p(keys), int(nkeys), _p(perm), _p(ptr))
    if rc:
        raise RuntimeError(f"orc_stable_sort failed: {rc}")
    return perm, ptr


def blocks(cams, pts, obs, cam_idx, pt_idx, loss="none", delta=0.0, with_E=False):
    """Hpp (nc,9,9), v (nc,9), Hll (np,3,3), w (np,3) [, E (n,9,3)]."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    Hpp, v = np.zeros((nc, 9, 9)), np.zeros((nc, 9))
    Hll, w = np.zeros((np_, 3, 3)), np.zeros((np_, 3))
    E = np.zeros((n, 9, 3)) if with_E else None
    rc = _load().orc_blocks(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss], float(delta),
                            _p(Hpp), _p(v), _p(Hll), _p(w), _p(E))
    if rc:
        raise RuntimeError(f"orc_blocks failed: {rc}")
    return (Hpp, v, Hll, w, E) if with_E else (Hpp, v, Hll, w)


def _fixed(mask, m):
    """A uint8 mask of m nodes held constant, or None."""
    if mask is None:
        return None
    a = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    if a.shape[0] != m:
        raise ValueError("fixed-node mask has the wrong length")
    return a


def step(cams, pts, obs, cam_idx, pt_idx, mu, loss="none", delta=0.0, damping="diag", schur="implicit_pcg",
         pcg_max=100, pcg_tol=1e-10, precond="block_jacobi", cam_fixed=None, pt_fixed=None,
         pcg_variant="standard"):
    """One damped Schur step: dict(dc (nc,9), dp (np,3), pcg_iters, rel_res, model_dec).
    cam_fixed / pt_fixed: optional masks of nodes held constant; pcg_variant:
    "standard" (Alg. 2) or "single_reduction" (Chronopoulos-Gear form)."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    cf, pf = _fixed(cam_fixed, nc), _fixed(pt_fixed, np_)
    dc, dp = np.zeros((nc, 9)), np.zeros((np_, 3))
    it, rr, md = C.c_int(), C.c_double(), C.c_double()
    rc = _load().orc_step(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss], float(delta),
                          float(mu), DAMPING[damping], SCHUR[schur], int(pcg_max), float(pcg_tol), _p(dc), _p(dp),
                          C.byref(it), C.byref(rr), C.byref(md), PRECOND[precond], _p(cf), _p(pf),
                          PCG_VARIANT[pcg_variant])
    if rc:
        raise RuntimeError(f"orc_step failed: {rc}")
    return dict(dc=dc, dp=dp, pcg_iters=it.value, rel_res=rr.value, model_dec=md.value)


def schur_jacobi_blocks(cams, pts, obs, cam_idx, pt_idx, mu, loss="none", delta=0.0, damping="diag"):
    """Schur-Jacobi camera blocks S~_ii (nc, 9, 9) at damping mu."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    out = np.zeros((nc, 9, 9))
    rc = _load().orc_schur_jacobi_blocks(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss],
                                         float(delta), float(mu), DAMPING[damping], _p(out))
    if rc:
        raise RuntimeError(f"orc_schur_jacobi_blocks failed: {rc}")
    return out


def schur(cams, pts, obs, cam_idx, pt_idx, mu, x=None, loss="none", delta=0.0, damping="diag", dense=False):
    """dict(y = S x (nc*9,) if x given, rhs (nc*9,), S (9nc, 9nc) if dense)."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    xv = None if x is None else _f64(x, (9 * nc,))
    y = None if x is None else np.zeros(9 * nc)
    rhs = np.zeros(9 * nc)
    S = np.zeros((9 * nc, 9 * nc)) if dense else None
    rc = _load().orc_schur(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss], float(delta),
                           float(mu), DAMPING[damping], _p(xv), _p(y), _p(rhs), _p(S))
    if rc:
        raise RuntimeError(f"orc_schur failed: {rc}")
    return dict(y=y, rhs=rhs, S=S)


def lm_solve(cams, pts, obs, cam_idx, pt_idx, max_iter=10, pcg_max=50, pcg_tol=1e-10, loss="none", delta=0.0,
             damping="diag", initial_radius=1e4, min_rel_dec=1e-3, function_tol=0.0, schur="implicit_pcg",
             precond="block_jacobi", forcing=False, cam_fixed=None, pt_fixed=None, pcg_variant="standard"):
    """Run the LM loop; returns dict(cameras, points, trace (list of dict), iterations, final_cost, radius).
    cam_fixed / pt_fixed: optional masks of nodes held constant."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    cf, pf = _fixed(cam_fixed, nc), _fixed(pt_fixed, np_)
    cams, pts = cams.copy(), pts.copy()
    tr = (Trace * max(1, max_iter))()
    it, fc, rad = C.c_int(), C.c_double(), C.c_double()
    rc = _load().orc_lm_solve(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss], float(delta),
                              int(max_iter), int(pcg_max), float(pcg_tol), DAMPING[damping], float(initial_radius),
                              float(min_rel_dec), float(function_tol), SCHUR[schur], C.cast(tr, C.c_void_p),
                              C.byref(it), C.byref(fc), C.byref(rad), PRECOND[precond], 1 if forcing else 0,
                              _p(cf), _p(pf), PCG_VARIANT[pcg_variant])
    if rc:
        raise RuntimeError(f"orc_lm_solve failed: {rc}")
    trace = [{f: getattr(tr[i], f) for f, _ in Trace._fields_} for i in range(it.value)]
    return dict(cameras=cams, points=pts, trace=trace, iterations=it.value, final_cost=fc.value, radius=rad.value)


def adjoint(cams, pts, obs, cam_idx, pt_idx, mu, gbar_c, gbar_p, loss="none", delta=0.0, damping="diag",
            pcg_max=500, pcg_tol=1e-14, precond="block_jacobi", pcg_variant="standard"):
    """dict(grad_obs (n,2), grad_c0 (nc,9), grad_p0 (np,3), pcg_iters) for upstream gradient (gbar_c, gbar_p)."""
    cams, pts, obs, ci, pi, nc, np_, n = _prob(cams, pts, obs, cam_idx, pt_idx)
    gc, gp = _f64(gbar_c, (nc, 9)), _f64(gbar_p, (np_, 3))
    go, gc0, gp0 = np.zeros((n, 2)), np.zeros((nc, 9)), np.zeros((np_, 3))
    it = C.c_int()
    rc = _load().orc_adjoint(nc, np_, n, _p(cams), _p(pts), _p(obs), _p(ci), _p(pi), LOSS[loss], float(delta),
                             float(mu), DAMPING[damping], int(pcg_max), float(pcg_tol), _p(gc), _p(gp), _p(go),
                             _p(gc0), _p(gp0), C.byref(it), PRECOND[precond], PCG_VARIANT[pcg_variant])
    if rc:
        raise RuntimeError(f"orc_adjoint failed: {rc}")
    return dict(grad_obs=go, grad_c0=gc0, grad_p0=gp0, pcg_iters=it.value)
