"""Python binding of the C ABI in include/mba.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arrays and structures; all computation runs in the CUDA
kernels of ``_build/libmba.so``.  There is no fallback: if the library is not
built, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

MBA_OK, MBA_ERR_INVALID_ARG, MBA_ERR_OOM, MBA_ERR_CUDA = 0, 1, 2, 3
MBA_ERR_NONFINITE, MBA_ERR_TIMEOUT, MBA_ERR_NOT_CONVERGED = 4, 5, 6
MBA_FP64, MBA_FP32_MIXED = 0, 1
MBA_LOSS_NONE, MBA_LOSS_HUBER = 0, 1
MBA_DAMP_DIAG, MBA_DAMP_IDENTITY = 0, 1

PRECISION = {"fp64": MBA_FP64, "fp32": MBA_FP32_MIXED, "fp32_mixed": MBA_FP32_MIXED}
LOSS = {"none": MBA_LOSS_NONE, "huber": MBA_LOSS_HUBER}
DAMPING = {"diag": MBA_DAMP_DIAG, "identity": MBA_DAMP_IDENTITY}
MBA_PRECOND_BLOCK_JACOBI, MBA_PRECOND_SCHUR_JACOBI = 0, 1
PRECONDITIONER = {"block_jacobi": MBA_PRECOND_BLOCK_JACOBI, "schur_jacobi": MBA_PRECOND_SCHUR_JACOBI}
MBA_JACOBIAN_ANALYTIC, MBA_JACOBIAN_AUTODIFF = 0, 1
JACOBIAN = {"analytic": MBA_JACOBIAN_ANALYTIC, "autodiff": MBA_JACOBIAN_AUTODIFF}
MBA_COST_FP64, MBA_COST_FLOAT_FLOAT = 0, 1
COST_ARITHMETIC = {"fp64": MBA_COST_FP64, "float-float": MBA_COST_FLOAT_FLOAT}
MBA_PCG_STANDARD, MBA_PCG_SINGLE_REDUCTION = 0, 1
PCG_VARIANT = {"standard": MBA_PCG_STANDARD, "single_reduction": MBA_PCG_SINGLE_REDUCTION}


class MbaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class ProblemOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("loss", C.c_int32), ("huber_delta", C.c_double),
                ("cuda_stream", C.c_void_p), ("jacobian", C.c_int32), ("pad", C.c_int32)]


class SolverOptions(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("pcg_max_iter", C.c_int32), ("pcg_rel_tol", C.c_double),
                ("damping", C.c_int32), ("initial_radius", C.c_double), ("min_relative_decrease", C.c_double),
                ("function_tol", C.c_double), ("barrier_spin_limit", C.c_int64), ("collect_timing", C.c_int32),
                ("preconditioner", C.c_int32), ("forcing", C.c_int32), ("cost_arithmetic", C.c_int32),
                ("pcg_variant", C.c_int32)]


class Iteration(C.Structure):
    _fields_ = [("cost", C.c_double), ("cost_new", C.c_double), ("model_decrease", C.c_double),
                ("mu", C.c_double), ("gain", C.c_double), ("accepted", C.c_int32), ("pcg_iters", C.c_int32),
                ("pcg_rel_residual", C.c_double)]


class Summary(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accepted", C.c_int32), ("pcg_iters_total", C.c_int32),
                ("status", C.c_int32), ("initial_cost", C.c_double), ("final_cost", C.c_double),
                ("final_mu", C.c_double), ("final_radius", C.c_double), ("ms_total", C.c_double),
                ("ms_linearize", C.c_double), ("ms_pcg", C.c_double), ("ms_other", C.c_double),
                ("kernel_launches", C.c_int32),
                ("trace", C.POINTER(Iteration)), ("trace_capacity", C.c_int32)]


class WindowSummary(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("accepted", C.c_int32), ("pcg_iters_total", C.c_int32),
                ("status", C.c_int32), ("initial_cost", C.c_double), ("final_cost", C.c_double),
                ("final_radius", C.c_double), ("mu_accepted", C.c_double), ("adjoint_pcg_iters", C.c_int32),
                ("pad", C.c_int32)]


class BatchSchedule(C.Structure):
    _fields_ = [("threads_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32), ("schur", C.c_int32)]


class BatchAdjoint(C.Structure):
    _fields_ = [("grad_cameras", C.c_void_p), ("grad_points", C.c_void_p), ("pcg_max_iter", C.c_int32),
                ("pad", C.c_int32), ("pcg_rel_tol", C.c_double), ("mu", C.c_double)]


_lock = threading.Lock()
_lib = None


_lib_path = None


def library_path() -> str:
    return _lib_path or _build.LIB


def load(path: str | None = None):
    """Load libmba.so (built in-tree by __graft_entry__.build()), or the
    library at path (a build with a user edge type, _build.build(edge=...)),
    once per process."""
    global _lib, _lib_path
    with _lock:
        if _lib is not None:
            if path is not None and os.path.abspath(path) != os.path.abspath(library_path()):
                raise RuntimeError(f"{library_path()} is already loaded in this process")
            return _lib
        target = path or _build.LIB
        if not os.path.exists(target):
            raise RuntimeError(f"{target} is missing: build the CUDA library first (__graft_entry__.build())")
        lib = C.CDLL(target)
        _lib_path = target
        P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "mba_problem_options_default": (None, [P]),
            "mba_solver_options_default": (None, [P]),
            "mba_problem_create": (C.c_int, [P, i32, P, i32, P, P, P, i64, P, P]),
            "mba_problem_destroy": (None, [P]),
            "mba_problem_info": (C.c_int, [P, P, P, P, P]),
            "mba_evaluate": (C.c_int, [P, P, P, P, P]),
            "mba_solve": (C.c_int, [P, P, P]),
            "mba_get_parameters": (C.c_int, [P, P, P]),
            "mba_set_parameters": (C.c_int, [P, P, P]),
            "mba_reset": (C.c_int, [P]),
            "mba_get_ordering": (C.c_int, [P, P, P, P, P]),
            "mba_linear_system": (C.c_int, [P, dbl, i32, P, P, P, P, P]),
            "mba_schur_matvec": (C.c_int, [P, dbl, i32, P, P]),
            "mba_step": (C.c_int, [P, dbl, P, P, P, P, P]),
            "mba_cost_noalloc": (C.c_int, [P, i32, P, i32, P, P, P, i64, i32, dbl, P, P]),
            "mba_adjoint": (C.c_int, [P, P, dbl, P, P, P, P, P, P]),
            "mba_batch_create": (C.c_int, [i32, P, P, P, P, P, P, P, P, P, P]),
            "mba_batch_destroy": (None, [P]),
            "mba_batch_info": (C.c_int, [P, P, P, P, P, P]),
            "mba_batch_set_schedule": (C.c_int, [P, P]),
            "mba_batch_get_schedule": (C.c_int, [P, P]),
            "mba_batch_autotune": (C.c_int, [P, P, P, P]),
            "mba_batch_solve": (C.c_int, [P, P, P, P, P]),
            "mba_batch_get_parameters": (C.c_int, [P, P, P]),
            "mba_batch_set_parameters": (C.c_int, [P, P, P]),
            "mba_batch_reset": (C.c_int, [P]),
            "mba_batch_get_gradients": (C.c_int, [P, P, P, P]),
            "mba_batch_window_times": (C.c_int, [P, P]),
            "mba_bal_read": (C.c_int, [C.c_char_p, P, P, P, P, P, P, P, P]),
            "mba_bal_write": (C.c_int, [C.c_char_p, i32, i32, i64, P, P, P, P, P]),
            "mba_status_string": (C.c_char_p, [C.c_int]),
            "mba_edge_name": (C.c_char_p, []),
            "mba_last_error": (C.c_char_p, []),
            "mba_set_device_memory_limit": (C.c_int, [C.c_size_t]),
            "mba_set_fixed": (C.c_int, [P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().mba_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return f"status {status}"


def _check(status: int):
    if status != MBA_OK:
        raise MbaError(status, load().mba_last_error().decode())


def _ptr(a, dtype):
    """Host pointer of a contiguous numpy array or CPU torch tensor of the given dtype."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch

        want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.is_cuda or a.dtype != want or not a.is_contiguous():
            raise ValueError("host tensor must be a contiguous CPU tensor of the right dtype")
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), arr


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def mba_problem_options_default() -> ProblemOptions:
    o = ProblemOptions()
    load().mba_problem_options_default(C.byref(o))
    return o


def mba_solver_options_default() -> SolverOptions:
    o = SolverOptions()
    load().mba_solver_options_default(C.byref(o))
    return o


def mba_problem_create(cameras, points, observations, cam_idx, pt_idx, precision="fp64", loss="none",
                       huber_delta=0.0, stream=None, jacobian="analytic") -> C.c_void_p:
    lib = load()
    pc, ac = _ptr(cameras, np.float64)
    pp, ap = _ptr(points, np.float64)
    po, ao = _ptr(observations, np.float64)
    pci, aci = _ptr(cam_idx, np.int32)
    ppi, api = _ptr(pt_idx, np.int32)
    nc, np_ = int(len(ac)), int(len(ap))
    n = int(len(ao))
    if int(np.prod(ac.shape)) != 9 * nc or int(np.prod(ap.shape)) != 3 * np_ or int(np.prod(ao.shape)) != 2 * n:
        raise ValueError("cameras must be (nc, 9), points (np, 3), observations (n, 2)")
    if len(aci) != n or len(api) != n:
        raise ValueError("cam_idx and pt_idx must have one entry per observation")
    o = mba_problem_options_default()
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.loss = LOSS[loss] if isinstance(loss, str) else int(loss)
    o.huber_delta = float(huber_delta)
    o.cuda_stream = _stream_handle(stream)
    o.jacobian = JACOBIAN[jacobian] if isinstance(jacobian, str) else int(jacobian)
    h = C.c_void_p()
    _check(lib.mba_problem_create(pc, nc, pp, np_, po, pci, ppi, n, C.byref(o), C.byref(h)))
    return h


def mba_problem_destroy(h):
    if h:
        load().mba_problem_destroy(h)


def mba_problem_info(h):
    nc, np_, n, b = C.c_int32(), C.c_int32(), C.c_int64(), C.c_size_t()
    _check(load().mba_problem_info(h, C.byref(nc), C.byref(np_), C.byref(n), C.byref(b)))
    return dict(nc=nc.value, np=np_.value, n=n.value, device_bytes=b.value)


def mba_evaluate(h, residuals=True, jacobians=True):
    info = mba_problem_info(h)
    n = info["n"]
    cost = C.c_double()
    e = np.zeros((n, 2)) if residuals else None
    jc = np.zeros((n, 2, 9)) if jacobians else None
    jp = np.zeros((n, 2, 3)) if jacobians else None
    f = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(load().mba_evaluate(h, C.byref(cost), f(e), f(jc), f(jp)))
    return cost.value, e, jc, jp


def solver_options(**kw) -> SolverOptions:
    o = mba_solver_options_default()
    for k, v in kw.items():
        if k == "damping" and isinstance(v, str):
            v = DAMPING[v]
        if k == "preconditioner" and isinstance(v, str):
            v = PRECONDITIONER[v]
        if k == "forcing":
            v = int(bool(v))
        if k == "cost_arithmetic" and isinstance(v, str):
            v = COST_ARITHMETIC[v]
        if k == "pcg_variant" and isinstance(v, str):
            v = PCG_VARIANT[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown solver option {k}")
        setattr(o, k, v)
    return o


def mba_solve(h, trace_capacity=0, **opts):
    o = solver_options(**opts)
    s = Summary()
    tr = None
    if trace_capacity > 0:
        tr = (Iteration * trace_capacity)()
        s.trace = C.cast(tr, C.POINTER(Iteration))
        s.trace_capacity = trace_capacity
    st = load().mba_solve(h, C.byref(o), C.byref(s))
    out = {f: getattr(s, f) for f, _ in Summary._fields_ if f not in ("trace", "trace_capacity")}
    if tr is not None:
        out["trace"] = [{f: getattr(tr[i], f) for f, _ in Iteration._fields_}
                        for i in range(min(s.iterations, trace_capacity))]
    _check(st)
    return out


def mba_get_parameters(h, cameras=None, points=None):
    info = mba_problem_info(h)
    cams = np.zeros((info["nc"], 9)) if cameras is None else cameras
    pts = np.zeros((info["np"], 3)) if points is None else points
    pc, _ = _ptr(cams, np.float64)
    pp, _ = _ptr(pts, np.float64)
    _check(load().mba_get_parameters(h, pc, pp))
    return cams, pts


def mba_set_parameters(h, cameras=None, points=None):
    pc, ac = _ptr(cameras, np.float64)
    pp, ap = _ptr(points, np.float64)
    _check(load().mba_set_parameters(h, pc, pp))


def mba_reset(h):
    _check(load().mba_reset(h))


def mba_get_ordering(h):
    info = mba_problem_info(h)
    n, nc, np_ = info["n"], info["nc"], info["np"]
    pt_perm, pt_ptr = np.zeros(n, np.int32), np.zeros(np_ + 1, np.int32)
    cam_perm, cam_ptr = np.zeros(n, np.int32), np.zeros(nc + 1, np.int32)
    f = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(load().mba_get_ordering(h, f(pt_perm), f(pt_ptr), f(cam_perm), f(cam_ptr)))
    return pt_perm, pt_ptr, cam_perm, cam_ptr


def mba_linear_system(h, mu, damping="diag"):
    info = mba_problem_info(h)
    nc, np_ = info["nc"], info["np"]
    Hpp, v = np.zeros((nc, 9, 9)), np.zeros((nc, 9))
    Hll, w = np.zeros((np_, 3, 3)), np.zeros((np_, 3))
    rhs = np.zeros((nc, 9))
    f = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(load().mba_linear_system(h, float(mu), DAMPING[damping], f(Hpp), f(v), f(Hll), f(w), f(rhs)))
    return dict(Hpp=Hpp, v=v, Hll=Hll, w=w, rhs=rhs)


def mba_schur_matvec(h, mu, x, damping="diag"):
    info = mba_problem_info(h)
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(info["nc"], 9)
    y = np.zeros_like(xx)
    _check(load().mba_schur_matvec(h, float(mu), DAMPING[damping], xx.ctypes.data_as(C.c_void_p),
                                   y.ctypes.data_as(C.c_void_p)))
    return y


def mba_step(h, mu, **opts):
    info = mba_problem_info(h)
    o = solver_options(**opts)
    dc, dp = np.zeros((info["nc"], 9)), np.zeros((info["np"], 3))
    it, md = C.c_int32(), C.c_double()
    _check(load().mba_step(h, float(mu), C.byref(o), dc.ctypes.data_as(C.c_void_p), dp.ctypes.data_as(C.c_void_p),
                           C.byref(it), C.byref(md)))
    return dict(dc=dc, dp=dp, pcg_iters=it.value, model_dec=md.value)


def mba_adjoint(h, grad_cameras, grad_points, mu=-1.0, **opts):
    """dict(grad_obs (n,2), grad_init_cam (nc,9), grad_init_pt (np,3), pcg_iters) for dL/dx* = (grad_cameras,
    grad_points); mu < 0 uses the damping of the last solve's last accepted step."""
    info = mba_problem_info(h)
    o = solver_options(**opts)
    gc = np.ascontiguousarray(grad_cameras, dtype=np.float64).reshape(info["nc"], 9)
    gp = np.ascontiguousarray(grad_points, dtype=np.float64).reshape(info["np"], 3)
    go = np.zeros((info["n"], 2))
    gc0, gp0 = np.zeros((info["nc"], 9)), np.zeros((info["np"], 3))
    it = C.c_int32()
    f = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(load().mba_adjoint(h, C.byref(o), float(mu), f(gc), f(gp), f(go), f(gc0), f(gp0), C.byref(it)))
    return dict(grad_obs=go, grad_init_cam=gc0, grad_init_pt=gp0, pcg_iters=it.value)


def mba_cost_noalloc(d_cameras, nc, d_points, np_, d_observations, d_cam_idx, d_pt_idx, n, loss="none",
                     huber_delta=0.0, d_cost=None, stream=None):
    """Cost from caller-owned device arrays (integer device addresses); no allocation.

    Enqueues the work on ``stream`` and returns; the cost lands in ``d_cost``.
    """
    lb = LOSS[loss] if isinstance(loss, str) else int(loss)
    _check(load().mba_cost_noalloc(C.c_void_p(d_cameras), int(nc), C.c_void_p(d_points), int(np_),
                                   C.c_void_p(d_observations), C.c_void_p(d_cam_idx), C.c_void_p(d_pt_idx), int(n),
                                   lb, float(huber_delta), C.c_void_p(d_cost), _stream_handle(stream)))


def mba_set_fixed(h, cam_fixed=None, pt_fixed=None):
    """Mark cameras / points constant (boolean masks of nc / np entries; None = none fixed)."""
    info = mba_problem_info(h)
    cf = None if cam_fixed is None else np.ascontiguousarray(cam_fixed, dtype=np.uint8).reshape(info["nc"])
    pf = None if pt_fixed is None else np.ascontiguousarray(pt_fixed, dtype=np.uint8).reshape(info["np"])
    f = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(load().mba_set_fixed(h, f(cf), f(pf)))


def mba_set_device_memory_limit(nbytes: int) -> None:
    """Cap the device memory one creation may allocate (0 = no cap); creations
    over the cap fail with MBA_ERR_OOM before allocating."""
    _check(load().mba_set_device_memory_limit(int(nbytes)))


class Problem:
    """Owning wrapper over one mba_problem handle."""

    def __init__(self, cameras, points, observations, cam_idx, pt_idx, precision="fp64", loss="none",
                 huber_delta=0.0, stream=None, jacobian="analytic"):
        self.handle = mba_problem_create(cameras, points, observations, cam_idx, pt_idx, precision, loss,
                                         huber_delta, stream, jacobian)
        self.info = mba_problem_info(self.handle)

    def close(self):
        if self.handle:
            mba_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def evaluate(self, residuals=True, jacobians=True):
        return mba_evaluate(self.handle, residuals, jacobians)

    def solve(self, trace_capacity=0, **opts):
        return mba_solve(self.handle, trace_capacity, **opts)

    def parameters(self):
        return mba_get_parameters(self.handle)

    def set_parameters(self, cameras=None, points=None):
        mba_set_parameters(self.handle, cameras, points)

    def reset(self):
        mba_reset(self.handle)

    def set_fixed(self, cam_fixed=None, pt_fixed=None):
        mba_set_fixed(self.handle, cam_fixed, pt_fixed)

    def ordering(self):
        return mba_get_ordering(self.handle)

    def linear_system(self, mu, damping="diag"):
        return mba_linear_system(self.handle, mu, damping)

    def schur_matvec(self, mu, x, damping="diag"):
        return mba_schur_matvec(self.handle, mu, x, damping)

    def step(self, mu, **opts):
        return mba_step(self.handle, mu, **opts)

    def adjoint(self, grad_cameras, grad_points, mu=-1.0, **opts):
        return mba_adjoint(self.handle, grad_cameras, grad_points, mu, **opts)


# ---------------------------------------------------------------------------
# batched windows
# ---------------------------------------------------------------------------
def _vp(a):
    return a.ctypes.data_as(C.c_void_p)


def mba_batch_create(cam_offsets, pt_offsets, obs_offsets, cameras, points, observations, cam_idx, pt_idx,
                     precision="fp32", loss="none", huber_delta=0.0, stream=None, jacobian="analytic") -> C.c_void_p:
    """Concatenated windows (offset arrays of n_windows + 1 entries; cam_idx / pt_idx local to the window)."""
    co = np.ascontiguousarray(cam_offsets, dtype=np.int64)
    po = np.ascontiguousarray(pt_offsets, dtype=np.int64)
    oo = np.ascontiguousarray(obs_offsets, dtype=np.int64)
    nw = len(co) - 1
    if nw < 1 or len(po) != nw + 1 or len(oo) != nw + 1:
        raise ValueError("offset arrays must have n_windows + 1 entries")
    cams = np.ascontiguousarray(cameras, dtype=np.float64).reshape(-1, 9)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    obs = np.ascontiguousarray(observations, dtype=np.float64).reshape(-1, 2)
    ci = np.ascontiguousarray(cam_idx, dtype=np.int32)
    pi = np.ascontiguousarray(pt_idx, dtype=np.int32)
    if len(cams) != co[-1] or len(pts) != po[-1] or len(obs) != oo[-1] or len(ci) != oo[-1] or len(pi) != oo[-1]:
        raise ValueError("array lengths must match the last offsets")
    o = mba_problem_options_default()
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.loss = LOSS[loss] if isinstance(loss, str) else int(loss)
    o.huber_delta = float(huber_delta)
    o.cuda_stream = _stream_handle(stream)
    o.jacobian = JACOBIAN[jacobian] if isinstance(jacobian, str) else int(jacobian)
    h = C.c_void_p()
    _check(load().mba_batch_create(nw, _vp(co), _vp(po), _vp(oo), _vp(cams), _vp(pts), _vp(obs), _vp(ci), _vp(pi),
                                   C.byref(o), C.byref(h)))
    return h


def mba_batch_destroy(h):
    if h:
        load().mba_batch_destroy(h)


def mba_batch_info(h):
    nw, mc = C.c_int32(), C.c_int32()
    nc, np_, n = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().mba_batch_info(h, C.byref(nw), C.byref(nc), C.byref(np_), C.byref(n), C.byref(mc)))
    return dict(n_windows=nw.value, nc=nc.value, np=np_.value, n=n.value, max_window_cameras=mc.value)


SCHUR = {"auto": 0, "implicit": 1, "explicit": 2}


def mba_batch_set_schedule(h, threads_per_cta=0, ctas_per_sm=0, schur="auto"):
    sc = BatchSchedule(int(threads_per_cta), int(ctas_per_sm), SCHUR[schur] if isinstance(schur, str) else int(schur))
    _check(load().mba_batch_set_schedule(h, C.byref(sc)))


def mba_batch_get_schedule(h):
    sc = BatchSchedule()
    _check(load().mba_batch_get_schedule(h, C.byref(sc)))
    return dict(threads_per_cta=sc.threads_per_cta, ctas_per_sm=sc.ctas_per_sm,
                schur={1: "implicit", 2: "explicit"}.get(sc.schur, "auto"))


def mba_batch_autotune(h, **opts):
    o = solver_options(**opts)
    sc = BatchSchedule()
    ms = C.c_double()
    _check(load().mba_batch_autotune(h, C.byref(o), C.byref(sc), C.byref(ms)))
    return dict(threads_per_cta=sc.threads_per_cta, ctas_per_sm=sc.ctas_per_sm,
                schur={1: "implicit", 2: "explicit"}.get(sc.schur, "auto"), ms=ms.value)


def _summaries(arr):
    names = [f[0] for f in WindowSummary._fields_ if f[0] != "pad"]
    return [{k: getattr(s, k) for k in names} for s in arr]


def mba_batch_solve(h, grad_cameras=None, grad_points=None, adjoint_pcg_max_iter=500, adjoint_pcg_rel_tol=1e-12,
                    adjoint_mu=-1.0, check=True, **opts):
    """Solves every window; with grad_cameras / grad_points also runs the adjoint.

    Returns dict(summaries=[per-window dict], ms=device time of the launch, status)."""
    info = mba_batch_info(h)
    o = solver_options(**opts)
    adj = None
    keep = []
    if grad_cameras is not None or grad_points is not None:
        gc = np.ascontiguousarray(grad_cameras, dtype=np.float64).reshape(info["nc"], 9)
        gp = np.ascontiguousarray(grad_points, dtype=np.float64).reshape(info["np"], 3)
        keep = [gc, gp]
        adj = BatchAdjoint(_vp(gc), _vp(gp), int(adjoint_pcg_max_iter), 0, float(adjoint_pcg_rel_tol),
                           float(adjoint_mu))
    arr = (WindowSummary * info["n_windows"])()
    ms = C.c_double()
    st = load().mba_batch_solve(h, C.byref(o), C.byref(adj) if adj is not None else None, arr, C.byref(ms))
    del keep
    if check:
        _check(st)
    return dict(summaries=_summaries(arr), ms=ms.value, status=st)


def mba_batch_get_parameters(h):
    info = mba_batch_info(h)
    cams, pts = np.zeros((info["nc"], 9)), np.zeros((info["np"], 3))
    _check(load().mba_batch_get_parameters(h, _vp(cams), _vp(pts)))
    return cams, pts


def mba_batch_set_parameters(h, cameras=None, points=None):
    info = mba_batch_info(h)
    c = None if cameras is None else np.ascontiguousarray(cameras, dtype=np.float64).reshape(info["nc"], 9)
    p = None if points is None else np.ascontiguousarray(points, dtype=np.float64).reshape(info["np"], 3)
    _check(load().mba_batch_set_parameters(h, None if c is None else _vp(c), None if p is None else _vp(p)))


def mba_batch_reset(h):
    _check(load().mba_batch_reset(h))


def mba_batch_get_gradients(h):
    info = mba_batch_info(h)
    go, gc, gp = np.zeros((info["n"], 2)), np.zeros((info["nc"], 9)), np.zeros((info["np"], 3))
    _check(load().mba_batch_get_gradients(h, _vp(go), _vp(gc), _vp(gp)))
    return dict(grad_obs=go, grad_init_cam=gc, grad_init_pt=gp)


def mba_edge_name() -> str:
    """The edge type of the loaded library's dual-number path ("BalEdge" or a user type)."""
    return load().mba_edge_name().decode()


def mba_batch_window_times(h):
    """Milliseconds each window took in the last solve (input order)."""
    ms = np.zeros(mba_batch_info(h)["n_windows"])
    _check(load().mba_batch_window_times(h, _vp(ms)))
    return ms


_COMPRESSED = {".bz2": "bz2", ".gz": "gzip", ".xz": "lzma"}


def _codec(path):
    """The standard-library module for a compressed BAL path (by suffix), or None."""
    ext = os.path.splitext(os.fspath(path))[1].lower()
    if ext not in _COMPRESSED:
        return None
    import importlib

    return importlib.import_module(_COMPRESSED[ext])


def mba_bal_read(path):
    """(cameras (nc, 9), points (np, 3), observations (n, 2), cam_idx (n,), pt_idx (n,)) of a BAL text file.

    Paths ending in .bz2, .gz or .xz (the BAL datasets are distributed
    bz2-compressed) are decompressed to a temporary file first; the parsing is
    always the C reader's."""
    codec = _codec(path)
    if codec is None:
        return _bal_read_text(path)
    import shutil
    import tempfile

    fd, tmp = tempfile.mkstemp(suffix=".txt")
    try:
        with os.fdopen(fd, "wb") as out, codec.open(os.fspath(path), "rb") as src:
            shutil.copyfileobj(src, out, 1 << 20)
        return _bal_read_text(tmp)
    finally:
        os.unlink(tmp)


def _bal_read_text(path):
    lib = load()
    bpath = os.fsencode(path)
    nc, np_, n = C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib.mba_bal_read(bpath, C.byref(nc), C.byref(np_), C.byref(n), None, None, None, None, None))
    cams, pts = np.zeros((nc.value, 9)), np.zeros((np_.value, 3))
    obs = np.zeros((n.value, 2))
    ci, pi = np.zeros(n.value, np.int32), np.zeros(n.value, np.int32)
    _check(lib.mba_bal_read(bpath, C.byref(nc), C.byref(np_), C.byref(n), _vp(cams), _vp(pts), _vp(obs), _vp(ci),
                            _vp(pi)))
    return cams, pts, obs, ci, pi


def mba_bal_write(path, cameras, points, observations, cam_idx, pt_idx):
    """Write a BAL text file (every double to 17 significant digits: it reads back bit for bit).

    Paths ending in .bz2, .gz or .xz are written through that compressor."""
    codec = _codec(path)
    if codec is not None:
        import shutil
        import tempfile

        fd, tmp = tempfile.mkstemp(suffix=".txt")
        os.close(fd)
        try:
            mba_bal_write(tmp, cameras, points, observations, cam_idx, pt_idx)
            with open(tmp, "rb") as src, codec.open(os.fspath(path), "wb") as out:
                shutil.copyfileobj(src, out, 1 << 20)
        finally:
            os.unlink(tmp)
        return
    cams = np.ascontiguousarray(cameras, dtype=np.float64).reshape(-1, 9)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    obs = np.ascontiguousarray(observations, dtype=np.float64).reshape(-1, 2)
    ci, pi = np.ascontiguousarray(cam_idx, dtype=np.int32), np.ascontiguousarray(pt_idx, dtype=np.int32)
    if len(ci) != len(obs) or len(pi) != len(obs):
        raise ValueError("cam_idx and pt_idx must have one entry per observation")
    _check(load().mba_bal_write(os.fsencode(path), len(cams), len(pts), len(obs), _vp(cams), _vp(pts), _vp(obs),
                                _vp(ci), _vp(pi)))


class Graph:
    """Graph-style declaration of a BA problem, after the g2o / Ceres convention
    the paper's API follows (Sec. 5.3): camera and point nodes, observation
    edges (the BAL reprojection edge), then one solver call.  Node ids are the
    return values of add_camera / add_point; the graph turns into the flat
    arrays of mba_problem_create."""

    def __init__(self):
        self._cams, self._pts, self._obs, self._ci, self._pi = [], [], [], [], []
        self._cfix, self._pfix = [], []

    def add_camera(self, params, fixed: bool = False) -> int:
        """9 parameters: angle-axis w (3), t (3), f, k1, k2; fixed=True holds the camera constant."""
        p = np.asarray(params, dtype=np.float64).reshape(9)
        self._cams.append(p)
        self._cfix.append(bool(fixed))
        return len(self._cams) - 1

    def add_point(self, xyz, fixed: bool = False) -> int:
        """3-D point; fixed=True holds it constant."""
        self._pts.append(np.asarray(xyz, dtype=np.float64).reshape(3))
        self._pfix.append(bool(fixed))
        return len(self._pts) - 1

    def fixed_masks(self):
        """(camera mask, point mask) of the nodes declared fixed."""
        return np.array(self._cfix, dtype=bool), np.array(self._pfix, dtype=bool)

    def add_edge(self, camera: int, point: int, uv) -> int:
        """Observation uv of point `point` in camera `camera` (residual pi(c, X) - uv)."""
        if not (0 <= camera < len(self._cams)) or not (0 <= point < len(self._pts)):
            raise IndexError("add the camera and point nodes before the edge")
        self._obs.append(np.asarray(uv, dtype=np.float64).reshape(2))
        self._ci.append(camera)
        self._pi.append(point)
        return len(self._obs) - 1

    def arrays(self):
        """(cameras, points, observations, cam_idx, pt_idx) in node and edge order."""
        return (np.array(self._cams).reshape(-1, 9), np.array(self._pts).reshape(-1, 3),
                np.array(self._obs).reshape(-1, 2), np.array(self._ci, np.int32), np.array(self._pi, np.int32))

    def problem(self, **opts) -> "Problem":
        """A device problem (mba_problem_create) of this graph, with its fixed
        nodes marked (mba_set_fixed); opts as Problem's."""
        pr = Problem(*self.arrays(), **opts)
        cf, pf = self.fixed_masks()
        if cf.any() or pf.any():
            pr.set_fixed(cf, pf)
        return pr

    @classmethod
    def from_bal(cls, path) -> "Graph":
        g = cls()
        cams, pts, obs, ci, pi = mba_bal_read(path)
        g._cams, g._pts, g._obs = list(cams), list(pts), list(obs)
        g._ci, g._pi = [int(i) for i in ci], [int(i) for i in pi]
        g._cfix, g._pfix = [False] * len(g._cams), [False] * len(g._pts)
        return g

    def to_bal(self, path):
        mba_bal_write(path, *self.arrays())


def concat_windows(windows):
    """Offsets and concatenated arrays of a list of (cameras, points, observations, cam_idx, pt_idx)."""
    co, po, oo = [0], [0], [0]
    for c, p, o, _, _ in windows:
        co.append(co[-1] + len(c))
        po.append(po[-1] + len(p))
        oo.append(oo[-1] + len(o))
    cat = lambda i, dt: np.concatenate([np.asarray(w[i], dtype=dt) for w in windows])  # noqa: E731
    return (np.array(co, np.int64), np.array(po, np.int64), np.array(oo, np.int64), cat(0, np.float64).reshape(-1, 9),
            cat(1, np.float64).reshape(-1, 3), cat(2, np.float64).reshape(-1, 2), cat(3, np.int32), cat(4, np.int32))


class Batch:
    """Owning wrapper over one mba_batch handle (windows given as a list of
    (cameras, points, observations, cam_idx, pt_idx) with window-local indices)."""

    def __init__(self, windows, precision="fp32", loss="none", huber_delta=0.0, stream=None):
        self.offsets = concat_windows(windows)[:3]
        self.handle = mba_batch_create(*concat_windows(windows), precision=precision, loss=loss,
                                       huber_delta=huber_delta, stream=stream)
        self.info = mba_batch_info(self.handle)

    def close(self):
        if self.handle:
            mba_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, grad_cameras=None, grad_points=None, **opts):
        return mba_batch_solve(self.handle, grad_cameras, grad_points, **opts)

    def autotune(self, **opts):
        return mba_batch_autotune(self.handle, **opts)

    def set_schedule(self, threads_per_cta=0, ctas_per_sm=0, schur="auto"):
        mba_batch_set_schedule(self.handle, threads_per_cta, ctas_per_sm, schur)

    def schedule(self):
        return mba_batch_get_schedule(self.handle)

    def parameters(self):
        return mba_batch_get_parameters(self.handle)

    def window_parameters(self, w):
        cams, pts = self.parameters()
        co, po, _ = self.offsets
        return cams[co[w]:co[w + 1]], pts[po[w]:po[w + 1]]

    def set_parameters(self, cameras=None, points=None):
        mba_batch_set_parameters(self.handle, cameras, points)

    def reset(self):
        mba_batch_reset(self.handle)

    def gradients(self):
        return mba_batch_get_gradients(self.handle)

    def window_times(self):
        return mba_batch_window_times(self.handle)
