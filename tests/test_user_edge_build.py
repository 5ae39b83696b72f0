"""The build-time user edge plug-in without a GPU: the library builds with a
user edge type (tests/user_edges/offset_bal_edge.cuh), reports it through
mba_edge_name, and refuses analytic-Jacobian problems before it touches the
device; the default library keeps the BAL edge.  The solve with the user edge
is checked against the oracle in tests/test_gpu_user_edge.py."""
import ctypes as C
import os

import numpy as np

from paper_2112_01349_gb300 import _build, mba

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "user_edges", "offset_bal_edge.cuh")


def _lib(path):
    lib = C.CDLL(path)
    lib.mba_edge_name.restype = C.c_char_p
    lib.mba_problem_create.restype = C.c_int
    lib.mba_problem_create.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.mba_problem_options_default.argtypes = [C.c_void_p]
    return lib


def _create(lib, jacobian):
    cams = np.zeros((2, 9))
    cams[:, 6] = 500.0
    pts = np.array([[0.0, 0.0, -5.0]])
    obs = np.zeros((2, 2))
    ci = np.array([0, 1], dtype=np.int32)
    pi = np.array([0, 0], dtype=np.int32)
    o = mba.ProblemOptions()
    lib.mba_problem_options_default(C.byref(o))
    o.jacobian = jacobian
    h = C.c_void_p()
    f = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    return lib.mba_problem_create(f(cams), 2, f(pts), 1, f(obs), f(ci), f(pi), 2, C.byref(o), C.byref(h))


def test_user_edge_library_builds_and_reports_its_edge():
    path = _build.build(edge=(HEADER, "OffsetBalEdge"))
    assert path == _build.edge_lib("OffsetBalEdge") and os.path.exists(path)
    user = _lib(path)
    assert user.mba_edge_name() == b"OffsetBalEdge"
    assert _create(user, mba.JACOBIAN["analytic"]) == mba.MBA_ERR_INVALID_ARG
    default = _lib(_build.build())
    assert default.mba_edge_name() == b"BalEdge"
    # the binding holds one library per process: the default one here, so a
    # request for the user-edge library is refused rather than mixed in
    mba.load()
    assert mba.mba_edge_name() == "BalEdge"
    try:
        mba.load(path)
        raised = False
    except RuntimeError:
        raised = True
    assert raised
