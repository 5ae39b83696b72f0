"""A user edge type compiled into the library (the g2o / Ceres-style edge of the
paper's graph API, Sec. 5.3, evaluated on the dual-number path of Sec. 3.2).

The library is built a second time with tests/user_edges/offset_bal_edge.cuh:
the BAL camera plus a principal point (cx, cy).  Solving a scene with that edge
and observations shifted by (cx, cy) is the BAL problem with the unshifted
observations, so the oracle pins it.  The user-edge library runs in a child
process (this process keeps the default library loaded)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from scenes import make_scene

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(HERE, "user_edges", "offset_bal_edge.cuh")
CX, CY = 320.0, 240.0

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2112_01349_gb300 import mba
from scenes import make_scene
mba.load({lib!r})
out = {{"edge": mba.mba_edge_name()}}
sc = make_scene(12, 600, sigma=0.5, seed=91)
obs = sc.observations + np.array([{cx}, {cy}])
args = (sc.cameras, sc.points, obs, sc.cam_idx, sc.pt_idx)
try:
    mba.Problem(*args)
    out["analytic_rejected"] = False
except mba.MbaError as e:
    out["analytic_rejected"] = e.status == mba.MBA_ERR_INVALID_ARG
try:
    mba.Batch([args])
    out["batch_rejected"] = False
except mba.MbaError as e:
    out["batch_rejected"] = e.status == mba.MBA_ERR_INVALID_ARG
for prec in ("fp64", "fp32"):
    with mba.Problem(*args, precision=prec, jacobian="autodiff") as pr:
        e0 = pr.evaluate()[0]
        s = pr.solve(trace_capacity=8, max_iter=8, pcg_max_iter=50)
        cams, pts = pr.parameters()
    out[prec] = dict(initial_cost=e0, final_cost=s["final_cost"], accepted=[t["accepted"] for t in s["trace"]],
                     cams=cams.tolist(), pts=pts.tolist())
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def child_result():
    from paper_2112_01349_gb300 import _build

    lib = _build.build(edge=(HEADER, "OffsetBalEdge"))
    code = CHILD.format(root=ROOT, lib=lib, cx=CX, cy=CY)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_user_edge_library_reports_its_edge_and_rejects_bal_only_paths(child_result):
    assert child_result["edge"] == "OffsetBalEdge"
    assert child_result["analytic_rejected"] and child_result["batch_rejected"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_user_edge_solve_matches_the_oracle(child_result, precision, tol):
    sc = make_scene(12, 600, sigma=0.5, seed=91)
    args = (sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx)
    F0 = oracle.evaluate(*args, jacobians=False)[0]
    ref = oracle.lm_solve(*args, max_iter=8, pcg_max=50)
    got = child_result[precision]
    assert got["initial_cost"] == pytest.approx(F0, rel=1e-12 if precision == "fp64" else 1e-5)
    assert got["final_cost"] == pytest.approx(ref["final_cost"], rel=tol)
    if precision == "fp64":
        # decisions once the model decrease reaches the rounding floor may differ
        # (the prediction carries the offset through its rounding)
        assert got["accepted"][:3] == [t["accepted"] for t in ref["trace"]][:3]
        np.testing.assert_allclose(np.array(got["pts"]), ref["points"], rtol=0, atol=1e-5 * np.abs(ref["points"]).max())
