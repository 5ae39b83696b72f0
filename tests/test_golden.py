"""Stored fixtures under tests/golden/.

- paper_bal_dataset_statistics.txt: the paper's BAL dataset statistics (Sec. 6).
  The synthetic workloads that stand in for Venice-1778 and Final-13682 must
  have the shape of those problems: cameras within 5 %, points within 1 %,
  observations per point (the mean track length) within 1 %, every point seen
  by at least two cameras, and the expected observation count within 2 %.
- oracle_tiny_lm.txt: the oracle's LM trajectory on the tiny workload, written
  by make_oracle_fixtures.py (which calls only the oracle).  The oracle must
  keep reproducing it: a change to the oracle's arithmetic shows up here and
  has to be made on purpose, with the fixture rewritten by that script.
  Iterations whose model decrease is at the rounding floor (below 1e-10 of the
  cost) are compared by cost only, since their accept decisions follow the
  last bits of the arithmetic."""
import os

import numpy as np
import pytest

import oracle
from scenes.generate import CONFIGS, _track_lengths

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _paper_table():
    rows = {}
    with open(os.path.join(HERE, "paper_bal_dataset_statistics.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, nc, npts, nobs = line.split()
                rows[name] = (int(nc), int(npts), int(nobs))
    return rows


def test_paper_table_is_consistent():
    rows = _paper_table()
    assert len(rows) == 5
    for name, (nc, npts, nobs) in rows.items():
        assert name.endswith(f"-{nc}")
        assert 2 * npts <= nobs <= 300 * npts  # every BAL point is seen at least twice


@pytest.mark.parametrize("cfg,dataset", [(2, "Venice-1778"), (3, "Final-13682")])
def test_workload_has_the_shape_of_the_paper_dataset(cfg, dataset):
    nc, npts, nobs = _paper_table()[dataset]
    c = CONFIGS[cfg]
    assert abs(c["nc"] / nc - 1) <= 0.05
    assert abs(c["np"] / npts - 1) <= 0.01
    rng = np.random.default_rng(12345)
    L = _track_lengths(rng, 400_000, c["nc"], c["track"])  # a sample of the workload's track lengths
    assert L.min() >= 2
    assert abs(L.mean() / (nobs / npts) - 1) <= 0.01
    assert abs(c["np"] * L.mean() / nobs - 1) <= 0.02


def _fixture():
    rows, final = [], None
    with open(os.path.join(HERE, "oracle_tiny_lm.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            v = line.split()
            if v[0] == "final_cost":
                final = float(v[1])
            else:
                rows.append(dict(cost=float(v[0]), cost_new=float(v[1]), model_dec=float(v[2]), mu=float(v[3]),
                                 accepted=int(v[5]), pcg_iters=int(v[6]), pcg_rel_res=float(v[7])))
    return rows, final


def test_oracle_reproduces_its_stored_trajectory():
    from tests.golden.make_oracle_fixtures import tiny_lm

    rows, final = _fixture()
    got = tiny_lm()
    assert got["iterations"] == len(rows) == 10
    assert got["final_cost"] == pytest.approx(final, rel=1e-12)
    for t, r in zip(got["trace"], rows):
        assert t["cost"] == pytest.approx(r["cost"], rel=1e-12)
        assert t["cost_new"] == pytest.approx(r["cost_new"], rel=1e-12)
        if r["model_dec"] > 1e-10 * r["cost"]:
            assert t["accepted"] == r["accepted"]
            assert t["mu"] == pytest.approx(r["mu"], rel=1e-12)
            assert t["pcg_iters"] == r["pcg_iters"]
            assert t["model_dec"] == pytest.approx(r["model_dec"], rel=1e-8)
            assert t["pcg_rel_res"] == pytest.approx(r["pcg_rel_res"], rel=1e-4)
