"""The dual-number header and the BAL edge functor, built as plain C++ on the
host: chain-rule identities against hand-derived gradients, and the functor's
forward-mode Jacobian against the oracle's analytic Jacobian (itself pinned
to finite differences and to scipy's rotation in test_oracle_pins.py).  Pass
widths 12, 5, 3 and 1 must give bit-identical Jacobians: each partial is the
same sequence of operations whatever the number of directions per pass."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("jet") / "jet_host_check")
    cmd = [gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wall", "-Wno-unknown-pragmas",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2112_01349_gb300", "csrc"),
           os.path.join(ROOT, "tests", "jet_host_check.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_jet_chain_rule_closed_forms(exe):
    r = subprocess.run([exe, "closed"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "closed ok" in r.stdout


def _cases(rng, m=40):
    """Cameras with large rotations, small rotations (1e-3 rad), an exactly zero
    rotation and a rotation below the first-order threshold (|w|^2 <= eps),
    each with a point in front of it."""
    rows = []
    for i in range(m):
        scale = (1.0, 1e-3, 0.0, 1e-9)[i % 4]
        w = rng.normal(0, 1, 3) * scale
        t = rng.normal(0, 0.3, 3) + np.array([0.0, 0.0, -6.0])
        cam = np.concatenate([w, t, [rng.uniform(500, 1500), rng.normal(0, 0.05), rng.normal(0, 0.05)]])
        X = rng.normal(0, 1.0, 3)
        rows.append((cam, X))
    return rows


def test_bal_functor_jacobian_matches_oracle(exe):
    rng = np.random.default_rng(17)
    cases = _cases(rng)
    text = "\n".join(" ".join(f"{v:.17g}" for v in np.concatenate([c, X])) for c, X in cases) + "\n"
    r = subprocess.run([exe, "bal"], input=text, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    assert len(lines) == len(cases)
    for (cam, X), line in zip(cases, lines):
        v = np.array([float(t) for t in line.split()]).reshape(4, 26)
        # every pass width gives the same bits
        for k in range(1, 4):
            np.testing.assert_array_equal(v[k], v[0])
        pix, Jc, Jp = v[0, :2], v[0, 2:20].reshape(2, 9), v[0, 20:26].reshape(2, 3)
        e, Jc_ref, Jp_ref = oracle.residual_jacobian(cam, X, np.zeros(2))
        np.testing.assert_allclose(pix, e, rtol=1e-13, atol=1e-9)
        scale_c = np.abs(Jc_ref).max()
        np.testing.assert_allclose(Jc, Jc_ref, rtol=1e-10, atol=1e-12 * scale_c)
        np.testing.assert_allclose(Jp, Jp_ref, rtol=1e-10, atol=1e-12 * np.abs(Jp_ref).max())
