"""Writes oracle_tiny_lm.txt: the oracle's LM trajectory on the tiny workload
(16 cameras, 2,000 points, 5 observations per point, 10 LM iterations, PCG up
to 50, seed 0).  Calls only the oracle and the seeded scene generator; run it
again, and commit the result with the reason, only when the oracle's
arithmetic changes on purpose.

    python tests/golden/make_oracle_fixtures.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from scenes import config_scene  # noqa: E402

FIELDS = ("cost", "cost_new", "model_dec", "mu", "gain", "accepted", "pcg_iters", "pcg_rel_res")


def tiny_lm():
    sc = config_scene(1)
    c = sc.meta
    return oracle.lm_solve(sc.cameras, sc.points, sc.observations, sc.cam_idx, sc.pt_idx, max_iter=c["lm_iters"],
                           pcg_max=c["pcg_max"], pcg_tol=c["pcg_tol"])


def main():
    r = tiny_lm()
    path = os.path.join(HERE, "oracle_tiny_lm.txt")
    with open(path, "w") as f:
        f.write("# oracle LM trajectory, tiny workload (16 cameras, 2,000 points, 10,000 observations,\n")
        f.write("# seed 0, 10 LM iterations, PCG <= 50, rel tol 1e-10); written by make_oracle_fixtures.py\n")
        f.write("# " + " ".join(FIELDS) + "\n")
        for t in r["trace"]:
            f.write(" ".join(repr(float(t[k])) if isinstance(t[k], float) else str(t[k]) for k in FIELDS) + "\n")
        f.write(f"final_cost {r['final_cost']!r}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
