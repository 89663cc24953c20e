"""Writes the stored expected values under tests/golden/ by calling only the oracle (and the
seeded input generator for its inputs).  Run from the repository root:

    python tests/golden/make_golden.py

The paper prints no worked example of the SF iteration, so these fixtures are the oracle's
own results on fixed seeded inputs: they pin the CUDA path to the oracle on a case that
never changes, and they flag any later change to the oracle's arithmetic (which must then
name, in its commit message, the passage of the paper that justifies it).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sfgen  # noqa: E402

RHO = 0.3
CASES = [
    # name, config, instance index, iterations, cost
    ("cfg1_projection_100it", 1, 0, 100, "projection"),
    ("cfg1_smoothness_60it", 1, 0, 60, "smoothness"),
]


def write(path, name, cid, idx, iters, cost):
    inst = sfgen.make_batch(cid, B=idx + 1)[idx]
    out = oracle.solve(inst, iters, rho=RHO, cost=cost, hist=True)
    res = oracle.residual(inst, out["xi"])
    with open(path, "w") as f:
        f.write("# %s: the oracle's SF iteration (Sec. IV-B, steps alpha .. xi_bar; Appendix closed forms)\n" % name)
        f.write("# input: sfgen config %d, instance %d (seed %d); rho %g; %d iterations; cost %s (dt %g s);"
                " xi0 = xi_cand, lambda0 = 0\n" % (cid, idx, 1000 * cid + idx, RHO, iters, cost, oracle.DEFAULT_DT))
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        f.write("shape %d %d %d\n" % out["xi"].shape)
        f.write("xi %s\n" % " ".join(repr(float(v)) for v in out["xi"].ravel()))
        f.write("lam %s\n" % " ".join(repr(float(v)) for v in out["lam"].ravel()))
        f.write("residual %s\n" % " ".join(repr(float(v)) for v in res[:3]))
        f.write("hist_max %s\n" % " ".join(repr(float(v)) for v in out["hist"][:, 1]))


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for name, cid, idx, iters, cost in CASES:
        write(os.path.join(here, name + ".txt"), name, cid, idx, iters, cost)
        print("wrote", name)


if __name__ == "__main__":
    main()
