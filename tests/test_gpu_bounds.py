"""The bounds-checked build (libsf_check.so, compiled with SF_BOUNDS_CHECK): every
data-dependent shared-memory index the kernels form (candidate-list entries and their
positions, the carve against the launch's dynamic shared memory) is checked, a violation
is recorded and skipped and the instance reports SF_EBOUNDS.  On the batches below (culled
and full loops, dense and structured projections, tensor cores, uneven shapes, 3-D
anisotropic bodies, moving obstacles, forward and adjoint) no check may fail, and the
results must agree with the unchecked build's tolerance against the oracle.

The library runs in a child process: one process loads one build of the library."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    from paper_2510_09204_b300 import build, sf
    sf.lib(build.build_check())
    import oracle, sfgen
    from paper_2510_09204_b300 import SFSolver
    from paper_2510_09204_b300.sf import SF_OPT_CULL

    def run(insts, precision, proj, iters, cull=1, cluster=None, check=None):
        s = SFSolver(insts, insts[0]["n_d"], insts[0]["n_xi"], rho=0.3, precision=precision, proj=proj,
                     max_iters=iters, ckpt_every=1, n_refine=1 if precision in ("tf32", "bf16x3") else 0)
        if cluster:
            s.set_launch(cluster, 0)
        if not cull:
            s.set_option(SF_OPT_CULL, 0)
        d = s.pack(insts)
        xo, lo, res = s.solve(d, d["xi"], iters)
        s.backward(torch.ones_like(xo) * 1e-2)
        torch.cuda.synchronize()
        st = s.status()
        assert (st == 0).all(), (precision, proj, st)
        if check is not None:
            inst = insts[check]
            ref = oracle.solve(inst, iters, rho=0.3)
            W = oracle.basis(inst["H"], inst["n_xi"])
            got = s.unpack(xo, check).double().cpu().numpy()
            err = np.abs(np.einsum("kc,dic->dik", W, got - ref["xi"])).max()
            assert err <= (1e-8 if precision == "fp64" else 1e-4), (precision, proj, err)
        s.close()

    c2 = sfgen.make_batch(2, B=4)
    crowded = [sfgen.custom_instance(n=12, n_obs=12, H=40, seed=s, extent=5.0, sigma=0.8) for s in range(2)]
    aniso = [sfgen.custom_instance(n=9, n_obs=12, H=50, n_d=3, seed=s, extent=(6.0, 6.0, 2.0)) for s in range(2)]
    for i in aniso:
        i["b"] = 0.7 * i["a"]
    dyn = [sfgen.custom_instance(n=10, n_obs=8, H=60, seed=20 + s, extent=7.0, dyn_obs=True) for s in range(2)]
    uneven = sfgen.make_batch(3, B=6)
    for proj in ("structured", "dense"):
        run(c2, "fp32", proj, 60, check=1)
        run(c2, "fp32", proj, 60, cluster=3)
        run(crowded, "fp32", proj, 40, check=0)
        run(crowded, "fp32", proj, 40, cull=0)
        run(aniso, "fp32", proj, 30)
        run(dyn, "fp64", proj, 30, check=1)
        run(uneven, "fp32", proj, 40)
    run(c2, "tf32", "dense", 40)
    run(aniso, "bf16x3", "dense", 30)
    run(c2, "bf16x3", "dense", 30, cluster=4)   # four instances in one cluster: the batched product
    print("bounds-checked runs: no violation")
""")


def test_bounds_checked_build_reports_no_violation():
    script = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no violation" in r.stdout
