"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py from the
oracle alone): the oracle must keep reproducing them, and the CUDA path must match them.
The paper prints no worked example of the iteration, so these are fixed-input regression
pins of the oracle, not independent pins (those are in test_oracle_pins.py)."""
import os

import numpy as np
import pytest

import oracle
import sfgen

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RHO = 0.3
CASES = [("cfg1_projection_100it", 1, 0, 100, "projection"), ("cfg1_smoothness_60it", 1, 0, 60, "smoothness")]


def load(name):
    out = {}
    with open(os.path.join(HERE, name + ".txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out[key] = np.array([float(v) for v in vals])
    shape = tuple(int(v) for v in out.pop("shape"))
    out["xi"] = out["xi"].reshape(shape)
    out["lam"] = out["lam"].reshape(shape)
    return out


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("name,cid,idx,iters,cost", CASES)
def test_oracle_reproduces_stored_values(name, cid, idx, iters, cost):
    g = load(name)
    inst = sfgen.make_batch(cid, B=idx + 1)[idx]
    out = oracle.solve(inst, iters, rho=RHO, cost=cost, hist=True)
    assert rel(out["xi"], g["xi"]) <= 1e-12
    assert rel(out["lam"], g["lam"]) <= 1e-12
    np.testing.assert_allclose(out["hist"][:, 1], g["hist_max"], rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(oracle.residual(inst, out["xi"])[:3], g["residual"], rtol=1e-10, atol=1e-13)
    # the fixture is a solve that moved the candidate and met the boundary equalities
    assert rel(g["xi"], inst["xi"]) > 1e-3
    np.testing.assert_allclose(g["xi"][:, :, 0], inst["bnd"][:, :, 0], atol=1e-12)
    np.testing.assert_allclose(g["xi"][:, :, -1], inst["bnd"][:, :, 1], atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("proj", ["dense", "structured"])
@pytest.mark.parametrize("name,cid,idx,iters,cost", CASES)
def test_cuda_path_matches_stored_values(name, cid, idx, iters, cost, proj):
    import torch
    from paper_2510_09204_b300 import SFSolver
    g = load(name)
    inst = sfgen.make_batch(cid, B=idx + 1)[idx]
    s = SFSolver([inst], inst["n_d"], inst["n_xi"], rho=RHO, precision="fp64", proj=proj, max_iters=iters,
                 cost=cost, dt=oracle.DEFAULT_DT)
    data = s.pack([inst])
    xo, lo, res = s.solve(data, data["xi"], iters)
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    assert rel(s.unpack(xo, 0).cpu().numpy(), g["xi"]) <= 1e-10
    assert rel(s.unpack(lo, 0).cpu().numpy(), g["lam"]) <= 1e-10
    np.testing.assert_allclose(res.cpu().numpy()[0, :2], g["residual"][:2], rtol=1e-9, atol=1e-12)
    s.close()
