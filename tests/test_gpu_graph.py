"""The whole differentiable solve (forward, FP64 residual check, adjoint) captured in
one CUDA graph.  Replays reproduce the eager calls bit for bit, and new inputs copied
into the captured buffers give the eager results for those inputs."""
import numpy as np
import pytest
import torch

import sfgen
from paper_2510_09204_b300 import SF_NRES, SFSolver
from paper_2510_09204_b300.sf import SF_OPT_TC_BATCH

pytestmark = pytest.mark.gpu
RHO = 0.3
ITERS = 30


def uneven_batch():
    """Six instances of different robot counts, obstacle counts and horizons."""
    spec = [(8, 10, 80), (13, 25, 100), (20, 12, 120), (9, 0, 100), (16, 40, 80), (11, 17, 120)]
    return [sfgen.custom_instance(n=n, n_obs=o, H=H, n_d=2, seed=40 + k, extent=15.0)
            for k, (n, o, H) in enumerate(spec)]


class Step:
    """Preallocated buffers and the call sequence of one differentiable solve."""

    def __init__(self, s, data):
        self.s, self.data = s, data
        x = data["xi"]
        self.xo, self.lo = torch.empty_like(x), torch.empty_like(x)
        self.res = torch.empty((s.B, SF_NRES), dtype=torch.float64, device=x.device)
        g = np.random.default_rng(3).normal(size=x.numel()) * 1e-2
        self.gxo = torch.as_tensor(g, dtype=x.dtype, device=x.device)
        self.grp2 = torch.ones(s.B, dtype=torch.float64, device=x.device)
        self.g = (torch.empty_like(x), torch.empty_like(x), torch.empty_like(x))

    def __call__(self):
        self.s.solve(self.data, self.data["xi"], ITERS, xi_out=self.xo, lam_out=self.lo, resid=self.res)
        self.s.backward(self.gxo, None, self.grp2, out=self.g)

    def outputs(self):
        return [t.clone() for t in (self.xo, self.lo, self.res) + self.g]


@pytest.mark.parametrize("precision,proj,n_refine", [("fp32", "dense", 0), ("fp64", "structured", 0),
                                                     ("bf16x3", "dense", 1), ("bf16x3+batched", "dense", 1)])
def test_graph_replay_matches_eager(precision, proj, n_refine):
    batched = precision.endswith("+batched")
    precision = precision.split("+")[0]
    insts = sfgen.make_batch(2, B=8) if batched else uneven_batch()
    s = SFSolver(insts, 2, 11, rho=RHO, precision=precision, proj=proj, max_iters=ITERS, ckpt_every=10,
                 n_refine=n_refine)
    s.autotune(s.pack(insts), s.pack(insts)["xi"], ITERS, reps=1)
    if batched:
        assert s.option(SF_OPT_TC_BATCH) > 1
    data = s.pack(insts)
    st = Step(s, data)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        st()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = st.outputs()

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st()
    for t in (st.xo, st.lo, st.res) + st.g:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert (s.status() == 0).all()
    for a, b in zip(eager, st.outputs()):
        assert torch.equal(a, b)

    # new candidate contents in the captured input buffer
    rng = np.random.default_rng(5)
    new = [dict(i, xi=i["xi"] + np.pad(rng.normal(0, 0.05, size=i["xi"][..., 1:-1].shape), ((0, 0), (0, 0), (1, 1))))
           for i in insts]
    data["xi"].copy_(s.pack(new)["xi"])
    g.replay()
    torch.cuda.synchronize()
    replayed = st.outputs()
    st()
    torch.cuda.synchronize()
    for a, b in zip(replayed, st.outputs()):
        assert torch.equal(a, b)
    assert not torch.equal(replayed[0], eager[0])
