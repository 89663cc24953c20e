"""Helpers shared by the GPU tests: run the CUDA solver on sfgen instances."""
import numpy as np
import torch

from paper_2510_09204_b300 import SFSolver


def pack_list(solver, arrays):
    flat = np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in arrays])
    return torch.as_tensor(flat, dtype=solver.dtype, device="cuda")


def gpu_solve(insts, iters, precision="fp64", proj="dense", rho=0.3, xi0=None, lam0=None, ckpt_every=0,
              tol=1e-3, max_iters=None, cluster=None, threads=0, n_refine=0):
    s = SFSolver(insts, insts[0]["n_d"], insts[0]["n_xi"], rho=rho, precision=precision, proj=proj,
                 max_iters=max(iters, 1) if max_iters is None else max_iters, ckpt_every=ckpt_every, tol=tol,
                 n_refine=n_refine)
    if cluster is not None:
        s.set_launch(cluster, threads)
    data = s.pack(insts)
    x0 = pack_list(s, xi0) if xi0 is not None else None
    l0 = pack_list(s, lam0) if lam0 is not None else None
    xo, lo, res = s.solve(data, data["xi"], iters, xi0=x0, lam0=l0)
    torch.cuda.synchronize()
    st = s.status()
    xs = [s.unpack(xo, k).double().cpu().numpy() for k in range(len(insts))]
    ls = [s.unpack(lo, k).double().cpu().numpy() for k in range(len(insts))]
    out = dict(xi=xs, lam=ls, resid=res.cpu().numpy(), status=st, solver=s, data=data)
    return out


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def max_pos_err(inst, xa, xb, W):
    return np.abs(np.einsum("kc,dic->dik", W, xa - xb)).max()
