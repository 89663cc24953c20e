"""sf_fit_positions (endpoint-pinned least-squares coefficients) against the oracle's
numpy restatement: instances of different robot counts and horizons, including the
square case H = n_xi and a long horizon."""
import numpy as np
import pytest

import oracle
from paper_2510_09204_b300.sf import fit_positions

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nd,nxi", [(2, 11), (3, 7)])
def test_fit_matches_oracle(nd, nxi):
    rng = np.random.default_rng(nd * 10 + nxi)
    shapes = [(4, 50), (1, nxi), (9, 100), (3, 777), (2, 50)]
    pos = [rng.normal(size=(nd, n, H)) * 3.0 for n, H in shapes]
    got = fit_positions(pos, nxi)
    for g, p in zip(got, pos):
        ref = oracle.fit_positions(p, nxi)
        W = oracle.basis(p.shape[2], nxi)
        # the library solves the normal equations (condition number squared); numpy's
        # least squares does not: coefficients agree to rounding at kappa^2
        kappa = np.linalg.cond(W[:, 1:-1])
        tol = max(1e-10, 1e-15 * kappa ** 2)
        assert np.abs(g - ref).max() <= tol * max(1.0, np.abs(ref).max()), (p.shape, kappa)
        assert np.array_equal(g[..., 0], p[..., 0]) and np.array_equal(g[..., -1], p[..., -1])
        f = lambda x: ((np.einsum("kc,dic->dik", W, x) - p) ** 2).sum()
        assert f(g) <= f(ref) * (1 + 1e-9) + 1e-12 * (p ** 2).sum()   # as good a fit as the oracle's


def test_fit_rejects_short_horizons():
    from paper_2510_09204_b300 import SFError
    with pytest.raises(SFError):
        fit_positions([np.zeros((2, 3, 5))], 11)
