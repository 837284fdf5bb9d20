"""The sketched least-squares step (Algorithm 2) through tk_sketched_ls, on both of its kernels:
reflectors applied in compact WY form (k <= 256 columns) and one at a time beyond.  Checked
against numpy's least squares, including an ill-conditioned M, where an unstable reduction
(normal equations: error ~ cond^2 eps) would fail and Householder's ~ cond eps passes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


def _solve(P, M, b):
    import torch
    y, res = P.tk_sketched_ls(P.to_fortran(M, "cuda"), P.to_fortran(b, "cuda"))
    torch.cuda.synchronize()
    return y.cpu().numpy(), res.item()


@pytest.mark.parametrize("s,k", [(96, 1), (128, 60), (300, 97), (1024, 256), (600, 300), (1024, 700)])
def test_sketched_ls_matches_numpy(P, s, k):
    """Gaussian M (well conditioned): y and the residual norm to rounding level; (600, 300) and
    (1024, 700) take the one-reflector-at-a-time kernel, the rest the compact WY kernel."""
    rng = np.random.default_rng(s * 1000 + k)
    M = rng.standard_normal((s, k))
    b = rng.standard_normal(s)
    y, res = _solve(P, M, b)
    yr, *_ = np.linalg.lstsq(M, b, rcond=None)
    assert np.linalg.norm(y - yr) <= 1e-11 * np.linalg.norm(yr)
    assert np.isclose(res, np.linalg.norm(M @ yr - b), rtol=1e-11)


def test_sketched_ls_ill_conditioned(P):
    """Consistent system b = M x0 with M = U diag(sigma) V^T, sigma from 1 to 1e-10 (cond 1e10):
    a backward-stable reduction recovers x0 to ~cond eps (the cond^2 term of least-squares
    sensitivity is multiplied by the zero residual), normal equations to ~cond^2 eps, i.e. not
    at all.  Bound: 100 cond eps."""
    rng = np.random.default_rng(7)
    s, k = 200, 60
    U, _ = np.linalg.qr(rng.standard_normal((s, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    sig = np.logspace(0, -10, k)
    M = (U * sig) @ V.T
    x0 = rng.standard_normal(k)
    b = M @ x0
    y, res = _solve(P, M, b)
    assert res <= 1e-13 * np.linalg.norm(b)
    assert np.linalg.norm(y - x0) <= 100 * 1e10 * 2.2e-16 * np.linalg.norm(x0)
