"""Gradients through the solve (adjoint system + adjoint contractions) on the GPU.

Checked against (i) exact gradients from dense LU solves (oracle/adjoint.py) at settings without
truncation, (ii) central finite differences of the GPU forward solve with common random numbers,
(iii) the FP64 oracle's own Tucker-form adjoint at a truncating setting."""
from functools import reduce

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as OA
from oracle import sgmres as OS
from oracle import tensor as OT
from tests.helpers import rel_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


def _dense_param_grads(mu, b):
    dG = OT.multi_ttm(mu, [u.T for u in b.factors])
    dU = []
    for k in range(b.d):
        kr = reduce(np.kron, [b.factors[j] for j in reversed(range(b.d)) if j != k])
        dU.append(OT.unfold(mu, k) @ kr @ OT.unfold(b.core, k).T)
    return dG, dU


def _small_problem(n=5, lam=0.5):
    wl = W.deblur3d(n, 3, None, lam=lam)
    xt = W.random_tucker([n] * 3, [2, 2, 2], 31)
    prm = W.SolverParams('rhosvd', n, 100, 5, 90, 1e-13, ktrunc=3, round_tol=1e-15, seed=2)
    return wl, xt, prm


def test_adjoint_matches_dense_gradients(P):
    wl, xt, prm = _small_problem()
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    opts = P.Options.from_params(prm)
    x, rep = P.tk_solve(dop, b, opts)
    g = P.autograd.tucker_difference(x, to_dev(xt))
    mu, rep_t = P.tk_solve(dop, g, P.Options.from_params(prm, transpose=True))
    dth, dG, dU = P.tk_adjoint_grads(dop, mu, x, b)
    _, mu_d, dth_d = OA.dense_gradients(wl.op, wl.b, OT.full(xt))
    assert np.allclose(dth, dth_d, rtol=1e-8, atol=1e-12)
    dG_d, dU_d = _dense_param_grads(mu_d, wl.b)
    assert np.allclose(dG.cpu().numpy(), dG_d, atol=1e-9 * np.abs(dG_d).max())
    for k in range(3):
        assert np.allclose(dU[k].cpu().numpy(), dU_d[k], atol=1e-9 * np.abs(dU_d[k]).max())


def test_autograd_function_gradients(P):
    import torch
    wl, xt, prm = _small_problem()
    dop = P.DeviceOperator(wl.op)
    b = to_dev(wl.b)
    theta = torch.tensor(wl.op.theta, dtype=torch.float64, requires_grad=True)
    core = b.core.clone().requires_grad_(True)
    facs = [u.clone().requires_grad_(True) for u in b.factors]
    loss = P.autograd.tucker_solve_mse(dop, theta, core, facs, to_dev(xt), P.Options.from_params(prm))
    loss.backward()
    xd, mu_d, dth_d = OA.dense_gradients(wl.op, wl.b, OT.full(xt))
    assert np.isclose(loss.item(), 0.5 * np.sum((xd - OT.full(xt)) ** 2), rtol=1e-9)
    assert np.allclose(theta.grad.numpy(), dth_d, rtol=1e-8, atol=1e-12)
    dG_d, dU_d = _dense_param_grads(mu_d, wl.b)
    assert np.allclose(core.grad.cpu().numpy(), dG_d, atol=1e-9 * np.abs(dG_d).max())
    for k in range(3):
        assert np.allclose(facs[k].grad.cpu().numpy(), dU_d[k], atol=1e-9 * np.abs(dU_d[k]).max())


def test_adjoint_against_finite_differences(P):
    wl, xt, prm = _small_problem(n=6, lam=0.3)
    dop, b, xr = P.DeviceOperator(wl.op), to_dev(wl.b), to_dev(xt)
    opts = P.Options.from_params(prm)

    def loss(theta):
        dop.set_theta(theta)
        x, _ = P.tk_solve(dop, b, opts)
        return 0.5 * P.tk_sum_norm([x, xr], [1.0, -1.0]) ** 2

    th0 = list(wl.op.theta)
    dop.set_theta(th0)
    x, _ = P.tk_solve(dop, b, opts)
    mu, _ = P.tk_solve(dop, P.autograd.tucker_difference(x, xr), P.Options.from_params(prm, transpose=True))
    dth, _, _ = P.tk_adjoint_grads(dop, mu, x, b)
    for t in range(len(th0)):
        h = 1e-6 * max(1.0, abs(th0[t]))
        tp, tm = list(th0), list(th0)
        tp[t] += h
        tm[t] -= h
        fd = (loss(tp) - loss(tm)) / (2 * h)
        assert np.isclose(dth[t], fd, rtol=1e-5, atol=1e-9)


def test_adjoint_parity_with_oracle_truncating(P):
    """Truncating setting (rank cap below n): GPU forward + adjoint + contractions against the
    oracle's Tucker-form computation with the same streams."""
    n = 24
    wl = W.deblur3d(n, 4, None, lam=0.2)
    xt = W.random_tucker([n] * 3, [3, 3, 3], 32)
    prm = W.SolverParams('rhosvd', 10, 64, 5, 8, 1e-10, seed=5)
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    x, _ = P.tk_solve(dop, b, P.Options.from_params(prm))
    mu, _ = P.tk_solve(dop, P.autograd.tucker_difference(x, to_dev(xt)), P.Options.from_params(prm, transpose=True))
    dth, dG, dU = P.tk_adjoint_grads(dop, mu, x, b)
    fx = OS.rhosvd_sgmres(wl.op, wl.b, prm).x
    fmu = OS.rhosvd_sgmres(wl.op, OT.concat_sum([(1.0, fx), (-1.0, xt)]), prm, transpose=True).x
    assert rel_diff(to_host(x), fx) <= 1e-10 and rel_diff(to_host(mu), fmu) <= 1e-9
    ref_th = OA.theta_gradients(wl.op, fx, fmu)
    assert np.allclose(dth, ref_th, rtol=1e-8)
    ref_G = OA.core_gradient(fmu, wl.b)
    assert np.allclose(dG.cpu().numpy(), ref_G, atol=1e-8 * np.abs(ref_G).max())
    ref_U = OA.factor_gradients(fmu, wl.b)
    for k in range(3):
        assert np.allclose(dU[k].cpu().numpy(), ref_U[k], atol=1e-8 * np.abs(ref_U[k]).max())


def test_sum_norm_is_accurate_for_small_differences(P):
    x = W.random_tucker([30, 31, 32], [4, 5, 3], 33)
    y = W.Tucker(x.core * (1 + 1e-9), x.factors)
    v = P.tk_sum_norm([to_dev(x), to_dev(y)], [1.0, -1.0])
    assert np.isclose(v, 1e-9 * OT.norm(x), rtol=1e-5)
