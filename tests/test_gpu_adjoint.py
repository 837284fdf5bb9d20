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


# ------------------------------------------------------------------------------ full size
def _blur_eig_inverse(n, lam, sigma=2.0):
    """A = G x G x G + lam I with G the symmetric Gaussian Toeplitz blur: G = Q diag(g) Q^T, so
    A^{-1} is diagonal in Q (x) Q (x) Q.  Returns a function applying A^{-1} to a dense tensor
    and ||A^{-1}||_2 = 1 / min |g_i g_j g_k + lam|."""
    g, q = np.linalg.eigh(W.gaussian_blur_dense(n, sigma))
    den = g[:, None, None] * g[None, :, None] * g[None, None, :] + lam

    def solve(t):
        return OT.multi_ttm(OT.multi_ttm(t, [q.T] * 3) / den, [q] * 3)
    return solve, 1.0 / np.min(np.abs(den))


def _unit_weight(n):
    return W.Tucker(np.ones((1, 1, 1)), [np.ones((n, 1)) / np.sqrt(n)] * 3)


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_adjoint_closed_form_deblur_n128(P, form):
    """The deblurring workload at full size (n = 128, G Gaussian blur sigma = 2, lam = 1e-2,
    b = A x_true with x_true of rank (6,6,6); rank cap 32, s = 256) and the quantity of interest
    l = <w, x>, w the smooth rank-1 tensor (1/sqrt(n))^(x)3.  Exact: mu* = A^{-T} w through G's
    eigenbasis (A^{-1} is diagonal in Q (x) Q (x) Q), dl/db = mu*, dl/dlam = -<mu*, x> at the
    computed x, dl/dG_b = mu* x_k U_bk^T.  The GPU's mu from the transposed solve differs from
    mu* by A^{-T} (A^T mu - w), so |<mu - mu*, v>| <= ||v|| ||A^{-1}|| ||A^T mu - w|| for any v,
    with the adjoint residual measured in Tucker form: every gradient is checked against its
    closed form within that bound, and the bound itself must be small (adjoint residual < 1e-6)."""
    n, lam = 128, 1e-2
    wl = W.workload("deblur3d_n128")
    prm = W.SolverParams('rhosvd', 32, 256, 5, 60, 1e-7, seed=0)
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    wq = _unit_weight(n)
    x, _ = P.tk_solve(dop, b, P.Options.from_params(prm, precision=form))
    mu, rep_t = P.tk_solve(dop, to_dev(wq), P.Options.from_params(prm, precision=form, transpose=True))
    r_mu = P.tk_residual(dop, mu, to_dev(wq), transpose=True)          # ||A^T mu - w|| / ||w||, ||w|| = 1
    assert r_mu < 1e-6
    dth, dG, _ = P.tk_adjoint_grads(dop, mu, x, b)
    ainv, ainv_norm = _blur_eig_inverse(n, lam)
    mu_star = ainv(OT.full(wq))
    err_bound = ainv_norm * r_mu                                        # >= ||mu - mu*||
    mu_d = OT.full(to_host(mu))
    assert np.linalg.norm(mu_d - mu_star) <= err_bound * (1 + 1e-6) + 1e-12 * np.linalg.norm(mu_star)
    xd = OT.full(to_host(x))
    dlam_star = -np.sum(mu_star * xd)
    assert abs(dth[1] - dlam_star) <= np.linalg.norm(xd) * err_bound * (1 + 1e-6) + 1e-12 * abs(dlam_star)
    dG_star = OT.multi_ttm(mu_star, [u.T for u in wl.b.factors])
    fac_norm = np.prod([np.linalg.norm(u, 2) for u in wl.b.factors])
    assert np.linalg.norm(dG.cpu().numpy() - dG_star) <= fac_norm * err_bound * (1 + 1e-6) + 1e-12 * np.linalg.norm(dG_star)


def test_adjoint_central_differences_n128(P):
    """Full size n = 128 with a well-conditioned blur system (lam = 1, rank cap 48, where the
    forward solve reaches a relative residual near 1e-8): the adjoint gradient of l = <w, x> along
    a core direction delta of b, <mu, [delta; U_b]> = <dl/dG_b, delta>, against central
    differences of the GPU forward solve (common random numbers), and the mixed form's gradient
    against the FP64 one.  l is linear in b, so the exact central difference equals the exact
    gradient at any step h; the computed ones differ only through the solves' errors, each at most
    ||A^-1|| times its residual:
        |grad - fd| <= ||w|| ||A^-1|| (|r+| + |r-|) / (2h) + ||delta_b|| ||A^-T|| |r_mu|,
    with |r| the true residual norms (A symmetric here: ||A^-T|| = ||A^-1||)."""
    n = 128
    lam = 1.0
    wl = W.deblur3d(n, 0, None, lam=lam)
    prm = W.SolverParams('rhosvd', 48, 128, 5, 30, 1e-13, seed=0)
    dop = P.DeviceOperator(wl.op)
    wq_np = _unit_weight(n)
    wq = to_dev(wq_np)
    rng = np.random.default_rng(41)
    delta = rng.standard_normal(wl.b.core.shape)
    delta *= np.linalg.norm(wl.b.core) / np.linalg.norm(delta)
    _, ainv_norm = _blur_eig_inverse(n, lam)

    def qoi(core):
        """l(b) and the absolute true residual norm of its forward solve"""
        bt = W.Tucker(core, wl.b.factors)
        bd = to_dev(bt)
        x, _ = P.tk_solve(dop, bd, P.Options.from_params(prm))
        return P.tk_inner(wq, x), P.tk_residual(dop, x, bd) * np.linalg.norm(OT.full(bt))

    grads = {}
    rmu = {}
    for form in ["fp64", "mixed"]:
        x, _ = P.tk_solve(dop, to_dev(wl.b), P.Options.from_params(prm, precision=form))
        mu, _ = P.tk_solve(dop, wq, P.Options.from_params(prm, precision=form, transpose=True))
        rmu[form] = P.tk_residual(dop, mu, wq, transpose=True) * np.linalg.norm(OT.full(wq_np))
        _, dG, _ = P.tk_adjoint_grads(dop, mu, x, to_dev(wl.b))
        grads[form] = float(np.sum(dG.cpu().numpy() * delta))
    # a large step keeps the forward solves' ~1e-8 errors from being divided by a small one
    h = 0.5
    lp, rp = qoi(wl.b.core + h * delta)
    lm, rm = qoi(wl.b.core - h * delta)
    fd = (lp - lm) / (2 * h)
    w_norm = np.linalg.norm(OT.full(wq_np))
    d_norm = np.linalg.norm(OT.full(W.Tucker(delta, wl.b.factors)))
    bound = w_norm * ainv_norm * (rp + rm) / (2 * h) + d_norm * ainv_norm * rmu["fp64"]
    assert abs(grads["fp64"] - fd) <= bound
    # the bound is not vacuous: it resolves the directional derivative to 0.2% of its size (a wrong
    # contraction or sign would miss by O(1))
    assert bound <= 2e-3 * abs(grads["fp64"])
    scale = abs(qoi(wl.b.core)[0])
    assert abs(grads["mixed"] - grads["fp64"]) <= 1e-6 * scale
