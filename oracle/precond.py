"""Exponential-sum approximation of the inverse Laplacian (Section 3.4).  Test infrastructure only.

Delta_d^{-1} ~ sum_{h=-q}^{q} c_h exp(-t_h Delta_1) x ... x exp(-t_h Delta_1) with c_h = eta t_h,
t_h = exp(h eta), eta = pi / sqrt(q).  Reading: the printed exp(+t_h Delta_1) is read as
exp(-t_h Delta_1) (1/lambda = int_0^inf exp(-t lambda) dt, sampled at t = e^{h eta}); Delta_1 is
the operator's own 1D matrix (T_n = tridiag(-1, 2, -1) for the Poisson workloads), applied through
its sine eigenpairs (the DST-I basis the paper names): exp(-t T_n) = V exp(-t Lambda) V^T.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def expsum_weights(q: int):
    eta = np.pi / np.sqrt(q)
    h = np.arange(-q, q + 1)
    t = np.exp(h * eta)
    return eta * t, t


def sine_eigenpairs(n: int):
    i = np.arange(1, n + 1)
    v = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * np.pi / (n + 1))
    lam = 2.0 - 2.0 * np.cos(i * np.pi / (n + 1))
    return v, lam


def expsum_preconditioner(n: int, d: int, q: int) -> W.Operator:
    """M = sum_h c_h exp(-t_h T_n)^{(x) d} as a separable operator with dense mode matrices."""
    c, t = expsum_weights(q)
    v, lam = sine_eigenpairs(n)
    mats, theta = [], []
    for ch, th in zip(c, t):
        e = (v * np.exp(-th * lam)) @ v.T
        m = W.ModeMat('D', n, 0, 0, e)
        mats.append([m] * d)
        theta.append(float(ch))
    return W.Operator(d, [n] * d, theta, mats)
