"""Gradients of a loss through the solve x = L^{-1}(b).  The paper has no counterpart.

Test infrastructure only.  For L = sum_t theta_t L_t and a loss l(x) with g = dl/dx:
  mu solves the adjoint system L^T(mu) = g (every mode matrix transposed);
  dl/db = mu;  dl/dtheta_t = -<mu, L_t(x)>;
  for b = [G_b; U_b]:  dl/dG_b = mu x_1 U_b1^T ... x_d U_bd^T,
                       dl/dU_bk = mu_(k) (kron_{j != k} U_bj) G_b(k)^T.
`dense_gradients` is the same computation by dense LU solves (small problems only).
"""
from __future__ import annotations

from typing import List

import numpy as np

from workloads import Operator, Tucker
from .operators import apply_term, dense_matrix, mode_dense
from .tensor import full, inner, multi_ttm, ttm, unfold


def theta_gradients(op: Operator, x: Tucker, mu: Tucker) -> np.ndarray:
    return np.array([-inner(mu, apply_term(op, t, x)) for t in range(op.nterms)])


def core_gradient(mu: Tucker, b: Tucker) -> np.ndarray:
    """dl/dG_b = mu x_k U_bk^T = G_mu x_k (U_bk^T U_mu,k)."""
    return multi_ttm(mu.core, [b.factors[k].T @ mu.factors[k] for k in range(b.d)])


def factor_gradients(mu: Tucker, b: Tucker) -> List[np.ndarray]:
    """dl/dU_bk = U_mu,k [G_mu x_{j != k} (U_bj^T U_mu,j)]_(k) G_b(k)^T."""
    out = []
    for k in range(b.d):
        g = mu.core
        for j in range(b.d):
            if j != k:
                g = ttm(g, b.factors[j].T @ mu.factors[j], j)
        out.append(mu.factors[k] @ unfold(g, k) @ unfold(b.core, k).T)
    return out


def dense_gradients(op: Operator, b: Tucker, x_true: np.ndarray):
    """Exact gradients of l = 0.5 ||x - x_true||^2, x = A^{-1} vec(b), by dense solves."""
    a = dense_matrix(op)
    bv = full(b).reshape(-1, order='F')
    x = np.linalg.solve(a, bv)
    g = x - x_true.reshape(-1, order='F')
    mu = np.linalg.solve(a.T, g)
    dtheta = []
    for t in range(op.nterms):
        from functools import reduce
        at = reduce(np.kron, [mode_dense(op.mats[t][k]) for k in range(op.d)][::-1])
        dtheta.append(-mu @ (at @ x))
    shape = b.n
    return x.reshape(shape, order='F'), mu.reshape(shape, order='F'), np.array(dtheta)
