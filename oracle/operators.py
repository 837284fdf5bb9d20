"""Separable operators L = sum_t theta_t A_1^(t) x ... x A_d^(t) (Section 1, Eq. (1.2)).

Test infrastructure only.  Reading of the paper's Kronecker order (Eq. (1.2) writes
A_1 x ... x A_d, Section 4.3 writes A_3 x A_2 x A_1 for the same mode products): the
operator is defined in mode-product form L(X) = sum_t theta_t X x_1 A_1^(t) ... x_d A_d^(t);
with column-major vec this is (sum_t theta_t A_d^(t) kron ... kron A_1^(t)) vec(X).
"""
from __future__ import annotations

from functools import reduce
from typing import List

import numpy as np

from workloads import ModeMat, Operator, Tucker
from .tensor import multi_ttm


def mode_dense(m: ModeMat) -> np.ndarray:
    """Dense n x n matrix of a mode matrix (band layout: data[ku + i - j, j] = A[i, j])."""
    n = m.n
    if m.kind == 'I':
        return np.eye(n)
    if m.kind == 'D':
        return np.array(m.data, dtype=np.float64)
    a = np.zeros((n, n))
    for j in range(n):
        for i in range(max(0, j - m.ku), min(n, j + m.kl + 1)):
            a[i, j] = m.data[m.ku + i - j, j]
    return a


def apply_mode(m: ModeMat, u: np.ndarray, transpose: bool = False) -> np.ndarray:
    """A U (or A^T U) for one mode matrix."""
    if m.kind == 'I':
        return u.copy()
    a = mode_dense(m)
    return (a.T if transpose else a) @ u


def apply_op(op: Operator, x: Tucker, transpose: bool = False) -> List[Tucker]:
    """L(X) for a Tucker X, Section 3.1: one Tucker term per operator term, all sharing X's
    core, theta_t folded into the core: term t = [theta_t G; A_1^(t) U_1, ..., A_d^(t) U_d].
    With transpose=True the adjoint L^T(X) (every A_k^(t) replaced by its transpose)."""
    out = []
    for t in range(op.nterms):
        fac = [apply_mode(op.mats[t][k], x.factors[k], transpose) for k in range(op.d)]
        out.append(Tucker(op.theta[t] * x.core, fac))
    return out


def apply_term(op: Operator, t: int, x: Tucker, transpose: bool = False) -> Tucker:
    """The unscaled term A_1^(t) x ... x A_d^(t) applied to X (theta_t not applied)."""
    fac = [apply_mode(op.mats[t][k], x.factors[k], transpose) for k in range(op.d)]
    return Tucker(x.core.copy(), fac)


def dense_matrix(op: Operator) -> np.ndarray:
    """The N x N matrix sum_t theta_t A_d^(t) kron ... kron A_1^(t) (small problems only)."""
    mats = []
    for t in range(op.nterms):
        dense = [mode_dense(op.mats[t][k]) for k in range(op.d)]
        mats.append(op.theta[t] * reduce(np.kron, dense[::-1]))
    return sum(mats)


def dense_apply(op: Operator, x: np.ndarray) -> np.ndarray:
    """L(X) for a dense tensor X by mode products."""
    out = np.zeros([op.n[k] for k in range(op.d)])
    for t in range(op.nterms):
        out += op.theta[t] * multi_ttm(x, [mode_dense(op.mats[t][k]) for k in range(op.d)])
    return out
