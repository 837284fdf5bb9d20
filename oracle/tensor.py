"""Tensor algebra of Section 2.2-2.3 (FP64, numpy).  Test infrastructure only.

Conventions.  A tensor X in R^{n_1 x ... x n_d} is a numpy array indexed X[i_1, ..., i_d];
vec(X) is column-major (i_1 fastest).  The mode-k unfolding X_(k) has rows i_k and columns
running over the remaining indices in increasing mode order, first remaining mode fastest.
With these conventions the Tucker tensor G x_1 U_1 ... x_d U_d has
vec = (U_d kron ... kron U_1) vec(G).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from workloads import Tucker


def unfold(x: np.ndarray, k: int) -> np.ndarray:
    """Mode-k unfolding X_(k) (Definition 2.2, matricized form)."""
    return np.moveaxis(x, k, 0).reshape(x.shape[k], -1, order='F')


def fold(m: np.ndarray, k: int, shape: Sequence[int]) -> np.ndarray:
    """Inverse of `unfold` for a tensor of the given shape."""
    rest = [shape[j] for j in range(len(shape)) if j != k]
    return np.moveaxis(m.reshape([shape[k]] + rest, order='F'), 0, k)


def ttm(x: np.ndarray, u: np.ndarray, k: int) -> np.ndarray:
    """Y = X x_k U, i.e. Y_(k) = U X_(k) (Definition 2.2)."""
    shape = list(x.shape)
    shape[k] = u.shape[0]
    return fold(u @ unfold(x, k), k, shape)


def multi_ttm(x: np.ndarray, us: Sequence[np.ndarray]) -> np.ndarray:
    """X x_1 U_1 x_2 U_2 ... x_d U_d (Definition 2.2, Eq. (2.1))."""
    for k, u in enumerate(us):
        x = ttm(x, u, k)
    return x


def khatri_rao(mats: Sequence[np.ndarray]) -> np.ndarray:
    """A_1 (.) A_2 (.) ... : column-wise Kronecker product (Definition 2.1)."""
    r = mats[0].shape[1]
    out = mats[0]
    for m in mats[1:]:
        assert m.shape[1] == r
        out = np.einsum('ir,jr->ijr', out, m).reshape(-1, r)
    return out


def mttkrp(x: np.ndarray, us: Sequence[np.ndarray], k: int) -> np.ndarray:
    """MTTKRP (Definition 2.3, Eq. (2.2)): X_(k) (U_d (.) ... (.) U_{k+1} (.) U_{k-1} (.) ... (.) U_1).

    us[j] has shape (x.shape[j], r); us[k] is ignored.  Result: x.shape[k] x r.
    """
    d = x.ndim
    order = [us[j] for j in reversed(range(d)) if j != k]
    return unfold(x, k) @ khatri_rao(order)


def full(t: Tucker) -> np.ndarray:
    """Dense tensor of a Tucker tensor, Eq. (2.3)."""
    return multi_ttm(t.core, t.factors)


def scale(t: Tucker, c: float) -> Tucker:
    return Tucker(c * t.core, list(t.factors))


def inner(x: Tucker, y: Tucker) -> float:
    """<X, Y>_F = <G_X, G_Y x_1 (U_1^T W_1) ... x_d (U_d^T W_d)> for X = [G_X; U], Y = [G_Y; W]."""
    g = y.core
    for k in range(x.d):
        g = ttm(g, x.factors[k].T @ y.factors[k], k)
    return float(np.sum(x.core * g))


def norm(x: Tucker) -> float:
    return float(np.sqrt(max(inner(x, x), 0.0)))


def concat_sum(terms: Sequence[tuple]) -> Tucker:
    """Exact Tucker form of sum_i c_i X_i: concatenated factors, block-diagonal core."""
    d = terms[0][1].d
    widths = [[t.r[k] for _, t in terms] for k in range(d)]
    shape = [sum(w) for w in widths]
    core = np.zeros(shape)
    offs = [np.concatenate([[0], np.cumsum(w)]) for w in widths]
    for i, (c, t) in enumerate(terms):
        sl = tuple(slice(offs[k][i], offs[k][i + 1]) for k in range(d))
        core[sl] += c * t.core
    factors = [np.concatenate([t.factors[k] for _, t in terms], axis=1) for k in range(d)]
    return Tucker(core, factors)


def storage(n: Sequence[int], r: Sequence[int]) -> int:
    """Floats stored by a Tucker tensor: sum_k n_k r_k + prod_k r_k (Section 4.3)."""
    return int(sum(a * b for a, b in zip(n, r)) + np.prod(r))
