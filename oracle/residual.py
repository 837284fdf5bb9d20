"""True relative residual ||L(X) - B||_F / ||B||_F in Tucker form (output contract of
Algorithms 1, 2 and 6), without forming any n_1 x ... x n_d tensor.

Test infrastructure only.  The residual is the sum of the N_t terms of L(X) and -B.  Its
exact Tucker form has the concatenated factors [U^(1) ... U^(N_t+1)] per mode and a
block-diagonal core; with Q_k R_k = the QR factorization of the concatenated factors, the
residual norm is the norm of the small dense core sum_i G^(i) x_k R_k[:, block_i].  Unlike
an expansion into pairwise inner products, this keeps full relative accuracy when
||L(X) - B|| << ||B||.
"""
from __future__ import annotations

import numpy as np

from workloads import Operator, Tucker
from .operators import apply_op, dense_apply
from .tensor import full, multi_ttm, norm


def tucker_sum_norm(terms) -> float:
    """||sum_i c_i X^(i)||_F through QR of the concatenated factors."""
    d = terms[0][1].d
    rs, offs = [], []
    for k in range(d):
        cat = np.concatenate([t.factors[k] for _, t in terms], axis=1)
        _, r = np.linalg.qr(cat)
        rs.append(r)
        offs.append(np.concatenate([[0], np.cumsum([t.r[k] for _, t in terms])]))
    core = 0.0
    for i, (c, t) in enumerate(terms):
        core = core + c * multi_ttm(t.core, [rs[k][:, offs[k][i]:offs[k][i + 1]] for k in range(d)])
    return float(np.linalg.norm(core))


def true_residual(op: Operator, x: Tucker, b: Tucker, transpose: bool = False) -> float:
    terms = [(1.0, t) for t in apply_op(op, x, transpose)] + [(-1.0, b)]
    return tucker_sum_norm(terms) / norm(b)


def dense_residual(op: Operator, x: Tucker, b: Tucker) -> float:
    """The same quantity by densification (small problems only)."""
    r = dense_apply(op, full(x)) - full(b)
    return float(np.linalg.norm(r) / np.linalg.norm(full(b)))
