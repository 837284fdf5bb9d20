"""Multilinear Nystrom (MLN) compression with Khatri-Rao structured sketches (Section 3.3).

Test infrastructure only.  Algorithms 3 (MLN_Sketch), 4 (MLN_Sum) and 5 (MLN_Recovery).
Psi_k in R^{n_k x (r+p)}; Psi-bar_k is its first r columns; Omega_k is the Khatri-Rao
product of the Psi-bar_j, j != k (Eq. (3.3)).  Readings:
  * Algorithm 3's "first r_k rows" is the first r rows, r the target rank (as in Section 3.3);
  * R_k^+ is the pseudo-inverse through an SVD of the r x r factor R_k, singular values
    below r * 2^-52 * sigma_max dropped (R_k is singular for low-rank inputs, e.g. the
    rank-one right-hand side at the first iteration).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from workloads import Tucker
from .tensor import mttkrp, multi_ttm

Sketch = Tuple[np.ndarray, List[np.ndarray]]      # (G_Psi, [F_Psi_k])


def mln_sketch(x: Tucker, psis: Sequence[np.ndarray], r: int) -> Sketch:
    """Algorithm 3 for one Tucker tensor: G_Psi = G x_k (Psi_k^T U_k), F_k = U_k MTTKRP(G, {Ubar^T}, k)."""
    d = x.d
    u_psi = [psis[k].T @ x.factors[k] for k in range(d)]          # (r+p) x r_k
    u_bar = [u_psi[k][:r, :] for k in range(d)]                    # r x r_k
    g_psi = multi_ttm(x.core, u_psi)
    f = [x.factors[k] @ mttkrp(x.core, [ub.T for ub in u_bar], k) for k in range(d)]
    return g_psi, f


def mln_diag(g_psi: np.ndarray) -> np.ndarray:
    """Superdiagonal of the sketched core, [diag(G_Psi)]_i = G_Psi[i, ..., i] (Eq. (3.7))."""
    m = min(g_psi.shape)
    idx = np.arange(m)
    return g_psi[(idx,) * g_psi.ndim].copy()


def mln_sum(items: Sequence[Tuple[float, Sketch]]) -> Sketch:
    """Algorithm 4: G_Psi = sum_j c_j G_Psi^(j), F_k = sum_j c_j F_k^(j)."""
    g = sum(c * s[0] for c, s in items)
    d = len(items[0][1][1])
    f = [sum(c * s[1][k] for c, s in items) for k in range(d)]
    return g, f


def pinv_upper(r_mat: np.ndarray) -> np.ndarray:
    """Pseudo-inverse of the small triangular factor via its SVD (reading stated above)."""
    u, s, vt = np.linalg.svd(r_mat)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros(r_mat.T.shape)
    keep = s > r_mat.shape[1] * 2.0 ** -52 * s[0]
    return (vt[keep].T / s[keep]) @ u[:, keep].T


def mln_recovery(sk: Sketch, psis: Sequence[np.ndarray]) -> Tucker:
    """Algorithm 5: Q_k R_k = qr(Psi_k^T F_k); U~_k = F_k R_k^+; G~ = G_Psi x_k Q_k^T."""
    g_psi, f = sk
    qs, us = [], []
    for k in range(len(f)):
        q, rr = np.linalg.qr(psis[k].T @ f[k])
        us.append(f[k] @ pinv_upper(rr))
        qs.append(q)
    return Tucker(multi_ttm(g_psi, [q.T for q in qs]), us)


def mln_downsample(sk: Sketch, rt_sol: int, r_sol: int) -> Sketch:
    """Memory-efficient truncation of a stored sketch (Section 3.3): the leading
    rt_sol x ... x rt_sol block of G_Psi and the leading r_sol columns of every F_k.  Equal to
    sketching with the leading rt_sol columns of each Psi_k from the start (the Khatri-Rao
    column l of F_k uses column l of every other Psi_j)."""
    g, f = sk
    return g[(slice(0, rt_sol),) * g.ndim].copy(), [fk[:, :r_sol].copy() for fk in f]
