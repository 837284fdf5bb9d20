"""RoundSum: Khatri-Rao sketched randomized HOSVD of a sum of Tucker tensors (Section 3.1).

Test infrastructure only.  Steps, in the paper's order (Section 3.1, Eq. (3.1)):
  1. factor sketches     M_j^(i) = U_j^(i)T S_j                      (r_j^(i) x s)
  2. range finder        Y_k = sum_i U_k^(i) G_(k)^(i) (KR_{j != k} M_j^(i))   (n_k x s)
  3. economy QR          Y_k = U^_k R_k
  4. core projection     C^ = sum_i G^(i) x_1 (U^_1^T U_1^(i)) ... x_d (U^_d^T U_d^(i))
  5. ST-HOSVD of C^ to the tolerance eps, ranks capped at rank_cap.
Readings (the paper leaves them open):
  * the Khatri-Rao order in step 2 is the one matching the unfolding (Eq. (2.2)); the
    paper's subscript M_{d-j+1} is read as that order;
  * ST-HOSVD: modes 1..d in order, SVD of the current unfolding, kept rank
    r_k = min(rank_cap, smallest r whose tail energy sum_{j>r} sigma_j^2 <= eps^2 ||C^||^2 / d);
  * adaptive sketch size: tail energy of the Gram eigenvalues of the energy-weighted
    concatenated factors below rank_tol^2 of their total, s = min(max_k r~_k, rank_cap) + p
    (rank_tol = the RoundSum tolerance; estimate formed when V_k has <= 96 rows or columns).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from workloads import Tucker
from .tensor import mttkrp, multi_ttm, ttm, unfold


def st_hosvd(c: np.ndarray, eps: float, rank_cap: int) -> Tuple[np.ndarray, List[np.ndarray]]:
    """Sequentially truncated HOSVD (Section 2.4.1 / 3.1): returns the truncated core and W_k."""
    norm2 = float(np.sum(c * c))
    d = c.ndim
    thr = eps * eps * norm2 / d
    ws = []
    for k in range(d):
        u, sv, _ = np.linalg.svd(unfold(c, k), full_matrices=False)
        e = sv * sv
        tail = np.concatenate([np.cumsum(e[::-1])[::-1], [0.0]])   # tail[r] = sum_{j >= r} e_j
        r = len(sv)
        for cand in range(1, len(sv) + 1):
            if tail[cand] <= thr:
                r = cand
                break
        r = max(1, min(r, rank_cap))
        w = u[:, :r]
        c = ttm(c, w.T, k)
        ws.append(w)
    return c, ws


GRAM_MAX = 96


def effective_sketch_size(terms: Sequence[Tuple[float, Tucker]], p: int, rank_cap: int,
                          rank_tol: float, gram_max: int = GRAM_MAX) -> int:
    """Sketch size from the effective rank of V_k = [|c_i| ||G^(i)||_F U_k^(i)]_i (Section 3.1):
    r~_k is the smallest r whose tail sum_{j > r} lambda_j of the eigenvalues of V_k^T V_k is at
    most rank_tol^2 sum_j lambda_j, and s = min(max_k r~_k, rank_cap) + p.  Reading of a size
    limit shared with the library: the estimate is formed only when V_k has at most gram_max
    columns or rows (min(n_k, sum_i r_k^(i)) <= gram_max); otherwise r~_k = rank_cap."""
    d = terms[0][1].d
    rt = []
    for k in range(d):
        n_k = terms[0][1].factors[k].shape[0]
        if min(n_k, sum(t.factors[k].shape[1] for _, t in terms)) > gram_max:
            rt.append(rank_cap)
            continue
        v = np.concatenate([abs(c) * np.linalg.norm(t.core) * t.factors[k] for c, t in terms], axis=1)
        # the eigenvalues of V_k^T V_k, taken as the squared singular values of V_k: the same
        # numbers without the rounding of forming V_k^T V_k (which would blur every eigenvalue
        # below ~1e-16 of the largest, and with it thresholds rank_tol < 1e-8)
        lam = np.linalg.svd(v, compute_uv=False) ** 2
        total = lam.sum()
        tail = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])
        r = len(lam)
        for cand in range(1, len(lam) + 1):
            if tail[cand] <= rank_tol * rank_tol * total:
                r = cand
                break
        rt.append(r)
    return min(max(rt), rank_cap) + p


def roundsum(terms: Sequence[Tuple[float, Tucker]], sketches: Sequence[np.ndarray],
             rank_cap: int, eps: float) -> Tucker:
    """RoundSum(sum_i c_i X^(i)) with Gaussian S_j = sketches[j] (n_j x s)."""
    d = terms[0][1].d
    # step 1: factor sketches
    ms = [[t.factors[j].T @ sketches[j] for j in range(d)] for _, t in terms]
    # steps 2-3: range finder and economy QR per mode
    uh = []
    for k in range(d):
        y = sum(c * (t.factors[k] @ mttkrp(t.core, ms[i], k)) for i, (c, t) in enumerate(terms))
        q, _ = np.linalg.qr(y)
        uh.append(q)
    # step 4: core projection
    chat = sum(c * multi_ttm(t.core, [uh[k].T @ t.factors[k] for k in range(d)]) for c, t in terms)
    # step 5: ST-HOSVD
    core, ws = st_hosvd(chat, eps, rank_cap)
    return Tucker(core, [uh[k] @ ws[k] for k in range(d)])


def kron_sketch(x: Tucker, sketches: Sequence[np.ndarray]) -> np.ndarray:
    """Kronecker-structured sketch of a Tucker tensor (Algorithm 2, lines b_s and M):
    m_l = X x_1 s_{1,l}^T ... x_d s_{d,l}^T = sum_a G[a] prod_k (U_k^T S_k)[a_k, l].
    Reading: sketch column l applies S_k's column l to mode k; with column-major vec this
    is (S_d (.) ... (.) S_1)^T vec(X)."""
    p = [x.factors[k].T @ sketches[k] for k in range(x.d)]
    z = mttkrp(x.core, p, 0)
    return np.sum(p[0] * z, axis=0)
