"""RHOSVD-Tucker GMRES (Algorithm 1), RHOSVD-Tucker sGMRES (Algorithm 2), MLN-Tucker sGMRES
(Algorithm 6), dense sGMRES (Eq. (2.8)).

Test infrastructure only.  Readings of points the paper leaves open:
  * x_0 = 0, so V_1 = B / ||B||;
  * breakdown "||W|| ~ 0" means ||W|| <= 1e-14 ||W_0||, W_0 the compressed L(V_k) before
    the short-recurrence orthogonalization; on breakdown the least-squares problem is still
    solved with the k columns gathered so far and the solve ends successfully;
  * the window orthogonalization is classical Gram-Schmidt: every h_j uses the same W;
  * the sketched least-squares problem is degenerate once k reaches the sketch size s, so
    at most s - 1 iterations run (status SKETCH_EXHAUSTED if that limit, not N_max, ends it);
  * RoundSum draws fresh Gaussian matrices on every call, from stream
    (seed, STREAM_ROUNDSUM, call, mode); the Krylov sketch S_k (or Psi_k) from
    (seed, STREAM_KRYLOV, 0, mode);
  * Algorithm 6: Psi_k has r + p columns (Section 3.3); b_s = ||B|| diag(G_Psi(V_1)) so that
    b_s = S^T vec(B) as in Algorithm 2; after the window's MLN_Sum the sum is recovered
    (MLN_Recovery) before its norm is taken and V_{i+1} is formed;
  * Algorithm 1: the same breakdown reading (the Hessenberg least-squares problem is solved
    with its zero last row, then the solve ends); it stops when res_k < tol (no eta factor).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from workloads import (STREAM_KRYLOV, STREAM_ROUNDSUM, Operator, SolverParams, Tucker,
                       sketch_matrix)
from .mln import mln_diag, mln_downsample, mln_recovery, mln_sketch, mln_sum
from .operators import apply_op
from .rhosvd import effective_sketch_size, kron_sketch, roundsum
from .tensor import inner, norm, scale

CONVERGED, NOT_CONVERGED, BREAKDOWN, SKETCH_EXHAUSTED = 0, 1, 2, 3


@dataclass
class Result:
    x: Tucker
    iters: int
    status: int
    res_hist: List[float]
    y: np.ndarray
    ranks: List[List[int]] = field(default_factory=list)
    sketch_sizes: List[int] = field(default_factory=list)
    basis: List[Tucker] = field(default_factory=list)


def _ls(mcols: List[np.ndarray], bs: np.ndarray):
    """y = argmin ||M y - b_s||_2 and ||M y - b_s||_2 (Algorithm 2, sketched residual)."""
    m = np.stack(mcols, axis=1)
    y = np.linalg.lstsq(m, bs, rcond=None)[0]
    return y, float(np.linalg.norm(m @ y - bs))


GCV_POINTS = 121


def gcv_grid(sigma_max: float) -> np.ndarray:
    """The lambda values GCV chooses from (reading: the paper does not state the search):
    sigma_max 10^(-12 + 12 g / 120), g = 0 .. 120."""
    return sigma_max * 10.0 ** (-12.0 + 12.0 * np.arange(GCV_POINTS) / (GCV_POINTS - 1))


def gcv_function(sig: np.ndarray, bhat: np.ndarray, rho2: float, m: int, lam: float) -> float:
    """GCV (Golub, Heath, Wahba 1979) of the Tikhonov problem min ||M y - b||^2 + lam^2 ||y||^2
    from the SVD of M (singular values sig, bhat = U^T b, rho2 = ||b||^2 - ||bhat||^2):
    ||(I - A_lam) b||^2 / trace(I - A_lam)^2, A_lam = M (M^T M + lam^2 I)^-1 M^T, m rows."""
    f = sig ** 2 / (sig ** 2 + lam ** 2)
    num = float(np.sum(((1.0 - f) * bhat) ** 2) + rho2)
    return num / (m - float(np.sum(f))) ** 2


def ls_tikhonov(m_mat: np.ndarray, b: np.ndarray, rows: Optional[int] = None):
    """Projected Tikhonov step (Section 4.3, Eq. for the sketched / Hessenberg problem): lambda by
    GCV over gcv_grid (ties: the smaller lambda), then y = V diag(sig / (sig^2 + lam^2)) U^T b.
    GCV counts the problem's rows (m_mat's, unless `rows` is given).  Returns y, ||M y - b||,
    lambda."""
    u, sig, vt = np.linalg.svd(m_mat, full_matrices=False)
    bhat = u.T @ b
    rho2 = max(float(b @ b - bhat @ bhat), 0.0)
    grid = gcv_grid(float(sig[0]) if sig.size else 0.0)
    m = m_mat.shape[0] if rows is None else rows
    vals = [gcv_function(sig, bhat, rho2, m, lam) for lam in grid]
    lam = float(grid[int(np.argmin(vals))])
    y = vt.T @ (sig / (sig ** 2 + lam ** 2) * bhat)
    return y, float(np.linalg.norm(m_mat @ y - b)), lam


def rhosvd_sgmres(op: Operator, b: Tucker, prm: SolverParams, transpose: bool = False,
                  bf16_sketch: bool = False, maxit: Optional[int] = None,
                  precond: Optional[Operator] = None, gcv_rows: Optional[str] = None) -> Result:
    """Algorithm 2.  bf16_sketch rounds RoundSum's Gaussian matrices to bfloat16 values (the
    mixed-precision form stores them so); the arithmetic stays FP64.

    gcv_rows (with prm.tikhonov; None: prm.gcv_rows): the row count m GCV uses for the sketched
    problem (Section 4.3 leaves it open), "projected" (k + 1, the dimension of the span of
    [M_k, S b] in which the sketched residual lives, as Algorithm 1's k + 1 x k Hessenberg
    problem has k + 1 rows) or "sketch" (s, every row of the sketched problem).

    precond: a separable operator M applied with truncation, Z_k = RoundSum(M(V_k)), in the
    flexible form of Section 3.4: the Krylov columns sketch RoundSum(L(Z_k)) and the solution is
    RoundSum(sum_i y_i Z_i)."""
    d, n = b.d, b.n
    s = prm.sketch_s
    maxit = prm.maxit if maxit is None else maxit
    gcv_rows = getattr(prm, "gcv_rows", "projected") if gcv_rows is None else gcv_rows
    call = [0]

    def draw(sr: int):
        mats = [sketch_matrix(prm.seed, STREAM_ROUNDSUM, call[0], k, n[k], sr, bf16_sketch)
                for k in range(d)]
        call[0] += 1
        return mats

    def rs(terms):
        sr = (effective_sketch_size(terms, prm.oversample_p, prm.rank_cap, prm.round_tol)
              if prm.adaptive_rank else prm.rank_cap + prm.oversample_p)
        out = roundsum(terms, draw(sr), prm.rank_cap, prm.round_tol)
        sizes.append(sr)
        return out

    sizes: List[int] = []
    beta = norm(b)
    v = [scale(b, 1.0 / beta)]
    sk = [sketch_matrix(prm.seed, STREAM_KRYLOV, 0, k, n[k], s) for k in range(d)]
    bs = kron_sketch(b, sk)
    beta_s = float(np.linalg.norm(bs))
    mcols: List[np.ndarray] = []
    hist: List[float] = []
    ranks: List[List[int]] = []
    kmax = min(maxit, s - 1)
    status = SKETCH_EXHAUSTED if kmax < maxit else NOT_CONVERGED
    y = np.zeros(0)
    k = 0
    zs: List[Tucker] = []
    for k in range(1, kmax + 1):
        if precond is not None:
            zs.append(rs([(1.0, t) for t in apply_op(precond, v[-1], transpose)]))
            w = rs([(1.0, t) for t in apply_op(op, zs[-1], transpose)])
        else:
            w = rs([(1.0, t) for t in apply_op(op, v[-1], transpose)])
        w0 = norm(w)
        mcols.append(kron_sketch(w, sk))
        window = range(max(1, k - prm.ktrunc + 1), k + 1)
        hs = [inner(v[j - 1], w) for j in window]
        w = rs([(1.0, w)] + [(-h, v[j - 1]) for h, j in zip(hs, window)])
        nw = norm(w)
        if prm.tikhonov:
            y, res, _ = ls_tikhonov(np.stack(mcols, axis=1), bs,
                                    rows=len(mcols) + 1 if gcv_rows == "projected" else None)
        else:
            y, res = _ls(mcols, bs)
        hist.append(res / beta_s)
        if nw <= 1e-14 * w0:
            status = BREAKDOWN
            break
        v.append(scale(w, 1.0 / nw))
        ranks.append(v[-1].r)
        if res / beta_s < prm.eta * prm.tol:
            status = CONVERGED
            break
    basis = zs if precond is not None else v
    x = rs([(float(y[i]), basis[i]) for i in range(k)])
    return Result(x, k, status, hist, y, ranks, sizes, v)


def rhosvd_gmres(op: Operator, b: Tucker, prm: SolverParams, transpose: bool = False,
                 bf16_sketch: bool = False, maxit: Optional[int] = None) -> Result:
    """Algorithm 1: GMRES with full Arnoldi orthogonalisation, every sum through RoundSum.
    h_{j,k} = <V_j, W> for all j <= k from the same W (classical Gram-Schmidt, one RoundSum of
    k + 1 terms); h_{k+1,k} = ||W||; y_k = argmin ||beta e_1 - H_{1:k+1,1:k} y||; the relative
    residual res_k = ||beta e_1 - H y_k|| / beta."""
    d, n = b.d, b.n
    maxit = prm.maxit if maxit is None else maxit
    call = [0]
    sizes: List[int] = []

    def rs(terms):
        sr = (effective_sketch_size(terms, prm.oversample_p, prm.rank_cap, prm.round_tol)
              if prm.adaptive_rank else prm.rank_cap + prm.oversample_p)
        mats = [sketch_matrix(prm.seed, STREAM_ROUNDSUM, call[0], k, n[k], sr, bf16_sketch)
                for k in range(d)]
        call[0] += 1
        sizes.append(sr)
        return roundsum(terms, mats, prm.rank_cap, prm.round_tol)

    beta = norm(b)
    v = [scale(b, 1.0 / beta)]
    h = np.zeros((maxit + 1, maxit))
    hist: List[float] = []
    ranks: List[List[int]] = []
    status = NOT_CONVERGED
    y = np.zeros(0)
    k = 0
    for k in range(1, maxit + 1):
        w = rs([(1.0, t) for t in apply_op(op, v[-1], transpose)])
        w0 = norm(w)
        hs = [inner(v[j], w) for j in range(k)]
        w = rs([(1.0, w)] + [(-hj, v[j]) for j, hj in enumerate(hs)])
        nw = norm(w)
        h[:k, k - 1] = hs
        h[k, k - 1] = nw
        rhs = np.zeros(k + 1)
        rhs[0] = beta
        if prm.tikhonov:
            y, res, _ = ls_tikhonov(h[:k + 1, :k], rhs)
            res /= beta
        else:
            y = np.linalg.lstsq(h[:k + 1, :k], rhs, rcond=None)[0]
            res = float(np.linalg.norm(rhs - h[:k + 1, :k] @ y)) / beta
        hist.append(res)
        if nw <= 1e-14 * w0:
            status = BREAKDOWN
            break
        v.append(scale(w, 1.0 / nw))
        ranks.append(v[-1].r)
        if res < prm.tol:
            status = CONVERGED
            break
    x = rs([(float(y[i]), v[i]) for i in range(k)])
    return Result(x, k, status, hist, y, ranks, sizes, v)


def mln_sgmres(op: Operator, b: Tucker, prm: SolverParams, transpose: bool = False,
               maxit: Optional[int] = None, gcv_rows: Optional[str] = None) -> Result:
    """Algorithm 6, r = rank_cap, r + p sketch columns.  With prm.r_sol > 0 (save_memory): once a
    basis tensor leaves the window (iteration i > k_trunc drops V_{i - k_trunc}) its stored
    sketch is cut to r_sol + p_sol (mln_downsample); at the end the sketches still in the
    window are cut too, and the solution is recovered at rank r_sol with the leading
    r_sol + p_sol columns of each Psi_k.  gcv_rows: as for rhosvd_sgmres ("sketch": r + p rows)."""
    d, n = b.d, b.n
    gcv_rows = getattr(prm, "gcv_rows", "projected") if gcv_rows is None else gcv_rows
    r = prm.rank_cap
    rp = r + prm.oversample_p
    maxit = prm.maxit if maxit is None else maxit
    psis = [sketch_matrix(prm.seed, STREAM_KRYLOV, 0, k, n[k], rp) for k in range(d)]
    save = prm.r_sol > 0
    rt_sol = prm.r_sol + prm.p_sol
    if save:
        assert prm.r_sol <= r and rt_sol <= rp, "r_sol <= r and r_sol + p_sol <= r + p"
    cut = {}
    beta = norm(b)
    v = [scale(b, 1.0 / beta)]
    sks = [mln_sketch(v[0], psis, r)]
    bs = beta * mln_diag(sks[0][0])
    beta_s = float(np.linalg.norm(bs))
    mcols: List[np.ndarray] = []
    hist: List[float] = []
    kmax = min(maxit, rp - 1)
    status = SKETCH_EXHAUSTED if kmax < maxit else NOT_CONVERGED
    y = np.zeros(0)
    i = 0
    for i in range(1, kmax + 1):
        gw = mln_sum([(1.0, mln_sketch(t, psis, r)) for t in apply_op(op, v[-1], transpose)])
        mcols.append(mln_diag(gw[0]))
        w = mln_recovery(gw, psis)
        w0 = norm(w)
        window = range(max(1, i - prm.ktrunc + 1), i + 1)
        hs = [inner(v[j - 1], w) for j in window]
        gw = mln_sum([(1.0, gw)] + [(-h, sks[j - 1]) for h, j in zip(hs, window)])
        w = mln_recovery(gw, psis)
        nw = norm(w)
        if prm.tikhonov:
            y, res, _ = ls_tikhonov(np.stack(mcols, axis=1), bs,
                                    rows=len(mcols) + 1 if gcv_rows == "projected" else None)
        else:
            y, res = _ls(mcols, bs)
        hist.append(res / beta_s)
        if nw <= 1e-14 * w0:
            status = BREAKDOWN
            break
        v.append(scale(w, 1.0 / nw))
        sks.append(mln_sketch(v[-1], psis, r))
        if save and i > prm.ktrunc:
            sks[i - prm.ktrunc - 1] = mln_downsample(sks[i - prm.ktrunc - 1], rt_sol, prm.r_sol)
            cut[i - prm.ktrunc - 1] = True
        if res / beta_s < prm.eta * prm.tol:
            status = CONVERGED
            break
    if save:
        for m in range(i):
            if not cut.get(m, False):
                sks[m] = mln_downsample(sks[m], rt_sol, prm.r_sol)
        x = mln_recovery(mln_sum([(float(y[m]), sks[m]) for m in range(i)]), [ps[:, :rt_sol] for ps in psis])
    else:
        x = mln_recovery(mln_sum([(float(y[m]), sks[m]) for m in range(i)]), psis)
    return Result(x, i, status, hist, y, basis=v)


def dense_sgmres(a: np.ndarray, b: np.ndarray, s_mat: np.ndarray, ktrunc: int, iters: int):
    """Matrix sGMRES (Eq. (2.8)) with the same window orthogonalization, no truncation:
    v_1 = b/||b||, w = A v_k, M[:, k] = S w, w -= sum_{window} (v_j^T w) v_j, v_{k+1} = w/||w||,
    y = argmin ||M y - S b||.  Returns x = V y and the sketched residual history."""
    beta = np.linalg.norm(b)
    v = [b / beta]
    bs = s_mat @ b
    mcols, hist = [], []
    y = np.zeros(0)
    for k in range(1, iters + 1):
        w = a @ v[-1]
        mcols.append(s_mat @ w)
        window = range(max(1, k - ktrunc + 1), k + 1)
        hs = [v[j - 1] @ w for j in window]
        for h, j in zip(hs, window):
            w = w - h * v[j - 1]
        y, res = _ls(mcols, bs)
        hist.append(res / np.linalg.norm(bs))
        v.append(w / np.linalg.norm(w))
    x = sum(y[i] * v[i] for i in range(len(y)))
    return x, hist
