"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published known-answer vectors, closed forms, brute force on small dense problems,
exact identities stated in the paper and invariants.  CPU only."""
import os
from functools import reduce

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A
from oracle import mln as M
from oracle import operators as O
from oracle import residual as RS
from oracle import rhosvd as R
from oracle import sgmres as S
from oracle import tensor as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _rand_tucker(n, r, seed):
    g = _rng(seed)
    return W.Tucker(g.standard_normal(tuple(r)), [g.standard_normal((a, b)) for a, b in zip(n, r)])


def _vec(x):
    return x.reshape(-1, order='F')


def _dst_basis(n):
    """Sine eigenvectors of tridiag(-1, 2, -1): V_ij = sqrt(2/(n+1)) sin(i j pi/(n+1)) (Section 3.4)."""
    i = np.arange(1, n + 1)
    v = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * np.pi / (n + 1))
    lam = 2.0 - 2.0 * np.cos(i * np.pi / (n + 1))
    return v, lam


# ------------------------------------------------------------------------------ RNG
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if l.strip() and l[0] != '#']
    for row in rows:
        w = [int(x, 16) for x in row]
        out = W.philox4x32_10([np.array([c]) for c in w[:4]], (w[4], w[5]))
        assert [int(o[0]) for o in out] == w[6:10]


def test_gaussian_stream_distribution():
    from scipy import stats
    z = W.gaussian_stream(11, W.stream_id(2, 3, 1), 200001)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert stats.kstest(z, 'norm').pvalue > 1e-3
    z2 = W.gaussian_stream(11, W.stream_id(2, 3, 2), 200001)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01
    # prefix property: element e does not depend on the requested count
    assert np.array_equal(W.gaussian_stream(11, 5, 7), W.gaussian_stream(11, 5, 1001)[:7])


def test_bf16_rounding_against_torch():
    import torch
    x = _rng(1).standard_normal(50000).astype(np.float32).astype(np.float64)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(W.round_to_bf16(x), ref)
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert W.round_to_bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    assert W.round_to_bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6


# ------------------------------------------------------------------------------ tensor algebra
def test_unfold_ttm_mttkrp_brute_force():
    g = _rng(2)
    x = g.standard_normal((3, 4, 5))
    # unfold: X_(2)[i2, i1 + 3*i3] = X[i1, i2, i3]
    u2 = T.unfold(x, 1)
    for i1 in range(3):
        for i2 in range(4):
            for i3 in range(5):
                assert u2[i2, i1 + 3 * i3] == x[i1, i2, i3]
    assert np.array_equal(T.fold(u2, 1, x.shape), x)
    u = g.standard_normal((6, 4))
    y = T.ttm(x, u, 1)
    assert np.allclose(y, np.einsum('ajc,bj->abc', x, u))
    us = [g.standard_normal((3, 7)), g.standard_normal((4, 7)), g.standard_normal((5, 7))]
    for k in range(3):
        m = T.mttkrp(x, us, k)
        ref = np.zeros((x.shape[k], 7))
        for idx in np.ndindex(*x.shape):
            for r in range(7):
                ref[idx[k], r] += x[idx] * np.prod([us[j][idx[j], r] for j in range(3) if j != k])
        assert np.allclose(m, ref, rtol=1e-13, atol=1e-13)
    kr = T.khatri_rao([us[0], us[1]])
    for r in range(7):
        assert np.allclose(kr[:, r], np.kron(us[0][:, r], us[1][:, r]))


def test_tucker_full_inner_norm():
    x = _rand_tucker([5, 4, 6], [2, 3, 2], 3)
    y = _rand_tucker([5, 4, 6], [3, 1, 2], 4)
    fx = T.full(x)
    vec_ref = reduce(np.kron, [u for u in x.factors][::-1]) @ _vec(x.core)
    assert np.allclose(_vec(fx), vec_ref)
    assert np.isclose(T.inner(x, y), np.sum(fx * T.full(y)), rtol=1e-13)
    assert np.isclose(T.norm(x), np.linalg.norm(fx), rtol=1e-13)
    q = [np.linalg.qr(u)[0] for u in x.factors]
    xo = W.Tucker(x.core, q)
    assert np.isclose(T.norm(xo), np.linalg.norm(x.core), rtol=1e-13)
    cs = T.concat_sum([(2.0, x), (-0.5, y)])
    assert np.allclose(T.full(cs), 2.0 * fx - 0.5 * T.full(y))


def test_storage_formula_golden():
    row = [l.split() for l in open(os.path.join(GOLDEN, "storage_deblur.txt")) if l[0] != '#'][0]
    n, r, dense, tucker = [int(v) for v in row[:3]], [int(v) for v in row[3:6]], int(row[6]), int(row[7])
    assert int(np.prod(n)) == dense
    assert T.storage(n, r) == tucker


# ------------------------------------------------------------------------------ operators
def test_band_layout_and_operator_bruteforce():
    n = 6
    t = O.mode_dense(W.second_difference(n))
    assert np.array_equal(t, 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    b = O.mode_dense(W.upwind_backward(n, 3.0))
    assert np.array_equal(b, 3.0 * (np.eye(n) - np.eye(n, k=-1)))
    assert np.allclose(O.mode_dense(W.gaussian_blur_band(n + 9)), W.gaussian_blur_dense(n + 9))
    for wl in [W.convdiff3d(n, 0, None), W.varcoef4d(n, 0, None), W.deblur3d(n, 0, None)]:
        op = wl.op
        x = _rand_tucker([n] * op.d, [2] * op.d, 5)
        lhs = sum(T.full(t) for t in O.apply_op(op, x))
        rhs = (O.dense_matrix(op) @ _vec(T.full(x))).reshape([n] * op.d, order='F')
        assert np.allclose(lhs, rhs, rtol=1e-13, atol=1e-12 * np.abs(rhs).max())
        lhs_t = sum(T.full(t) for t in O.apply_op(op, x, transpose=True))
        rhs_t = (O.dense_matrix(op).T @ _vec(T.full(x))).reshape([n] * op.d, order='F')
        assert np.allclose(lhs_t, rhs_t, rtol=1e-13, atol=1e-12 * np.abs(rhs_t).max())


def test_poisson_sine_eigentensors():
    n = 9
    v, lam = _dst_basis(n)
    assert np.allclose(O.mode_dense(W.second_difference(n)) @ v, v * lam)
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    for (i, j, k) in [(0, 0, 0), (2, 5, 8), (4, 1, 3)]:
        e = W.Tucker(np.ones((1, 1, 1)), [v[:, [i]], v[:, [j]], v[:, [k]]])
        lx = sum(T.full(t) for t in O.apply_op(op, e))
        assert np.allclose(lx, (lam[i] + lam[j] + lam[k]) * T.full(e), atol=1e-13)


# ------------------------------------------------------------------------------ RoundSum
def test_st_hosvd_exact_rank_and_bound():
    g = _rng(6)
    c = T.multi_ttm(g.standard_normal((2, 3, 2)), [g.standard_normal((7, 2)), g.standard_normal((8, 3)),
                                                      g.standard_normal((6, 2))])
    core, ws = R.st_hosvd(c, 1e-13, 10)
    assert core.shape == (2, 3, 2)
    assert np.allclose(T.multi_ttm(core, ws), c, atol=1e-12)
    c2 = g.standard_normal((8, 7, 6))
    for eps in [0.3, 0.1]:
        core, ws = R.st_hosvd(c2, eps, 100)
        err = np.linalg.norm(T.multi_ttm(core, ws) - c2)
        assert err <= eps * np.linalg.norm(c2) * (1 + 1e-12)
    core, ws = R.st_hosvd(c2, 0.0, 3)
    assert core.shape == (3, 3, 3)


def test_roundsum_exact_on_low_rank_sums():
    n = [9, 8, 10]
    x1 = _rand_tucker(n, [2, 2, 1], 7)
    x2 = _rand_tucker(n, [1, 2, 2], 8)
    g = _rng(9)
    sk = [g.standard_normal((nk, 4 + 5)) for nk in n]
    out = R.roundsum([(1.5, x1), (-2.0, x2)], sk, 4, 1e-14)
    ref = 1.5 * T.full(x1) - 2.0 * T.full(x2)
    assert np.linalg.norm(T.full(out) - ref) <= 1e-13 * np.linalg.norm(ref)
    # output factors orthonormal, so ||out|| = ||core||
    for u in out.factors:
        assert np.allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)
    # idempotent on its own output
    again = R.roundsum([(1.0, out)], [g.standard_normal((nk, 9)) for nk in n], 4, 1e-14)
    assert np.linalg.norm(T.full(again) - T.full(out)) <= 1e-13 * np.linalg.norm(ref)
    # X + (-1) X = 0
    zero = R.roundsum([(1.0, x1), (-1.0, x1)], sk, 4, 1e-14)
    assert T.norm(zero) <= 1e-13 * T.norm(x1)


def test_roundsum_randomized_bound_vs_hosvd():
    """Truncating a full-rank sum: the randomized result is within a modest factor of the
    deterministic truncated HOSVD of the dense sum (Halko-Martinsson-Tropp range finder)."""
    n, r, p = [12, 12, 12], 4, 5
    g = _rng(10)
    terms = []
    for i in range(3):
        t = _rand_tucker(n, [4, 4, 4], 20 + i)
        t.core *= 0.5 ** i
        terms.append((1.0, t))
    dense = sum(T.full(t) for _, t in terms)
    core, ws = R.st_hosvd(dense, 0.0, r)
    best = np.linalg.norm(T.multi_ttm(core, ws) - dense)
    errs = []
    for trial in range(5):
        sk = [g.standard_normal((12, r + p)) for _ in range(3)]
        out = R.roundsum(terms, sk, r, 0.0)
        errs.append(np.linalg.norm(T.full(out) - dense))
    assert np.median(errs) <= 3.0 * best


def test_kron_sketch_explicit():
    n = [4, 5, 3]
    x = _rand_tucker(n, [2, 3, 2], 11)
    g = _rng(12)
    sk = [g.standard_normal((nk, 7)) for nk in n]
    explicit = T.khatri_rao([sk[2], sk[1], sk[0]])        # (S_3 (.) S_2 (.) S_1)
    assert np.allclose(R.kron_sketch(x, sk), explicit.T @ _vec(T.full(x)), rtol=1e-13)
    y = _rand_tucker(n, [1, 2, 2], 13)
    lin = R.kron_sketch(T.concat_sum([(2.0, x), (-3.0, y)]), sk)
    assert np.allclose(lin, 2 * R.kron_sketch(x, sk) - 3 * R.kron_sketch(y, sk))


def test_effective_sketch_size():
    n = [10, 10, 10]
    x = _rand_tucker(n, [3, 2, 4], 14)
    assert R.effective_sketch_size([(1.0, x)], 5, 50, 1e-10) == 4 + 5
    assert R.effective_sketch_size([(1.0, x)], 5, 3, 1e-10) == 3 + 5


def test_effective_sketch_size_known_gram_spectrum():
    """A sum whose weighted factor Gram matrix V_k^T V_k is known exactly: three terms whose
    mode-k factors are disjoint column blocks of one orthogonal matrix (so V_k^T V_k is diagonal),
    cores of chosen Frobenius norms and chosen coefficients.  Its eigenvalues are
    (c_i ||G_i||)^2 with multiplicity r_i = 2, 3, 4: 100, 1 and 0.01, total 203.04; the tails
    after 2 and 5 eigenvalues are 3.04 and 0.04.  A threshold between two tail energies fixes
    r~ exactly: rank_tol^2 = 2.5e-3 lies between 0.04/203.04 and 3.04/203.04, so r~ = 5 (a
    weighting by ||G|| instead of ||G||^2 in the eigenvalues, or c instead of c^2, gives 2);
    rank_tol^2 = 0.04 gives 2; 1e-4 gives 7 (tails 0.03 and 0.02 after 6 and 7 eigenvalues);
    2.5e-5, below one 0.01 eigenvalue's share, gives 9; then the cap and the oversampling apply."""
    n, rs = 12, [2, 3, 4]
    rng = np.random.default_rng(3)
    qs = [np.linalg.qr(rng.standard_normal((n, n)))[0] for _ in range(3)]
    weights = [10.0, 1.0, 0.1]                 # c_i ||G_i||
    coefs = [2.0, -0.5, 4.0]
    terms, off = [], 0
    for r, wgt, c in zip(rs, weights, coefs):
        core = rng.standard_normal((r, r, r))
        core *= (wgt / abs(c)) / np.linalg.norm(core)
        fac = [q[:, off:off + r] for q in qs]
        terms.append((c, W.Tucker(core, fac)))
        off += r
    assert R.effective_sketch_size(terms, 5, 50, 0.05) == 5 + 5
    assert R.effective_sketch_size(terms, 5, 50, 0.2) == 2 + 5
    assert R.effective_sketch_size(terms, 5, 50, 0.01) == 7 + 5
    assert R.effective_sketch_size(terms, 5, 50, 0.005) == 9 + 5
    assert R.effective_sketch_size(terms, 5, 4, 0.05) == 4 + 5
    assert R.effective_sketch_size(terms, 7, 50, 0.05, gram_max=8) == 50 + 7   # beyond the size limit


# ------------------------------------------------------------------------------ MLN
def test_mln_diag_is_khatri_rao_sketch():
    n, r, p = [5, 4, 6], 2, 3
    x = _rand_tucker(n, [2, 3, 2], 15)
    g = _rng(16)
    psis = [g.standard_normal((nk, r + p)) for nk in n]
    gp, _ = M.mln_sketch(x, psis, r)
    explicit = T.khatri_rao([psis[2], psis[1], psis[0]])
    assert np.allclose(M.mln_diag(gp), explicit.T @ _vec(T.full(x)), rtol=1e-12)
    assert np.allclose(gp, T.multi_ttm(T.full(x), [p.T for p in psis]))


def test_mln_sketch_factor_is_unfolding_times_omega():
    n, r, p = [5, 4, 6], 2, 3
    x = _rand_tucker(n, [2, 3, 2], 17)
    g = _rng(18)
    psis = [g.standard_normal((nk, r + p)) for nk in n]
    _, f = M.mln_sketch(x, psis, r)
    bars = [ps[:, :r] for ps in psis]
    for k in range(3):
        omega = T.khatri_rao([bars[j] for j in reversed(range(3)) if j != k])   # Eq. (3.3)
        assert np.allclose(f[k], T.unfold(T.full(x), k) @ omega, rtol=1e-12)


def test_mln_recovery_exact_for_low_rank():
    n, r, p = [8, 7, 9], 3, 3
    x = _rand_tucker(n, [3, 2, 3], 19)
    g = _rng(20)
    psis = [g.standard_normal((nk, r + p)) for nk in n]
    out = M.mln_recovery(M.mln_sketch(x, psis, r), psis)
    assert np.linalg.norm(T.full(out) - T.full(x)) <= 1e-11 * np.linalg.norm(T.full(x))
    # Algorithm 4 is linear
    y = _rand_tucker(n, [1, 2, 1], 21)
    s = M.mln_sum([(2.0, M.mln_sketch(x, psis, r)), (-1.0, M.mln_sketch(y, psis, r))])
    ref = M.mln_sketch(T.concat_sum([(2.0, x), (-1.0, y)]), psis, r)
    assert np.allclose(s[0], ref[0]) and all(np.allclose(a, b) for a, b in zip(s[1], ref[1]))


def test_pinv_identity():
    g = _rng(22)
    a = g.standard_normal((9, 4))
    q, rr = np.linalg.qr(a)
    assert np.allclose(M.pinv_upper(rr) @ q.T, np.linalg.pinv(a))
    a1 = np.outer(g.standard_normal(9), g.standard_normal(4))     # rank one
    q, rr = np.linalg.qr(a1)
    assert np.allclose(M.pinv_upper(rr) @ q.T, np.linalg.pinv(a1), atol=1e-12)


# ------------------------------------------------------------------------------ solvers
def test_dense_sgmres_full_window_is_gmres():
    g = _rng(23)
    nn = 30
    a = np.eye(nn) * 3 + g.standard_normal((nn, nn)) * 0.3
    b = g.standard_normal(nn)
    k = 6
    x, _ = S.dense_sgmres(a, b, np.eye(nn), ktrunc=k, iters=k)
    kry = np.stack([np.linalg.matrix_power(a, j) @ b for j in range(k)], axis=1)
    c = np.linalg.lstsq(a @ kry, b, rcond=None)[0]
    assert np.allclose(x, kry @ c, rtol=1e-9)


@pytest.mark.parametrize("variant", ["rhosvd", "mln"])
def test_untruncated_tucker_sgmres_equals_dense(variant):
    n = 6
    wl = W.convdiff3d(n, 1, None)
    b = W.random_tucker([n] * 3, [1, 2, 1], 24)
    if variant == "rhosvd":
        prm = W.SolverParams('rhosvd', n, 40, 5, 14, 1e-15, ktrunc=2, round_tol=1e-15, seed=3)
        res = S.rhosvd_sgmres(wl.op, b, prm)
        sk = [W.sketch_matrix(3, W.STREAM_KRYLOV, 0, k, n, 40) for k in range(3)]
    else:
        prm = W.SolverParams('mln', n, 0, 20, 14, 1e-15, ktrunc=2, round_tol=1e-15, seed=3)
        res = S.mln_sgmres(wl.op, b, prm)
        sk = [W.sketch_matrix(3, W.STREAM_KRYLOV, 0, k, n, n + 20) for k in range(3)]
    smat = T.khatri_rao([sk[2], sk[1], sk[0]]).T
    xd, hd = S.dense_sgmres(O.dense_matrix(wl.op), _vec(T.full(b)), smat, 2, res.iters)
    assert np.allclose(res.res_hist, hd, rtol=1e-9)
    assert np.linalg.norm(_vec(T.full(res.x)) - xd) <= 1e-10 * np.linalg.norm(xd)


def test_poisson_solution_against_sine_closed_form():
    n = 12
    v, lam = _dst_basis(n)
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    b = W.random_tucker([n] * 3, [1, 1, 1], 25)
    prm = W.SolverParams('rhosvd', 12, 64, 5, 60, 1e-9, ktrunc=2, round_tol=1e-13)
    res = S.rhosvd_sgmres(op, b, prm)
    bh = T.multi_ttm(T.full(b), [v.T] * 3)
    xs = T.multi_ttm(bh / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :]), [v] * 3)
    tr = RS.true_residual(op, res.x, b)
    assert np.isclose(tr, RS.dense_residual(op, res.x, b), rtol=1e-6, atol=1e-14)
    kappa = (3 * lam.max()) / (3 * lam.min())
    err = np.linalg.norm(T.full(res.x) - xs) / np.linalg.norm(xs)
    assert err <= kappa * tr * 1.0001
    assert tr < 1e-7


def test_breakdown_on_eigentensor_rhs():
    n = 8
    v, lam = _dst_basis(n)
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    b = W.Tucker(np.full((1, 1, 1), 2.0), [v[:, [1]], v[:, [2]], v[:, [0]]])
    prm = W.SolverParams('rhosvd', 4, 16, 5, 10, 1e-12)
    res = S.rhosvd_sgmres(op, b, prm)
    assert res.status == S.BREAKDOWN and res.iters == 1
    assert np.allclose(T.full(res.x), T.full(b) / (lam[1] + lam[2] + lam[0]), atol=1e-13)


def test_sketched_residual_monotone_and_exhaustion():
    wl = W.convdiff3d(8, 2, None)
    prm = W.SolverParams('rhosvd', 4, 10, 5, 40, 1e-14)
    res = S.rhosvd_sgmres(wl.op, wl.b, prm)
    h = np.array(res.res_hist)
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))
    assert res.status == S.SKETCH_EXHAUSTED and res.iters == 9


def test_symmetric_window_two_is_lanczos():
    """Symmetric operator, k_trunc = 2, no truncation: the three-term recurrence keeps the
    whole basis orthonormal in exact arithmetic (Lanczos)."""
    n = 6
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    b = W.random_tucker([n] * 3, [2, 2, 2], 26)
    prm = W.SolverParams('rhosvd', n, 60, 5, 8, 1e-15, ktrunc=2, round_tol=1e-15)
    res = S.rhosvd_sgmres(op, b, prm)
    vs = res.basis[:8]
    gram = np.array([[T.inner(a, c) for c in vs] for a in vs])
    assert np.allclose(gram, np.eye(len(vs)), atol=1e-9)


def test_true_residual_tucker_form_keeps_relative_accuracy():
    n = 8
    v, lam = _dst_basis(n)
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    b = W.random_tucker([n] * 3, [2, 2, 2], 27)
    bh = T.multi_ttm(b.core, [v.T @ u for u in b.factors])
    x = W.Tucker(bh / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :]), [v] * 3)
    tr = RS.true_residual(op, x, b)
    assert tr < 1e-14
    x.core[0, 0, 0] += 1e-6
    ref = RS.dense_residual(op, x, b)
    assert np.isclose(RS.true_residual(op, x, b), ref, rtol=1e-8)


# ------------------------------------------------------------------------------ adjoint
def test_dense_gradients_against_finite_differences():
    n = 4
    wl = W.deblur3d(n, 3, None, lam=0.3)
    xt = T.full(W.random_tucker([n] * 3, [2, 2, 2], 28))
    x, mu, dth = A.dense_gradients(wl.op, wl.b, xt)

    def loss(op):
        a = O.dense_matrix(op)
        xx = np.linalg.solve(a, _vec(T.full(wl.b)))
        return 0.5 * np.sum((xx - _vec(xt)) ** 2)

    for t in range(wl.op.nterms):
        h = 1e-6
        op_p = W.Operator(3, wl.op.n, list(wl.op.theta), wl.op.mats)
        op_m = W.Operator(3, wl.op.n, list(wl.op.theta), wl.op.mats)
        op_p.theta[t] += h
        op_m.theta[t] -= h
        fd = (loss(op_p) - loss(op_m)) / (2 * h)
        assert np.isclose(dth[t], fd, rtol=1e-6)


def test_tucker_adjoint_gradients_match_dense():
    n = 5
    wl = W.deblur3d(n, 4, None, lam=0.5)
    xt = W.random_tucker([n] * 3, [2, 2, 2], 29)
    prm = W.SolverParams('rhosvd', n, 100, 5, 60, 1e-13, ktrunc=3, round_tol=1e-15)
    fwd = S.rhosvd_sgmres(wl.op, wl.b, prm)
    g = T.concat_sum([(1.0, fwd.x), (-1.0, xt)])
    adj = S.rhosvd_sgmres(wl.op, g, prm, transpose=True)
    dth = A.theta_gradients(wl.op, fwd.x, adj.x)
    _, mu_d, dth_d = A.dense_gradients(wl.op, wl.b, T.full(xt))
    assert np.allclose(dth, dth_d, rtol=1e-7)
    assert np.allclose(T.full(adj.x), mu_d, atol=1e-9 * np.abs(mu_d).max())
    # b = [G_b; U_b]: chain rule through the Tucker parameters against the dense mu
    gcore = A.core_gradient(adj.x, wl.b)
    assert np.allclose(gcore, T.multi_ttm(mu_d, [u.T for u in wl.b.factors]), atol=1e-9)
    gf = A.factor_gradients(adj.x, wl.b)
    for k in range(3):
        ref = T.unfold(mu_d, k) @ reduce(np.kron, [wl.b.factors[j] for j in reversed(range(3)) if j != k]) \
            @ T.unfold(wl.b.core, k).T
        assert np.allclose(gf[k], ref, atol=1e-9 * np.abs(ref).max())


# ------------------------------------------------------------------------------ preconditioner
def test_expsum_mode_matrices_are_matrix_exponentials():
    from scipy.linalg import expm
    from oracle import precond as OP
    n, q = 12, 4
    m = OP.expsum_preconditioner(n, 3, q)
    c, t = OP.expsum_weights(q)
    tn = O.mode_dense(W.second_difference(n))
    for h in [0, 3, 2 * q]:
        assert np.allclose(m.mats[h][0].data, expm(-t[h] * tn), atol=1e-12)
        assert np.isclose(m.theta[h], c[h])


def test_expsum_approximates_inverse_laplacian_spectrum():
    """sum_h c_h exp(-t_h lambda) ~ 1/lambda over the 3D Poisson spectrum; the error falls
    quickly with q (sinc quadrature of 1/lambda = int exp(-t lambda) dt)."""
    from oracle import precond as OP
    n = 32
    _, lam = OP.sine_eigenpairs(n)
    L = (lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).ravel()
    errs = []
    for q in [4, 8, 16]:
        c, t = OP.expsum_weights(q)
        approx = (c[None, :] * np.exp(-np.outer(L, t))).sum(axis=1)
        errs.append(np.max(np.abs(approx * L - 1.0)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-2 and errs[2] < 1e-3


def test_flexible_sgmres_with_exact_inverse_converges_at_once():
    """Flexible sGMRES with M = L^{-1} exactly (dense inverse as one mode-matrix term of a d = 3
    Kronecker-product operator is not separable; use the 1D-separable operator
    L = T (x) T (x) T whose inverse is T^{-1} (x) T^{-1} (x) T^{-1})."""
    n = 6
    t = O.mode_dense(W.second_difference(n))
    op = W.Operator(3, [n] * 3, [1.0], [[W.ModeMat('D', n, 0, 0, t)] * 3])
    inv = W.Operator(3, [n] * 3, [1.0], [[W.ModeMat('D', n, 0, 0, np.linalg.inv(t))] * 3])
    b = W.random_tucker([n] * 3, [2, 1, 2], 40)
    prm = W.SolverParams('rhosvd', n, 40, 5, 5, 1e-12, round_tol=1e-15)
    res = S.rhosvd_sgmres(op, b, prm, precond=inv)
    assert res.iters <= 2 and res.res_hist[0] < 1e-12
    xs = T.full(b)
    for k in range(3):
        xs = T.ttm(xs, np.linalg.inv(t), k)
    assert np.linalg.norm(T.full(res.x) - xs) <= 1e-11 * np.linalg.norm(xs)


def test_preconditioned_poisson_reaches_1e6_quickly():
    from oracle import precond as OP
    n = 32
    wl = W.workload("poisson3d_n32")
    prm = W.SolverParams('rhosvd', 12, 64, 5, 20, 1e-6, seed=0)
    res = S.rhosvd_sgmres(wl.op, wl.b, prm, precond=OP.expsum_preconditioner(n, 3, 8))
    assert res.status == S.CONVERGED and res.iters <= 12
    assert RS.true_residual(wl.op, res.x, wl.b) < 1e-5


# ------------------------------------------------------------------------------ Algorithm 1
def _dense_op(n, seed):
    rng = np.random.default_rng(seed)
    mats = []
    for k in range(3):
        a = rng.standard_normal((n, n)) / np.sqrt(n) + 3.0 * np.eye(n)
        mats.append(W.ModeMat('D', n, 0, 0, a))
    return W.Operator(
        3, [n] * 3, [1.0, 1.0, 1.0],
        [[mats[0], W.identity(n), W.identity(n)], [W.identity(n), mats[1], W.identity(n)],
         [W.identity(n), W.identity(n), mats[2]]])


def test_tucker_gmres_untruncated_matches_scipy_gmres():
    """Untruncated Algorithm 1 (rank cap = n, tiny tolerance) is exact GMRES: its residual
    history equals scipy's unrestarted GMRES on the dense Kronecker matrix (an independent
    Arnoldi implementation)."""
    from scipy.sparse.linalg import gmres
    n = 6
    op = _dense_op(n, 3)
    b = W.random_tucker([n] * 3, [2, 2, 2], 41)
    prm = W.SolverParams('gmres', n, 0, n, 12, 1e-14, round_tol=1e-15, seed=1)
    res = S.rhosvd_gmres(op, b, prm)
    a = O.dense_matrix(op)
    bv = T.full(b).reshape(-1, order='F')
    hist = []
    gmres(a, bv, rtol=1e-14, atol=0.0, restart=200, maxiter=1, callback=lambda r: hist.append(r),
          callback_type='pr_norm')
    k = min(len(hist), len(res.res_hist))
    assert k >= 8
    assert np.allclose(res.res_hist[:k], hist[:k], rtol=1e-6, atol=1e-12)


def test_tucker_gmres_two_eigenvalues_converges_in_two_steps():
    """A diagonalisable operator with two distinct eigenvalues: the minimal polynomial has
    degree 2, so GMRES is exact at iteration 2 (and the solution is the exact inverse)."""
    n = 5
    dvals = np.where(np.arange(n) % 2 == 0, 1.0, 3.0)
    d0 = W.ModeMat('D', n, 0, 0, np.diag(dvals))
    op = W.Operator(3, [n] * 3, [1.0], [[d0, W.identity(n), W.identity(n)]])   # eigenvalues 1, 3
    b = W.random_tucker([n] * 3, [2, 2, 2], 42)
    prm = W.SolverParams('gmres', n, 0, n, 10, 1e-12, round_tol=1e-15, seed=2)
    res = S.rhosvd_gmres(op, b, prm)
    assert res.iters <= 2 and res.res_hist[-1] < 1e-12
    xs = T.ttm(T.full(b), np.diag(1.0 / dvals), 0)
    assert np.linalg.norm(T.full(res.x) - xs) <= 1e-11 * np.linalg.norm(xs)


def test_tucker_gmres_residuals_do_not_increase_and_beat_short_recurrence():
    """Full GMRES minimises the residual over the whole Krylov space: its history is
    non-increasing, and (untruncated) never above the sketched short-recurrence method's
    true residual at the same iteration."""
    n = 6
    op = _dense_op(n, 4)
    b = W.random_tucker([n] * 3, [1, 2, 1], 43)
    prm = W.SolverParams('gmres', n, 0, n, 15, 1e-14, round_tol=1e-15, seed=3)
    res = S.rhosvd_gmres(op, b, prm)
    hsts = np.array(res.res_hist)
    assert np.all(np.diff(hsts) <= 1e-12)
    prm2 = W.SolverParams('rhosvd', n, 64, n, 15, 1e-14, ktrunc=2, round_tol=1e-15, seed=3)
    for k in [3, 6, 10]:
        r2 = S.rhosvd_sgmres(op, b, prm2, maxit=k)
        assert hsts[k - 1] <= RS.true_residual(op, r2.x, b) * (1 + 1e-8)


# ------------------------------------------------------------------------------ memory-efficient MLN
def test_mln_downsample_equals_sketch_with_leading_columns():
    """Cutting a stored sketch to (r_sol + p_sol, r_sol) equals sketching with the leading
    r_sol + p_sol columns of every Psi_k and target rank r_sol (Section 3.3)."""
    from oracle import mln as M
    n = [9, 8, 7]
    x = W.random_tucker(n, [3, 4, 2], 51)
    rng = np.random.default_rng(52)
    r, p, r_sol, p_sol = 5, 6, 3, 2
    psis = [rng.standard_normal((nk, r + p)) for nk in n]
    full = M.mln_downsample(M.mln_sketch(x, psis, r), r_sol + p_sol, r_sol)
    small = M.mln_sketch(x, [ps[:, :r_sol + p_sol] for ps in psis], r_sol)
    assert np.allclose(full[0], small[0], atol=1e-13)
    for a, b in zip(full[1], small[1]):
        assert np.allclose(a, b, atol=1e-13)


def test_mln_save_memory_exact_for_low_rank_solution():
    """A problem whose Krylov vectors stay within multilinear rank r_sol: the memory-efficient
    variant returns the same solution as the full one (the cut sketches still determine the
    rank-r_sol tensors exactly), with every stored sketch cut."""
    n = 7
    d0 = W.ModeMat('D', n, 0, 0, np.diag(np.linspace(1.0, 2.0, n)))
    op = W.Operator(3, [n] * 3, [1.0], [[d0, W.identity(n), W.identity(n)]])
    b = W.random_tucker([n] * 3, [1, 1, 1], 53)
    prm_full = W.SolverParams('mln', 4, 0, 8, 6, 1e-12, ktrunc=2, seed=5)
    prm_save = W.SolverParams('mln', 4, 0, 8, 6, 1e-12, ktrunc=2, seed=5, r_sol=3, p_sol=3)
    a = S.mln_sgmres(op, b, prm_full)
    s_ = S.mln_sgmres(op, b, prm_save)
    assert a.iters == s_.iters and np.allclose(a.res_hist, s_.res_hist, rtol=1e-12)
    xa, xs = T.full(a.x), T.full(s_.x)
    assert np.linalg.norm(xa - xs) <= 1e-10 * np.linalg.norm(xa)
    assert max(s_.x.r) <= 3


# ------------------------------------------------------------------------------ Tikhonov + GCV
def test_gcv_function_matches_influence_matrix_definition():
    """The SVD form of the GCV function equals its definition with the explicit influence
    matrix A = M (M^T M + lam^2 I)^-1 M^T (dense), at several lambda."""
    rng = np.random.default_rng(61)
    m_mat = rng.standard_normal((40, 9)) @ np.diag(10.0 ** -np.arange(9))
    b = rng.standard_normal(40)
    u, sig, vt = np.linalg.svd(m_mat, full_matrices=False)
    bhat = u.T @ b
    rho2 = b @ b - bhat @ bhat
    for lam in [1e-6, 1e-3, 1e-1, 1.0]:
        a = m_mat @ np.linalg.solve(m_mat.T @ m_mat + lam ** 2 * np.eye(9), m_mat.T)
        r = b - a @ b
        ref = (r @ r) / np.trace(np.eye(40) - a) ** 2
        assert np.isclose(S.gcv_function(sig, bhat, rho2, 40, lam), ref, rtol=1e-8)


def test_tikhonov_solution_is_the_augmented_least_squares_solution():
    """y_lambda solves min ||[M; lambda I] y - [b; 0]|| (the normal equations of the penalised
    problem), and the chosen lambda minimises GCV over the grid."""
    rng = np.random.default_rng(62)
    m_mat = rng.standard_normal((30, 8)) @ np.diag(10.0 ** -(0.5 * np.arange(8)))
    b = m_mat @ rng.standard_normal(8) + 1e-3 * rng.standard_normal(30)
    y, res, lam = S.ls_tikhonov(m_mat, b)
    aug = np.vstack([m_mat, lam * np.eye(8)])
    ref = np.linalg.lstsq(aug, np.concatenate([b, np.zeros(8)]), rcond=None)[0]
    assert np.allclose(y, ref, rtol=1e-9, atol=1e-12)
    assert np.isclose(res, np.linalg.norm(m_mat @ y - b), rtol=1e-12)
    u, sig, vt = np.linalg.svd(m_mat, full_matrices=False)
    bhat = u.T @ b
    vals = [S.gcv_function(sig, bhat, b @ b - bhat @ bhat, 30, l) for l in S.gcv_grid(sig[0])]
    assert np.isclose(S.gcv_function(sig, bhat, b @ b - bhat @ bhat, 30, lam), min(vals))
    assert 0 < lam < sig[0]


def test_tikhonov_gcv_regularises_a_noisy_ill_posed_solve():
    """Noisy deblurring (n = 12): with GCV-Tikhonov in the least-squares step the error to the
    true solution after many iterations stays near its best value, while the unregularised
    iteration drifts away (semi-convergence)."""
    n = 12
    wl = W.deblur3d(n, 0, None, lam=1e-4, x_rank=2)
    rng = np.random.default_rng(63)
    bf = T.full(wl.b)
    bf = bf + 0.02 * np.linalg.norm(bf) / np.sqrt(bf.size) * rng.standard_normal(bf.shape)
    core = bf.copy()
    facs = [np.eye(n) for _ in range(3)]
    b = W.Tucker(core, facs)
    xt = T.full(wl.x_true)
    errs = {}
    for tik in [False, True]:
        prm = W.SolverParams('gmres', n, 0, 5, 30, 1e-14, round_tol=1e-15, seed=1, tikhonov=tik)
        res = S.rhosvd_gmres(wl.op, b, prm)
        errs[tik] = np.linalg.norm(T.full(res.x) - xt) / np.linalg.norm(xt)
    assert errs[True] < 0.5 * errs[False]


def test_coarse_rhs_compression_removes_semi_convergence():
    """Section 4.3: compressing the noisy data by a truncated HOSVD whose tolerance matches the
    noise level regularises by itself.  Noisy deblurring (n = 32, 2% noise): Algorithm 2 on the
    data as given semi-converges (the error grows from 20 to 40 iterations); on the data
    compressed at tolerance 0.05 the error decreases monotonically and ends below the
    uncompressed run's best."""
    wl = W.deblur3d_noisy(32, 0, None)
    xt = T.full(wl.x_true)
    bf = T.full(wl.b)
    core, facs = R.st_hosvd(bf, 0.05, 32)
    assert np.linalg.norm(T.full(W.Tucker(core, facs)) - bf) <= 0.05 * np.linalg.norm(bf)
    errs = {}
    for label, b in [("raw", wl.b), ("compressed", W.Tucker(core, facs))]:
        errs[label] = []
        for it in [10, 20, 40]:
            prm = W.SolverParams('rhosvd', 32, 128, 5, it, 1e-12, seed=0)
            x = S.rhosvd_sgmres(wl.op, b, prm).x
            errs[label].append(np.linalg.norm(T.full(x) - xt) / np.linalg.norm(xt))
    raw, comp = errs["raw"], errs["compressed"]
    assert raw[2] > raw[1]                       # semi-convergence without compression
    assert comp[0] > comp[1] > comp[2]           # monotone with compression
    assert comp[2] < min(raw)


def test_gcv_counting_projected_rows_regularises_the_sketched_solve():
    """Section 4.3 for the sketched variants: the sketched residual lives in the (k + 1)-dimensional
    span of [M_k, S b].  GCV counting those k + 1 rows, as it counts Algorithm 1's k + 1 Hessenberg
    rows, keeps Algorithm 2's error flat from 20 to 40 iterations on noisy deblurring (n = 32);
    counting the sketch's s = 128 rows (the reading the library implements) lets it grow."""
    wl = W.deblur3d_noisy(32, 0, None)
    xt = T.full(wl.x_true)
    errs = {}
    for rows in ["sketch", "projected"]:
        errs[rows] = []
        for it in [20, 40]:
            prm = W.SolverParams('rhosvd', 32, 128, 5, it, 1e-12, seed=0, tikhonov=True)
            x = S.rhosvd_sgmres(wl.op, wl.b, prm, gcv_rows=rows).x
            errs[rows].append(np.linalg.norm(T.full(x) - xt) / np.linalg.norm(xt))
    assert errs["sketch"][1] > 1.1 * errs["sketch"][0]
    assert errs["projected"][1] < 1.02 * errs["projected"][0]
