"""Parity of each C-ABI entry point against the FP64 oracle on the same seeded inputs.

Sizes span several 32 x 32 GEMM tiles with ragged tails (n = 37, 70, 131), d = 3 and 4,
n smaller than the sketch size, rank-one and rank-deficient inputs."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import mln as OM
from oracle import operators as OO
from oracle import residual as ORS
from oracle import rhosvd as OR
from oracle import tensor as OT
from tests.helpers import rand_tucker, rel_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


# ------------------------------------------------------------------------------ RNG
def test_philox_bitwise(P):
    for seed, sid, first, nb in [(0, 0, 0, 1000), (2 ** 40 + 7, W.stream_id(2, 123456, 3), 5, 777),
                                 (2 ** 64 - 1, 2 ** 64 - 1, 2 ** 32 - 3, 10)]:
        dev = P.tk_philox(seed, sid, first, nb).cpu().numpy().view(np.uint32).reshape(-1, 4)
        ref = W.philox_words(seed, sid, first, nb).astype(np.uint32)
        assert np.array_equal(dev, ref)


@pytest.mark.parametrize("bf16", [False, True])
def test_gaussian_stream(P, bf16):
    for seed, sid, cnt in [(0, W.stream_id(1, 0, 0), 1001), (99, W.stream_id(2, 17, 2), 65536)]:
        dev = P.tk_gaussian(seed, sid, cnt, bf16).cpu().numpy()
        ref = W.gaussian_stream(seed, sid, cnt)
        if bf16:
            ref = W.round_to_bf16(ref)
            # rounding of values within an ulp of a bfloat16 midpoint may differ: allow none here
            assert np.mean(dev != ref) < 1e-4
            assert np.max(np.abs(dev - ref)) <= 2.0 ** -7 * np.max(np.abs(ref))
        else:
            assert np.max(np.abs(dev - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


# ------------------------------------------------------------------------------ matvec
def _ops(n):
    return {"convdiff": W.convdiff3d(n, 0, None).op, "varcoef4d": W.varcoef4d(n, 0, None).op,
            "deblur": W.deblur3d(n, 0, None).op,
            "dense": W.Operator(3, [n] * 3, [0.7, -1.3],
                                [[W.ModeMat('D', n, 0, 0, np.random.default_rng(1).standard_normal((n, n))),
                                  W.identity(n), W.second_difference(n)],
                                 [W.identity(n), W.ModeMat('D', n, 0, 0, np.random.default_rng(2).standard_normal((n, n))),
                                  W.gaussian_blur_band(n)]])}


@pytest.mark.parametrize("name", ["convdiff", "varcoef4d", "deblur", "dense"])
@pytest.mark.parametrize("transpose", [False, True])
def test_apply_operator(P, name, transpose):
    n = 37
    op = _ops(n)[name]
    x = rand_tucker([n] * op.d, [3, 5, 2, 4][:op.d], 3)
    out = P.tk_apply(P.DeviceOperator(op), to_dev(x), transpose)
    ref = OO.apply_op(op, x, transpose)
    for t in range(op.nterms):
        for k in range(op.d):
            a = out[t][k].cpu().numpy()
            b = ref[t].factors[k]
            assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("shape", [([37, 70, 9], [3, 5, 2], [4, 1, 6]), ([131, 5, 33, 12], [2, 3, 4, 5], [5, 2, 3, 1]),
                                   ([64, 64, 64], [32, 32, 32], [32, 32, 32])])
def test_inner(P, shape):
    n, r1, r2 = shape
    x = rand_tucker(n, r1, 4)
    y = rand_tucker(n, r2, 5)
    v = P.tk_inner(to_dev(x), to_dev(y))
    ref = OT.inner(x, y)
    assert abs(v - ref) <= 1e-12 * (OT.norm(x) * OT.norm(y))


@pytest.mark.parametrize("n,r,s", [([37, 70, 9], [3, 5, 2], 64), ([20, 21, 22, 23], [2, 3, 4, 2], 50)])
def test_kron_sketch(P, n, r, s):
    import torch
    x = rand_tucker(n, r, 6)
    S = [W.sketch_matrix(1, 1, 0, k, n[k], s) for k in range(len(n))]
    out = P.tk_kron_sketch(to_dev(x), [P.to_fortran(m, "cuda") for m in S]).cpu().numpy()
    ref = OR.kron_sketch(x, S)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


# ------------------------------------------------------------------------------ RoundSum
def _rs_case(name):
    if name == "exact_lowrank":
        n = [37, 70, 9]
        return [(1.5, rand_tucker(n, [2, 2, 1], 7)), (-2.0, rand_tucker(n, [1, 2, 2], 8))], 6, 5
    if name == "truncating":
        n = [70, 40, 131]
        ts = [(1.0, rand_tucker(n, [6, 6, 6], 9)), (0.5, rand_tucker(n, [5, 6, 4], 10)),
              (-0.25, rand_tucker(n, [6, 3, 6], 11))]
        return ts, 8, 5
    if name == "small_n":
        n = [6, 6, 6]
        return [(1.0, rand_tucker(n, [3, 3, 3], 12)), (1.0, rand_tucker(n, [2, 4, 1], 13))], 6, 5
    if name == "matvec_terms":
        n = 33
        op = W.convdiff3d(n, 0, None).op
        v = rand_tucker([n] * 3, [8, 8, 8], 14, orth=True)
        return [(1.0, t) for t in OO.apply_op(op, v)], 8, 5
    if name == "order4":
        n = [12, 11, 10, 9]
        return [(1.0, rand_tucker(n, [3, 3, 3, 3], 15)), (2.0, rand_tucker(n, [2, 2, 2, 2], 16))], 4, 3
    if name == "point_source":
        # L(b) for the Poisson operator and b = (ones / sqrt(n)) (x) e_1 (x) e_1: factors with
        # identical interior rows and exact zeros, so every range-finder matrix has exact rank
        # 2 and the Householder steps past it act on rounding noise that shrinks step by step
        n = 64
        wl = W.poisson3d_point(n, None, 8, "p")
        return [(1.0, t) for t in OO.apply_op(wl.op, wl.b)], 32, 5
    if name in ("tall_g2", "tall_g3"):
        # exact rank below the cap with a sketch of 50 (69) columns: the ST-HOSVD unfoldings of
        # the 50^3 (69^3) core have 2500 and 2100 (4761, 4140, 3600) rows, so the QR runs on two
        # (three) clusters that exchange their sums through global memory
        n = [90, 80, 100]
        r, R = (14, 45) if name == "tall_g2" else (20, 64)
        ts = [(1.0, rand_tucker(n, [r] * 3, 17)), (-0.5, rand_tucker(n, [r] * 3, 18)),
              (0.25, rand_tucker(n, [r] * 3, 19))]
        return ts, R, 5
    raise KeyError(name)


@pytest.mark.parametrize("case", ["exact_lowrank", "truncating", "small_n", "matvec_terms", "order4", "point_source",
                                  "tall_g2", "tall_g3"])
def test_roundsum(P, case):
    terms, R, p = _rs_case(case)
    n = terms[0][1].n
    d = len(n)
    seed, call, eps = 3, 7, 1e-12
    sk = [W.sketch_matrix(seed, W.STREAM_ROUNDSUM, call, k, n[k], R + p) for k in range(d)]
    ref = OR.roundsum(terms, sk, R, eps)
    opts = P.Options(rank_cap=R, oversample_p=p, round_tol=eps, seed=seed)
    out, ranks = P.tk_roundsum([to_dev(t) for _, t in terms], [c for c, _ in terms], opts, call)
    assert ranks == ref.r
    assert rel_diff(to_host(out), ref) <= 1e-11
    # output factors orthonormal (zero-padded columns aside)
    for u, rk in zip(to_host(out).factors, ranks):
        g = u[:, :rk].T @ u[:, :rk]
        assert np.allclose(g, np.eye(rk), atol=1e-12)


@pytest.mark.parametrize("case,cap,smaller", [("exact_lowrank", 6, True), ("point_source", 32, True),
                                              ("truncating", 8, False), ("matvec_terms", 30, True),
                                              ("order4", 4, False), ("small_n", 6, False)])
def test_adaptive_roundsum(P, case, cap, smaller):
    """RoundSum with the effective-rank sketch size (Section 3.1): the same size as the oracle's
    estimate (so the same Gaussian draws), the same ranks, the same tensor (1e-11).  `smaller`:
    the estimate is below rank_cap + p (exact low-rank sums; the convection-diffusion matvec,
    whose factors span 3 r directions per mode, formed through the transposed V_k)."""
    terms, _, p = _rs_case(case)
    n = terms[0][1].n
    d = len(n)
    seed, call, eps = 3, 7, 1e-12
    sr = OR.effective_sketch_size(terms, p, cap, eps)
    assert (sr < cap + p) == smaller
    sk = [W.sketch_matrix(seed, W.STREAM_ROUNDSUM, call, k, n[k], sr) for k in range(d)]
    ref = OR.roundsum(terms, sk, cap, eps)
    opts = P.Options(rank_cap=cap, oversample_p=p, round_tol=eps, seed=seed, adaptive_rank=True)
    out, ranks = P.tk_roundsum([to_dev(t) for _, t in terms], [c for c, _ in terms], opts, call)
    assert ranks == ref.r
    assert rel_diff(to_host(out), ref) <= 1e-11


# ------------------------------------------------------------------------------ MLN
@pytest.mark.parametrize("n,r,p,ranks", [([30, 31, 32], 5, 4, [[2, 3, 2], [5, 5, 5]]),
                                         ([12, 13, 14, 15], 4, 3, [[3, 3, 3, 3], [1, 1, 1, 1]])])
def test_mln_roundsum(P, n, r, p, ranks):
    terms = [(1.0, rand_tucker(n, ranks[0], 17)), (-0.5, rand_tucker(n, ranks[1], 18))]
    psis = [W.sketch_matrix(5, W.STREAM_KRYLOV, 0, k, n[k], r + p) for k in range(len(n))]
    ref = OM.mln_recovery(OM.mln_sum([(c, OM.mln_sketch(t, psis, r)) for c, t in terms]), psis)
    out = P.tk_mln_roundsum([to_dev(t) for _, t in terms], [c for c, _ in terms],
                            [P.to_fortran(m, "cuda") for m in psis], r, p)
    assert rel_diff(to_host(out), ref) <= 1e-11


# ------------------------------------------------------------------------------ least squares
@pytest.mark.parametrize("s,k", [(64, 1), (64, 37), (256, 150), (13, 12)])
def test_sketched_ls(P, s, k):
    g = np.random.default_rng(s + k)
    M = g.standard_normal((s, k))
    b = g.standard_normal(s)
    y, res = P.tk_sketched_ls(P.to_fortran(M, "cuda"), P.to_fortran(b, "cuda"))
    yr = np.linalg.lstsq(M, b, rcond=None)[0]
    assert np.allclose(y.cpu().numpy(), yr, rtol=1e-10, atol=1e-12)
    assert np.isclose(res.item(), np.linalg.norm(M @ yr - b), rtol=1e-10)


# ------------------------------------------------------------------------------ residual
@pytest.mark.parametrize("transpose", [False, True])
def test_true_residual(P, transpose):
    n = 40
    wl = W.convdiff3d(n, 0, None)
    x = rand_tucker([n] * 3, [5, 5, 5], 19)
    b = rand_tucker([n] * 3, [3, 3, 3], 20)
    v = P.tk_residual(P.DeviceOperator(wl.op), to_dev(x), to_dev(b), transpose)
    assert np.isclose(v, ORS.true_residual(wl.op, x, b, transpose), rtol=1e-11)


@pytest.mark.parametrize("mode", [1, 2])
def test_qr_bounded_wait_reports_and_context_stays_usable(P, mode):
    """Failure detection without a fault: a two-cluster QR with one exchange made to go missing
    (mode 1 inside a cluster, mode 2 between the clusters) gives up after its bounded wait, sets
    the error flag and finishes; the same context then runs a multi-cluster RoundSum to parity."""
    t0 = time.time()
    P.tk_selftest_qr_wait(mode)
    assert time.time() - t0 < 30.0
    with pytest.raises(P.TuckerError):
        P.tk_selftest_qr_wait(3)
    test_roundsum(P, "tall_g2")


def test_invalid_arguments_fail_loudly(P):
    x = rand_tucker([10, 10, 10], [2, 2, 2], 21)
    opts = P.Options(rank_cap=4, oversample_p=5)
    bad = P.DeviceTucker.empty([10, 10, 10], [3, 3, 3])     # ranks must equal rank_cap
    with pytest.raises(P.TuckerError):
        P.tk_roundsum([to_dev(x)], [1.0], opts, 0, out=bad)
    with pytest.raises(P.TuckerError):
        P.tk_roundsum([to_dev(x)], [1.0], P.Options(rank_cap=120, oversample_p=5), 0)
