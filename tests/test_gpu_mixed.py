"""Mixed-precision form (precision='mixed').

What runs on tensor cores: the range finder of every RoundSum (factor sketches U^T S with
RoundSum's Gaussian matrices rounded to BF16 when drawn, the MTTKRP, rotated sketches), the whole
preconditioner application in the flexible form (any Z_k is a valid preconditioned direction), and
in MLN-Tucker sGMRES the sketch of L(V_i).  Each product uses the sliced tensor-core GEMM (FP64
operands cut into five exact BF16 digit planes, FP32 accumulation exact per chunk, about 2^-40
relative error per product).  Everything that builds the Krylov tensors and the solution (the
FP64 projections, the ST-HOSVD, QR, SVD, least squares, inner products) stays FP64.

Parity: against the FP64 oracle drawing the same BF16-rounded sketch matrices
(oracle.sgmres.rhosvd_sgmres(..., bf16_sketch=True)), MLN against the plain FP64 oracle: 1e-6
relative on the compressed tensors, on the solution and on every sketched residual, at full length
(the oracle moves by at most ~1e-10 under 1e-12 perturbations of every compression,
tests/golden/mixed_sensitivity.json, written by tests/golden/make_solver_sensitivity.py --mixed).
In the flexible preconditioned form the whole preconditioner application runs on tensor cores:
its Z_k carries ~1e-12 relative error, a valid flexible direction but a different one, and the
residual sees that difference through L (condition number ~4e5 at n = 1024), so there the
sketched residual values (already relative to ||b_s||) are held to 1e-6 absolute, the solution to
1e-6 relative.  The error of every mixed result against the plain FP64 oracle (other sketch
matrices, so the randomized compression differs at its own truncation level) is checked
separately: the mixed solve reaches the FP64 solve's true residual to within 2x or 1e-6."""
import copy
import json
import os
import numpy as np
import pytest

import workloads as W
from oracle import precond as OPC
from oracle import residual as ORS
from oracle import rhosvd as OR
from oracle import sgmres as OS
from tests.helpers import rand_tucker, rel_diff, to_dev, to_host
from tests.solver_cases import MIXED_CASES
from tests.test_gpu_kernels import _rs_case

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


@pytest.mark.parametrize("case", ["exact_lowrank", "truncating", "small_n", "matvec_terms", "order4",
                                  "tall_g2", "tall_g3"])
def test_mixed_roundsum(P, case):
    terms, R, p = _rs_case(case)
    n = terms[0][1].n
    seed, call, eps = 3, 7, 1e-12
    sk = [W.sketch_matrix(seed, W.STREAM_ROUNDSUM, call, k, n[k], R + p, bf16=True) for k in range(len(n))]
    ref = OR.roundsum(terms, sk, R, eps)
    opts = P.Options(rank_cap=R, oversample_p=p, round_tol=eps, seed=seed, precision="mixed")
    out, ranks = P.tk_roundsum([to_dev(t) for _, t in terms], [c for c, _ in terms], opts, call)
    assert ranks == ref.r
    assert rel_diff(to_host(out), ref) <= MIXED_TOL


def test_mixed_tensor_core_products_are_accurate(P):
    """A sum whose multilinear rank is within the sketch: any sketch spans the range, so the
    compressed tensor is exact but for the products' own error.  Every mode product of the mixed
    compression runs on tensor cores with operands sliced to ~40 bits (about 2^-40 of the row and
    column maxima per reduction index): the result must be exact to 1e-10."""
    terms, R, p = _rs_case("exact_lowrank")
    opts = P.Options(rank_cap=R, oversample_p=p, round_tol=1e-14, seed=1, precision="mixed")
    out, _ = P.tk_roundsum([to_dev(t) for _, t in terms], [c for c, _ in terms], opts, 0)
    from oracle import tensor as OT
    exact = OT.concat_sum(terms)
    assert rel_diff(to_host(out), exact) <= 1e-10


SENS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mixed_sensitivity.json")))


def _compare(x, rep, ref, tol=MIXED_TOL, hist_absolute=False):
    assert rep.iters == ref.iters
    h, hr = np.array(rep.res_hist), np.array(ref.res_hist)
    dev = np.abs(h - hr) if hist_absolute else np.abs(h - hr) / hr
    assert np.max(dev) <= tol, dev
    assert rel_diff(to_host(x), ref.x) <= tol


@pytest.mark.parametrize("case", list(MIXED_CASES))
def test_mixed_solver_parity(P, case):
    build, prm = MIXED_CASES[case]
    assert SENS[case]["prefix"] == SENS[case]["iters"], "stable over the whole solve"
    wl = build()
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    _compare(x, rep, OS.rhosvd_sgmres(wl.op, wl.b, prm, bf16_sketch=True))


@pytest.mark.parametrize("case", list(MIXED_CASES))
def test_mixed_error_against_the_fp64_oracle(P, case):
    """The mixed result against the plain FP64 oracle: the true residual it reaches is the FP64
    solve's to within 2x (or 1e-6 absolute): the reduced-precision products cost no accuracy."""
    build, prm = MIXED_CASES[case]
    wl = build()
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm)
    tr_mixed = ORS.true_residual(wl.op, to_host(x), wl.b)
    tr_fp64 = ORS.true_residual(wl.op, ref.x, wl.b)
    assert tr_mixed <= 2.0 * tr_fp64 + 1e-6, (tr_mixed, tr_fp64)


@pytest.mark.parametrize("name,prm", [
    ("mln_varcoef4d_n16", W.SolverParams('mln', 6, 0, 6, 10, 1e-8, seed=7)),
    # chaotic in FP64 already (the oracle moves 1e-9 under 1e-14 perturbations at 16
    # iterations): the stable prefix
    ("mln_convdiff_n40", W.SolverParams('mln', 10, 0, 12, 8, 1e-8, seed=8)),
])
def test_mixed_mln_parity(P, name, prm):
    """MLN-Tucker sGMRES (Algorithm 6) in the mixed form: the sketch of L(V_i) on tensor cores,
    against the FP64 oracle (same Psi), 1e-6."""
    wl = W.varcoef4d(16, 1, None) if name.startswith("mln_varcoef") else W.convdiff3d(40, 2, None)
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    _compare(x, rep, OS.mln_sgmres(wl.op, wl.b, prm))


@pytest.mark.parametrize("n,q,maxit,cap", [(32, 8, 6, 12), (64, 16, 4, 24)])
def test_mixed_expsum_parity(P, n, q, maxit, cap):
    """The flexible solve with the sine-basis exponential-sum preconditioner in the mixed form
    (the whole preconditioner application on tensor cores) against the oracle's flexible
    iteration with the dense E_h and the same BF16-rounded sketches, 1e-6."""
    wl = W.workload("poisson3d_n32") if n == 32 else W.workload("poisson3d_smooth_n64")
    prm = W.SolverParams('rhosvd', cap, 64, 5, maxit, 1e-9, seed=3)
    x, rep = P.tk_solve_expsum(P.DeviceOperator(wl.op), q, to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, bf16_sketch=True, precond=OPC.expsum_preconditioner(n, 3, q))
    _compare(x, rep, ref, hist_absolute=True)


def test_mixed_full_size_poisson_n1024_prefix(P):
    """The benchmark workload at full size (n = 1024, smooth rank-8 right-hand side, cap 64,
    s = 256, q = 16) in the mixed form, its first two iterations against the oracle (1e-6)."""
    wl = W.workload("poisson3d_n1024")
    prm = copy.copy(wl.params)
    prm.maxit = 2
    x, rep = P.tk_solve_expsum(P.DeviceOperator(wl.op), 16, to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, bf16_sketch=True, precond=OPC.expsum_preconditioner(1024, 3, 16))
    _compare(x, rep, ref, hist_absolute=True)
