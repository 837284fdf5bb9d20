"""Exponential-sum preconditioner and flexible RHOSVD-Tucker sGMRES (Section 3.4) on the GPU.

The mode matrices E_h = exp(-t_h T_n) built by tk_expsum_laplacian are checked against the
oracle's (sine eigenpairs in numpy) and against the matrix exponential; the preconditioned solver
against the oracle's flexible iteration with the same preconditioner and random streams, with
the bounds of tests/parity.py (1e-10 on the stable prefix and, for these cases, at full length;
tests/golden/precond_sensitivity.json, written by tests/golden/make_solver_sensitivity.py --precond).
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import operators as OO
from oracle import precond as OPC
from oracle import residual as ORS
from oracle import sgmres as OS
from tests import parity as PT
from tests.helpers import rel_diff, to_dev, to_host
from tests.solver_cases import PRECOND_CASES

pytestmark = pytest.mark.gpu

SENS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "precond_sensitivity.json")))


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


@pytest.mark.parametrize("n,q", [(1, 1), (7, 2), (37, 4), (130, 8)])
def test_expsum_mode_matrices(P, n, q):
    dop = P.tk_expsum_laplacian(n, 3, q)
    ref = OPC.expsum_preconditioner(n, 3, q)
    assert dop.nterms == 2 * q + 1
    assert np.allclose(dop.theta_values, ref.theta, rtol=1e-15, atol=0)
    for h in range(2 * q + 1):
        got = dop._keep[0][h * 3].cpu().numpy()
        assert np.max(np.abs(got - ref.mats[h][0].data)) <= 1e-14


def test_expsum_against_matrix_exponential(P):
    from scipy.linalg import expm
    n, q = 24, 3
    dop = P.tk_expsum_laplacian(n, 3, q)
    tn = OO.mode_dense(W.second_difference(n))
    c, t = OPC.expsum_weights(q)
    for h in range(2 * q + 1):
        assert np.allclose(dop._keep[0][h * 3].cpu().numpy(), expm(-t[h] * tn), atol=1e-13)


@pytest.mark.parametrize("case", list(PRECOND_CASES))
def test_preconditioned_solver_parity(P, case):
    build, prm, q = PRECOND_CASES[case]
    wl = build()
    prm = prm or wl.params
    x_tol, h_tol = PT.full_length_bounds(case, SENS[case])
    n = wl.b.n[0]
    x, rep = P.tk_solve_precond(P.DeviceOperator(wl.op), P.tk_expsum_laplacian(n, wl.b.d, q), to_dev(wl.b),
                                P.Options.from_params(prm))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, precond=OPC.expsum_preconditioner(n, wl.b.d, q))
    assert rep.out_rank == list(ref.x.r)
    PT.check(rep, x, ref, x_tol, h_tol, prefix_hist=SENS[case]["prefix"])


@pytest.mark.parametrize("case", list(PRECOND_CASES))
def test_preconditioned_solver_parity_prefix(P, case):
    """The preconditioned solve stopped at its stable prefix: 1e-10 in the solution and history."""
    build, prm, q = PRECOND_CASES[case]
    wl = build()
    prm = PT.with_maxit(prm or wl.params, SENS[case]["prefix"])
    n = wl.b.n[0]
    x, rep = P.tk_solve_precond(P.DeviceOperator(wl.op), P.tk_expsum_laplacian(n, wl.b.d, q), to_dev(wl.b),
                                P.Options.from_params(prm))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, precond=OPC.expsum_preconditioner(n, wl.b.d, q))
    PT.check(rep, x, ref, PT.TOL, PT.TOL)


@pytest.mark.parametrize("case", list(PRECOND_CASES))
def test_expsum_sine_basis_solver_parity(P, case):
    """tk_solve_expsum (the preconditioner applied in the sine eigenbasis, RoundSum with rotated
    sketches) against the oracle's flexible iteration with the dense E_h: equal in exact
    arithmetic, so the bounds are those of the dense path (prefix and full length)."""
    build, prm, q = PRECOND_CASES[case]
    wl = build()
    prm = prm or wl.params
    n = wl.b.n[0]
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, precond=OPC.expsum_preconditioner(n, wl.b.d, q))
    x, rep = P.tk_solve_expsum(P.DeviceOperator(wl.op), q, to_dev(wl.b), P.Options.from_params(prm))
    x_tol, h_tol = PT.full_length_bounds(case, SENS[case])
    PT.check(rep, x, ref, x_tol, h_tol, prefix_hist=SENS[case]["prefix"])
    pm = PT.with_maxit(prm, SENS[case]["prefix"])
    ref = OS.rhosvd_sgmres(wl.op, wl.b, pm, precond=OPC.expsum_preconditioner(n, wl.b.d, q))
    x, rep = P.tk_solve_expsum(P.DeviceOperator(wl.op), q, to_dev(wl.b), P.Options.from_params(pm))
    PT.check(rep, x, ref, PT.TOL, PT.TOL)


def test_expsum_sine_basis_transposed_and_mixed(P):
    """The adjoint (transposed) solve and the mixed form through the sine-basis path: transposed
    against the oracle's transposed flexible iteration (1e-10); mixed reaches the FP64 solve's
    true residual to within 2x."""
    wl = W.poisson3d(24, 2, 7, None, "p24")
    prm = W.SolverParams('rhosvd', 12, 48, 5, 8, 1e-9, seed=6)
    pc = OPC.expsum_preconditioner(24, 3, 6)
    dop = P.DeviceOperator(wl.op)
    p4 = PT.with_maxit(prm, 3)      # residuals still far above their rounding floor
    x, rep = P.tk_solve_expsum(dop, 6, to_dev(wl.b), P.Options.from_params(p4, transpose=True))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, p4, transpose=True, precond=pc)
    PT.check(rep, x, ref, PT.TOL, PT.TOL)
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, precond=pc)
    xm, repm = P.tk_solve_expsum(dop, 6, to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    tr_m, tr_f = P.tk_residual(dop, xm, to_dev(wl.b)), ORS.true_residual(wl.op, ref.x, wl.b)
    assert tr_m <= 2 * tr_f + 1e-9


def test_preconditioned_point_source_true_residual(P):
    """The paper's Poisson setting (n = 1000, rank-1 point-source right-hand side): the flexible
    solver stops on the sketched residual and the true relative residual agrees with it."""
    wl = W.workload("poisson3d_point_n1000")
    dop = P.DeviceOperator(wl.op)
    b = to_dev(wl.b)
    x, rep = P.tk_solve_precond(dop, P.tk_expsum_laplacian(1000, 3, wl.extra["precond_q"]), b,
                                P.Options.from_params(wl.params))
    assert rep.status == "converged"
    true = P.tk_residual(dop, x, b)
    assert true < 3 * wl.params.tol
    assert np.isclose(true, ORS.true_residual(wl.op, to_host(x), wl.b), rtol=1e-6)


def test_precond_rejects_mln(P):
    wl = W.poisson3d(12, 1, 0, None, "p12")
    opts = P.Options(variant="mln", rank_cap=4, oversample_p=4, maxit=3)
    with pytest.raises(P.TuckerError):
        P.tk_solve_precond(P.DeviceOperator(wl.op), P.tk_expsum_laplacian(12, 3, 2), to_dev(wl.b), opts)
