"""Whole-solver parity: RHOSVD-Tucker sGMRES (Algorithm 2), MLN-Tucker sGMRES (Algorithm 6) and
RHOSVD-Tucker GMRES (Algorithm 1) on the GPU against the FP64 oracle with the same seeded inputs
and the same Gaussian streams.  Bounds: tests/parity.py (1e-10 relative on every stable prefix;
at full length 1e-10 except the listed chaotic cases).  Iteration counts and exit status must
match exactly."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import residual as ORS
from oracle import sgmres as OS
from tests import parity as PT
from tests.helpers import rel_diff, to_dev, to_host
from tests.solver_cases import CASES

pytestmark = pytest.mark.gpu

SENS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "solver_sensitivity.json")))


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


def _run(P, wl, params, transpose=False):
    opts = P.Options.from_params(params, transpose=transpose)
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), opts)
    if params.variant == "rhosvd":
        ref = OS.rhosvd_sgmres(wl.op, wl.b, params, transpose=transpose)
    elif params.variant == "gmres":
        ref = OS.rhosvd_gmres(wl.op, wl.b, params, transpose=transpose)
    else:
        ref = OS.mln_sgmres(wl.op, wl.b, params, transpose=transpose)
    return x, rep, ref


def _check(x, rep, ref, tol=1e-10):
    PT.check(rep, x, ref, tol, tol)


@pytest.mark.parametrize("case", list(CASES))
def test_solver_parity_prefix(P, case):
    """The solve stopped at the case's stable prefix: 1e-10 in the solution and the history."""
    build, params, transpose = CASES[case]
    wl = build()
    params = params or wl.params
    m = SENS[case]["prefix"]
    assert m >= 1
    x, rep, ref = _run(P, wl, PT.with_maxit(params, m), transpose)
    PT.check(rep, x, ref, PT.TOL, PT.TOL)


@pytest.mark.parametrize("case", list(CASES))
def test_solver_parity(P, case):
    """Full length: exact iteration count and status, 1e-10 over the prefix, 1e-10 beyond it
    except for the listed chaotic cases (10x the oracle's own 1e-14 movement)."""
    build, params, transpose = CASES[case]
    wl = build()
    params = params or wl.params
    x_tol, h_tol = PT.full_length_bounds(case, SENS[case])
    x, rep, ref = _run(P, wl, params, transpose)
    PT.check(rep, x, ref, x_tol, h_tol, prefix_hist=SENS[case]["prefix"])


def test_breakdown_on_eigentensor(P):
    n = 24
    i = np.arange(1, n + 1)
    v = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * np.pi / (n + 1))
    lam = 2 - 2 * np.cos(i * np.pi / (n + 1))
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    b = W.Tucker(np.full((1, 1, 1), 3.0), [v[:, [2]], v[:, [0]], v[:, [5]]])
    params = W.SolverParams('rhosvd', 4, 16, 5, 10, 1e-12)
    x, rep = P.tk_solve(P.DeviceOperator(op), to_dev(b), P.Options.from_params(params))
    assert rep.status == "breakdown" and rep.iters == 1
    ref = W.Tucker(b.core / (lam[2] + lam[0] + lam[5]), b.factors)
    assert rel_diff(to_host(x), ref) <= 1e-12


def test_true_residual_of_solution(P):
    wl = W.workload("poisson3d_n32")
    params = W.SolverParams('rhosvd', 12, 64, 5, 60, 1e-9, seed=0)
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), P.Options.from_params(params))
    tr = P.tk_residual(P.DeviceOperator(wl.op), x, to_dev(wl.b))
    assert np.isclose(tr, ORS.true_residual(wl.op, to_host(x), wl.b), rtol=1e-8)


def test_rejects_bad_options(P):
    wl = W.workload("poisson3d_n32")
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    for over in [dict(rank_cap=200), dict(ktrunc=0), dict(sketch_s=1), dict(tol=-1.0)]:
        with pytest.raises(P.TuckerError):
            P.tk_solve(dop, b, P.Options.from_params(wl.params, **over))


def test_gmres_breakdown_on_eigentensor(P):
    """Algorithm 1 on an eigentensor of the 3-D Laplacian: L(V_1) is a multiple of V_1, so W
    vanishes after the first orthogonalisation (lucky breakdown) and x is exact."""
    n = 24
    i = np.arange(1, n + 1)
    v = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * np.pi / (n + 1))
    lam = 2 - 2 * np.cos(i * np.pi / (n + 1))
    op = W.kronecker_sum_operator([W.second_difference(n)], 3)
    b = W.Tucker(np.full((1, 1, 1), 3.0), [v[:, [2]], v[:, [0]], v[:, [5]]])
    params = W.SolverParams('gmres', 4, 0, 5, 10, 1e-12)
    x, rep = P.tk_solve(P.DeviceOperator(op), to_dev(b), P.Options.from_params(params))
    assert rep.status == "breakdown" and rep.iters == 1
    ref = W.Tucker(b.core / (lam[2] + lam[0] + lam[5]), b.factors)
    assert rel_diff(to_host(x), ref) <= 1e-12


@pytest.mark.parametrize("name,iters", [("convdiff3d_n256", 12), ("poisson3d_n1024", 3), ("deblur3d_n128", 6),
                                        ("varcoef4d_n128", 3)])
def test_full_size_prefix_parity(P, name, iters):
    """The headline workloads at full size, first iterations (the oracle's cost bounds the count)."""
    wl = W.workload(name)
    params = wl.params
    params.maxit = iters
    x, rep, ref = _run(P, wl, params)
    _check(x, rep, ref)


def test_gmres_full_size_prefix_parity(P):
    """Algorithm 1 on the convection-diffusion workload at full size (n = 256, 6 terms, cap 32):
    the first iterations, every one orthogonalised against the whole basis."""
    wl = W.workload("convdiff3d_n256")
    params = W.SolverParams('gmres', 32, 0, 5, 8, 1e-6, seed=0)
    x, rep, ref = _run(P, wl, params)
    _check(x, rep, ref)


def test_mln_save_memory_full_size_prefix(P):
    """The 4D variable-coefficient workload (n = 128, r = 24, p = 36) in the memory-efficient
    form with r_sol = p_sol = 12 (the paper's p_sol = r_sol), first iterations at full size; the
    stored sketches shrink from 60^4 to 24^4 and the workspace with them."""
    wl = W.workload("varcoef4d_n128")
    params = wl.params
    params.maxit = 4
    params.r_sol, params.p_sol = 12, 12
    x, rep, ref = _run(P, wl, params)
    _check(x, rep, ref)
    assert rep.out_rank == [12, 12, 12, 12]
