"""Suspend, save, load and resume a solve (tk_checkpoint_save / tk_checkpoint_load).

A solve stopped after k iterations (opts.stop_after) keeps the loop state of Algorithms 1, 2 or 6
in the handle; the state is copied out as bytes, loaded back (possibly after other solves have
used the handle) and continued with opts.resume.  The continued solve must be the uninterrupted
one bit for bit: same iteration count, status and residual history, and the same solution core
and factors to the last bit.  Also: a resume with other options is refused, and so is a resume
without a suspended solve."""
import copy

import numpy as np
import pytest

import workloads as W
from tests.helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_11091_b300 as P
    return P


CASES = {
    "sgmres_convdiff_n30": (lambda: W.convdiff3d(30, 4, None), W.SolverParams('rhosvd', 10, 64, 5, 14, 1e-12, seed=9),
                            None, (4, 5)),
    "sgmres_precond_poisson_n20": (lambda: W.poisson3d(20, 1, 3, None, "p20"),
                                   W.SolverParams('rhosvd', 12, 64, 5, 8, 1e-13, seed=4), 4, (2, 3)),
    "sgmres_expsum_poisson_n20": (lambda: W.poisson3d(20, 1, 3, None, "p20"),
                                  W.SolverParams('rhosvd', 12, 64, 5, 8, 1e-13, seed=4), -4, (2, 3)),
    "gmres_convdiff_n30": (lambda: W.convdiff3d(30, 4, None), W.SolverParams('gmres', 10, 0, 5, 12, 1e-12, seed=9),
                           None, (3, 4)),
    "mln_varcoef4d_n16": (lambda: W.varcoef4d(16, 1, None), W.SolverParams('mln', 6, 0, 6, 10, 1e-12, seed=7),
                          None, (3, 2)),
    "mln_save_convdiff_n40": (lambda: W.convdiff3d(40, 2, None),
                              W.SolverParams('mln', 10, 0, 12, 14, 1e-12, ktrunc=3, seed=8, r_sol=8, p_sol=8),
                              None, (5, 3)),
}


def _solve(P, dop, pc, b, opts):
    if pc is None:
        return P.tk_solve(dop, b, opts)
    if isinstance(pc, int):            # the sine-basis exponential sum of q terms
        return P.tk_solve_expsum(dop, pc, b, opts)
    return P.tk_solve_precond(dop, pc, b, opts)


@pytest.mark.parametrize("case", list(CASES))
def test_resume_is_bit_for_bit(P, case):
    import torch
    build, prm, q, (k1, k2) = CASES[case]
    wl = build()
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    pc = None if not q else (-q if q < 0 else P.tk_expsum_laplacian(wl.b.n[0], wl.b.d, q))
    opts = P.Options.from_params(prm)
    x_ref, rep_ref = _solve(P, dop, pc, b, opts)
    assert rep_ref.iters > k1 + k2, "the case must run past both suspensions"

    o1 = copy.copy(opts)
    o1.stop_after = k1
    _, r1 = _solve(P, dop, pc, b, o1)
    assert r1.status == "suspended" and r1.iters == k1
    state1 = P.tk_checkpoint_save()
    # the handle is used by an unrelated solve in between; the state comes back from bytes
    other = W.poisson3d(12, 1, 5, None, "p12")
    P.tk_solve(P.DeviceOperator(other.op), to_dev(other.b), P.Options(rank_cap=4, sketch_s=16, maxit=3))
    P.tk_checkpoint_load(state1)
    o2 = copy.copy(opts)
    o2.stop_after, o2.resume = k2, True
    _, r2 = _solve(P, dop, pc, b, o2)
    assert r2.status == "suspended" and r2.iters == k1 + k2
    state2 = P.tk_checkpoint_save()
    P.tk_checkpoint_load(state2)
    o3 = copy.copy(opts)
    o3.resume = True
    x, rep = _solve(P, dop, pc, b, o3)
    torch.cuda.synchronize()
    assert rep.status == rep_ref.status and rep.iters == rep_ref.iters
    assert rep.res_hist == rep_ref.res_hist
    assert torch.equal(x.core, x_ref.core)
    for u, v in zip(x.factors, x_ref.factors):
        assert torch.equal(u, v)


def test_resume_refuses_other_options_and_missing_state(P):
    wl = W.convdiff3d(20, 1, None)
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    prm = W.SolverParams('rhosvd', 8, 48, 5, 10, 1e-12, seed=1)
    o = P.Options.from_params(prm, stop_after=2)
    _, r = P.tk_solve(dop, b, o)
    assert r.status == "suspended"
    state = P.tk_checkpoint_save()
    bad = P.Options.from_params(prm, resume=True, rank_cap=9)
    with pytest.raises(P.TuckerError):
        P.tk_solve(dop, b, bad)
    P.tk_checkpoint_load(state)
    _, r = P.tk_solve(dop, b, P.Options.from_params(prm, resume=True))
    assert r.status in ("converged", "not_converged")
    with pytest.raises(P.TuckerError):      # the state was consumed by the resume
        P.tk_solve(dop, b, P.Options.from_params(prm, resume=True))
    with pytest.raises(P.TuckerError):
        P.tk_checkpoint_load(b"not a checkpoint of this library at all")


def test_true_residual_in_report(P):
    from oracle import residual as ORS
    from tests.helpers import to_host
    wl = W.convdiff3d(24, 3, None)
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    x, rep = P.tk_solve(dop, b, P.Options.from_params(W.SolverParams('rhosvd', 8, 48, 5, 12, 1e-10, seed=2),
                                                     true_residual=True))
    assert rep.true_res > 0
    assert np.isclose(rep.true_res, ORS.true_residual(wl.op, to_host(x), wl.b), rtol=1e-8)


def test_workspace_limit_gives_enomem_and_leaves_the_handle_usable(P):
    """Allocation failure injected through the handle's workspace cap: the solve fails with
    TK_ENOMEM (a status, no partial result is trusted) and the same handle solves again once
    the cap is lifted."""
    import paper_2608_11091_b300._lib as L
    wl = W.convdiff3d(24, 3, None)
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    opts = P.Options.from_params(W.SolverParams('rhosvd', 8, 48, 5, 6, 1e-10, seed=2))
    h = P.handle()
    # a fresh handle holds no workspace yet: a 16 KiB cap is below what this solve needs
    fresh = P.Handle(h.device)
    try:
        rc = fresh.lib.tk_set_workspace_limit(fresh.h, 16 << 10)
        assert rc == 0
        x = P.DeviceTucker.empty(b.n, [opts.rank_cap] * b.d)
        rep = L.tk_report()
        opc, bc, oc, xc = dop.c(), b.c(), opts.c(), x.c()
        import ctypes
        rc = fresh.lib.tk_solve(fresh.h, ctypes.byref(opc), ctypes.byref(bc), ctypes.byref(oc), ctypes.byref(xc),
                                ctypes.byref(rep), None)
        assert rc == L.TK_ENOMEM
        assert b"limit" in fresh.lib.tk_last_error(fresh.h)
        assert fresh.lib.tk_set_workspace_limit(fresh.h, 0) == 0
        rc = fresh.lib.tk_solve(fresh.h, ctypes.byref(opc), ctypes.byref(bc), ctypes.byref(oc), ctypes.byref(xc),
                                ctypes.byref(rep), None)
        assert rc >= 0 and rep.iters == 6
    finally:
        fresh.close()


@pytest.mark.parametrize("where", ["core", "factor", "mode_matrix"])
def test_non_finite_inputs_return_an_error_status(P, where):
    """NaN or Inf in the right-hand side's core, one of its factors, or a mode matrix of the
    operator: the solve returns an error status and the handle keeps working."""
    wl = W.convdiff3d(20, 1, None)
    b_np = copy.deepcopy(wl.b)
    op = copy.deepcopy(wl.op)
    if where == "core":
        b_np.core[1, 0, 0] = np.nan
    elif where == "factor":
        b_np.factors[2][5, 1] = np.inf
    else:
        m = op.mats[0][0]              # term 0: the scaled second difference in mode 1 (banded)
        assert m.kind == 'B'
        data = np.array(m.data, dtype=np.float64)
        data[1, 7] = np.nan
        op.mats[0][0] = W.ModeMat(m.kind, m.n, m.kl, m.ku, data)
    prm = W.SolverParams('rhosvd', 8, 48, 5, 6, 1e-10, seed=1)
    with pytest.raises(P.TuckerError, match="not finite"):
        P.tk_solve(P.DeviceOperator(op), to_dev(b_np), P.Options.from_params(prm))
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), P.Options.from_params(prm))
    assert rep.iters == 6 and np.isfinite(rep.sketched_res)


def test_concurrent_solves_equal_the_serial_ones(P):
    """tk_solve_concurrent: a forward and a transposed sine-basis solve and a plain solve run at
    the same time on three handles and streams give, bit for bit, what each gives alone; a job with
    bad options fails with its own status while the others complete."""
    import torch
    wl = W.poisson3d(24, 2, 7, None, "p24")
    dop, b = P.DeviceOperator(wl.op), to_dev(wl.b)
    prm = W.SolverParams('rhosvd', 12, 48, 5, 6, 1e-10, seed=6)
    o = P.Options.from_params(prm)
    ot = P.Options.from_params(prm, transpose=True)
    jobs = [dict(op=dop, b=b, opts=o, expsum_q=6), dict(op=dop, b=b, opts=ot, expsum_q=6), dict(op=dop, b=b, opts=o)]
    got = P.tk_solve_concurrent(jobs)
    ref = [P.tk_solve_expsum(dop, 6, b, o), P.tk_solve_expsum(dop, 6, b, ot), P.tk_solve(dop, b, o)]
    torch.cuda.synchronize()
    for (x, rep), (xr, rr) in zip(got, ref):
        assert rep.iters == rr.iters and rep.res_hist == rr.res_hist
        assert torch.equal(x.core, xr.core) and all(torch.equal(u, v) for u, v in zip(x.factors, xr.factors))
    bad = P.Options.from_params(prm, rank_cap=200)
    with pytest.raises(P.TuckerError, match="job 1"):
        P.tk_solve_concurrent([dict(op=dop, b=b, opts=o), dict(op=dop, b=b, opts=bad)])
