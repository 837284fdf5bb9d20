"""Mixed-precision form (precision='mixed'): RoundSum's Gaussian matrices are rounded to BF16
when drawn and the range finder's factor sketches U^T S and the leading MTTKRP contraction run
on tcgen05 tensor cores (BF16 products, FP32 accumulation); everything else stays FP64.

Parity: against the FP64 oracle that draws the same BF16-rounded sketch matrices
(oracle.sgmres.rhosvd_sgmres(..., bf16_sketch=True)); bound 1e-6 relative on the compressed
tensors, the solution and the sketched-residual history, except where the iteration amplifies
perturbations of its compressions: there 10x the oracle's own movement under 1e-7
perturbations of every compression (the FP32-level accuracy of the tensor-core range finder;
tests/golden/mixed_sensitivity.json, written by tests/golden/make_solver_sensitivity.py --mixed)."""
import json
import os
import numpy as np
import pytest

import workloads as W
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


@pytest.mark.parametrize("case", ["exact_lowrank", "truncating", "small_n", "matvec_terms", "order4"])
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


def test_mixed_tensor_core_products_are_fp32_accurate(P):
    """A sum whose multilinear rank is within the sketch: any sketch spans the range, so the
    compressed tensor is exact in FP64 whatever the tensor-core rounding (1e-12)."""
    terms, R, p = _rs_case("exact_lowrank")
    opts = P.Options(rank_cap=R, oversample_p=p, round_tol=1e-14, seed=1, precision="mixed")
    out, _ = P.tk_roundsum([to_dev(t) for _, t in terms], [c for c, _ in terms], opts, 0)
    from oracle import tensor as OT
    exact = OT.concat_sum(terms)
    assert rel_diff(to_host(out), exact) <= 1e-12


SENS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mixed_sensitivity.json")))


def mixed_tolerance(case: str) -> float:
    sn = SENS[case]
    return max(MIXED_TOL, 10.0 * max(sn["x"], sn["hist"]))


@pytest.mark.parametrize("case", list(MIXED_CASES))
def test_mixed_solver_parity(P, case):
    build, prm = MIXED_CASES[case]
    tol = mixed_tolerance(case)
    wl = build()
    x, rep = P.tk_solve(P.DeviceOperator(wl.op), to_dev(wl.b), P.Options.from_params(prm, precision="mixed"))
    ref = OS.rhosvd_sgmres(wl.op, wl.b, prm, bf16_sketch=True)
    assert rep.iters == ref.iters
    h, hr = np.array(rep.res_hist), np.array(ref.res_hist)
    assert np.max(np.abs(h - hr) / hr) <= tol
    assert rel_diff(to_host(x), ref.x) <= tol
