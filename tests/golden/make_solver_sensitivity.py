"""Writes tests/golden/solver_sensitivity.json: for each whole-solver parity case, how far the
FP64 oracle's own output moves when every compression output core (RoundSum, MLN_Recovery)
carries a relative 1e-14 perturbation (five draws, maximum taken).  1e-14 is the rounding
level of the FP64 reductions on the path (length up to ~1e4: sqrt(1e4) x 2^-53), so this
models a second correct FP64 implementation that sums in another order; the GPU parity
tolerance of a case is max(1e-10, 10 x this value).  Calls only the oracle and the input
generators.

Run: python tests/golden/make_solver_sensitivity.py [--mixed | --precond]
(--mixed writes tests/golden/mixed_sensitivity.json for the mixed-precision cases instead;
--precond writes tests/golden/precond_sensitivity.json for the preconditioned cases, 1e-14.)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import residual as ORS  # noqa: E402
from oracle import rhosvd as ORH  # noqa: E402
from oracle import sgmres as OS  # noqa: E402
from oracle import mln as OM  # noqa: E402
from oracle import precond as OP  # noqa: E402
import workloads as W  # noqa: E402
from tests.solver_cases import CASES, MIXED_CASES, PRECOND_CASES  # noqa: E402


def _solve(wl, prm, noise, seed, transpose=False, bf16=False, precond=None):
    rng = np.random.default_rng(seed)
    rs, rec = OS.roundsum, OS.mln_recovery

    def noisy_rs(terms, sk, cap, eps):
        out = rs(terms, sk, cap, eps)
        return W.Tucker(out.core * (1 + noise * rng.standard_normal(out.core.shape)), out.factors)

    def noisy_rec(sk, psis):
        out = rec(sk, psis)
        return W.Tucker(out.core * (1 + noise * rng.standard_normal(out.core.shape)), out.factors)

    if noise:
        OS.roundsum, OS.mln_recovery = noisy_rs, noisy_rec
    try:
        if prm.variant == "rhosvd":
            return OS.rhosvd_sgmres(wl.op, wl.b, prm, transpose=transpose, bf16_sketch=bf16, precond=precond)
        if prm.variant == "gmres":
            return OS.rhosvd_gmres(wl.op, wl.b, prm, transpose=transpose, bf16_sketch=bf16)
        return OS.mln_sgmres(wl.op, wl.b, prm, transpose=transpose)
    finally:
        OS.roundsum, OS.mln_recovery = rs, rec


def _movement(wl, prm, noise, transpose=False, bf16=False, precond=None):
    base = _solve(wl, prm, 0.0, 0, transpose, bf16, precond)
    xs, hs = [], []
    for s in range(5):
        alt = _solve(wl, prm, noise, s + 1, transpose, bf16, precond)
        n = min(len(alt.res_hist), len(base.res_hist))
        hs.append(float(np.max(np.abs(np.array(alt.res_hist[:n]) - np.array(base.res_hist[:n]))
                               / np.array(base.res_hist[:n]))))
        xs.append(ORS.tucker_sum_norm([(1.0, alt.x), (-1.0, base.x)]) / ORS.tucker_sum_norm([(1.0, base.x)]))
    return {"x": max(xs), "hist": max(hs), "iters": base.iters}


def main_mixed():
    """Mixed form: BF16-rounded sketches, 1e-7 perturbations (the FP32-level accuracy of the
    tensor-core range finder) -> tests/golden/mixed_sensitivity.json."""
    out = {}
    for name, (build, prm) in MIXED_CASES.items():
        out[name] = _movement(build(), prm, 1e-7, bf16=True)
        print(name, out[name], flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "mixed_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def main_precond():
    """Preconditioned cases: FP64, 1e-14 perturbations -> tests/golden/precond_sensitivity.json."""
    out = {}
    for name, (build, prm, q) in PRECOND_CASES.items():
        wl = build()
        out[name] = _movement(wl, prm or wl.params, 1e-14, precond=OP.expsum_preconditioner(wl.b.n[0], wl.b.d, q))
        print(name, out[name], flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "precond_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def main():
    out = {}
    for name, (build, prm, transpose) in CASES.items():
        wl = build()
        prm = prm or wl.params
        base = _solve(wl, prm, 0.0, 0, transpose)
        xs, hs = [], []
        for s in range(5):
            alt = _solve(wl, prm, 1e-14, s + 1, transpose)
            n = min(len(alt.res_hist), len(base.res_hist))
            hs.append(float(np.max(np.abs(np.array(alt.res_hist[:n]) - np.array(base.res_hist[:n]))
                                   / np.array(base.res_hist[:n]))))
            xs.append(ORS.tucker_sum_norm([(1.0, alt.x), (-1.0, base.x)]) / ORS.tucker_sum_norm([(1.0, base.x)]))
        out[name] = {"x": max(xs), "hist": max(hs), "iters": base.iters}
        print(name, out[name], flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "solver_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    if "--mixed" in sys.argv:
        main_mixed()
    elif "--precond" in sys.argv:
        main_precond()
    else:
        main()
