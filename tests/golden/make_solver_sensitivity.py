"""Writes tests/golden/solver_sensitivity.json: for each whole-solver parity case, how far the
FP64 oracle's own output moves when every compression output core (RoundSum, MLN_Recovery)
carries a relative perturbation (five draws, maximum taken): "x"/"hist" at 1e-14 (the
rounding level of the FP64 reductions on the path, length up to ~1e4: sqrt(1e4) x 2^-53, a
second correct FP64 implementation summing in another order) and "x15"/"hist15" at 1e-15, for
the full iteration count; and "prefix", the largest iteration count m whose 1e-14 movement of
the history (iterations 1..m) and of the solution of the solve stopped after m iterations both
stay <= 1e-11 ("x_prefix" is that solution movement).  The GPU parity tests hold 1e-10 on the
prefix; the full-length comparison of a case whose movement exceeds that is listed, with its
numbers, in the design notes.  Calls only the oracle and the input generators.

Run: python tests/golden/make_solver_sensitivity.py [--mixed | --precond]
(--mixed writes tests/golden/mixed_sensitivity.json for the mixed-precision cases instead;
--precond writes tests/golden/precond_sensitivity.json for the preconditioned cases, 1e-14.)
"""
import json
import os
import sys

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

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


def _one_mixed(name):
    build, prm = MIXED_CASES[name]
    return name, case_entry(build(), prm, noise=1e-12, noise2=1e-13, threshold=1e-7, bf16=True)


def main_mixed():
    """Mixed form: BF16-rounded sketches, 1e-12 perturbations of every compression (the accuracy
    of the sliced tensor-core products, ~2^-40 per product; "x15"/"hist15" hold the 1e-13
    movement here) and the longest prefix whose movement stays <= 1e-7, a tenth of the mixed
    bound 1e-6 -> tests/golden/mixed_sensitivity.json."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    out = {}
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn")) as ex:
        for name, ent in ex.map(_one_mixed, list(MIXED_CASES)):
            out[name] = ent
            print(name, ent, flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "mixed_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


def _one_precond(name):
    build, prm, q = PRECOND_CASES[name]
    wl = build()
    return name, case_entry(wl, prm or wl.params, precond=OP.expsum_preconditioner(wl.b.n[0], wl.b.d, q))


def main_precond():
    """Preconditioned cases: FP64, as main() -> tests/golden/precond_sensitivity.json."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    out = {}
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn")) as ex:
        for name, ent in ex.map(_one_precond, list(PRECOND_CASES)):
            out[name] = ent
            print(name, ent, flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "precond_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


PREFIX_MOVEMENT = 1e-11


def _per_iter(wl, prm, noise, transpose, precond=None, bf16=False):
    """(x movement, per-iteration history movement, base result) under `noise`, five draws."""
    base = _solve(wl, prm, 0.0, 0, transpose, bf16=bf16, precond=precond)
    xs, hs = [], []
    for s in range(5):
        alt = _solve(wl, prm, noise, s + 1, transpose, bf16=bf16, precond=precond)
        n = min(len(alt.res_hist), len(base.res_hist))
        hs.append(np.abs(np.array(alt.res_hist[:n]) - np.array(base.res_hist[:n])) / np.array(base.res_hist[:n]))
        xs.append(ORS.tucker_sum_norm([(1.0, alt.x), (-1.0, base.x)]) / ORS.tucker_sum_norm([(1.0, base.x)]))
    n = min(len(h) for h in hs)
    return max(xs), np.max(np.stack([h[:n] for h in hs]), axis=0), base


def case_entry(wl, prm, transpose=False, precond=None, noise=1e-14, noise2=1e-15, threshold=PREFIX_MOVEMENT,
               bf16=False):
    import copy
    x14, h14, base = _per_iter(wl, prm, noise, transpose, precond, bf16)
    x15, h15, _ = _per_iter(wl, prm, noise2, transpose, precond, bf16)
    ent = {"x": x14, "hist": float(np.max(h14)), "x15": x15, "hist15": float(np.max(h15)), "iters": base.iters}
    # longest prefix m with history movement <= threshold on 1..m and solution movement of the
    # m-iteration solve <= threshold
    ok = np.cumprod(h14 <= threshold).astype(bool)
    m = int(np.sum(ok))
    while m >= 1:
        p2 = copy.copy(prm)
        p2.maxit = m
        xm, _, _ = _per_iter(wl, p2, noise, transpose, precond, bf16)
        if xm <= threshold:
            ent["prefix"], ent["x_prefix"] = m, xm
            break
        m = m - 1 if m <= 4 else int(m * 0.75)
    else:
        ent["prefix"], ent["x_prefix"] = 0, None
    return ent


def _one(name):
    build, prm, transpose = CASES[name]
    wl = build()
    return name, case_entry(wl, prm or wl.params, transpose)


def main():
    """Cases in parallel worker processes (spawned; one BLAS thread each); names given on the
    command line restrict the run to those cases and merge them into the existing file."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    out = {}
    only = [a for a in sys.argv[1:] if not a.startswith("--")]
    path = os.path.join(ROOT, "tests", "golden", "solver_sensitivity.json")
    if only and os.path.exists(path):
        out = json.load(open(path))
    names = [n for n in CASES if not only or n in only]
    with ProcessPoolExecutor(max_workers=os.cpu_count(), mp_context=mp.get_context("spawn")) as ex:
        for name, ent in ex.map(_one, names):
            out[name] = ent
            print(name, ent, flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "solver_sensitivity.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    if "--mixed" in sys.argv:
        main_mixed()
    elif "--precond" in sys.argv:
        main_precond()
    else:
        main()
