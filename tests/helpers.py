"""Shared helpers for the GPU parity tests (conversion between the oracle's numpy Tucker
tensors and the library's device tensors, and accurate Tucker-form differences)."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import residual as ORS
from oracle import tensor as OT


def to_dev(t: W.Tucker):
    import paper_2608_11091_b300 as P
    return P.DeviceTucker.from_numpy(t.core, t.factors)


def to_host(x) -> W.Tucker:
    core, facs = x.numpy()
    return W.Tucker(np.asarray(core), [np.asarray(f) for f in facs])


def rel_diff(a: W.Tucker, b: W.Tucker) -> float:
    """||A - B||_F / ||B||_F in Tucker form (QR of concatenated factors: no cancellation)."""
    return ORS.tucker_sum_norm([(1.0, a), (-1.0, b)]) / max(OT.norm(b), 1e-300)


def rand_tucker(n, r, seed, orth=False) -> W.Tucker:
    g = np.random.default_rng(seed)
    fac = [g.standard_normal((a, b)) for a, b in zip(n, r)]
    if orth:
        fac = [np.linalg.qr(f)[0] for f in fac]
    return W.Tucker(g.standard_normal(tuple(r)), fac)
