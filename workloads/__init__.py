"""Seeded synthetic inputs for the Tucker-format sketched GMRES solvers.

This module is shared by the FP64 oracle, the tests and the benchmark.  It holds
problem definitions and random streams only, none of the solvers' arithmetic:

* the mode matrices of the separable operators L = sum_t theta_t A_1^(t) x ... x A_d^(t)
  (Section 1, Eq. (1.2)) for the five synthetic workloads, stored in LAPACK band
  layout or dense column-major layout;
* seeded Tucker right-hand sides (Section 2.3: a core plus one factor per mode);
* the counter-based Gaussian stream the solvers draw their sketch matrices from.

Gaussian stream.  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11) maps a 128-bit counter and a 64-bit key to
four 32-bit words.  Two words give a 53-bit integer m, u1 = (m + 1) 2^-53 lies in
(0, 1]; the other two give u2 = m' 2^-53 in [0, 1).  Box-Muller turns (u1, u2)
into z0 = sqrt(-2 ln u1) cos(2 pi u2) and z1 = sqrt(-2 ln u1) sin(2 pi u2).
Element e of stream (seed, stream_id) comes from counter
(e // 2 mod 2^32, e // 2 >> 32, stream_id mod 2^32, stream_id >> 32) under key
(seed mod 2^32, seed >> 32); even e takes z0, odd e takes z1.  The CUDA library
implements the same published generator on its own; tests compare the two.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ----------------------------------------------------------------------------------
# Philox4x32-10 + Box-Muller
# ----------------------------------------------------------------------------------
_M32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)

# stream_id = (purpose << 48) | (call << 8) | mode
STREAM_KRYLOV = 1      # Krylov sketch S_k (Alg. 2) or Nystrom sketch Psi_k (Alg. 6)
STREAM_ROUNDSUM = 2    # Gaussian matrices of one RoundSum call (Section 3.1)


def stream_id(purpose: int, call: int, mode: int) -> int:
    """64-bit stream identifier of one sketch matrix."""
    assert 0 <= mode < 256 and 0 <= call < (1 << 40) and 0 <= purpose < (1 << 16)
    return (purpose << 48) | (call << 8) | mode


def philox4x32_10(c: Sequence[np.ndarray], k: Tuple[int, int]) -> List[np.ndarray]:
    """Ten Philox4x32 rounds on arrays of 32-bit counters (held in uint64)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _M32 for x in c)
    k0 = np.uint64(k[0]) & _M32
    k1 = np.uint64(k[1]) & _M32
    for r in range(10):
        if r:
            k0 = (k0 + _PHILOX_W0) & _M32
            k1 = (k1 + _PHILOX_W1) & _M32
        p0 = c0 * _PHILOX_M0          # 32x32 -> 64 bit, exact in uint64
        p1 = c2 * _PHILOX_M1
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return [c0, c1, c2, c3]


def philox_words(seed: int, sid: int, first_block: int, nblocks: int) -> np.ndarray:
    """Raw 32-bit words of counter blocks [first_block, first_block + nblocks), shape (nblocks, 4)."""
    b = np.arange(first_block, first_block + nblocks, dtype=np.uint64)
    sid = int(sid)
    seed = int(seed)
    c = [b & _M32, b >> np.uint64(32),
         np.full_like(b, sid & 0xFFFFFFFF), np.full_like(b, (sid >> 32) & 0xFFFFFFFF)]
    out = philox4x32_10(c, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    return np.stack(out, axis=1)


def gaussian_stream(seed: int, sid: int, count: int) -> np.ndarray:
    """First `count` N(0,1) values (float64) of stream (seed, sid)."""
    nblk = (count + 1) // 2
    w = philox_words(seed, sid, 0, nblk).astype(np.uint64)
    m1 = (w[:, 0] >> np.uint64(5)) * np.uint64(1 << 26) + (w[:, 1] >> np.uint64(6))
    m2 = (w[:, 2] >> np.uint64(5)) * np.uint64(1 << 26) + (w[:, 3] >> np.uint64(6))
    u1 = (m1.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = m2.astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * nblk, dtype=np.float64)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 value (ties to even), returned as float64.

    bfloat16 keeps 8 significant bits and the float32 exponent range; the sketch
    values are O(1) so the result is always a normal number.
    """
    x = np.asarray(x, dtype=np.float64)
    bits = x.view(np.uint64)
    drop = np.uint64(52 - 7)                  # mantissa bits removed
    half = np.uint64(1) << (drop - np.uint64(1))
    lsb = (bits >> drop) & np.uint64(1)
    rounded = (bits + half - np.uint64(1) + lsb) >> drop << drop
    out = rounded.view(np.float64).copy()
    out[x == 0] = 0.0
    return out


def sketch_matrix(seed: int, purpose: int, call: int, mode: int, n: int, s: int,
                  bf16: bool = False) -> np.ndarray:
    """Gaussian n x s matrix, column-major fill: entry (i, j) is stream element j*n + i."""
    g = gaussian_stream(seed, stream_id(purpose, call, mode), n * s)
    if bf16:
        g = round_to_bf16(g)
    return g.reshape((s, n)).T.copy()


# ----------------------------------------------------------------------------------
# Operators: lists of per-mode matrix tuples (Section 1, Eq. (1.2))
# ----------------------------------------------------------------------------------
@dataclass
class ModeMat:
    """One mode matrix A in R^{n x n}.

    kind 'I': identity, data None.
    kind 'B': banded with kl sub- and ku super-diagonals, LAPACK band layout:
              data[ku + i - j, j] = A[i, j], array shape (kl + ku + 1, n).
    kind 'D': dense, data[i, j] = A[i, j], array shape (n, n).
    """
    kind: str
    n: int
    kl: int = 0
    ku: int = 0
    data: Optional[np.ndarray] = None


@dataclass
class Operator:
    """L(X) = sum_t theta[t] * X x_1 A_1^(t) ... x_d A_d^(t)."""
    d: int
    n: List[int]
    theta: List[float]
    mats: List[List[ModeMat]]          # mats[t][k]

    @property
    def nterms(self) -> int:
        return len(self.theta)


@dataclass
class Tucker:
    """Tucker tensor: core G (shape r_1 x ... x r_d) and factors U_k (n_k x r_k)."""
    core: np.ndarray
    factors: List[np.ndarray]

    @property
    def d(self) -> int:
        return len(self.factors)

    @property
    def n(self) -> List[int]:
        return [u.shape[0] for u in self.factors]

    @property
    def r(self) -> List[int]:
        return [u.shape[1] for u in self.factors]


def identity(n: int) -> ModeMat:
    return ModeMat('I', n)


def tridiag(n: int, sub: float, diag: float, sup: float) -> ModeMat:
    band = np.zeros((3, n))
    band[0, 1:] = sup
    band[1, :] = diag
    band[2, :-1] = sub
    return ModeMat('B', n, 1, 1, band)


def second_difference(n: int, scale: float = 1.0) -> ModeMat:
    """scale * tridiag(-1, 2, -1), the 1D second-difference matrix T_n."""
    return tridiag(n, -scale, 2.0 * scale, -scale)


def upwind_backward(n: int, scale: float = 1.0) -> ModeMat:
    """scale * (I - subdiagonal shift): the upwind backward difference (Section 4.2)."""
    band = np.zeros((2, n))
    band[0, :] = scale
    band[1, :-1] = -scale
    return ModeMat('B', n, 1, 0, band)


def diagonal(values: np.ndarray) -> ModeMat:
    v = np.asarray(values, dtype=np.float64)
    return ModeMat('B', v.size, 0, 0, v.reshape(1, -1).copy())


def gaussian_blur_band(n: int, sigma: float = 2.0, half_width: int = 7) -> ModeMat:
    """Symmetric Gaussian Toeplitz blur, taps exp(-t^2/(2 sigma^2))/Z for |t| <= half_width,
    Z the sum of the taps, zero boundary."""
    t = np.arange(-half_width, half_width + 1)
    taps = np.exp(-t.astype(np.float64) ** 2 / (2.0 * sigma * sigma))
    taps /= taps.sum()
    w = half_width
    band = np.zeros((2 * w + 1, n))
    for j in range(n):
        for i in range(max(0, j - w), min(n, j + w + 1)):
            band[w + i - j, j] = taps[i - j + w]
    return ModeMat('B', n, w, w, band)


def gaussian_blur_dense(n: int, sigma: float = 2.0, half_width: int = 7) -> np.ndarray:
    """The same blur matrix as `gaussian_blur_band`, formed densely from its definition."""
    t = np.arange(-half_width, half_width + 1)
    taps = np.exp(-t.astype(np.float64) ** 2 / (2.0 * sigma * sigma))
    taps /= taps.sum()
    g = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - half_width), min(n, i + half_width + 1)):
            g[i, j] = taps[i - j + half_width]
    return g


def kronecker_sum_operator(mats_1d: Sequence[ModeMat], d: int,
                           thetas: Optional[Sequence[float]] = None) -> Operator:
    """sum_k theta_k I x .. x M_k x .. x I: one term per mode per 1D matrix."""
    n = mats_1d[0].n
    terms, theta = [], []
    for idx, m in enumerate(mats_1d):
        for k in range(d):
            terms.append([m if j == k else identity(n) for j in range(d)])
            theta.append(1.0 if thetas is None else float(thetas[idx]))
    return Operator(d, [n] * d, theta, terms)


def random_tucker(n: Sequence[int], r: Sequence[int], seed: int) -> Tucker:
    """Core i.i.d. N(0,1); factor columns i.i.d. N(0,1) scaled to unit 2-norm."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(r))
    factors = []
    for nk, rk in zip(n, r):
        u = rng.standard_normal((nk, rk))
        u /= np.linalg.norm(u, axis=0, keepdims=True)
        factors.append(u)
    return Tucker(core, factors)


def smooth_tucker(n: Sequence[int], r: Sequence[int], seed: int, decay: float = 2.0) -> Tucker:
    """Tucker tensor with i.i.d. N(0,1) core and smooth factors: column c of U_k is
    sum_j g_jc j^(-decay) sqrt(2/(n+1)) sin(j i pi/(n+1)) (i, j = 1..n_k, g_jc i.i.d. N(0,1)),
    normalised to unit norm: a seeded random function whose sine coefficients decay like
    j^(-decay), the kind of source a PDE right-hand side is."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(r))
    factors = []
    for nk, rk in zip(n, r):
        i = np.arange(1, nk + 1)
        basis = np.sqrt(2.0 / (nk + 1)) * np.sin(np.outer(i, i) * np.pi / (nk + 1))
        coef = rng.standard_normal((nk, rk)) * (i[:, None].astype(float) ** -decay)
        u = basis @ coef
        u /= np.linalg.norm(u, axis=0, keepdims=True)
        factors.append(u)
    return Tucker(core, factors)


# ----------------------------------------------------------------------------------
# The five synthetic workloads
# ----------------------------------------------------------------------------------
@dataclass
class SolverParams:
    variant: str            # 'rhosvd' (Alg. 2) or 'mln' (Alg. 6)
    rank_cap: int           # r: multilinear rank cap (RHOSVD) / Nystrom target rank (MLN)
    sketch_s: int           # s: Krylov sketch size (RHOSVD); MLN uses r + p
    oversample_p: int       # p: RoundSum oversampling (RHOSVD) / Nystrom oversampling (MLN)
    maxit: int
    tol: float
    eta: float = 0.3
    ktrunc: int = 2
    round_tol: float = 1e-12
    seed: int = 0
    adaptive_rank: bool = False
    r_sol: int = 0          # MLN memory-efficient variant (Section 3.3): solution rank r_sol,
    p_sol: int = 0          # stored sketches cut to r_sol + p_sol (0: off)
    tikhonov: bool = False  # projected Tikhonov with the GCV parameter in every least-squares step
    gcv_rows: str = "projected"  # GCV's row count for the sketched variants: 'projected' (k + 1) or
                                 # 'sketch' (every row of the sketch, s or r + p)


@dataclass
class Workload:
    name: str
    op: Operator
    b: Tucker
    params: SolverParams
    x_true: Optional[Tucker] = None
    extra: dict = field(default_factory=dict)


def poisson3d(n: int, rhs_rank: int, seed: int, params: SolverParams, name: str) -> Workload:
    op = kronecker_sum_operator([second_difference(n)], 3)
    b = random_tucker([n] * 3, [rhs_rank] * 3, seed)
    return Workload(name, op, b, params)


def point_source_rhs(n: int, d: int = 3) -> Tucker:
    """Rank-1 right-hand side (ones / sqrt(n)) (x) e_1 (x) .. (x) e_1 of the Poisson and
    convection-diffusion experiments (Section 4)."""
    ones = np.ones((n, 1)) / np.sqrt(n)
    fac = [ones] + [np.eye(n, 1) for _ in range(d - 1)]
    return Tucker(np.ones((1,) * d), fac)


def poisson3d_point(n: int, params: SolverParams, q: int, name: str) -> Workload:
    """3-D Poisson (T_n per mode) with the rank-1 point-source right-hand side, solved with the
    exponential-sum preconditioner of q (2q+1 terms)."""
    op = kronecker_sum_operator([second_difference(n)], 3)
    return Workload(name, op, point_source_rhs(n), params, extra={"precond_q": q})


def convdiff3d(n: int, seed: int, params: SolverParams, weight: float = 10.0,
               rhs_rank: int = 4) -> Workload:
    """Six terms: per mode (1/h^2) T_n and weight * (1/h) B_n, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    op = kronecker_sum_operator([second_difference(n, 1.0 / h ** 2),
                                 upwind_backward(n, weight / h)], 3)
    b = random_tucker([n] * 3, [rhs_rank] * 3, seed)
    return Workload(f"convdiff3d_n{n}", op, b, params)


def varcoef4d(n: int, seed: int, params: SolverParams, rhs_rank: int = 3) -> Workload:
    """Term i: T_n in mode i, D_j = diag(U[1, 10]) (seeded, one per mode) in the other modes."""
    rng = np.random.default_rng(seed + 7919)
    dmats = [diagonal(rng.uniform(1.0, 10.0, size=n)) for _ in range(4)]
    t = second_difference(n)
    terms = [[t if j == i else dmats[j] for j in range(4)] for i in range(4)]
    op = Operator(4, [n] * 4, [1.0] * 4, terms)
    b = random_tucker([n] * 4, [rhs_rank] * 4, seed)
    return Workload(f"varcoef4d_n{n}", op, b, params)


def deblur3d(n: int, seed: int, params: SolverParams, lam: float = 1e-2, sigma: float = 2.0,
             x_rank: int = 6) -> Workload:
    """A = G x G x G + lam I; b = A(x_true) written exactly as a Tucker tensor of rank 2*x_rank
    (factors [G U_k, U_k], block-diagonal core diag(G_x, lam G_x))."""
    g = gaussian_blur_band(n, sigma)
    op = Operator(3, [n] * 3, [1.0, lam], [[g, g, g], [identity(n)] * 3])
    xt = random_tucker([n] * 3, [x_rank] * 3, seed)
    gd = gaussian_blur_dense(n, sigma)
    r = x_rank
    core = np.zeros((2 * r,) * 3)
    core[:r, :r, :r] = xt.core
    core[r:, r:, r:] = lam * xt.core
    factors = [np.concatenate([gd @ u, u], axis=1) for u in xt.factors]
    return Workload(f"deblur3d_n{n}", op, Tucker(core, factors), params, x_true=xt,
                    extra={"lam": lam, "sigma": sigma})


def deblur3d_noisy(n: int, seed: int, params: SolverParams, noise: float = 0.02, lam: float = 1e-4,
                   x_rank: int = 2) -> Workload:
    """Deblurring with a noisy right-hand side: b = A x_true + e, e i.i.d. Gaussian scaled to
    noise ||A x_true|| / sqrt(N), given as a full tensor (core = the noisy data, identity
    factors).  The setting of the paper's regularisation study (Section 4.3), synthetic."""
    wl = deblur3d(n, seed, params, lam=lam, x_rank=x_rank)
    g = wl.b.core
    for k, u in enumerate(wl.b.factors):
        g = np.moveaxis(np.tensordot(u, np.moveaxis(g, k, 0), axes=(1, 0)), 0, k)
    rng = np.random.default_rng(seed + 104729)
    g = g + noise * np.linalg.norm(g) / np.sqrt(g.size) * rng.standard_normal(g.shape)
    b = Tucker(g, [np.eye(n) for _ in range(3)])
    return Workload(f"deblur3d_noisy_n{n}", wl.op, b, params, x_true=wl.x_true)


def workload(name: str, seed: int = 0) -> Workload:
    """The synthetic workloads by name (sizes as the headline configurations state them)."""
    if name == "poisson3d_n32":
        p = SolverParams('rhosvd', 8, 64, 5, 50, 1e-8, seed=seed)
        return poisson3d(32, 1, seed, p, name)
    if name == "convdiff3d_n256":
        p = SolverParams('rhosvd', 32, 128, 5, 60, 1e-6, seed=seed)
        return convdiff3d(256, seed, p)
    if name == "varcoef4d_n128":
        p = SolverParams('mln', 24, 60, 36, 30, 1e-6, seed=seed)
        return varcoef4d(128, seed, p)
    if name == "deblur3d_n128":
        p = SolverParams('rhosvd', 32, 256, 5, 150, 1e-6, seed=seed)
        return deblur3d(128, seed, p)
    if name == "poisson3d_n1024":
        # rank (8,8,8) seeded smooth right-hand side, solved with the exponential-sum
        # preconditioner of q = 8 (2q+1 = 17 terms)
        p = SolverParams('rhosvd', 64, 256, 5, 40, 1e-6, seed=seed)
        op = kronecker_sum_operator([second_difference(1024)], 3)
        return Workload(name, op, smooth_tucker([1024] * 3, [8] * 3, seed), p, extra={"precond_q": 8})
    if name == "poisson3d_smooth_n64":
        # a small instance of the same problem (test size)
        p = SolverParams('rhosvd', 24, 64, 5, 20, 1e-6, seed=seed)
        op = kronecker_sum_operator([second_difference(64)], 3)
        return Workload(name, op, smooth_tucker([64] * 3, [4] * 3, seed), p, extra={"precond_q": 16})
    if name == "poisson3d_n1024_gaussian":
        # the same problem with white-noise (i.i.d. Gaussian, unit-norm) factors: its solution
        # is not representable at rank 64 to 1e-6 (iteration speed only)
        p = SolverParams('rhosvd', 64, 256, 5, 100, 1e-6, seed=seed)
        return Workload(name, kronecker_sum_operator([second_difference(1024)], 3),
                        random_tucker([1024] * 3, [8] * 3, seed), p, extra={"precond_q": 8})
    if name == "poisson3d_point_n1000":
        p = SolverParams('rhosvd', 40, 64, 40, 20, 1e-7, eta=0.4, ktrunc=1, seed=seed)
        return poisson3d_point(1000, p, 8, name)
    raise KeyError(name)


WORKLOADS = ["poisson3d_n32", "convdiff3d_n256", "varcoef4d_n128", "deblur3d_n128",
             "poisson3d_n1024"]
