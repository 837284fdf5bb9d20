"""Python binding of the C ABI: argument marshalling only.

Device memory and the stream come from PyTorch; every step of the solvers runs in the CUDA
library.  Tensors cross the boundary column-major: a core of logical shape (r_1, .., r_d) is
held in a torch tensor with Fortran strides (element [i_1, .., i_d] at i_1 + r_1 (i_2 + ...)),
and a factor n x r likewise.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L

STATUS = {L.TK_OK: "converged", L.TK_NOT_CONVERGED: "not_converged", L.TK_BREAKDOWN: "breakdown",
          L.TK_SKETCH_EXHAUSTED: "sketch_exhausted", L.TK_SUSPENDED: "suspended"}


class TuckerError(RuntimeError):
    pass


def fortran_empty(shape: Sequence[int], device) -> torch.Tensor:
    """Uninitialised float64 tensor of `shape` with column-major strides."""
    shape = [int(s) for s in shape]
    t = torch.empty(shape[::-1], dtype=torch.float64, device=device)
    return t.permute(*reversed(range(len(shape))))


def to_fortran(x, device) -> torch.Tensor:
    """Copy an array (numpy or torch) to `device` as float64 with column-major strides."""
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.asarray(x, dtype=np.float64))
    x = x.to(dtype=torch.float64)
    nd = x.dim()
    rev = list(reversed(range(nd)))
    return x.permute(*rev).contiguous().to(device).permute(*rev)


def is_fortran(t: torch.Tensor) -> bool:
    stride = 1
    for size, st in zip(t.shape, t.stride()):
        if size > 1 and st != stride:
            return False
        stride *= size
    return True


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """Library handle bound to one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0):
        self.lib = L.load()
        self.device = int(device)
        h = ctypes.c_void_p()
        rc = self.lib.tk_create(ctypes.byref(h), self.device)
        if rc != 0:
            raise TuckerError(f"tk_create failed with status {rc}")
        self.h = h

    def check(self, rc: int, what: str) -> int:
        if rc < 0:
            msg = self.lib.tk_last_error(self.h).decode()
            raise TuckerError(f"{what} failed ({rc}): {msg}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.tk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_HANDLES: Dict[int, Handle] = {}


def handle(device: Optional[int] = None) -> Handle:
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _HANDLES:
        _HANDLES[dev] = Handle(dev)
    return _HANDLES[dev]


@dataclass
class DeviceTucker:
    """Tucker tensor on the GPU: core (r_1 x .. x r_d) and factors (n_k x r_k), column-major."""
    core: torch.Tensor
    factors: List[torch.Tensor]

    @staticmethod
    def from_numpy(core: np.ndarray, factors: Sequence[np.ndarray], device="cuda") -> "DeviceTucker":
        return DeviceTucker(to_fortran(core, device), [to_fortran(u, device) for u in factors])

    @staticmethod
    def empty(n: Sequence[int], r: Sequence[int], device="cuda") -> "DeviceTucker":
        return DeviceTucker(fortran_empty(r, device), [fortran_empty((a, b), device) for a, b in zip(n, r)])

    @property
    def d(self) -> int:
        return len(self.factors)

    @property
    def n(self) -> List[int]:
        return [int(u.shape[0]) for u in self.factors]

    @property
    def r(self) -> List[int]:
        return [int(u.shape[1]) for u in self.factors]

    def numpy(self):
        return (self.core.cpu().numpy(), [u.cpu().numpy() for u in self.factors])

    def c(self) -> L.tk_tucker:
        for t in [self.core, *self.factors]:
            if t.dtype != torch.float64 or not t.is_cuda or not is_fortran(t):
                raise TuckerError("Tucker tensors must be float64 CUDA tensors in column-major layout")
        s = L.tk_tucker()
        s.d = self.d
        for k in range(self.d):
            s.n[k] = self.n[k]
            s.r[k] = self.r[k]
            s.factor[k] = self.factors[k].data_ptr()
        s.core = self.core.data_ptr()
        return s


class DeviceOperator:
    """L = sum_t theta_t A_1^(t) x .. x A_d^(t) with its mode matrices on the GPU.

    `op` has attributes d, n, theta and mats[t][k] with kind ('I', 'B', 'D'), n, kl, ku and
    data (band layout (kl+ku+1) x n, or dense n x n)."""

    _KIND = {'I': L.TK_IDENTITY, 'B': L.TK_BANDED, 'D': L.TK_DENSE}

    def __init__(self, op, device="cuda", theta: Optional[Sequence[float]] = None):
        self.d = int(op.d)
        self.n = [int(v) for v in op.n]
        self.nterms = len(op.mats)
        self._keep = []
        cache = {}
        mats = (L.tk_modemat * (self.nterms * self.d))()
        for t in range(self.nterms):
            for k in range(self.d):
                m = op.mats[t][k]
                e = mats[t * self.d + k]
                e.kind = self._KIND[m.kind]
                e.kl, e.ku, e.n = int(m.kl), int(m.ku), int(m.n)
                if m.kind == 'I':
                    e.data = None
                    continue
                key = id(m.data)
                if key not in cache:
                    cache[key] = to_fortran(np.asarray(m.data, dtype=np.float64), device)
                e.data = cache[key].data_ptr()
        self._keep.append(cache)
        self.mats = mats
        self.set_theta(op.theta if theta is None else theta)

    @classmethod
    def from_device(cls, d: int, n: Sequence[int], theta: Sequence[float], mats) -> "DeviceOperator":
        """Operator from mode matrices already on the GPU: mats[t][k] = (kind, tensor, kl, ku) with
        kind 'I' (tensor None), 'B' (band layout (kl+ku+1) x n) or 'D' (dense n x n), float64 and
        column-major.  The tensors are referenced, not copied."""
        self = cls.__new__(cls)
        self.d, self.n, self.nterms = int(d), [int(v) for v in n], len(mats)
        mm = (L.tk_modemat * (self.nterms * self.d))()
        keep = []
        for t in range(self.nterms):
            for k in range(self.d):
                kind, data, kl, ku = mats[t][k]
                e = mm[t * self.d + k]
                e.kind, e.kl, e.ku, e.n = cls._KIND[kind], int(kl), int(ku), self.n[k]
                if kind == 'I':
                    e.data = None
                    continue
                if data.dtype != torch.float64 or not data.is_cuda or not is_fortran(data):
                    raise TuckerError("mode matrices must be float64 CUDA tensors in column-major layout")
                e.data = data.data_ptr()
                keep.append(data)
        self._keep, self.mats = [keep], mm
        self.set_theta(theta)
        return self

    def set_theta(self, theta: Sequence[float]):
        self.theta_values = [float(v) for v in theta]
        self.theta = (ctypes.c_double * self.nterms)(*self.theta_values)

    def c(self) -> L.tk_operator:
        s = L.tk_operator()
        s.nterms = self.nterms
        s.d = self.d
        s.theta = ctypes.cast(self.theta, ctypes.POINTER(ctypes.c_double))
        s.mats = ctypes.cast(self.mats, ctypes.POINTER(L.tk_modemat))
        return s


@dataclass
class Options:
    variant: str = "rhosvd"          # 'rhosvd' (Algorithm 2), 'mln' (Algorithm 6) or 'gmres' (Algorithm 1)
    rank_cap: int = 8
    sketch_s: int = 64
    oversample_p: int = 5
    ktrunc: int = 2
    maxit: int = 50
    tol: float = 1e-8
    eta: float = 0.3
    round_tol: float = 1e-12
    seed: int = 0
    adaptive_rank: bool = False
    precision: str = "fp64"          # 'fp64' or 'mixed'
    transpose: bool = False
    r_sol: int = 0                   # MLN memory-efficient variant: solution rank (0: off)
    p_sol: int = 0                   # ... and the stored sketches' extra columns
    tikhonov: bool = False           # projected Tikhonov with the GCV parameter (Section 4.3)
    gcv_rows: str = "projected"      # GCV's row count for the sketched variants: 'projected' (k + 1) or 'sketch'
    stop_after: int = 0              # > 0: suspend after this many iterations (tk_checkpoint_save)
    resume: bool = False             # continue the solve suspended in the handle
    true_residual: bool = False      # report the true relative residual of x

    @staticmethod
    def from_params(p, **over) -> "Options":
        o = Options(variant=p.variant, rank_cap=p.rank_cap, sketch_s=p.sketch_s,
                    oversample_p=p.oversample_p, ktrunc=p.ktrunc, maxit=p.maxit, tol=p.tol,
                    eta=p.eta, round_tol=p.round_tol, seed=p.seed, adaptive_rank=p.adaptive_rank,
                    r_sol=getattr(p, "r_sol", 0), p_sol=getattr(p, "p_sol", 0),
                    tikhonov=bool(getattr(p, "tikhonov", False)),
                    gcv_rows=getattr(p, "gcv_rows", "projected"))
        for k, v in over.items():
            setattr(o, k, v)
        return o

    def c(self) -> L.tk_opts:
        s = L.tk_opts()
        s.variant = {"rhosvd": L.TK_RHOSVD_SGMRES, "mln": L.TK_MLN_SGMRES, "gmres": L.TK_RHOSVD_GMRES}[self.variant]
        s.rank_cap, s.sketch_s, s.oversample_p = self.rank_cap, self.sketch_s, self.oversample_p
        s.ktrunc, s.maxit, s.adaptive_rank = self.ktrunc, self.maxit, int(self.adaptive_rank)
        s.precision = L.TK_MIXED if self.precision == "mixed" else L.TK_FP64
        s.transpose = int(self.transpose)
        s.mln_r_sol, s.mln_p_sol = int(self.r_sol), int(self.p_sol)
        s.gcv_tikhonov = int(self.tikhonov)
        if self.gcv_rows not in ("projected", "sketch"):
            raise TuckerError("gcv_rows must be 'projected' or 'sketch'")
        s.gcv_rows = 0 if self.gcv_rows == "projected" else 1
        s.stop_after, s.resume, s.true_residual = int(self.stop_after), int(self.resume), int(self.true_residual)
        s.tol, s.eta, s.round_tol, s.seed = self.tol, self.eta, self.round_tol, self.seed
        return s


@dataclass
class Report:
    iters: int
    status: str
    sketched_res: float
    res_hist: List[float]
    out_rank: List[int]
    ms_total: float
    workspace_bytes: int
    kernel_launches: int
    true_res: float = -1.0


def tk_solve(op: DeviceOperator, b: DeviceTucker, opts: Options, x: Optional[DeviceTucker] = None,
             stream=None, device: Optional[int] = None):
    """RHOSVD-Tucker sGMRES (Algorithm 2), MLN-Tucker sGMRES (Algorithm 6) or RHOSVD-Tucker GMRES
    (Algorithm 1), by opts.variant. Returns (x, Report)."""
    h = handle(device)
    if x is None:
        x = DeviceTucker.empty(b.n, [opts.rank_cap] * b.d, device=b.core.device)
    hist = (ctypes.c_double * max(1, opts.maxit))()
    rep = L.tk_report()
    rep.res_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    rep.res_hist_len = opts.maxit
    opc, bc, oc, xc = op.c(), b.c(), opts.c(), x.c()
    rc = h.lib.tk_solve(h.h, ctypes.byref(opc), ctypes.byref(bc), ctypes.byref(oc), ctypes.byref(xc),
                        ctypes.byref(rep), _stream(stream))
    h.check(rc, "tk_solve")
    r = Report(rep.iters, STATUS[rep.status], rep.sketched_res, list(hist[:rep.iters]),
               list(rep.out_rank[:b.d]), rep.ms_total, rep.workspace_bytes, rep.kernel_launches, rep.true_res)
    return x, r


def tk_solve_precond(op: DeviceOperator, precond: DeviceOperator, b: DeviceTucker, opts: Options,
                     x: Optional[DeviceTucker] = None, stream=None, device: Optional[int] = None):
    """RHOSVD-Tucker sGMRES with flexible preconditioning by the separable operator `precond`
    (Section 3.4). Returns (x, Report)."""
    h = handle(device)
    if x is None:
        x = DeviceTucker.empty(b.n, [opts.rank_cap] * b.d, device=b.core.device)
    hist = (ctypes.c_double * max(1, opts.maxit))()
    rep = L.tk_report()
    rep.res_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    rep.res_hist_len = opts.maxit
    opc, pc, bc, oc, xc = op.c(), precond.c(), b.c(), opts.c(), x.c()
    rc = h.lib.tk_solve_precond(h.h, ctypes.byref(opc), ctypes.byref(pc), ctypes.byref(bc), ctypes.byref(oc),
                                ctypes.byref(xc), ctypes.byref(rep), _stream(stream))
    h.check(rc, "tk_solve_precond")
    r = Report(rep.iters, STATUS[rep.status], rep.sketched_res, list(hist[:rep.iters]),
               list(rep.out_rank[:b.d]), rep.ms_total, rep.workspace_bytes, rep.kernel_launches, rep.true_res)
    return x, r


def tk_solve_expsum(op: DeviceOperator, q: int, b: DeviceTucker, opts: Options, x: Optional[DeviceTucker] = None,
                    stream=None, device: Optional[int] = None):
    """Flexible RHOSVD-Tucker sGMRES preconditioned by the exponential-sum inverse Laplacian of
    2q+1 terms, applied in the sine eigenbasis (Section 3.4). Returns (x, Report)."""
    h = handle(device)
    if x is None:
        x = DeviceTucker.empty(b.n, [opts.rank_cap] * b.d, device=b.core.device)
    hist = (ctypes.c_double * max(1, opts.maxit))()
    rep = L.tk_report()
    rep.res_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    rep.res_hist_len = opts.maxit
    opc, bc, oc, xc = op.c(), b.c(), opts.c(), x.c()
    rc = h.lib.tk_solve_expsum(h.h, ctypes.byref(opc), int(q), ctypes.byref(bc), ctypes.byref(oc), ctypes.byref(xc),
                               ctypes.byref(rep), _stream(stream))
    h.check(rc, "tk_solve_expsum")
    r = Report(rep.iters, STATUS[rep.status], rep.sketched_res, list(hist[:rep.iters]),
               list(rep.out_rank[:b.d]), rep.ms_total, rep.workspace_bytes, rep.kernel_launches, rep.true_res)
    return x, r


_POOL: Dict[int, List[tuple]] = {}


def _pool(device: int, count: int) -> List[tuple]:
    """(handle, stream) pairs for concurrent solves on `device`: the device's default handle
    with a stream of its own, then extra handles, each with its own stream (created once)."""
    lst = _POOL.setdefault(device, [])
    while len(lst) < count:
        h = handle(device) if not lst else Handle(device)
        lst.append((h, torch.cuda.Stream(device=device)))
    return lst[:count]


def tk_solve_concurrent(jobs: Sequence[dict], device: Optional[int] = None):
    """Independent solves at the same time (tk_solve_concurrent): each job is a dict with op, b,
    opts and optionally precond (DeviceOperator), expsum_q (int) and x (output DeviceTucker).
    The jobs run on their own handles and streams, after the current stream's pending work.
    Returns [(x, Report)] in job order; raises on the first failed job."""
    dev = torch.cuda.current_device() if device is None else int(device)
    pool = _pool(dev, len(jobs))
    cur = torch.cuda.current_stream(dev)
    keep, arr = [], (L.tk_solve_job * len(jobs))()
    for i, (job, (h, st)) in enumerate(zip(jobs, pool)):
        st.wait_stream(cur)
        b, opts = job["b"], job["opts"]
        x = job.get("x") or DeviceTucker.empty(b.n, [opts.rank_cap] * b.d, device=b.core.device)
        hist = (ctypes.c_double * max(1, opts.maxit))()
        rep = L.tk_report()
        rep.res_hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        rep.res_hist_len = opts.maxit
        opc, bc, oc, xc = job["op"].c(), b.c(), opts.c(), x.c()
        pcc = job["precond"].c() if job.get("precond") is not None else None
        keep.append((x, hist, rep, opc, bc, oc, xc, pcc))
        J = arr[i]
        J.h, J.op, J.b, J.opts, J.x_out = h.h, ctypes.addressof(opc), ctypes.addressof(bc), ctypes.addressof(oc), \
            ctypes.addressof(xc)
        J.precond = ctypes.addressof(pcc) if pcc is not None else None
        J.expsum_q = int(job.get("expsum_q", 0))
        J.report = ctypes.addressof(rep)
        J.stream = st.cuda_stream
    lib = L.load()
    lib.tk_solve_concurrent(len(jobs), arr)
    out = []
    for i, (x, hist, rep, *_rest) in enumerate(keep):
        h = pool[i][0]
        h.check(arr[i].status, f"tk_solve_concurrent job {i}")
        out.append((x, Report(rep.iters, STATUS[rep.status], rep.sketched_res, list(hist[:rep.iters]),
                              list(rep.out_rank[:x.d]), rep.ms_total, rep.workspace_bytes, rep.kernel_launches,
                              rep.true_res)))
    return out


def tk_checkpoint_save(device: Optional[int] = None) -> bytes:
    """The Krylov state of the solve suspended in this device's handle (opts.stop_after), as bytes."""
    h = handle(device)
    size = ctypes.c_int64()
    h.check(h.lib.tk_checkpoint_save(h.h, None, 0, ctypes.byref(size)), "tk_checkpoint_save")
    buf = ctypes.create_string_buffer(size.value)
    h.check(h.lib.tk_checkpoint_save(h.h, buf, size.value, ctypes.byref(size)), "tk_checkpoint_save")
    return buf.raw[:size.value]


def tk_checkpoint_load(state: bytes, device: Optional[int] = None):
    """Install a saved Krylov state in this device's handle; a solve with opts.resume continues it."""
    h = handle(device)
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    h.check(h.lib.tk_checkpoint_load(h.h, buf, len(state)), "tk_checkpoint_load")


def tk_fma_peak(fp64: bool = True, device: Optional[int] = None, stream=None) -> float:
    """Measured FMA throughput of the device in TFLOP/s (FP64 or FP32), the ALU roofline's peak."""
    h = handle(device)
    out = ctypes.c_double()
    h.check(h.lib.tk_fma_peak(h.h, int(bool(fp64)), ctypes.byref(out), _stream(stream)), "tk_fma_peak")
    return out.value


def tk_selftest_qr_wait(mode: int, device: Optional[int] = None, stream=None):
    """Failure detection of the multi-cluster QR (tk_selftest_qr_wait): one exchange made to go
    missing (mode 1: a byte count inside a cluster, 2: a publication to the other cluster); raises
    TuckerError unless the kernel gave up waiting, reported it and finished."""
    h = handle(device)
    h.check(h.lib.tk_selftest_qr_wait(h.h, int(mode), _stream(stream)), "tk_selftest_qr_wait")


def tk_set_workspace_limit(nbytes: int, device: Optional[int] = None):
    """Cap the device workspace of this device's handle (0: no cap); beyond it calls fail with TK_ENOMEM."""
    h = handle(device)
    h.check(h.lib.tk_set_workspace_limit(h.h, int(nbytes)), "tk_set_workspace_limit")


def tk_expsum_laplacian(n: int, d: int, q: int, device="cuda", stream=None) -> DeviceOperator:
    """Exponential-sum approximation of the inverse of the d-dimensional Laplacian
    T_n (+) .. (+) T_n, T_n = tridiag(-1, 2, -1): 2q+1 separable terms c_h E_h x .. x E_h with
    E_h = exp(-t_h T_n) formed on the GPU (Section 3.4)."""
    h = handle()
    mats = [fortran_empty((n, n), device) for _ in range(2 * q + 1)]
    ptrs = (ctypes.c_void_p * (2 * q + 1))(*[m.data_ptr() for m in mats])
    coef = (ctypes.c_double * (2 * q + 1))()
    h.check(h.lib.tk_expsum_laplacian(h.h, int(n), int(q), ptrs, coef, _stream(stream)), "tk_expsum_laplacian")
    return DeviceOperator.from_device(d, [n] * d, list(coef), [[('D', m, 0, 0)] * d for m in mats])


def tk_profile(enable: bool, device: Optional[int] = None):
    """Enable or disable per-kernel CUDA-event timing inside the library."""
    h = handle(device)
    h.check(h.lib.tk_profile(h.h, int(enable)), "tk_profile")


def tk_profile_report(device: Optional[int] = None) -> Dict[str, tuple]:
    """{kernel name: (launches, total ms, algorithmic flops, algorithmic bytes)} since the last
    report (then reset)."""
    h = handle(device)
    txt = h.lib.tk_profile_report(h.h).decode()
    out = {}
    for line in txt.strip().splitlines():
        name, n, ms, fl, by = line.split()
        out[name] = (int(n), float(ms), float(fl), float(by))
    return out


def tk_apply(op: DeviceOperator, x: DeviceTucker, transpose: bool = False, stream=None) -> List[List[torch.Tensor]]:
    """Factors A_k^(t) U_k of every term (Eq. (1.2)); the terms share x's core scaled by theta_t."""
    h = handle()
    outs = [[fortran_empty((x.n[k], x.r[k]), x.core.device) for k in range(x.d)] for _ in range(op.nterms)]
    ptrs = (ctypes.c_void_p * (op.nterms * x.d))(*[outs[t][k].data_ptr() for t in range(op.nterms) for k in range(x.d)])
    opc, xc = op.c(), x.c()
    h.check(h.lib.tk_apply(h.h, ctypes.byref(opc), ctypes.byref(xc), int(transpose), ptrs, _stream(stream)), "tk_apply")
    return outs


def tk_roundsum(terms: Sequence[DeviceTucker], coef: Sequence[float], opts: Options, call_index: int = 0,
                out: Optional[DeviceTucker] = None, stream=None):
    """RoundSum (Section 3.1) of sum_i coef_i terms_i. Returns (out, ranks)."""
    h = handle()
    d = terms[0].d
    if out is None:
        out = DeviceTucker.empty(terms[0].n, [opts.rank_cap] * d, device=terms[0].core.device)
    arr = (L.tk_tucker * len(terms))(*[t.c() for t in terms])
    cf = (ctypes.c_double * len(terms))(*[float(c) for c in coef])
    ranks = (ctypes.c_int32 * d)()
    oc, outc = opts.c(), out.c()
    rc = h.lib.tk_roundsum(h.h, len(terms), arr, cf, ctypes.byref(oc), int(call_index), ctypes.byref(outc),
                           ranks, _stream(stream))
    h.check(rc, "tk_roundsum")
    return out, list(ranks)


def tk_kron_sketch(x: DeviceTucker, S: Sequence[torch.Tensor], stream=None) -> torch.Tensor:
    """Kronecker-structured sketch out[l] = X x_1 S_1[:,l]^T ... x_d S_d[:,l]^T (Algorithm 2)."""
    h = handle()
    s = int(S[0].shape[1])
    out = torch.empty(s, dtype=torch.float64, device=x.core.device)
    for m in S:
        if not is_fortran(m):
            raise TuckerError("sketch matrices must be column-major")
    ptrs = (ctypes.c_void_p * x.d)(*[m.data_ptr() for m in S])
    xc = x.c()
    h.check(h.lib.tk_kron_sketch(h.h, ctypes.byref(xc), ptrs, s, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
            "tk_kron_sketch")
    return out


def tk_inner(x: DeviceTucker, y: DeviceTucker, stream=None) -> float:
    h = handle()
    out = ctypes.c_double()
    xc, yc = x.c(), y.c()
    h.check(h.lib.tk_inner(h.h, ctypes.byref(xc), ctypes.byref(yc), ctypes.byref(out), _stream(stream)), "tk_inner")
    return out.value


def tk_residual(op: DeviceOperator, x: DeviceTucker, b: DeviceTucker, transpose: bool = False, stream=None) -> float:
    """True relative residual ||L(X) - B|| / ||B|| computed in Tucker form."""
    h = handle()
    out = ctypes.c_double()
    opc, xc, bc = op.c(), x.c(), b.c()
    h.check(h.lib.tk_residual(h.h, ctypes.byref(opc), ctypes.byref(xc), ctypes.byref(bc), int(transpose),
                              ctypes.byref(out), _stream(stream)), "tk_residual")
    return out.value


def tk_sum_norm(terms: Sequence[DeviceTucker], coef: Sequence[float], stream=None) -> float:
    """||sum_i coef_i terms_i||_F computed in Tucker form (QR of concatenated factors)."""
    h = handle()
    arr = (L.tk_tucker * len(terms))(*[t.c() for t in terms])
    cf = (ctypes.c_double * len(terms))(*[float(c) for c in coef])
    out = ctypes.c_double()
    h.check(h.lib.tk_sum_norm(h.h, len(terms), arr, cf, ctypes.byref(out), _stream(stream)), "tk_sum_norm")
    return out.value


def tk_adjoint_grads(op: DeviceOperator, mu: DeviceTucker, x: DeviceTucker, b: DeviceTucker, stream=None):
    """(dl/dtheta (list), dl/dG_b, [dl/dU_bk]) from the adjoint solution mu and forward solution x."""
    h = handle()
    dth = (ctypes.c_double * op.nterms)()
    dcore = fortran_empty(b.r, b.core.device)
    dfac = [fortran_empty((b.n[k], b.r[k]), b.core.device) for k in range(b.d)]
    ptrs = (ctypes.c_void_p * b.d)(*[t.data_ptr() for t in dfac])
    opc, muc, xc, bc = op.c(), mu.c(), x.c(), b.c()
    h.check(h.lib.tk_adjoint_grads(h.h, ctypes.byref(opc), ctypes.byref(muc), ctypes.byref(xc), ctypes.byref(bc),
                                   dth, ctypes.c_void_p(dcore.data_ptr()), ptrs, _stream(stream)), "tk_adjoint_grads")
    return list(dth), dcore, dfac


def tk_gaussian(seed: int, stream_id: int, count: int, bf16_round: bool = False, device="cuda", stream=None):
    h = handle()
    out = torch.empty(max(count, 1), dtype=torch.float64, device=device)
    h.check(h.lib.tk_gaussian(h.h, int(seed), int(stream_id), int(count), int(bf16_round),
                              ctypes.c_void_p(out.data_ptr()), _stream(stream)), "tk_gaussian")
    return out[:count]


def tk_philox(seed: int, stream_id: int, first: int, nblocks: int, device="cuda", stream=None):
    h = handle()
    out = torch.empty(max(4 * nblocks, 4), dtype=torch.int32, device=device)
    h.check(h.lib.tk_philox(h.h, int(seed), int(stream_id), int(first), int(nblocks),
                            ctypes.c_void_p(out.data_ptr()), _stream(stream)), "tk_philox")
    return out[:4 * nblocks]


def _check_ls_args(M: torch.Tensor, b: torch.Tensor):
    """M: float64 CUDA s x k column-major; b: float64 CUDA contiguous vector of length s, same device."""
    if M.dim() != 2 or M.dtype != torch.float64 or not M.is_cuda or not is_fortran(M):
        raise TuckerError("M must be a float64 CUDA matrix in column-major layout")
    if b.dtype != torch.float64 or not b.is_cuda or b.device != M.device or not b.is_contiguous():
        raise TuckerError("b must be a contiguous float64 CUDA vector on M's device")
    if b.numel() != M.shape[0]:
        raise TuckerError(f"b has {b.numel()} entries, M has {M.shape[0]} rows")


def tk_sketched_ls(M: torch.Tensor, b: torch.Tensor, stream=None):
    """y = argmin ||M y - b|| (Householder), M s x k column-major. Returns (y, residual norm)."""
    h = handle()
    _check_ls_args(M, b)
    s, k = int(M.shape[0]), int(M.shape[1])
    y = torch.empty(k, dtype=torch.float64, device=M.device)
    res = torch.empty(1, dtype=torch.float64, device=M.device)
    h.check(h.lib.tk_sketched_ls(h.h, ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(b.data_ptr()), s, k,
                                 ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(res.data_ptr()), _stream(stream)),
            "tk_sketched_ls")
    return y, res


def tk_sketched_ls_static(M: torch.Tensor, b: torch.Tensor, stream=None):
    """tk_sketched_ls without any device allocation by the library (fixed device workspace;
    s <= 512, k <= 128; concurrent calls race).  Returns (y, residual norm)."""
    lib = L.load()
    _check_ls_args(M, b)
    s, k = int(M.shape[0]), int(M.shape[1])
    y = torch.empty(k, dtype=torch.float64, device=M.device)
    res = torch.empty(1, dtype=torch.float64, device=M.device)
    rc = lib.tk_sketched_ls_static(ctypes.c_void_p(M.data_ptr()), ctypes.c_void_p(b.data_ptr()), s, k,
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(res.data_ptr()), _stream(stream))
    if rc != 0:
        raise TuckerError(f"tk_sketched_ls_static failed ({rc})")
    return y, res


def tk_mln_roundsum(terms: Sequence[DeviceTucker], coef: Sequence[float], psi: Sequence[torch.Tensor], r: int,
                    p: int, out: Optional[DeviceTucker] = None, stream=None) -> DeviceTucker:
    """MLN_Sketch + MLN_Sum + MLN_Recovery (Algorithms 3-5)."""
    h = handle()
    d = terms[0].d
    if out is None:
        out = DeviceTucker.empty(terms[0].n, [r] * d, device=terms[0].core.device)
    arr = (L.tk_tucker * len(terms))(*[t.c() for t in terms])
    cf = (ctypes.c_double * len(terms))(*[float(c) for c in coef])
    ptrs = (ctypes.c_void_p * d)(*[m.data_ptr() for m in psi])
    outc = out.c()
    h.check(h.lib.tk_mln_roundsum(h.h, len(terms), arr, cf, ptrs, int(r), int(p), ctypes.byref(outc),
                                  _stream(stream)), "tk_mln_roundsum")
    return out
