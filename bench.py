#!/usr/bin/env python
"""Time to relative residual 1e-6 of Tucker-format sketched GMRES on B300, mixed+adjoint vs FP64.

Workload (the largest configuration): 3-D Poisson, n = 1024 per mode (N = 1.07e9, never formed),
right-hand side of multilinear rank (8,8,8) with seeded smooth factors, rank cap 64, Krylov
sketch s = 256, RoundSum oversampling 5, flexible RHOSVD-Tucker sGMRES (Algorithm 2) with the
exponential-sum inverse-Laplacian preconditioner of Section 3.4 (q = 16, 33 terms), tol 1e-6.

One step = one gradient evaluation: the forward solve to the tolerance and the adjoint solve
L^T mu = w of the quantity of interest l = <w, x> (w smooth, rank 1) to the same tolerance, run
at the same time on two streams (tk_solve_concurrent; they are independent), then the adjoint
contractions dl/dtheta, dl/dG_b, dl/dU_b (every step of the path in the library's kernels).  `value` is the seconds per step of the mixed form (BF16 sketches and tensor-core
products with FP32 accumulation, FP64 QR/SVD/least squares); `config.fp64_seconds` is the same
step in plain FP64 and `config.mixed_speedup` their ratio.  Inputs are resident in HBM and L2 is
flushed (256 MiB write) between steps; `e2e` repeats the step through the public API with the
right-hand side, operator and weight copied from pinned host memory and x, mu and the gradients
read back inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

--impl reference times the FP64 CPU oracle on the same step.  Under torchrun every rank runs
independent replicas (different seeds); there is no data-path collective.
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "poisson3d_n1024"
PRECOND_Q = 16
TOL = 1e-6
METRIC = "time to rel. residual 1e-6 and iters/s: mixed+adjoint vs plain FP64 on 1 B300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-extras", action="store_true", help="skip the cpu_baseline and secondary workloads")
    ap.add_argument("--profile-only", action="store_true", help="one step of each form with the kernel profile")
    ap.add_argument("--maxit", type=int, default=0, help="--profile-only on another workload: iteration cap (0 = its own)")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(t_local: float, units_local: float, device) -> tuple:
    """Whole-job figures of independent replicas: (max over ranks of the timed seconds, sum over
    ranks of the units processed).  One process per rank; `device` is where the reduction tensor
    lives ("cuda" under NCCL, "cpu" under gloo).  A single process returns its own figures."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_local), float(units_local)
    tmax = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    usum = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(usum, op=dist.ReduceOp.SUM)
    return tmax.item(), usum.item()


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------------------------------
def host_cpu() -> dict:
    model = platform.processor() or ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    try:
        import numpy  # noqa: F401  (loads the BLAS whose thread pool the oracle uses)
        from threadpoolctl import threadpool_info
        cores = max([int(i.get("num_threads", 1)) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return {"cpu_model": model, "cores": cores, "nproc": os.cpu_count()}


def qoi_weight_np(n: int, d: int):
    """w of the quantity of interest l = <w, x>: the smooth rank-1 tensor (1/sqrt(n))^(x)d."""
    import numpy as np
    import workloads as W
    return W.Tucker(np.ones((1,) * d), [np.ones((n, 1)) / np.sqrt(n)] * d)


def oracle_step(name: str, seed: int, maxit=None):
    """The FP64 oracle as it stands on this host: the step the GPU arm times (forward solve to the
    tolerance, adjoint solve, adjoint contractions) with the same preconditioner and streams.
    Returns (seconds, forward iterations, adjoint iterations)."""
    import workloads as W
    from oracle import adjoint as OA
    from oracle import precond as OP
    from oracle import sgmres as OS
    wl = W.workload(name, seed=seed)
    prm = copy.copy(wl.params)
    prm.tol = TOL
    if maxit:
        prm.maxit = maxit
    t0 = time.perf_counter()
    pc = OP.expsum_preconditioner(wl.b.n[0], wl.b.d, PRECOND_Q)
    fw = OS.rhosvd_sgmres(wl.op, wl.b, prm, precond=pc)
    ad = OS.rhosvd_sgmres(wl.op, qoi_weight_np(wl.b.n[0], wl.b.d), prm, transpose=True, precond=pc)
    OA.theta_gradients(wl.op, fw.x, ad.x)
    OA.core_gradient(ad.x, wl.b)
    OA.factor_gradients(ad.x, wl.b)
    return time.perf_counter() - t0, fw.iters, ad.iters


def oracle_baseline(name: str, budget_s: float, gpu_iters: int):
    """Bounded sample for cpu_baseline: oracle steps cut at 1 iteration per solve until the budget
    is used, giving seconds per Krylov iteration; scaled to the seconds the full step needs at the
    iteration count the GPU FP64 step took."""
    host = host_cpu()
    t, its, n = 0.0, 0, 0
    while t < budget_s or n == 0:
        dt, fi, ai = oracle_step(name, 0, maxit=1)
        t += dt
        its += fi + ai
        n += 1
    per_it = t / its
    return {"value": per_it * gpu_iters, "unit": "s", "cores": host["cores"], "kind": "oracle",
            "cpu_model": host["cpu_model"], "nproc": host["nproc"],
            "sample": f"{n} oracle step(s) of {name} cut at 1 forward + 1 adjoint iteration (numpy FP64, "
                      f"{t:.1f} s, {per_it:.3f} s per Krylov iteration), scaled to the {gpu_iters} iterations "
                      f"of the GPU FP64 step"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    host = host_cpu()
    budget, times, its = 240.0, [], []
    t_start = time.perf_counter()
    for _ in range(args.warmup):       # warm-up steps, untimed (at most half the budget)
        if time.perf_counter() - t_start > budget / 2:
            break
        oracle_step(args.workload, 0)
    for _ in range(args.steps):        # exactly the requested steps unless the budget runs out
        if times and time.perf_counter() - t_start > budget:
            break                      # bounded: at least one full step is always timed
        dt, fi, ai = oracle_step(args.workload, 0)
        times.append(dt)
        its.append(fi + ai)
    value = statistics.median(times)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": len(times),
            "warmup": args.warmup, "ms_per_step": 1000.0 * value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "solver": "flexible RHOSVD-Tucker sGMRES (Algorithm 2), "
                                                             "exponential-sum preconditioner q = 16",
                       "step": "forward solve + adjoint solve + adjoint contractions to rel. residual 1e-6",
                       "iters_per_step": statistics.median(its), "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": host["cores"], "kind": "oracle",
                             "cpu_model": host["cpu_model"],
                             "sample": f"{len(times)} full oracle step(s) (numpy FP64; the run is cut after "
                                       f"{budget:.0f} s, at least one step)"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
def tucker_bytes(t) -> int:
    return 8 * (t.core.numel() + sum(u.numel() for u in t.factors))


class Problem:
    """The benchmark problem on the device: operator, right-hand side, preconditioner, weight w."""

    def __init__(self, P, W, name, seed):
        import numpy as np
        self.wl = W.workload(name, seed=seed)
        self.prm = copy.copy(self.wl.params)
        self.prm.tol = TOL
        n, d = self.wl.b.n[0], self.wl.b.d
        self.dop = P.DeviceOperator(self.wl.op)
        self.b = P.DeviceTucker.from_numpy(self.wl.b.core, self.wl.b.factors)
        wq = qoi_weight_np(n, d)
        self.w = P.DeviceTucker.from_numpy(wq.core, wq.factors)
        R = self.prm.rank_cap
        self.x = P.DeviceTucker.empty(self.b.n, [R] * d)
        self.mu = P.DeviceTucker.empty(self.b.n, [R] * d)
        self.np = np

    def step(self, P, form, concurrent=True):
        """Forward and adjoint solves at the same time (independent: the adjoint right-hand side
        is w), then the adjoint contractions.  concurrent=False runs them one after the other on
        the default handle (the kernel profile is per handle)."""
        opts = P.Options.from_params(self.prm, precision=form)
        adj = copy.copy(opts)
        adj.transpose = True
        if concurrent:
            (x, rep), (mu, rep_a) = P.tk_solve_concurrent(
                [dict(op=self.dop, b=self.b, opts=opts, expsum_q=PRECOND_Q, x=self.x),
                 dict(op=self.dop, b=self.w, opts=adj, expsum_q=PRECOND_Q, x=self.mu)])
        else:
            x, rep = P.tk_solve_expsum(self.dop, PRECOND_Q, self.b, opts, x=self.x)
            mu, rep_a = P.tk_solve_expsum(self.dop, PRECOND_Q, self.w, adj, x=self.mu)
        grads = P.tk_adjoint_grads(self.dop, mu, x, self.b)
        return rep, rep_a, grads


def kernel_table(prof, peaks):
    """Per kernel: launches, device time, share, and its roofline: FP64 pipe (GEMM, QR, SVD and
    contraction kernels, algorithmic FP64 flops), BF16 tensor pipe (gemm_tc) or HBM (streaming
    kernels, algorithmic bytes).  Small launches are latency bound far below these peaks."""
    total = sum(v[1] for v in prof.values()) or 1.0
    out = {}
    for name, (n, ms, fl, by) in sorted(prof.items(), key=lambda kv: -kv[1][1]):
        e = {"launches": n, "ms": round(ms, 4), "share": round(ms / total, 4), "avg_us": round(1000 * ms / n, 2)}
        if name == "gemm_tc" and fl > 0:
            a = fl / (ms * 1e-3) / 1e12
            e.update({"bound": "tensor", "achieved": round(a, 4), "unit": "TFLOP/s",
                      "frac": round(a / peaks["bf16_tflops"], 5)})
        elif fl > 0 and (name.startswith("gemm") or name in ("qr", "svd", "tikhonov", "hadamard", "qr_wy_solve", "ls")):
            a = fl / (ms * 1e-3) / 1e12
            e.update({"bound": "alu", "achieved": round(a, 4), "unit": "TFLOP/s",
                      "frac": round(a / peaks["fp64_tflops"], 5)})
        elif by > 0:
            a = by / (ms * 1e-3) / 1e9
            e.update({"bound": "hbm", "achieved": round(a, 2), "unit": "GB/s", "frac": round(a / peaks["hbm_gbs"], 5)})
        out[name] = e
    return out


def run_native(args):
    import numpy as np
    import torch

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2608_11091_b300 as P
    import workloads as W

    name = args.workload
    prob = Problem(P, W, name, seed=rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    mp = _peaks()
    # the FMA-rate probes: best of three (a single run reads a few percent low now and then)
    peaks = {"fp64_tflops": max(P.tk_fma_peak(True) for _ in range(3)),
             "fp32_tflops": max(P.tk_fma_peak(False) for _ in range(3)),
             "bf16_tflops": mp.get("bf16_tflops", 1800.0), "hbm_gbs": mp.get("hbm_gbs", 6400.0)}

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(form, steps):
        evs, its, launches, reps = [], 0, 0, None
        for i in range(steps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep, rep_a, _ = prob.step(P, form)
            e1.record(stream)
            evs.append((e0, e1))
            its += rep.iters + rep_a.iters
            launches += rep.kernel_launches + rep_a.kernel_launches
            reps = (rep, rep_a)
        barrier()
        return sum(a.elapsed_time(bb) for a, bb in evs) / 1000.0, its, launches, reps

    for _ in range(args.warmup):
        prob.step(P, "mixed")
        prob.step(P, "fp64")
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    t_mixed, it_mixed, launches, (rep_m, rep_ma) = timed("mixed", args.steps)
    k64 = max(1, min(args.steps, 5))
    t_fp64, it_fp64, _, (rep_f, rep_fa) = timed("fp64", k64)
    clocks = sampler.stop()
    t_all, steps_all = aggregate_over_ranks(t_mixed, args.steps, "cuda")
    sec_mixed = t_all / args.steps            # max over ranks of the per-step time
    sec_fp64 = t_fp64 / k64
    # the 1e-6 the step reached: true relative residuals of the last step's x and mu
    prob.step(P, "mixed")
    tr_x = P.tk_residual(prob.dop, prob.x, prob.b)
    tr_mu = P.tk_residual(prob.dop, prob.mu, prob.w, transpose=True)
    prob.step(P, "fp64")
    tr_x64 = P.tk_residual(prob.dop, prob.x, prob.b)
    tr_mu64 = P.tk_residual(prob.dop, prob.mu, prob.w, transpose=True)

    # ---------------- e2e through the public API with host buffers
    host_b = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
              for a in [np.asfortranarray(prob.wl.b.core).ravel(order='F')] +
              [f.ravel(order='F') for f in prob.wl.b.factors]]
    dev_b = [prob.b.core] + prob.b.factors
    wq = qoi_weight_np(prob.wl.b.n[0], prob.wl.b.d)
    host_w = [torch.from_numpy(np.ascontiguousarray(a.ravel(order='F'))).pin_memory()
              for a in [wq.core] + wq.factors]
    dev_w = [prob.w.core] + prob.w.factors
    host_ops = []
    for key, t in prob.dop._keep[0].items():
        host_ops.append((torch.from_numpy(np.ascontiguousarray(t.cpu().numpy().ravel(order='F'))).pin_memory(), t))
    outs_shape = [prob.x.core] + prob.x.factors + [prob.mu.core] + prob.mu.factors
    host_out = [torch.empty(t.numel(), dtype=torch.float64).pin_memory() for t in outs_shape]
    nb = prob.wl.b
    host_g = [torch.empty(int(np.prod(nb.core.shape)), dtype=torch.float64).pin_memory()] + \
             [torch.empty(f.size, dtype=torch.float64).pin_memory() for f in nb.factors]

    def flat(d):
        return d.permute(*reversed(range(d.dim()))).reshape(-1)

    h2d = sum(h.numel() * 8 for h in host_b + host_w) + sum(h.numel() * 8 for h, _ in host_ops)
    d2h = sum(h.numel() * 8 for h in host_out + host_g) + 8 * prob.wl.op.nterms
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        for h, d in list(zip(host_b, dev_b)) + list(zip(host_w, dev_w)):
            flat(d).copy_(h, non_blocking=True)
        for h, d in host_ops:
            flat(d).copy_(h, non_blocking=True)
        _, _, (dth, dcore, dfac) = prob.step(P, "mixed")
        for h, d in zip(host_out, outs_shape):
            h.copy_(flat(d), non_blocking=True)
        for h, d in zip(host_g, [dcore] + dfac):
            h.copy_(flat(d), non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_t, _ = aggregate_over_ranks(e0.elapsed_time(e1) / 1000.0, args.steps, "cuda")
    e2e_val = e2e_t / args.steps

    # ---------------- per-kernel device time (library event profiler), one step of each form
    profs = {}
    for form in ("mixed", "fp64"):
        P.tk_profile(True)
        P.tk_profile_report()
        prob.step(P, form, concurrent=False)
        profs[form] = P.tk_profile_report()
        P.tk_profile(False)
    kernels = kernel_table(profs["mixed"], peaks)
    roofline = roofline_from_profile(profs["mixed"], peaks)

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = secondary(P, W, torch, peaks)
        extras["kernels_fp64_step"] = kernel_table(profs["fp64"], peaks)

    if rank == 0:
        cpu = None if args.no_extras else oracle_baseline(name, 20.0, rep_f.iters + rep_fa.iters)
        line = {
            "metric": METRIC, "value": sec_mixed, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * sec_mixed, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16/fp32 products, f64 QR/SVD/LS",
            "data": "synthetic",
            "config": {"workload": name, "solver": "flexible RHOSVD-Tucker sGMRES (Algorithm 2), exponential-sum "
                                                   f"preconditioner q = {PRECOND_Q} ({2 * PRECOND_Q + 1} terms)",
                       "step": "forward solve + adjoint solve + adjoint contractions to rel. residual 1e-6",
                       "n": prob.wl.b.n, "rhs_rank": prob.wl.b.r, "rhs": "seeded smooth factors",
                       "rank_cap": prob.prm.rank_cap, "sketch_s": prob.prm.sketch_s,
                       "oversample_p": prob.prm.oversample_p, "ktrunc": prob.prm.ktrunc, "tol": TOL,
                       "mixed_seconds": round(sec_mixed, 5), "fp64_seconds": round(sec_fp64, 5),
                       "mixed_speedup": round(sec_fp64 / sec_mixed, 4),
                       "mixed_iters": [rep_m.iters, rep_ma.iters], "fp64_iters": [rep_f.iters, rep_fa.iters],
                       "mixed_iters_per_s": round(it_mixed / t_mixed, 2), "fp64_iters_per_s": round(it_fp64 / t_fp64, 2),
                       "true_rel_residual": {"mixed_x": tr_x, "mixed_mu": tr_mu, "fp64_x": tr_x64, "fp64_mu": tr_mu64},
                       "reached_1e-6": bool(max(tr_x, tr_mu, tr_x64, tr_mu64) <= TOL),
                       "solves_per_s_all_ranks": round(2 * steps_all / t_all, 3),
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": {"value": e2e_val, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "peaks": {k: round(v, 3) for k, v in peaks.items()},
            "kernels": kernels,
            "cpu_baseline": cpu,
            "extras": extras,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


def roofline_from_profile(prof, peaks):
    """Dominant kernel (by device time) of the step with its algorithmic rate against its pipe's
    measured peak: FP64 FMA rate (tk_fma_peak, measured in this run), BF16 tensor (MEASURED_PEAKS
    burst figure) or HBM copy bandwidth."""
    if not prof:
        return None
    tab = kernel_table(prof, peaks)
    name = max(prof.items(), key=lambda kv: kv[1][1])[0]
    e = tab[name]
    n, ms, fl, by = prof[name]
    # DRAM bytes per launch of the dominant kernel from the ncu capture of this workload
    # (profiles/qr_svd_gemm_tc_poisson3d_n1024.md: the two ST-HOSVD QRs captured on three
    # clusters, 2.79 and 2.63 MB)
    traffic = {"qr": 2.71e6}.get(name)
    out = {"kernel": name, "launches": n, "avg_us": e["avg_us"], "share": e["share"], "traffic": traffic,
           "bound": e.get("bound"), "achieved": e.get("achieved"), "unit": e.get("unit"), "frac": e.get("frac")}
    if e.get("bound") == "alu":
        out.update({"peak": round(peaks["fp64_tflops"], 4), "flops_per_launch": fl / max(n, 1),
                    "peak_source": "FP64 FMA rate measured in this run (tk_fma_peak, 8 DFMA chains per thread, best of three)"})
    elif e.get("bound") == "tensor":
        out.update({"peak": peaks["bf16_tflops"], "flops_per_launch": fl / max(n, 1),
                    "peak_source": "MEASURED_PEAKS bf16_tflops (cuBLAS bf16 GEMM burst)"})
    elif e.get("bound") == "hbm":
        out.update({"peak": peaks["hbm_gbs"], "bytes_per_launch": by / max(n, 1),
                    "peak_source": "MEASURED_PEAKS hbm_gbs (copy)"})
    return out


def _timed_solve(P, torch, dop, b, opts):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, rep = P.tk_solve(dop, b, opts)
    torch.cuda.synchronize()
    return x, rep, time.perf_counter() - t0


def regularisation_study(P, W, torch):
    """Noisy deblurring (n = 32, 2% noise): relative reconstruction error after 10 / 20 / 40
    iterations of Algorithms 2 and 1, with and without projected Tikhonov + GCV in the
    least-squares step (Section 4.3), on the noisy data as given and after the data are compressed
    by a truncated HOSVD of relative tolerance tau, as the paper compresses its data before
    solving.  The compression is RoundSum with rank cap n, so the range finder spans every mode
    exactly and only the ST-HOSVD truncation (tail energy <= tau^2 ||B||^2) acts."""
    wl = W.deblur3d_noisy(32, 0, None)
    dop = P.DeviceOperator(wl.op)
    b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
    xt = P.DeviceTucker.from_numpy(wl.x_true.core, wl.x_true.factors)
    xt_norm = P.tk_sum_norm([xt], [1.0])
    b_norm = P.tk_sum_norm([b], [1.0])
    reg = {}
    rhs = [("", b)]
    for tau in (0.01, 0.05):
        bc, ranks = P.tk_roundsum([b], [1.0], P.Options(rank_cap=32, oversample_p=5, round_tol=tau, seed=11))
        reg[f"compressed_rhs_tol{tau}"] = {"ranks": ranks, "rel_compression_error":
                                           round(P.tk_sum_norm([bc, b], [1.0, -1.0]) / b_norm, 4)}
        rhs.append((f"tol{tau}_rhs ", bc))
    for rhs_label, r in rhs:
        for label, variant, s_, tik in [("sgmres", 'rhosvd', 128, False), ("sgmres+tikhonov_gcv", 'rhosvd', 128, True),
                                        ("gmres", 'gmres', 0, False), ("gmres+tikhonov_gcv", 'gmres', 0, True)]:
            errs = {}
            for it in [10, 20, 40]:
                prm = W.SolverParams(variant, 32, s_, 5, it, 1e-12, seed=0, tikhonov=tik)
                x, rep, dt = _timed_solve(P, torch, dop, r, P.Options.from_params(prm))
                errs[f"rre_at_{it}"] = round(P.tk_sum_norm([x, xt], [1.0, -1.0]) / xt_norm, 4)
                errs[f"seconds_{it}"] = round(dt, 4)
            reg[rhs_label + label] = errs
    return reg


def secondary(P, W, torch, peaks):
    """Other workloads of the method, FP64 and mixed form, one solve each after a warm-up
    (reported, not the headline): iterations/s, true residual, and the mixed result's distance
    from the FP64 one (relative Tucker-form difference of the solutions; the two forms draw
    different sketch matrices, so this is the randomized compression's own spread plus the
    reduced-precision error).  The convection-diffusion and 4-D MLN workloads also get a
    per-kernel table (one more solve of each form with the library's event profiler on)."""
    profiled = ("convdiff3d_n256", "varcoef4d_n128")
    out = {}
    for name in ["convdiff3d_n256", "poisson3d_n32", "deblur3d_n128", "varcoef4d_n128", "poisson3d_n1024_gaussian"]:
        wl = W.workload(name)
        prm = wl.params
        pc = None
        if name == "poisson3d_n1024_gaussian":
            prm.maxit = 10
            pc = PRECOND_Q
        dop = P.DeviceOperator(wl.op)
        b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
        entry = {"variant": prm.variant}
        forms = ["fp64", "mixed"]
        xs = {}
        for form in forms:
            opts = P.Options.from_params(prm, precision=form)

            def solve():
                if pc is None:
                    return P.tk_solve(dop, b, opts)
                return P.tk_solve_expsum(dop, pc, b, opts)
            solve()                     # warm-up (workspace, module load)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, rep = solve()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            xs[form] = x
            tr = P.tk_residual(dop, x, b)
            entry[form] = {"iters": rep.iters, "status": rep.status, "seconds": round(dt, 4),
                           "iters_per_s": round(rep.iters / dt, 2), "sketched_res": float(f"{rep.sketched_res:.4g}"),
                           "true_rel_residual": float(f"{tr:.4g}")}
            if name in profiled:
                P.tk_profile(True)
                P.tk_profile_report()
                solve()
                torch.cuda.synchronize()
                out[f"kernels_{name}_{form}"] = kernel_table(P.tk_profile_report(), peaks)
                P.tk_profile(False)
        if len(xs) == 2:
            entry["mixed_vs_fp64_rel_diff_x"] = float(f"{P.tk_sum_norm([xs['mixed'], xs['fp64']], [1.0, -1.0]) / P.tk_sum_norm([xs['fp64']], [1.0]):.3g}")
        out[name] = entry
    # the paper's preconditioned Poisson setting: exponential-sum preconditioner (Section 3.4),
    # flexible iteration, rank-1 point-source right-hand side, n = 1000
    wl = W.workload("poisson3d_point_n1000")
    q = wl.extra["precond_q"]
    dop = P.DeviceOperator(wl.op)
    b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
    P.tk_expsum_laplacian(wl.b.n[0], 3, q)              # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pc = P.tk_expsum_laplacian(wl.b.n[0], 3, q)
    torch.cuda.synchronize()
    entry = {"precond_terms": 2 * q + 1, "precond_build_s": round(time.perf_counter() - t0, 4),
             "tol": wl.params.tol}
    for form in ["fp64", "mixed"]:
        opts = P.Options.from_params(wl.params, precision=form)
        for how, run in [("dense E_h", lambda: P.tk_solve_precond(dop, pc, b, opts)),
                         ("sine basis", lambda: P.tk_solve_expsum(dop, q, b, opts))]:
            run()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, rep = run()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            entry[f"{form} ({how})"] = {"iters": rep.iters, "status": rep.status, "seconds": round(dt, 4),
                                        "true_rel_residual": float(f"{P.tk_residual(dop, x, b):.4g}"),
                                        "ranks": rep.out_rank}
    opts = P.Options.from_params(wl.params)
    x, rep, dt = _timed_solve(P, torch, dop, b, opts)
    entry["unpreconditioned"] = {"iters": rep.iters, "status": rep.status, "seconds": round(dt, 4),
                                 "true_rel_residual": P.tk_residual(dop, x, b)}
    out["poisson3d_point_n1000_expsum_q8"] = entry
    out["regularisation_deblur3d_noisy_n32"] = regularisation_study(P, W, torch)
    # MLN-Tucker sGMRES, full vs memory-efficient sketches (Section 3.3, r_sol = p_sol = 12)
    wl = W.workload("varcoef4d_n128")
    dop = P.DeviceOperator(wl.op)
    b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
    mem = {}
    r, p, n, d = wl.params.rank_cap, wl.params.oversample_p, wl.b.n[0], wl.b.d
    for label, rs, ps in [("full", 0, 0), ("save_memory r_sol=12 p_sol=12", 12, 12)]:
        prm = copy.copy(wl.params)
        prm.r_sol, prm.p_sol = rs, ps
        opts = P.Options.from_params(prm)
        P.tk_solve(dop, b, opts)
        x, rep, dt = _timed_solve(P, torch, dop, b, opts)
        side, cols = (r + p, r) if rs == 0 else (rs + ps, rs)
        mem[label] = {"iters": rep.iters, "seconds": round(dt, 4), "iters_per_s": round(rep.iters / dt, 2),
                      "stored_sketch_bytes_per_iteration": 8 * (side ** d + d * n * cols),
                      "true_rel_residual": P.tk_residual(dop, x, b), "out_rank": rep.out_rank}
    out["mln_memory_varcoef4d_n128"] = mem
    # Algorithm 1 (full Arnoldi) against Algorithm 2 (short recurrence), same RoundSum settings
    wl = W.workload("convdiff3d_n256")
    dop = P.DeviceOperator(wl.op)
    b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
    cmp = {}
    for variant, prm in [("gmres (Algorithm 1)", W.SolverParams('gmres', 32, 0, 5, 30, 1e-6, seed=0)),
                         ("sgmres (Algorithm 2)", W.SolverParams('rhosvd', 32, 128, 5, 30, 1e-6, seed=0))]:
        opts = P.Options.from_params(prm)
        P.tk_solve(dop, b, opts)
        x, rep, dt = _timed_solve(P, torch, dop, b, opts)
        cmp[variant] = {"iters": rep.iters, "seconds": round(dt, 4), "iters_per_s": round(rep.iters / dt, 2),
                        "res_hist_last": rep.res_hist[-1], "true_rel_residual": P.tk_residual(dop, x, b)}
    out["gmres_vs_sgmres_convdiff3d_n256_30it"] = cmp
    # gradient of the quantity of interest l = <w, x> (w smooth, rank 1) on the deblurring workload
    # (n = 128, lam = 1e-2, cap 32): forward solve and adjoint solve L^T mu = w run concurrently,
    # then the contractions; the adjoint's true residual shows the gradient's accuracy (its closed
    # form through the blur's eigenbasis is checked in the tests)
    wl = W.workload("deblur3d_n128")
    prm = W.SolverParams('rhosvd', 32, 256, 5, 60, 1e-7, seed=0)
    dop = P.DeviceOperator(wl.op)
    b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
    wq = qoi_weight_np(wl.b.n[0], wl.b.d)
    w = P.DeviceTucker.from_numpy(wq.core, wq.factors)
    grads = {}
    for form in ["fp64", "mixed"]:
        opts = P.Options.from_params(prm, precision=form)
        adj = copy.copy(opts)
        adj.transpose = True
        for _ in range(2):      # the first pass warms up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            (x, rep), (mu, rep_a) = P.tk_solve_concurrent([dict(op=dop, b=b, opts=opts), dict(op=dop, b=w, opts=adj)])
            dth, _, _ = P.tk_adjoint_grads(dop, mu, x, b)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        grads[form] = {"seconds": round(dt, 4), "forward_iters": rep.iters, "adjoint_iters": rep_a.iters,
                       "adjoint_true_rel_residual": float(f"{P.tk_residual(dop, mu, w, transpose=True):.3g}"),
                       "dl_dtheta": [float(f"{v:.8g}") for v in dth]}
    out["gradient_qoi_deblur3d_n128"] = grads
    return out


def run_profile_target(args):
    """One gradient step of each form, run serially on the default handle, nothing timed: the
    command the kernel captures (ncu) profile."""
    import torch
    import paper_2608_11091_b300 as P
    import workloads as W
    torch.cuda.set_device(0)
    if args.workload != DEFAULT_WORKLOAD:
        # another workload: one solve of each form with its own parameters (no preconditioner)
        wl = W.workload(args.workload)
        if args.maxit > 0:
            wl.params.maxit = args.maxit
        dop = P.DeviceOperator(wl.op)
        b = P.DeviceTucker.from_numpy(wl.b.core, wl.b.factors)
        for form in ("mixed", "fp64"):
            _, rep = P.tk_solve(dop, b, P.Options.from_params(wl.params, precision=form))
            torch.cuda.synchronize()
            print(f"{form}: {rep.iters} iterations, {rep.kernel_launches} launches, {rep.ms_total:.2f} ms")
        return
    prob = Problem(P, W, args.workload, seed=0)
    for form in ("mixed", "fp64"):
        rep, rep_a, _ = prob.step(P, form, concurrent=False)
        torch.cuda.synchronize()
        print(f"{form}: forward {rep.iters} / adjoint {rep_a.iters} iterations, {rep.kernel_launches + rep_a.kernel_launches}"
              f" launches, {rep.ms_total + rep_a.ms_total:.2f} ms")


def main():
    args = parse()
    if args.impl == "native" and args.profile_only:
        run_profile_target(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
