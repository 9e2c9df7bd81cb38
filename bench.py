#!/usr/bin/env python3
"""Benchmark: IsoMP steps/s at N=4096 on GB300, split-precision form vs plain FP64.

Workload (synthetic, seeded): N = 4096, h = 0.005, W0 from the seeded recipe
(complex Gaussian, (1+|j-k|)^-2 decay, spectral norm 1, traceless
skew-Hermitian), fixed-point tol 1e-12 (Frobenius), at most 50 sweeps.  A
"step" is one full IsoMP step: stream solves, complex products, updates and
residuals until convergence, then the W_{n+1} assembly.

Prints one JSON line.  `--impl reference` times the CPU oracle instead (the
paper has no GPU code), on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IsoMP steps/s @N=4096, split-prec vs FP64; ensemble steps/s, p99 step latency"
N_DEFAULT = 4096
H = 0.005
TOL = 1e-12
MAXIT = 50
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (non-tensor) nominal rate; no measured FP64 peak is available

# DRAM traffic of the split product kernel per launch (mean over one IsoMP step's
# full and lower-triangle products), from an ncu capture of dram__bytes_read.sum +
# dram__bytes_write.sum at N = 2048 scaled to N = 4096 by the tile count (x4 for the
# full product, x528/136 for the lower one); valid only for the kernel source it was
# taken on (sha256 of csrc/zt_split.cu), null otherwise.
TRAFFIC = {"sha256": "25c42489b964d7f5429b585415bd53a10b52306b458e69eb9df6f77a6e5730c9",
           "bytes_per_launch": 1414305445, "captured_n": 2048}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


_T0 = time.perf_counter()


def _log(msg):
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier_max(value: float, ws: int):
    """Maximum of a per-rank value over all ranks (the slowest rank's time)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank: int, seconds_max: float, ws: int) -> float:
    """Whole-job throughput of replicas: units every rank processed over the slowest rank's time."""
    return ws * units_per_rank / seconds_max


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def _oracle_steps(W0, nsteps):
    import oracle

    W = W0.copy()
    t0 = time.perf_counter()
    iters = []
    for _ in range(nsteps):
        W, info = oracle.isomp_step(W, H, TOL, MAXIT)
        iters.append(info.iters)
    return W, time.perf_counter() - t0, iters


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2206_05466_gb300.inputs import vorticity_w0

    N = args.n
    W0 = vorticity_w0(N, seed=0)
    # each step is one full oracle IsoMP step; the count is bounded so the run ends in minutes
    est = None
    nwarm = min(args.warmup, 1)
    W = W0
    if nwarm:
        W, t, _ = _oracle_steps(W, 1)
        est = t
    nsteps = args.steps
    if est is not None and est * nsteps > 240.0:
        nsteps = max(1, int(240.0 / est))
    W, t, iters = _oracle_steps(W, nsteps)
    v = nsteps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": ws,
            "steps": nsteps, "warmup": nwarm, "ms_per_step": 1e3 * t / nsteps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"IsoMP N={N} h={H} seeded W0, tol {TOL} Frobenius, maxit {MAXIT}",
                       "N": N, "h": H, "impl": "CPU oracle (NumPy/SciPy complex128)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": _cores(), "kind": "oracle",
                             "sample": f"{nsteps} IsoMP steps at N={N} from the seeded W0 (after {nwarm} warm-up)"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sweeps": iters}
    print(json.dumps(line), flush=True)
    return 0


def _tuning(args, N, h=H):
    """Split-product tuning: autotuned (cached per N, step size and GPU) or fixed from the flags."""
    if args.tuning == "auto":
        from paper_2206_05466_gb300 import autotune

        res = autotune.autotune(N, target=args.tune_target, step_h=h)
        timed = sorted((t for t in res["trials"] if "ms" in t), key=lambda t: t["ms"])
        return dict(res["tuning"]), {"mode": "auto", "target_rel_err": args.tune_target,
                                     "probe_rel_err": res["rel_err"], "probe_ms": res["ms"],
                                     "second_product": res.get("gemm2"),
                                     "candidates": len(res["trials"]),
                                     "fastest": [{**t["tuning"], "ms": round(t["ms"], 3),
                                                  "rel_err": t["rel_err"]} for t in timed[:6]]}
    tun = dict(slices=args.slices, digit_bits=args.digit_bits, exact_groups=args.exact_groups,
               tile_order=args.tile_order, no_persistent=args.no_persistent, slices2=args.slices2)
    return tun, {"mode": "fixed"}


def run_profile(args):
    """Kernels only, for profiler captures: --warmup + --steps IsoMP steps of the
    bench workload with a fixed tuning (or the FP64 form), nothing else."""
    import torch

    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import vorticity_w0

    torch.cuda.set_device(0)
    N = args.n
    if args.fp64:
        plan, tun = z.Plan(N, z.PRECISION_FP64), {}
    else:
        tun, _ = _tuning(args, N)
        plan = z.Plan(N, z.PRECISION_SPLIT, **tun)
    W = torch.from_numpy(vorticity_w0(N, seed=0)).cuda()
    iters = []
    for _ in range(args.warmup + args.steps):
        iters.append(z.isomp_step(plan, W, H, TOL, MAXIT)["iters"])
    torch.cuda.synchronize()
    print(json.dumps({"mode": "profile", "N": N, "precision": "fp64" if args.fp64 else "split", "tuning": tun,
                      "steps": args.warmup + args.steps, "sweeps": iters, "launches": plan.launch_count()}),
          flush=True)
    plan.close()
    return 0


def _casimir_drift(W0, W1, ks=(2, 3, 4)):
    """Relative drift of C_k = tr(W^k) and of the spectrum (eigenvalues i mu of W)."""
    import numpy as np

    mu0 = np.linalg.eigvalsh(-1j * W0)
    mu1 = np.linalg.eigvalsh(-1j * W1)
    out = {}
    for k in ks:
        out[f"C{k}"] = float(abs(np.sum(mu1 ** k) - np.sum(mu0 ** k)) / np.sum(np.abs(mu0) ** k))
    out["spectrum_max_abs"] = float(np.max(np.abs(mu1 - mu0)))
    return out


def run_casimir(args):
    """Long run: Casimir, eigenvalue and energy drift after --steps steps, split and (optionally) FP64
    form, with the on-device Casimirs and kinetic-energy spectrum timed."""
    import torch

    import numpy as np

    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import vorticity_w0

    N, steps = args.n, args.steps
    W0 = vorticity_w0(N, seed=0)
    res = {"mode": "casimir", "N": N, "h": H, "steps": steps, "tol": TOL, "data": "synthetic"}
    forms = [("split", z.PRECISION_SPLIT)] + ([("fp64", z.PRECISION_FP64)] if args.fp64_steps > 0 else [])
    for name, prec in forms:
        if prec == z.PRECISION_SPLIT:
            tun, info = _tuning(args, N)
            plan = z.Plan(N, prec, **tun)
            res["split_tuning"] = tun
        else:
            plan = z.Plan(N, prec)
        W = torch.from_numpy(W0).cuda()
        c0 = z.zeitlin_casimirs(plan, W)   # on the device, the plan's products
        E0 = z.zeitlin_energy_spectrum(plan, W).cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = z.isomp_run(plan, W, H, steps, TOL, MAXIT)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        tc = time.perf_counter()
        c1 = z.zeitlin_casimirs(plan, W)
        t_cas = time.perf_counter() - tc
        st = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(st)
        E1 = z.zeitlin_energy_spectrum(plan, W)
        ev1.record(st)
        torch.cuda.synchronize()
        t_spec = ev0.elapsed_time(ev1)
        E1 = E1.cpu().numpy()
        W1 = W.cpu().numpy()
        drift = _casimir_drift(W0, W1)
        mu0 = np.abs(np.linalg.eigvalsh(-1j * W0))
        dev = {f"C{k}": float(abs(c1[k] - c0[k]) / np.sum(mu0 ** k)) for k in (2, 3, 4, 5)}
        res[name] = {"steps_per_s": steps / dt, "run_stats": r, "drift": drift,
                     "device_casimir_drift": dev, "device_casimirs_ms": t_cas * 1e3,
                     "device_spectrum_ms": t_spec,
                     "energy_rel_drift": float(abs(E1.sum() - E0.sum()) / E0.sum()),
                     "spectrum_l_peak": [int(np.argmax(E0)), int(np.argmax(E1))],
                     "trace_abs": float(abs(W1.trace())), "skew_err": float(abs(W1 + W1.conj().T).max())}
        plan.close()
    print(json.dumps(res), flush=True)
    return 0


def run_spectrum(args):
    """Kinetic-energy spectrum alone (zeitlin_energy_spectrum at --n): time per call on the
    stream with CUDA events, and its FP64 rate against the nominal FP64 peak."""
    import torch

    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import vorticity_w0

    torch.cuda.set_device(0)
    N = args.n
    plan = z.Plan(N)
    W = torch.from_numpy(vorticity_w0(N, seed=0)).cuda()
    E = torch.empty(N, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        z.zeitlin_energy_spectrum(plan, W, E)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(args.steps):
        z.zeitlin_energy_spectrum(plan, W, E)
    ev1.record(st)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    # algorithmic FP64 work per (l, m): half accumulation steps (3 FMA: the complex dot
    # product with the folded lower diagonal and the norm) and half - 1 recurrence steps
    # (2 FMA + 2 MUL) over the half diagonal, half = ceil((N - m) / 2)
    flops = 0
    for m in range(N):
        half = (N - m + 1) // 2
        flops += (N - m) * (6 * half + 6 * (half - 1))
    tf = flops / (ms * 1e-3) / 1e12
    out = {"mode": "spectrum", "N": N, "calls": args.steps, "warmup": args.warmup, "ms_per_call": ms,
           "gpu_launches_per_call": 2, "fp64_flop_per_call": flops,
           "roofline": {"bound": "fp64", "achieved": tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                        "frac": tf / FP64_NOMINAL_TFLOPS, "peak_kind": "nominal"},
           "total_energy": float(E.sum().item()), "clocks": clocks, "data": "synthetic"}
    plan.close()
    print(json.dumps(out), flush=True)
    return 0


def _ensemble(args, tun, steps, graph=True):
    """Ensemble of independent instances advanced by grouped (batched) steps."""
    import numpy as np
    import torch

    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import ensemble_sizes, vorticity_w0

    sizes = ensemble_sizes(args.ens_count, seed=0)
    # the tuning is the one chosen for the largest member size at the ensemble's step
    # size (the second product's digits depend on h); with fixed flags the members keep
    # the full digit count for both products
    if args.tuning == "auto":
        tun, _ = _tuning(args, max(sizes), h=0.01)
    else:
        tun = {k: v for k, v in tun.items() if k != "slices2"}
    cache = {}
    plans, Ws = [], []
    for k, N in enumerate(sizes):
        key = (N, k % 8)   # W0 recipe, 8 seeds per size (generation is host-side and slow at large N)
        if key not in cache:
            cache[key] = vorticity_w0(N, seed=key[1])
        plans.append(z.Plan(N, z.PRECISION_SPLIT, **tun))
        Ws.append(torch.from_numpy(cache[key]).cuda())
    b = z.Batch(plans, Ws, [0.01] * len(plans))
    b.set_graph(graph)
    for _ in range(2):
        b.step()
    torch.cuda.synchronize()
    l0 = b.launch_count()
    t0 = time.perf_counter()
    r = b.run(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    launches = b.launch_count() - l0
    # the same instances stepped one plan at a time (a few steps) for comparison
    seq_steps = 2
    t1 = time.perf_counter()
    for _ in range(seq_steps):
        for p, W in zip(plans, Ws):
            z.isomp_step(p, W, 0.01)
    torch.cuda.synchronize()
    dts = time.perf_counter() - t1
    b.close()
    for p in plans:
        p.close()
    n = len(plans)
    # FP64-equivalent rate: the algorithmic flops of both products of every sweep and of
    # the final assembly (8 N^3 + 4 N^2 (N + 1) each), with the mean sweep count
    mean_sweeps = r["total_iters"] / (n * steps)
    alg = sum((mean_sweeps + 1) * (8.0 * N ** 3 + 4.0 * N * N * (N + 1.0)) for N in sizes) * steps
    return {"instances": n, "sizes": {str(N): sizes.count(N) for N in sorted(set(sizes))}, "h": 0.01,
            "tuning": tun, "fp64_equivalent_tflops": alg / dt / 1e12, "mean_sweeps": mean_sweeps,
            "steps": steps, "graph": graph, "value": n * steps / dt, "unit": "instance-steps/s",
            "batched_steps_per_s": steps / dt, "ms_per_batched_step": 1e3 * dt / steps,
            "launches_per_batched_step": launches / steps, "all_converged": r["all_converged"],
            "max_sweeps": r["max_iters"],
            "one_plan_at_a_time": {"value": n * seq_steps / dts, "unit": "instance-steps/s"}}


def _serving(args, duration):
    """Poisson job stream, admission by device footprint and class step latency, continuous batching."""
    import numpy as np

    from paper_2206_05466_gb300 import serving
    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import serving_jobs, vorticity_w0

    stream = serving_jobs(duration, rate_per_s=50.0, seed=0)
    cache = {}
    jobs = []
    for (t, N, nsteps, jid) in stream:
        key = (N, jid % 4)
        if key not in cache:
            cache[key] = vorticity_w0(N, seed=key[1])
        prec = z.PRECISION_SPLIT if jid % 2 == 0 else z.PRECISION_FP64
        jobs.append(serving.Job(jid=jid, N=N, nsteps=nsteps, h=0.01, precision=prec, arrival=t, W0=cache[key]))
    rep = serving.Server(int(args.serve_budget_gb * 1e9), target_step_ms=args.serve_target_ms).run(
        jobs, time_limit=duration)
    rep.pop("results", None)
    rep.update({"arrivals": len(jobs), "rate_per_s": 50.0, "duration_s": duration,
                "budget_gb": args.serve_budget_gb, "precision_mix": "even job ids split, odd FP64",
                "sizes": "N in {256,512,1024,2048} w.p. .4/.3/.2/.1, 200-2000 steps"})
    return rep


def _drift_leg(N, prec, h, steps, tun=None):
    """`steps` IsoMP steps from the seeded W0; relative drift of the Casimirs C2..C5
    (device, with an FP64 plan's products) and of the spectrum (host eigenvalues)."""
    import numpy as np
    import torch

    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import vorticity_w0

    W0 = vorticity_w0(N, seed=0)
    plan = z.Plan(N, prec, **(tun or {}))
    meas = z.Plan(N, z.PRECISION_FP64)   # Casimirs with FP64 products: rounding far below the drift bound
    W = torch.from_numpy(W0).cuda()
    c0 = z.zeitlin_casimirs(meas, W)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = z.isomp_run(plan, W, h, steps, TOL, MAXIT)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    c1 = z.zeitlin_casimirs(meas, W)
    W1 = W.cpu().numpy()
    plan.close()
    meas.close()
    mu0 = np.linalg.eigvalsh(-1j * W0)
    mu1 = np.linalg.eigvalsh(-1j * W1)
    scale = {k: float(np.sum(np.abs(mu0) ** k)) for k in (2, 3, 4, 5)}
    per = 1000.0 / steps
    dev = {f"C{k}": float(abs(c1[k] - c0[k]) / scale[k]) * per for k in (2, 3, 4, 5)}
    host = {f"C{k}": float(abs(np.sum(mu1 ** k) - np.sum(mu0 ** k)) / scale[k]) * per for k in (2, 3, 4)}
    return {"N": N, "precision": "split" if prec == z.PRECISION_SPLIT else "fp64", "h": h, "steps": steps,
            "steps_per_s": steps / dt, "sweeps_total": r["total_iters"], "all_converged": r["all_converged"],
            "per_1000_steps": dev, "max_per_1000_steps": max(dev.values()),
            "host_eig_per_1000_steps": host,
            "spectrum_max_abs_per_1000_steps": float(np.max(np.abs(mu1 - mu0))) * per,
            "measure": "C_k = tr(W^k) on the device with FP64 products, relative to sum_j |lambda_j|^k of W0; "
                       "host: power sums of eigvalsh(-i W)",
            "bound": 1e-10}


def _dense_product(N, tun):
    """Throughput of the split product with every digit pair multiplied (dense=1): the
    kernel's efficiency without the zero-tile skipping the decaying workload allows."""
    import torch

    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import vorticity_w0

    t = dict(tun)
    t["dense"] = 1
    plan = z.Plan(N, z.PRECISION_SPLIT, **t)
    W = torch.from_numpy(vorticity_w0(N, seed=0)).cuda()
    P = torch.empty_like(W)
    C = torch.empty_like(W)
    z.zeitlin_stream_solve(plan, W, P)
    for _ in range(2):
        z.zt_zgemm_skew(plan, P, W, C)
    torch.cuda.synchronize()
    plan.set_timing(True)
    reps = 5
    for _ in range(reps):
        z.zt_zgemm_skew(plan, P, W, C)
    torch.cuda.synchronize()
    k = plan.kernel_time(z.KERNEL_PRODUCT)
    plan.set_timing(False)
    plan.close()
    tf = k["work"] / (k["total_ms"] / 1e3) / 1e12
    peak = _peaks()["bf16_tflops"]   # timed alone, back to back: the burst peak
    return {"N": N, "launches": k["launches"], "avg_launch_ms": k["total_ms"] / k["launches"],
            "achieved_tflops": tf, "peak_tflops": peak, "frac": tf / peak,
            "peak_source": f"{_peaks()['source']} bf16 burst",
            "fp64_equivalent_tflops": k["work_alg"] / (k["total_ms"] / 1e3) / 1e12}


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2206_05466_gb300 import zeitlin as z
    from paper_2206_05466_gb300.inputs import vorticity_w0

    N = args.n
    peaks = _peaks()
    W0 = vorticity_w0(N, seed=rank)   # replicas: each rank its own seeded instance
    tun, tune_info = _tuning(args, N)
    plan = z.Plan(N, z.PRECISION_SPLIT, **tun)
    Wd = torch.from_numpy(W0).cuda()
    stream = torch.cuda.current_stream()

    # ---- warm-up ----
    _log('warm-up')
    iters = []
    for _ in range(args.warmup):
        iters.append(z.isomp_step(plan, Wd, H, TOL, MAXIT)["iters"])
    torch.cuda.synchronize()

    # ---- timed region: exactly K steps, inputs resident in HBM ----
    _log('timed region')
    clk = ClockSampler(local)
    clk.start()
    plan.set_timing(True)
    launches0 = plan.launch_count()
    _barrier(ws)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step_iters, host_ms = [], []
    for _ in range(args.steps):
        th = time.perf_counter()
        step_iters.append(z.isomp_step(plan, Wd, H, TOL, MAXIT)["iters"])
        host_ms.append(1e3 * (time.perf_counter() - th))
    ev1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    gpu_launches = plan.launch_count() - launches0
    t_ms = ev0.elapsed_time(ev1)
    clocks = clk.stop()
    prod = plan.kernel_time(z.KERNEL_PRODUCT)
    solve = plan.kernel_time(z.KERNEL_SOLVE)
    split = plan.kernel_time(z.KERNEL_SPLIT)
    upd = plan.kernel_time(z.KERNEL_UPDATE)
    plan.set_timing(False)
    t_max = _barrier_max(t_ms, ws)
    value = _job_rate(args.steps, t_max / 1e3, ws)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed: a
    # trajectory whose state lives on the host (each step's input is the previous
    # step's output, copied in; its result copied out) ----
    _log('e2e')
    Wh = torch.from_numpy(W0.copy()).pin_memory()
    Wout = torch.empty_like(Wh).pin_memory()
    Wd2 = torch.empty_like(Wd)
    e2e_steps = max(1, args.steps)   # as many as the timed region: a host-side stall of one step stays a small share
    for _ in range(2):   # untimed: the plan's history for this buffer
        Wd2.copy_(Wh, non_blocking=True)
        z.isomp_step(plan, Wd2, H, TOL, MAXIT)
        Wh.copy_(Wd2, non_blocking=True)
        torch.cuda.synchronize()
    _barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Wd2.copy_(Wh, non_blocking=True)
        z.isomp_step(plan, Wd2, H, TOL, MAXIT)
        Wout.copy_(Wd2, non_blocking=True)
        torch.cuda.synchronize()
        Wh, Wout = Wout, Wh
    t_e2e = _barrier_max(time.perf_counter() - t0, ws)
    e2e = {"value": _job_rate(e2e_steps, t_e2e, ws), "unit": "steps/s", "h2d_bytes_per_step": int(Wh.numel() * 16),
           "d2h_bytes_per_step": int(Wout.numel() * 16), "steps": e2e_steps}

    # ---- plain FP64 form on the same GPU (same workload) ----
    _log('fp64 form')
    fp64 = None
    if args.fp64_steps > 0:
        plan64 = z.Plan(N, z.PRECISION_FP64)
        W64 = torch.from_numpy(W0).cuda()
        z.isomp_step(plan64, W64, H, TOL, MAXIT)
        torch.cuda.synchronize()
        plan64.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            z.isomp_step(plan64, W64, H, TOL, MAXIT)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        p64 = plan64.kernel_time(z.KERNEL_PRODUCT)
        fp64 = {"value": args.fp64_steps / (t64 / 1e3), "unit": "steps/s", "ms_per_step": t64 / args.fp64_steps,
                "steps": args.fp64_steps, "warmup": 1,
                "product_fp64_tflops": p64["work"] / (p64["total_ms"] / 1e3) / 1e12 if p64["total_ms"] else None}
        plan64.close()
        del W64

    # ---- accuracy and CPU baseline (rank 0): oracle vs both forms after the same steps ----
    _log('oracle baseline')
    cpu_baseline, accuracy = None, None
    if rank == 0 and args.oracle_steps > 0:
        k = args.oracle_steps
        Wo, t_or, or_iters = _oracle_steps(W0, k)
        cpu_baseline = {"value": k / t_or, "unit": "steps/s", "cores": _cores(), "kind": "oracle",
                        "sample": f"{k} IsoMP steps at N={N} from the seeded W0 (same workload)"}
        acc = {}
        for name, prec in (("split", z.PRECISION_SPLIT), ("fp64", z.PRECISION_FP64)):
            if name == "fp64" and args.fp64_steps <= 0:
                continue
            pl = plan if prec == z.PRECISION_SPLIT else z.Plan(N, z.PRECISION_FP64)
            Wc = torch.from_numpy(W0).cuda()
            for _ in range(k):
                z.isomp_step(pl, Wc, H, TOL, MAXIT)
            got = Wc.cpu().numpy()
            acc[f"{name}_rel_fro_err_after_{k}_steps"] = float(np.linalg.norm(got - Wo) / np.linalg.norm(Wo))
            if pl is not plan:
                pl.close()
        accuracy = acc

    drift = dense = None
    if rank == 0 and args.casimir_steps > 0:
        _log("casimir drift (split)")
        drift = {"split": _drift_leg(N, z.PRECISION_SPLIT, H, args.casimir_steps, tun)}
        if args.casimir_n2 > 0 and args.casimir_n2 != N:   # the workload's second precision-form size
            _log(f"casimir drift (split, N={args.casimir_n2})")
            tun2, _ = _tuning(args, args.casimir_n2)
            drift[f"split_n{args.casimir_n2}"] = _drift_leg(args.casimir_n2, z.PRECISION_SPLIT, H,
                                                            args.casimir_steps, tun2)
            drift[f"split_n{args.casimir_n2}"]["tuning"] = tun2
        if args.casimir_fp64_steps > 0:
            _log("casimir drift (fp64)")
            drift["fp64"] = _drift_leg(args.casimir_fp64_n, z.PRECISION_FP64, 0.01, args.casimir_fp64_steps)
    if rank == 0 and args.dense_product:
        _log("dense product")
        dense = _dense_product(N, tun)
    ens = serve = None
    _log("ensemble")
    if rank == 0 and args.ens_steps > 0:
        ens = _ensemble(args, tun, args.ens_steps)
    if rank == 0 and args.serve_seconds > 0:
        _log("serving")
        serve = _serving(args, args.serve_seconds)
    _log("done")
    if rank != 0:
        return 0
    s1 = tun["slices"]
    s2 = tun.get("slices2") or s1
    pairs = {"first": s1 * (s1 + 1) / 2, "second": s2 * (s2 + 1) / 2}
    # dense equivalent: every digit pair on every computed tile of the timed launches (the
    # full products are 8 N^3 of the 8 N^3 + 4 N^2 (N + 1) algorithmic flops of a sweep)
    f1 = 8.0 * N ** 3 / (8.0 * N ** 3 + 4.0 * N * N * (N + 1.0))
    dense_work = (pairs["first"] * f1 + pairs["second"] * (1 - f1)) * prod["work_alg"] if prod["work_alg"] else None
    achieved = prod["work"] / (prod["total_ms"] / 1e3) / 1e12 if prod["total_ms"] else None
    peak = peaks["bf16_tflops_sustained"]
    src = open(os.path.join(ROOT, "paper_2206_05466_gb300", "csrc", "zt_split.cu"), "rb").read()
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["sha256"] == hashlib.sha256(src).hexdigest() else None
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (products: bf16 digit slices, fp32/int64 accumulate)",
        "data": "synthetic",
        "config": {"workload": f"IsoMP N={N} h={H} seeded W0 (decay 2, spectral norm 1), tol {TOL} Frobenius, "
                               f"maxit {MAXIT}, split-precision products s={tun['slices']} beta={tun['digit_bits']}"
                               f" (second product s={tun.get('slices2') or tun['slices']})",
                   "N": N, "h": H, "precision": "split", "tuning": tun, "tuning_source": tune_info,
                   "parallelism": f"replicas x{ws}",
                   "l2": "working set > L2 (digit planes ~1.4 GB + 6 matrices of 268 MB)"},
        "sweeps_per_step": statistics.mean(step_iters) if step_iters else None,
        "step_host_ms": {"min": min(host_ms), "median": statistics.median(host_ms), "max": max(host_ms)}
        if host_ms else None,
        "gpu_launches": gpu_launches,
        "e2e": e2e,
        "fp64_form": fp64,
        "roofline": {"bound": "tensor", "kernel": "zgemm_split_kernel", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": (f"ncu DRAM bytes at N={TRAFFIC['captured_n']}, scaled by tile count"
                                        if traffic else "source changed since the capture"),
                     "peak_source": f"{peaks['source']} bf16 sustained",
                     "work": "BF16 digit-pair MMA units issued (2 x 128 x 256 x 64 flops each, counted on the "
                             "device; exactly-zero digit tiles are skipped)",
                     "dense_units_fraction_issued": prod["work"] / dense_work if dense_work else None,
                     "launches": prod["launches"], "avg_launch_ms": prod["total_ms"] / max(1, prod["launches"]),
                     "fp64_equivalent_tflops": prod["work_alg"] / (prod["total_ms"] / 1e3) / 1e12
                     if prod["total_ms"] else None,
                     "pairs": pairs},
        "kernels_ms_per_step": {"product": prod["total_ms"] / args.steps, "solve": solve["total_ms"] / args.steps,
                                "split": split["total_ms"] / args.steps, "update": upd["total_ms"] / args.steps},
        "solve_hbm": {"achieved_gbs": solve["work"] / (solve["total_ms"] / 1e3) / 1e9 if solve["total_ms"] else None,
                      "peak_gbs": peaks["hbm_gbs"]},
        "cpu_baseline": cpu_baseline,
        "accuracy": accuracy,
        "ensemble": ens,
        "serving": serve,
        "casimir_drift_per_1000": drift,
        "dense_product": dense,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--mode", default="bench", choices=["bench", "casimir", "ensemble", "serving", "profile", "spectrum"])
    ap.add_argument("--ens-count", type=int, default=256)
    ap.add_argument("--ens-steps", type=int, default=20)
    ap.add_argument("--serve-seconds", type=float, default=120.0)
    ap.add_argument("--casimir-steps", type=int, default=1000,
                    help="split steps at --n for the Casimir drift (0: skip)")
    ap.add_argument("--casimir-fp64-n", type=int, default=1024)
    ap.add_argument("--casimir-n2", type=int, default=2048,
                    help="split-form drift leg at this second size too (0: skip)")
    ap.add_argument("--casimir-fp64-steps", type=int, default=1000,
                    help="FP64-form steps at --casimir-fp64-n, h = 0.01, for its Casimir drift (0: skip)")
    ap.add_argument("--dense-product", type=int, default=1, help="time the product with dense=1 (0: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-target-ms", type=float, default=100.0,
                    help="step latency above which a serving class admits no further job")
    ap.add_argument("--tuning", default="auto", choices=["auto", "fixed"])
    ap.add_argument("--tune-target", type=float, default=1e-11)
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--digit-bits", type=int, default=8)
    ap.add_argument("--slices2", type=int, default=0, help="fixed tuning: digits of the second product (0: slices)")
    ap.add_argument("--exact-groups", type=int, default=2)
    ap.add_argument("--tile-order", type=int, default=6)
    ap.add_argument("--no-persistent", type=int, default=0, help="fixed tuning: 1 = one tile per CTA")
    ap.add_argument("--fp64", action="store_true", help="profile mode: the FP64 form")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--oracle-steps", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "casimir":
        return run_casimir(args)
    if args.mode == "profile":
        return run_profile(args)
    if args.mode == "spectrum":
        return run_spectrum(args)
    if args.mode in ("ensemble", "serving"):
        import torch

        torch.cuda.set_device(0)
        if args.mode == "ensemble":
            tun, _ = _tuning(args, 512)
            out = _ensemble(args, tun, args.steps)
        else:
            out = _serving(args, args.serve_seconds)
        out["mode"] = args.mode
        print(json.dumps(out), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
