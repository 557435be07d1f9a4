"""Benchmark of the FS-QRPPA hot path on one GB300 (and N replicas).

Workload (geno_int8): n = 5,000 samples, p = 100,000 int8 genotypes
Bin(2, MAF), MAF ~ U(0.05, 0.5), standardised on the fly, intercept plus 5
dense N(0,1) covariates (unpenalised), G = 32 equal feature blocks,
quantiles tau in {0.1, 0.5, 0.9}, lambda = 0.1 lambda_max(tau). One step =
the whole hot path for the 3 fits: lambda_max per tau, column statistics,
eta_g by the power method, and FS-QRPPA (Algorithm 1) from a cold start to
KKT <= 1e-6. The metric is fits per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (oracle/) on a bounded sample of
the same workload. Under torchrun (N > 1) every rank runs an independent
replica (the method is not sharded across GPUs); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tau x lambda PQR fits/s to KKT<=1e-6"
UNIT = "fits/s"
TAUS = [0.1, 0.5, 0.9]
LAMBDA_FRAC = 0.1
TOL = 1e-6


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel_src_hash: str):
    """Per-launch DRAM bytes of the column pass from the committed ncu summary,
    or None when absent or taken on a different kernel source."""
    p = os.path.join(ROOT, "profiles", "k_col_tc_geno_int8.md")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_hash():
    """Hash of the sources of the column pass the committed counters describe."""
    h = hashlib.sha256()
    for f in ("k_tc.cu", "sm103_ops.cuh", "fsqr_device.cuh", "fsqr_internal.h"):
        with open(os.path.join(ROOT, "paper_2601_02826_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over the ranks (x itself without torch.distributed):
    the timed region of a multi-rank run is its slowest rank's."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def make_workload():
    from paper_2601_02826_gb300 import synth
    return synth.geno_int8()


# ------------------------------------------------------------------ GB300 arm

def fp64_plain_leg(ctx, step, B, mixed_iters, n_short, dev):
    """Plain FP64 FS-QRPPA on the GPU, one fit at a time (the metric's comparison)."""
    import torch

    from paper_2601_02826_gb300 import fsqr, synth
    from paper_2601_02826_gb300.device import upload
    walls = []
    for n_it in (n_short, 3 * n_short):
        opts = dict(tol=0.0, max_iter=n_it, precision=fsqr.FP64, max_group=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(opts)
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
    s_per_iter = max(walls[1] - walls[0], 1e-9) / (B * 2 * n_short)
    setup_s = max(walls[0] - B * n_short * s_per_iter, 0.0)
    # iteration ratio FP64 / mixed on a small problem, both solved to the tolerance
    w = synth.tiny_geno(7, 300, 500, c=2, fmt=synth.FMT_INT8, G=4, taus=(0.5,))
    dw = upload(ctx, w, device=dev)
    lam = 0.3 * ctx.lambda_max(dw.design, dw.y, 0.5, dw.omega)
    its = {}
    for prec in (fsqr.FP64, fsqr.MIXED):
        b = torch.zeros(w.P, dtype=torch.float64, device=dev)
        z = torch.zeros(w.n, dtype=torch.float64, device=dev)
        th = torch.zeros(w.n, dtype=torch.float64, device=dev)
        _, info = ctx.fit(dw.design, dw.y, 0.5, lam, dw.omega, w.block_ptr(), b, z, th,
                          opts=dict(tol=TOL, max_iter=1_000_000, precision=prec))
        its[prec] = info.iters
    ratio = its[fsqr.FP64] / max(1, its[fsqr.MIXED])
    need = float(np.mean(mixed_iters)) * ratio
    step_s = setup_s + B * need * s_per_iter
    return {"value": B / step_s, "unit": UNIT, "ms_per_iteration": s_per_iter * 1e3,
            "setup_s_per_step": setup_s, "iterations_per_fit": need,
            "iteration_ratio_fp64_over_mixed": ratio,
            "sample": (f"{B} fits one at a time, timed at {n_short} and {3 * n_short} iterations each; "
                       f"per-iteration time from the difference, set-up once per step; iterations = "
                       f"mean mixed count x FP64/mixed ratio ({its[fsqr.FP64]}/{its[fsqr.MIXED]}) of a "
                       f"300 x 500 fit solved to the tolerance in this run"),
            "precision": "fp64", "max_group": 1}



def grid_leg(ctx, dev, stream, iters, slots):
    """The tau x lambda grid (9 tau x 20 lambda from lambda_max to 0.01
    lambda_max = 180 fits; n = 10,000, p = 500,000 int8 genotypes, ragged
    feature blocks U(5k, 30k)) solved as one wide batched solve: every fit
    streams through `slots` slots sharing each X pass, and takes `iters`
    steps of Algorithm 1 (tolerance 0; a throughput sample, since fits near
    lambda_max need more than 3e5 steps to reach KKT <= 1e-6). Kernel times
    come from a profiled 20-step run before the timed one."""
    import torch

    from paper_2601_02826_gb300 import fsqr, synth
    from paper_2601_02826_gb300.device import upload
    t0 = time.perf_counter()
    w = synth.grid_int8()
    t_gen = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        dw = upload(ctx, w, device=dev)
    stream.synchronize()
    taus = w.taus
    fr = np.asarray(w.lambda_fracs)
    lm = [ctx.lambda_max(dw.design, dw.y, t, dw.omega) for t in taus]
    lam = np.array([[f * l for f in fr] for l in lm])
    B = lam.size
    beta = torch.zeros(B * w.P, dtype=torch.float64, device=dev)
    z = torch.zeros(B * w.n, dtype=torch.float64, device=dev)
    th = torch.zeros(B * w.n, dtype=torch.float64, device=dev)
    opts = dict(tol=0.0, max_iter=iters, precision=fsqr.MIXED, max_group=slots)
    ctx.profile(enable=True, reset=True)
    ctx.fit_batch(dw.design, dw.y, taus, lam, dw.omega, w.block_ptr(), beta, z, th, opts=dict(opts, max_iter=20))
    kp = ctx.profile(enable=False)
    ctx.profile(reset=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc, infos = ctx.fit_batch(dw.design, dw.y, taus, lam, dw.omega, w.block_ptr(), beta, z, th, opts=opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    p = ctx.profile()
    col_ms = kp.col_ms / max(1, kp.col_samples)
    peak, kind = measured_peaks()
    gbs = kp.col_bytes / (col_ms / 1e3) / 1e9
    fit_its = sum(i.iters for i in infos)
    setup_ms = float(np.mean([i.t_setup_ms for i in infos]))
    solve_ms = ms - setup_ms
    del dw, beta, z, th
    torch.cuda.empty_cache()
    return {"workload": "grid_int8", "n": w.n, "p": w.p, "G": len(w.block_sizes), "fits": B,
            "slots": slots, "iterations_per_fit": iters, "steps": int(p.iterations), "ms": ms,
            "setup_ms": setup_ms, "fit_iterations_per_s": fit_its / (solve_ms / 1e3),
            "ms_per_step": solve_ms / max(1, p.iterations),
            "col": {"kernel": f"k_wcol<{slots}> (X~^T Theta over all slots + beta prox)",
                    "avg_launch_ms": col_ms, "bytes_per_launch": kp.col_bytes, "achieved_gbs": gbs,
                    "peak_gbs": peak, "frac": gbs / peak, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({kind})"},
            "xbeta_and_vector_update_ms": kp.xb_ms / max(1, kp.xb_samples),
            "wide_groups": int(p.wide_groups), "gpu_launches": int(p.kernel_launches),
            "generate_s": t_gen,
            "note": "throughput sample: every fit takes the fixed number of steps (tolerance 0); "
                    "setup (column statistics, 9 lambda_max, eta) inside ms"}



def run_gb300(args, rank, world, local_rank):
    import torch

    from paper_2601_02826_gb300 import fsqr
    from paper_2601_02826_gb300.device import upload

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    stream = torch.cuda.Stream(device=dev)
    ctx = fsqr.Context(local_rank, stream.cuda_stream)
    w = make_workload()
    with torch.cuda.stream(stream):
        dw = upload(ctx, w, device=dev)
    stream.synchronize()
    gh_keep = None
    B = len(TAUS)
    bp = w.block_ptr()
    beta = torch.zeros(B * w.P, dtype=torch.float64, device=dev)
    z = torch.zeros(B * w.n, dtype=torch.float64, device=dev)
    th = torch.zeros(B * w.n, dtype=torch.float64, device=dev)
    mixed = dict(tol=TOL, max_iter=1_000_000, precision=fsqr.MIXED, digits=4, max_group=B)
    if args.profile_iters:
        # bounded run for profilers: fixed iteration count, no stop at tol
        mixed.update(tol=0.0, max_iter=args.profile_iters)

    def step(opts, infos_out=None):
        lam = [LAMBDA_FRAC * ctx.lambda_max(dw.design, dw.y, t, dw.omega) for t in TAUS]
        rc, infos = ctx.fit_batch(dw.design, dw.y, TAUS, lam, dw.omega, bp, beta, z, th, opts=opts)
        if infos_out is not None:
            infos_out.extend(infos)
        return rc

    # Kernel times come from events inside the solver, sampled during the last
    # warm-up step only; the timed steps run with the sampling off.
    for w_i in range(args.warmup):
        if w_i == args.warmup - 1:
            ctx.profile(enable=True, reset=True)
        step(mixed)
    kprof = ctx.profile(enable=False)
    if args.warmup == 0:  # no warm-up step to sample: take one extra, untimed
        ctx.profile(enable=True, reset=True)
        step(mixed)
        kprof = ctx.profile(enable=False)
    ctx.profile(enable=False, reset=True)
    infos = []
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clocks:
        e0.record(stream)
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            rc = step(mixed, infos)
            assert rc == fsqr.OK or args.profile_iters, (rc, [i.as_dict() for i in infos[-B:]])
        e1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()  # launches and iterations of the timed steps
    ms_max = max_over_ranks(ms, dev)
    fits = B * args.steps * world
    value = fits / (ms_max / 1e3)

    # roofline of the dominant kernel: the column pass (X~^T theta + prox)
    col_avg_ms = kprof.col_ms / max(1, kprof.col_samples)
    achieved = kprof.col_bytes / (col_avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = ncu_traffic(kernel_hash())

    # accuracy of the returned fits (their own stop test) and iteration counts
    iters = [i.iters for i in infos[-B:]]
    kkts = [i.kkt for i in infos[-B:]]
    # set-up inside each timed solve (column statistics, eta), reported apart
    setup_ms = [i.t_setup_ms for i in infos[::B]]

    # plain FP64 GPU FS-QRPPA: one fit at a time, cold start (comparison).
    # Per-iteration time from two run lengths (their difference removes the
    # set-up), the set-up added once per step, and FP64's own iteration count
    # estimated as the mixed fits' count times the FP64/mixed iteration ratio
    # of the same fits solved to the tolerance on a small problem in this run.
    fp64 = None
    if not args.skip_fp64 and rank == 0 and not args.profile_iters:
        fp64 = fp64_plain_leg(ctx, step, B, iters, args.fp64_iters, dev)

    # end to end through the host-buffer entry point (copies inside the call)
    e2e = None
    if not args.skip_e2e and not args.profile_iters:
        gh = torch.from_numpy(np.ascontiguousarray(w.geno).view(np.uint8)).pin_memory()
        ch = torch.from_numpy(np.ascontiguousarray(w.cov)).pin_memory()
        yh = torch.from_numpy(w.y.copy()).pin_memory()
        oh = torch.from_numpy(w.omega.copy()).pin_memory()
        bh = torch.zeros(B * w.P, dtype=torch.float64).pin_memory()
        zh = torch.zeros(B * w.n, dtype=torch.float64).pin_memory()
        thh = torch.zeros(B * w.n, dtype=torch.float64).pin_memory()
        dh = ctx.design(w.n, w.p, w.c, w.fmt, gh, w.ld, cov=ch, host=True)
        lam = [LAMBDA_FRAC * ctx.lambda_max(dw.design, dw.y, t, dw.omega) for t in TAUS]
        # warm-up: the host-buffer path allocates its device copies once
        ctx.fit_batch(dh, yh, TAUS, lam, oh, bp, bh, zh, thh, opts=dict(mixed, max_iter=20, tol=0.0), host=True)
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for _ in range(n_e2e):
            ctx.fit_batch(dh, yh, TAUS, lam, oh, bp, bh, zh, thh, opts=mixed, host=True)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, dev)
        h2d = gh.numel() + 8 * (ch.numel() + yh.numel() + oh.numel())
        d2h = 8 * (bh.numel() + zh.numel() + thh.numel())
        e2e = {"value": B * n_e2e * world / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "steps": n_e2e,
               "note": "fsqr_fit_batch_host from pinned host buffers; lambda from a device call"}

    cpu = None
    if rank == 0 and not args.skip_cpu and not args.profile_iters:
        cpu = cpu_baseline(w, iters)

    grid = None
    if not args.skip_grid and not args.profile_iters:
        del dw, gh_keep
        torch.cuda.empty_cache()
        grid = grid_leg(ctx, dev, stream, args.grid_iters, args.grid_slots)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "e4m3 x e4m3 -> f32 (exact integer digit products), f64 state",
        "data": "synthetic (seeded Bin(2,MAF) genotypes, heteroscedastic normal noise)",
        "config": {"workload": "geno_int8", "n": w.n, "p": w.p, "covariates": w.c, "G": len(bp) - 1,
                   "taus": TAUS, "lambda": "0.1 lambda_max(tau)", "fits_per_step": B,
                   "precision": "mixed: tensor-core digit products (7 base-16 digits of theta, "
                                "11 of a_j beta_j), FP64 state and stop test",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (X = 500 MB int8)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_col_tc (column pass: X~^T theta on tcgen05 + beta prox)",
                     "bytes_per_launch": kprof.col_bytes, "avg_launch_ms": col_avg_ms,
                     "samples": kprof.col_samples, "sampled_in": "last warm-up step (timed steps unsampled)", "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"},
        "kernels_ms": {"col": col_avg_ms,
                       "xbeta_and_vector_update": kprof.xb_ms / max(1, kprof.xb_samples),
                       "vec": (kprof.vec_ms / kprof.vec_samples) if kprof.vec_samples else None},
        "iters": iters, "kkt": kkts, "iterations_timed": prof.iterations,
        "setup_ms_per_step": float(np.mean(setup_ms)) if setup_ms else None,
        "gpu_launches": int(prof.kernel_launches),
        "clocks": clocks.summary(),
        "e2e": e2e,
        "fp64_plain": fp64,
        "cpu_baseline": cpu,
        "grid": grid,
        "wall_s": t_wall,
    }
    if fp64:
        out["vs_fp64_plain"] = value / fp64["value"]
    if args.profile_iters:
        out["profile_run"] = f"fixed {args.profile_iters} iterations per fit; not a benchmark result"

    if rank == 0:
        print(json.dumps(out))
    ctx.close()


# ------------------------------------------------------------ CPU baseline

class OracleSample:
    """The FP64 oracle (oracle/) on the full standardised design of the
    workload, for timing a bounded number of Algorithm 1 iterations of the
    tau = 0.5 fit. Building the dense design is set-up, outside the timing."""

    def __init__(self, w):
        from oracle import fsqrppa as O
        self.O = O
        self.w = w
        g = O.decode_stored(w.geno, w.fmt, w.n)
        self.d = O.build_design(g, w.cov)
        self.bp = w.block_ptr()
        self.mu = O.default_mu(w.y)
        self.tau = 0.5
        self.lmax = O.lambda_max(self.d.Xt, w.y, self.tau, w.omega)
        self.lam = LAMBDA_FRAC * self.lmax * w.omega
        # eta only sets step sizes; the cost of an iteration does not depend on it
        self.eta = np.full(len(self.bp) - 1, self.mu * float(w.n))

    def seconds_per_iteration(self, iters):
        t0 = time.perf_counter()
        self.O.fsqrppa(self.d.Xt, self.w.y, self.tau, self.lam, self.bp, self.eta, self.mu, tol=0.0,
                       max_iter=iters, check_every=10, lam_norm=self.lmax)
        return (time.perf_counter() - t0) / iters

    def describe(self, iters, s_per_iter, mean_iters):
        return (f"oracle Algorithm 1 (numpy FP64, dense standardised X~ {self.w.n}x{self.w.P}) timed for "
                f"{iters} iterations of the tau=0.5 fit ({s_per_iter * 1e3:.1f} ms/iter), scaled by "
                f"{mean_iters:.0f} iterations per fit (the count the fits need); design build excluded; "
                f"threads = numpy BLAS default")


def cpu_baseline(w, iters_needed, sample_iters=40):
    """The FP64 oracle timed on the host on a bounded sample, scaled to fits/s:
    with the BLAS default threads (all host cores) and, in a child process
    with every BLAS pool set to one thread, single-threaded."""
    o = OracleSample(w)
    spi = o.seconds_per_iteration(sample_iters)
    mean_iters = float(np.mean(iters_needed))
    single = oracle_single_thread(sample_iters // 2, mean_iters)
    return {"value": 1.0 / (spi * mean_iters), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": o.describe(sample_iters, spi, mean_iters), "single_thread": single}


def oracle_single_thread(sample_iters, mean_iters):
    """Seconds per oracle iteration with one BLAS thread (child process)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "o = bench.OracleSample(bench.make_workload()); "
            "print(json.dumps(o.seconds_per_iteration(%d)))" % (ROOT, sample_iters))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        spi = float(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": 1.0 / (spi * mean_iters), "unit": UNIT, "cores": 1, "ms_per_iteration": spi * 1e3,
            "sample": f"{sample_iters} iterations of the tau=0.5 fit, one BLAS thread"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = make_workload()
    o = OracleSample(w)
    iters = 20
    for _ in range(args.warmup):
        o.seconds_per_iteration(2)
    times = []
    for _ in range(args.steps):
        times.append(o.seconds_per_iteration(iters))
    spi = statistics.median(times)
    v = 1.0 / (spi * args.ref_iters)
    sample = o.describe(iters, spi, args.ref_iters)
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": spi * iters * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded Bin(2,MAF) genotypes, heteroscedastic normal noise)",
           "config": {"workload": "geno_int8", "n": w.n, "p": w.p, "covariates": w.c,
                      "G": len(w.block_sizes), "taus": TAUS, "lambda": "0.1 lambda_max(tau)",
                      "fits_per_step": len(TAUS),
                      "precision": "FP64 oracle (numpy, dense standardised design)",
                      "parallelism": "rank 0 only (host cores)",
                      "l2": "inputs larger than L2 (X = 500 MB int8)"},
           "impl": "reference",
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_grid_sample(args, local_rank):
    """Batched-grid sample (not the contract line, and the small case for
    profilers): the tau x lambda grid generator at n = 10,000 and p =
    --grid-p columns (default 500,000), int8 or (--grid-2bit) 2-bit storage,
    --grid-slots fits (taus 0.1..0.9, lambdas 0.3..0.03 lambda_max) advanced
    together on the tensor cores for --profile-iters steps each (default
    400). Reports the time per step, the fit-steps per second and the column
    pass against the HBM roofline."""
    import torch

    from paper_2601_02826_gb300 import fsqr, synth
    from paper_2601_02826_gb300.device import upload

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    stream = torch.cuda.Stream(device=dev)
    ctx = fsqr.Context(local_rank, stream.cuda_stream)
    t0 = time.perf_counter()
    slots = args.grid_slots
    n_l = max(1, (slots + 8) // 9)
    w = synth.grid_int8(p=args.grid_p, n_lambda=n_l)
    if args.grid_2bit:
        g = synth.unpack_int8(w.geno, w.n)
        w.geno, w.ld = synth.pack_2bit(g)
        w.fmt = synth.FMT_2BIT
    t_gen = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        dw = upload(ctx, w, device=dev)
    stream.synchronize()
    taus = w.taus[:slots] if slots < 9 else w.taus
    fr = np.geomspace(0.3, 0.03, n_l)
    lm = [ctx.lambda_max(dw.design, dw.y, t, dw.omega) for t in taus]
    lam = np.array([[f * l for f in fr] for l in lm])
    B = lam.size
    beta = torch.zeros(B * w.P, dtype=torch.float64, device=dev)
    z = torch.zeros(B * w.n, dtype=torch.float64, device=dev)
    th = torch.zeros(B * w.n, dtype=torch.float64, device=dev)
    iters = args.profile_iters or 400
    opts = dict(tol=0.0, max_iter=iters, precision=fsqr.MIXED, max_group=slots)
    ctx.fit_batch(dw.design, dw.y, taus, lam, dw.omega, w.block_ptr(), beta, z, th,
                  opts=dict(opts, max_iter=20))
    ctx.profile(enable=True, reset=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, infos = ctx.fit_batch(dw.design, dw.y, taus, lam, dw.omega, w.block_ptr(), beta, z, th, opts=opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile(enable=False)
    col_ms = prof.col_ms / max(1, prof.col_samples)
    peak, kind = measured_peaks()
    gbs = prof.col_bytes / (col_ms / 1e3) / 1e9
    out = {"sample": "batched grid, fixed steps per fit (setup included); not a bench line",
           "workload": "grid_int8" + (" (2-bit storage)" if args.grid_2bit else ""), "n": w.n, "p": w.p,
           "G": len(w.block_sizes), "fits": B, "slots": slots, "iterations": iters, "ms": ms,
           "steps": prof.iterations, "fit_iterations_per_s": sum(i.iters for i in infos) / (ms / 1e3),
           "col": {"avg_launch_ms": col_ms, "bytes_per_launch": prof.col_bytes, "achieved_gbs": gbs,
                   "peak_gbs": peak, "frac": gbs / peak, "peak_source": kind},
           "xbeta_and_vector_update_ms": prof.xb_ms / max(1, prof.xb_samples),
           "groups": {"tc": prof.tc_groups, "wide": prof.wide_groups, "simt": prof.simt_groups},
           "kkt_after": [i.kkt for i in infos][:4], "generate_s": t_gen}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    # mean iterations per fit of this workload measured on the GB300 path
    # (144110, 182730, 146700 for tau = 0.1, 0.5, 0.9; same algorithm)
    ap.add_argument("--ref-iters", type=int, default=157847)
    ap.add_argument("--fp64-iters", type=int, default=400)
    ap.add_argument("--skip-grid", action="store_true")
    ap.add_argument("--grid-iters", type=int, default=500,
                    help="iterations per fit of the tau x lambda grid leg (a throughput sample)")
    ap.add_argument("--grid-slots", type=int, default=32)
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiling run: every fit stops after this many iterations (not a bench line)")
    ap.add_argument("--grid-p", type=int, default=500_000)
    ap.add_argument("--grid-2bit", action="store_true")
    ap.add_argument("--grid-sample", action="store_true",
                    help="batched-grid sample on the 10,000 x 500,000 workload (not a bench line)")
    args = ap.parse_args()
    if args.grid_sample:
        run_grid_sample(args, int(os.environ.get("LOCAL_RANK", 0)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gb300(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
