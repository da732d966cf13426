"""Benchmark of the B-KFAC preconditioning hot path on one GB300.

Headline workload (the one-wide-FC-layer configuration): forward factor A at
d = 4097 (4096 inputs + bias), backward factor Gamma at d = 4096, rank r = 256,
n = 256 new columns per step, rho = 0.95, lambda = 1e-2, FP32 plain per-factor
path.  One step = Brand update of A + Brand update of Gamma + damped inverse
application to a fresh 4096 x 4097 FP32 gradient.  Inputs are seeded synthetic
power-law batches (exponent 1.2) and N(0, 1) gradients, resident in HBM before
the timed region (config["inputs"]).

Metric: factor updates per second (two per step); the preconditioned gradients
per second are reported beside it.  The same JSON line carries, besides the
headline's dominant-kernel roofline, its composed roofline (each phase's
algorithmic work at its pipe's peak, summed, over the measured time), and:
  * batched:   the same layer through the batch API (CUDA graph), FP32 and mixed;
  * workloads: the small FP64 factor (d = 512 / 256, r = 64, n = 32, 50 steps),
               the 16-layer uneven batch (plain FP32 per-layer calls vs batched
               FP32 vs batched mixed, and mixed with the FP64 CholeskyQR and
               eigensolve) and the 8-layer MLP step (plain vs batched), each with
               a composed roofline;
  * cpu_baseline: the FP64 oracle on the host cores (all cores and one thread).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bkfac|reference]
       python bench.py --workload mlp         (the MLP step as the headline)
       python bench.py --profile-case ...     (one factor's updates, for profilers)
Under torchrun (N > 1) the ranks take whole layers (shard.assign_layers) and
all-gather the preconditioned steps in every timed step; timing is the max over
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "K-factor Brand updates/sec + preconditioned grads/sec (1 GB300), batched vs plain"
D_A, D_G, R, N, RHO, LAM, ALPHA = 4097, 4096, 256, 256, 0.95, 1e-2, 1.2
WORKLOAD = "one wide FC layer: A d=4097, Gamma d=4096, r=256, n=256, rho=0.95, lambda=1e-2, G 4096x4097"
POOL_X, POOL_G = 8, 3


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------------------- reference arm: the oracle on the host


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_2210_08494_gb300 import synth

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    step_cap_s = float(os.environ.get("BKFAC_REF_BUDGET_S", "150"))
    seedA, seedG = synth.factor_seed(2, 0, "A"), synth.factor_seed(2, 0, "G")
    XA = [synth.powerlaw_batch(D_A, N, ALPHA, seedA, t) for t in range(2)]
    XG = [synth.powerlaw_batch(D_G, N, ALPHA, seedG, t) for t in range(2)]
    G = synth.gradient(D_G, D_A, seedA, 0)
    UA, sA, iA = oracle.init(XA[0], R)
    UG, sG, iG = oracle.init(XG[0], R)
    times = []
    t_all = time.time()
    total = max(1, args.warmup) + args.steps
    for i in range(total):
        t0 = time.perf_counter()
        UA2, sA2, _ = oracle.update(UA, sA, iA["r_new"], XA[1], RHO, R)
        UG2, sG2, _ = oracle.update(UG, sG, iG["r_new"], XG[1], RHO, R)
        oracle.apply(UA2, sA2, LAM, UG2, sG2, LAM, G)
        dt = time.perf_counter() - t0
        if i >= total - args.steps:
            times.append(dt)
        if time.time() - t_all > step_cap_s and len(times) >= 1:
            break
    t_step = float(np.mean(times))
    value = 2.0 / t_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "factor-updates/s", "n_gpus": world,
        "steps": len(times), "warmup": total - len(times) if len(times) < args.steps else max(1, args.warmup),
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "path": "FP64 CPU oracle (Householder QR, two-sided Jacobi, direct apply)"},
        "preconditioned_grads_per_s": 1.0 / t_step,
        "cpu_baseline": {"value": value, "unit": "factor-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(times)} full step(s): 2 factor updates + 1 apply at the full shapes"},
        "e2e": {"value": value, "unit": "factor-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample():
    """The oracle as it stands, timed on the host cores on bounded samples (about 20-30 s):
    two full steps of the wide layer (two factor updates at d = 4097 / 4096, r = n = 256,
    and the apply to a 4096 x 4097 gradient) on all cores -- the line's value -- and five
    steps of the small FP64 factor (d = 512 / 256, r = 64, n = 32, with the apply to a
    256 x 512 gradient) on one thread and on all cores."""
    import oracle
    from paper_2210_08494_gb300 import synth

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    seedA, seedG = synth.factor_seed(2, 0, "A"), synth.factor_seed(2, 0, "G")
    steps = 2
    XA = [synth.powerlaw_batch(D_A, N, ALPHA, seedA, t) for t in range(steps + 1)]
    XG = [synth.powerlaw_batch(D_G, N, ALPHA, seedG, t) for t in range(steps + 1)]
    G = synth.gradient(D_G, D_A, seedA, 0)
    UA, sA, iA = oracle.init(XA[0], R)
    UG, sG, iG = oracle.init(XG[0], R)
    kA, kG = iA["r_new"], iG["r_new"]
    t0 = time.perf_counter()
    for t in range(1, steps + 1):
        UA, sA, iA = oracle.update(UA[:kA], sA[:kA], kA, XA[t], RHO, R)
        UG, sG, iG = oracle.update(UG[:kG], sG[:kG], kG, XG[t], RHO, R)
        kA, kG = iA["r_new"], iG["r_new"]
        oracle.apply(UA[:kA], sA[:kA], LAM, UG[:kG], sG[:kG], LAM, G)
    dt = (time.perf_counter() - t0) / steps

    def small(threads, nsteps=5):
        oracle.set_threads(threads)
        xa = [synth.powerlaw_batch(512, 32, 1.5, 1000, t) for t in range(nsteps + 1)]
        xg = [synth.powerlaw_batch(256, 32, 1.5, 1001, t) for t in range(nsteps + 1)]
        g = synth.gradient(256, 512, 1002, 0)
        ua, sa, ia = oracle.init(xa[0], 64)
        ug, sg, ig = oracle.init(xg[0], 64)
        ka, kg = ia["r_new"], ig["r_new"]
        t1 = time.perf_counter()
        for t in range(1, nsteps + 1):
            ua, sa, ia = oracle.update(ua[:ka], sa[:ka], ka, xa[t], RHO, 64)
            ug, sg, ig = oracle.update(ug[:kg], sg[:kg], kg, xg[t], RHO, 64)
            ka, kg = ia["r_new"], ig["r_new"]
            oracle.apply(ua[:ka], sa[:ka], 0.1, ug[:kg], sg[:kg], 0.1, g)
        return (time.perf_counter() - t1) / nsteps

    s1, sN = small(1), small(cores)
    oracle.set_threads(cores)
    return {"value": 2.0 / dt, "unit": "factor-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} full steps of the wide layer (2 factor updates at d=4097/4096, r=n=256 + 1 apply "
                      f"to 4096x4097), {dt:.1f} s per step on {cores} threads",
            "small_fp64_factor": {
                "workload": "A d=512, Gamma d=256, r=64, n=32 (+ apply to 256x512), 5 steps",
                "single_thread": {"value": 2.0 / s1, "unit": "factor-updates/s", "cores": 1, "ms_per_step": s1 * 1e3},
                "all_cores": {"value": 2.0 / sN, "unit": "factor-updates/s", "cores": cores,
                              "ms_per_step": sN * 1e3}}}


# --------------------------------------------------------------------------- GPU arm


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of the
# kernel on this workload, None when the kernel has changed since the capture (the
# eigensolve's angle normalisation changed after its last capture, 1.21 MB read and
# 0 written per 512-column launch; the blocks live in shared memory and registers).
DRAM_BYTES_PER_LAUNCH = {"jacobi": None}


def algorithmic_work(phase, ms, counts, sweeps):
    """Algorithmic bytes / flops per launch of a phase at the benchmark shapes (both factors)."""
    d = (D_A + D_G) / 2.0
    Nc = R + N
    if phase == "jacobi":
        # one-sided Jacobi, FP32: per sweep every column pair costs 3 dot products and a
        # rotation over Nc rows = 12 * Nc flops; per launch (one factor) x sweeps
        flops = sweeps * (Nc * (Nc - 1) / 2.0) * 12.0 * Nc
        return {"bound": "alu", "flops": flops}
    if phase == "apply_pass2":
        return {"bound": "hbm", "bytes": 2.0 * D_G * D_A * 4, "flops": 2.0 * D_G * D_A * 2 * R}
    if phase == "apply_pass1":
        return {"bound": "hbm", "bytes": D_G * D_A * 4 + D_A * R * 4, "flops": 2.0 * D_G * D_A * R}
    if phase == "chol":
        return {"bound": "alu64", "flops": N ** 3 / 3.0}
    if phase == "gram":
        return {"bound": "alu64", "flops": 2.0 * d * N * N}
    if phase == "trinv":
        return {"bound": "alu", "flops": N ** 3 / 3.0}
    return None


# --------------------------------------------------------------------------- composed roofline
# The update's roofline is the composed bound of its phases: each phase's algorithmic
# work at the peak of the pipe it needs (or its algorithmic bytes at the HBM peak,
# whichever is longer), summed over the phases of the step, over the measured time.


def pipe_peaks(torch, dev):
    """Peaks per second of the pipes the step uses, with where each comes from."""
    pk, src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2070.0
    try:
        q = subprocess.run(["nvidia-smi", f"--id={dev.index or 0}", "--query-gpu=clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        mhz = float(q.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    return {
        "hbm": pk["hbm_gbs"] * 1e9,
        "fp32": sms * 128 * 2 * mhz * 1e6,
        "fp64": 1.25e12,
        "bf16": pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * 1e12,
    }, {"hbm": f"{src} copy bandwidth", "fp32": f"derived: {sms} SMs x 128 lanes x 2 flops x {mhz:.0f} MHz",
        "fp64": "nominal 1.25 TFLOP/s", "bf16": f"{src} cuBLAS bf16 (sustained)"}


def update_work(d, k, n, r, prec, sweeps, eig64=False, chol64=False):
    """Phases of one factor update as (name, flops, bytes, pipe): the Brand path (Algorithm 3:
    projection, residual, CholeskyQR2, core, eigensolve, rotation) or, when r + n >= d, the
    dense path (Jacobi on the d x (k + n) factor).  prec: 'f64', 'f32' or 'mixed'."""
    e = 8 if prec == "f64" else 4
    mm = {"f64": "fp64", "f32": "fp32", "mixed": "bf16"}[prec]
    f32 = "fp64" if prec == "f64" else "fp32"
    eig = "fp64" if (prec == "f64" or eig64) else "fp32"
    chol = "fp64" if (prec == "f64" or chol64) else "fp32"
    N = k + n
    if r + n >= d:  # dense path: one-sided Jacobi on N columns of length d
        return [("dense_jacobi", 7.0 * N * N * d * sweeps, e * d * (k + n + r), eig)]
    rn = min(r, N)
    items = [("colnorm", 0.0, e * d * n, "hbm"),
             ("proj", 2.0 * d * k * n, e * d * (k + n), mm),
             ("resid", 2.0 * d * k * n, e * d * (k + 2 * n), mm),
             ("gram", 2.0 * d * n * (n + 1), 2.0 * e * d * n, f32),
             ("chol", 2.0 * n ** 3 / 3.0, 0.0, chol),
             ("trinv", 2.0 * n ** 3 / 3.0, 0.0, f32),
             ("trmm", 2.0 * d * n * n, 4.0 * e * d * n, f32)]
    if eig == "fp32" and N >= 128:
        items.append(("precond", N ** 3 + N ** 3 / 3.0, 0.0, "fp32"))
    items += [("jacobi", 7.0 * N ** 3 * sweeps, 0.0, eig),
              ("rotate", 2.0 * d * N * rn, e * d * (N + rn), mm),
              ("finalize", 0.0, 2.0 * e * d * rn, "hbm")]
    return items


def apply_work(dA, dG, rA, rG, prec):
    """Phases of Algorithm 1 on a dG x dA gradient: pass 1 reads G (T1 = G U_A, T2 = U_G^T G),
    pass 2 reads G and writes S."""
    e = 8 if prec == "f64" else 4
    mm = {"f64": "fp64", "f32": "fp32", "mixed": "bf16"}[prec]
    fl = 2.0 * dG * dA * (rA + rG)
    return [("apply_pass1", fl, e * dG * dA, mm), ("apply_pass2", fl, 2.0 * e * dG * dA, mm)]


def composed_roofline(items, measured_ms, peaks, sources):
    """Sum over phases of max(flops / pipe peak, bytes / HBM peak) against the measured time."""
    t_bound, by_pipe = 0.0, {}
    for name, flops, nbytes, pipe in items:
        t_c = flops / peaks[pipe] if pipe != "hbm" and flops else 0.0
        t_m = nbytes / peaks["hbm"]
        t = max(t_c, t_m)
        key = "hbm" if t_m >= t_c else pipe
        by_pipe[key] = by_pipe.get(key, 0.0) + t
        t_bound += t
    return {"kind": "composed: sum over phases of max(work / pipe peak, bytes / HBM peak), over the measured time",
            "bound_ms": t_bound * 1e3, "measured_ms": measured_ms,
            "frac": t_bound * 1e3 / measured_ms if measured_ms else None,
            "bound_ms_by_pipe": {k: v * 1e3 for k, v in sorted(by_pipe.items())},
            "peaks_per_s": {k: peaks[k] for k in sorted(peaks)}, "peak_sources": sources}


def factor_sweeps(bkfac, f, n):
    """Jacobi sweeps of the factor's last update (diagnostic word in its workspace)."""
    try:
        off = bkfac.bkfac_debug_offsets(f, n)[7]
        return int(f.ws(n)[off:off + 4].view(__import__("torch").int32).item())
    except Exception:
        return None


def timed_steps(torch, stream, fn, steps, flush):
    """CUDA-event time per step of fn(t) on `stream`, the L2 flushed outside the events."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for t in range(steps):
            flush.zero_()
            evs[t][0].record(stream)
            fn(t)
            evs[t][1].record(stream)
    stream.synchronize()
    return float(sum(a.elapsed_time(b) for a, b in evs)) / steps


def tune_products(bkfac, torch, fn, cache):
    """Run fn() once (untimed) with the library noting the FP32 product shapes it
    launches, then time the candidates of each new shape and keep the fastest."""
    torch.cuda.synchronize()
    bkfac.bkfac_gemm_tune_begin()
    try:
        fn()
    finally:
        torch.cuda.synchronize()
        bkfac.bkfac_gemm_tune_end(cache)


def run_workload_batch(args, bkfac, torch, dev, flush, peaks, sources, shapes, n, inputs, grads, name,
                       plain=True, variants=(("batched_f32_graph", "f32", 0),
                                             ("batched_mixed_bf16_graph", "mixed", 0))):
    """One multi-layer workload: the plain FP32 per-layer path (per-factor calls in sequence on
    one stream) and batched graph paths, each timed per step with a composed roofline.
    shapes: [(dA, dG, r)]; inputs(t) -> (XA list, XG list) device columns for step t."""
    L = len(shapes)
    DT = {"f32": bkfac.F32, "mixed": bkfac.MIXED_BF16}
    out = {}
    sweeps = {}
    stream = torch.cuda.Stream(device=dev)

    def work_for(prec, eig64=False, chol64=False):
        items = []
        for l, (dA, dG, r) in enumerate(shapes):
            for w, d in ((0, dA), (1, dG)):
                rr = min(r, d)
                sw = sweeps.get((l, w)) or 9
                items += update_work(d, rr, n, rr, prec, sw, eig64, chol64)
            items += apply_work(dA, dG, min(r, dA), min(r, dG), prec)
        return items

    if plain:
        layers = [(bkfac.Factor(dA, min(r, dA), bkfac.F32, device=dev), bkfac.Factor(dG, min(r, dG), bkfac.F32,
                                                                                   device=dev))
                  for dA, dG, r in shapes]
        # the eigensolve's launch shapes, tuned once per shape (untimed; cached per machine)
        tune_cache = os.path.join(ROOT, "paper_2210_08494_gb300", "_build", "tune_cache.txt")
        tuned = set()
        for a, g in layers:
            for f in (a, g):
                if (f.d, f.r) not in tuned:
                    bkfac.bkfac_tune(f, n, tune_cache)
                    tuned.add((f.d, f.r))
        S = [bkfac.grad_tensor(g.shape[0], g.shape[1], torch.float32, dev) for g in grads]

        def plain_step(t):
            XA, XG = inputs(t)
            for l, (a, g) in enumerate(layers):
                for f, X in ((a, XA[l]), (g, XG[l])):
                    if f.r_cur == 0:
                        bkfac.bkfac_init(f, X)
                    else:
                        bkfac.bkfac_update(f, X, RHO)
                bkfac.bkfac_apply(a, g, LAM, LAM, grads[l], S[l])

        with torch.cuda.stream(stream):
            plain_step(0)
            # the products' tile shapes and K splits, tuned on the step's own shapes
            tune_products(bkfac, torch, lambda: plain_step(1), tune_cache)
            for t in range(2, args.warmup + 1):
                plain_step(t)
        stream.synchronize()
        bkfac.bkfac_trace_enable(True)
        _, l0 = bkfac.bkfac_trace_read()
        ms = timed_steps(torch, stream, lambda t: plain_step(args.warmup + 1 + t), args.steps, flush)
        trace, l1 = bkfac.bkfac_trace_read()
        bkfac.bkfac_trace_enable(False)
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} plain: {bkfac.strerror(st)}")
        for l, (a, g) in enumerate(layers):
            for w, f in ((0, a), (1, g)):
                sweeps[(l, w)] = factor_sweeps(bkfac, f, n)
        out["plain_f32"] = {"ms_per_step": ms, "value": 2 * L * 1000.0 / ms, "unit": "factor-updates/s",
                            "preconditioned_grads_per_s": L * 1000.0 / ms, "gpu_launches_per_step": (l1 - l0) / args.steps,
                            "path": "plain FP32 per-layer calls", "parity_bound": 1e-4,
                            "phases_ms_per_step": {k: v[0] / args.steps for k, v in trace.items() if v[1]},
                            "roofline": composed_roofline(work_for("f32"), ms, peaks, sources)}
    for vname, prec, flags in variants:
        layers_b = [(bkfac.Factor(dA, min(r, dA), DT[prec], device=dev, flags=flags),
                     bkfac.Factor(dG, min(r, dG), DT[prec], device=dev, flags=flags)) for dA, dG, r in shapes]
        tune_cache = os.path.join(ROOT, "paper_2210_08494_gb300", "_build", "tune_cache.txt")
        batch = bkfac.Batch(layers_b, n, DT[prec], tune_cache=tune_cache)
        XA0, XG0 = inputs(0)
        xa = [bkfac.cols_tensor(n, x.shape[1], torch.float32, dev) for x in XA0]
        xg = [bkfac.cols_tensor(n, x.shape[1], torch.float32, dev) for x in XG0]
        Sb = [bkfac.grad_tensor(g.shape[0], g.shape[1], torch.float32, dev) for g in grads]

        def load(t):
            XA, XG = inputs(t)
            for dst, src in zip(xa + xg, XA + XG):
                dst.copy_(src)

        with torch.cuda.stream(stream):
            load(0)
            batch.update(xa, xg, RHO)
            load(1)

            def eager_step():
                batch.update(xa, xg, RHO)
                batch.apply(grads, Sb, [LAM] * L, [LAM] * L)

            tune_products(bkfac, torch, eager_step, tune_cache)
            load(2)
            batch.step_graph(xa, xg, RHO, grads, Sb, [LAM] * L, [LAM] * L, capture=True)
            for t in range(args.warmup):
                load(3 + t)
                batch.step_graph()
        stream.synchronize()
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} {vname} warm-up: {bkfac.strerror(st)}")
        steps = args.steps if not (flags & bkfac.FLAG_EIG_FP64) else max(3, min(args.steps, 8))

        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for t in range(steps):
                load(t)
                flush.zero_()
                evs[t][0].record(stream)
                batch.step_graph()
                evs[t][1].record(stream)
        stream.synchronize()
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} {vname} timed: {bkfac.strerror(st)}")
        ms = float(sum(a.elapsed_time(b) for a, b in evs)) / steps
        eig64 = bool(flags & bkfac.FLAG_EIG_FP64)
        chol64 = bool(flags & bkfac.FLAG_CHOL_FP64)
        out[vname] = {"ms_per_step": ms, "value": 2 * L * 1000.0 / ms, "unit": "factor-updates/s",
                      "preconditioned_grads_per_s": L * 1000.0 / ms, "steps": steps,
                      "path": ("batch API, one CUDA graph per step, " +
                               ("FP32" if prec == "f32" else "BF16-rounded tall-skinny operands, FP32 accumulation") +
                               (", FP64 CholeskyQR factorisations" if chol64 else "") +
                               (", FP64 core eigensolve" if eig64 else "")),
                      "parity_bound": 1e-4 if prec == "f32" else 1e-2,
                      "roofline": composed_roofline(work_for(prec, eig64, chol64), ms, peaks, sources)}
        batch.close()
    if plain:
        for k, v in out.items():
            if k != "plain_f32":
                v["speedup_vs_plain"] = out["plain_f32"]["ms_per_step"] / v["ms_per_step"]
    out["jacobi_sweeps"] = {f"{l}{'AG'[w]}": s for (l, w), s in sorted(sweeps.items())}
    return out


UNEVEN_PAIRS = [(513, 1024), (1025, 2048), (2049, 4096), (4097, 4096), (4097, 10)]
UNEVEN_RANKS = [64, 128, 256]
UNEVEN_N = 128


def uneven_workload(args, bkfac, synth, torch, dev, flush, peaks, sources):
    """16 FC layers of uneven (d_in + bias, d_out) and r, n = 128: plain vs batched FP32 vs
    batched mixed, and the mixed path with the FP64 CholeskyQR and eigensolve."""
    shapes = [(UNEVEN_PAIRS[l % 5][0], UNEVEN_PAIRS[l % 5][1], UNEVEN_RANKS[l % 3]) for l in range(16)]
    gens = {}
    pool = 4
    bufs = []
    for t in range(pool):
        XA, XG = [], []
        for l, (dA, dG, r) in enumerate(shapes):
            for d, lst, w in ((dA, XA, 0), (dG, XG, 1)):
                if d not in gens:
                    gens[d] = synth.DevicePowerlaw(d, ALPHA, 3000 + d, dev)
                x = bkfac.cols_tensor(UNEVEN_N, d, torch.float32, dev)
                gens[d].draw(x, UNEVEN_N, 100 * t + 2 * l + w)
                lst.append(x)
        bufs.append((XA, XG))
    gg = torch.Generator(device=dev).manual_seed(3100)
    grads = []
    for dA, dG, r in shapes:
        g = bkfac.grad_tensor(dG, dA, torch.float32, dev, zero=False)
        g.normal_(generator=gg)
        grads.append(g)
    res = run_workload_batch(args, bkfac, torch, dev, flush, peaks, sources, shapes, UNEVEN_N,
                             lambda t: bufs[t % pool], grads, "uneven",
                             variants=(("batched_f32_graph", "f32", 0),
                                       ("batched_mixed_bf16_graph", "mixed", 0),
                                       ("batched_mixed_fp64_core_graph", "mixed",
                                        bkfac.FLAG_EIG_FP64 | bkfac.FLAG_CHOL_FP64)))
    res["workload"] = ("16 FC layers, (d_in+bias, d_out) cycling (513,1024),(1025,2048),(2049,4096),(4097,4096),"
                       "(4097,10), r cycling 64,128,256, n=128, rho=0.95, lambda=1e-2")
    return res


def mlp_workload(args, bkfac, synth, torch, dev, flush, peaks, sources):
    """The full synthetic preconditioning step: an 8-layer ReLU MLP of width 4096 (output 10),
    minibatch 256, r = 220."""
    L = len(MLP_WIDTHS) - 1
    pool = mlp_inputs(torch, bkfac, synth, dev, 4)
    shapes = [(MLP_WIDTHS[l] + 1, MLP_WIDTHS[l + 1], MLP_R) for l in range(L)]
    grads = [bkfac.grad_tensor(g.shape[0], g.shape[1], torch.float32, dev) for g in pool[0][2]]
    for g, src in zip(grads, pool[0][2]):
        g.copy_(src)
    res = run_workload_batch(args, bkfac, torch, dev, flush, peaks, sources, shapes, MLP_N,
                             lambda t: (pool[t % len(pool)][0], pool[t % len(pool)][1]), grads, "mlp")
    res["workload"] = MLP_WORKLOAD
    return res


def small_fp64_workload(args, bkfac, synth, torch, dev, flush, peaks, sources):
    """The small FP64 factor: A at d = 512, Gamma at d = 256, r = 64, n = 32, 50 updates of
    each (plain per-factor calls), then the damped inverse application (lambda = 0.1) to a
    256 x 512 N(0, 1) gradient; per-step time over the 50 steps."""
    dA, dG, r, n, steps = 512, 256, 64, 32, 50
    fA = bkfac.Factor(dA, r, bkfac.F64, device=dev)
    fG = bkfac.Factor(dG, r, bkfac.F64, device=dev)
    XA, XG = [], []
    for t in range(steps + 1):
        for d, lst, sd in ((dA, XA, 1000), (dG, XG, 1001)):
            x = bkfac.cols_tensor(n, d, torch.float64, dev)
            x.copy_(torch.from_numpy(synth.powerlaw_batch(d, n, 1.5, sd, t)))
            lst.append(x)
    G = bkfac.grad_tensor(dG, dA, torch.float64, dev)
    G.copy_(torch.from_numpy(synth.gradient(dG, dA, 1002, 0)))
    S = bkfac.grad_tensor(dG, dA, torch.float64, dev)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        bkfac.bkfac_init(fA, XA[0])
        bkfac.bkfac_init(fG, XG[0])

    def step(t):
        bkfac.bkfac_update(fA, XA[1 + t], RHO)
        bkfac.bkfac_update(fG, XG[1 + t], RHO)

    ms = timed_steps(torch, stream, step, steps, flush)
    ms_apply = timed_steps(torch, stream, lambda t: bkfac.bkfac_apply(fA, fG, 0.1, 0.1, G, S), 5, flush)
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"small FP64 workload: {bkfac.strerror(st)}")
    sw = [factor_sweeps(bkfac, f, n) or 9 for f in (fA, fG)]
    items = update_work(dA, r, n, r, "f64", sw[0]) + update_work(dG, r, n, r, "f64", sw[1])
    return {"workload": "small FP64 factor: A d=512, Gamma d=256, r=64, n=32, rho=0.95, 50 steps; "
                        "apply (Gamma+0.1I)^-1 G (A+0.1I)^-1 to a 256x512 gradient",
            "ms_per_step": ms, "value": 2 * 1000.0 / ms, "unit": "factor-updates/s",
            "apply_ms": ms_apply, "preconditioned_grads_per_s": 1000.0 / ms_apply, "parity_bound": 1e-10,
            "jacobi_sweeps": sw, "path": "plain FP64 per-factor calls",
            "roofline": composed_roofline(items, ms, peaks, sources)}


def run_batched(args, bkfac, synth, torch, dev, seedA, seedG, dtype, flush):
    """The same one-layer step through the batch API: both factor updates forked onto
    worker streams, then the apply, captured once into a CUDA graph and replayed.
    Each replay gets fresh inputs, copied into the graph's buffers outside the
    timed events (like the L2 flush)."""
    layers = [(bkfac.Factor(D_A, R, dtype, device=dev), bkfac.Factor(D_G, R, dtype, device=dev))]
    batch = bkfac.Batch(layers, N, dtype)
    pool = min(POOL_X, 4)
    XA = [bkfac.cols_tensor(N, D_A, torch.float32, dev) for _ in range(pool)]
    XG = [bkfac.cols_tensor(N, D_G, torch.float32, dev) for _ in range(pool)]
    for t in range(pool):
        XA[t].copy_(torch.from_numpy(synth.powerlaw_batch(D_A, N, ALPHA, seedA, 20 + t)))
        XG[t].copy_(torch.from_numpy(synth.powerlaw_batch(D_G, N, ALPHA, seedG, 20 + t)))
    xa, xg = bkfac.cols_tensor(N, D_A, torch.float32, dev), bkfac.cols_tensor(N, D_G, torch.float32, dev)
    G = bkfac.grad_tensor(D_G, D_A, torch.float32, dev, zero=False)
    G.normal_(generator=torch.Generator(device=dev).manual_seed(seedA + 600))
    S = bkfac.grad_tensor(D_G, D_A, torch.float32, dev)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        for t in range(2):  # init, then reach the steady rank before capturing
            xa.copy_(XA[t % pool])
            xg.copy_(XG[t % pool])
            batch.update([xa], [xg], RHO)
        batch.step_graph([xa], [xg], RHO, [G], [S], [LAM], [LAM], capture=True)
        for t in range(args.warmup):
            xa.copy_(XA[t % pool])
            xg.copy_(XG[t % pool])
            batch.step_graph()
    stream.synchronize()
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"batched warm-up: {bkfac.strerror(st)}")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for t in range(args.steps):
            xa.copy_(XA[t % pool])
            xg.copy_(XG[t % pool])
            flush.zero_()
            evs[t][0].record(stream)
            batch.step_graph()
            evs[t][1].record(stream)
    stream.synchronize()
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"batched timed region: {bkfac.strerror(st)}")
    ms = float(sum(a.elapsed_time(b) for a, b in evs)) / args.steps
    batch.close()
    return {"value": 2.0 * 1000.0 / ms, "unit": "factor-updates/s", "ms_per_step": ms,
            "preconditioned_grads_per_s": 1000.0 / ms,
            "path": ("batch API, CUDA graph replay, " +
                     ("FP32" if dtype == bkfac.F32 else "BF16-rounded tall-skinny operands, FP32 accumulation")),
            "parity_bound": 1e-4 if dtype == bkfac.F32 else 1e-2}


MLP_WIDTHS = [4096] * 8 + [10]
MLP_R, MLP_N = 220, 256
MLP_WORKLOAD = ("full synthetic preconditioning step: 8-layer ReLU MLP 7x(4096->4096)+(4096->10), batch 256, "
                "r=220, rho=0.95, lambda=1e-2; 16 factor updates + 8 preconditioned gradients per step")


def mlp_inputs(torch, bkfac, synth, dev, steps):
    """Activations, pre-activation gradients and weight gradients of the seeded MLP for
    `steps` batches, copied into 16-byte aligned (padded) device buffers."""
    out = []
    for t in range(steps):
        acts, grads, wgrads = synth.mlp_batches(MLP_WIDTHS, MLP_N, 5000, 5001, t, device=dev)
        XA, XG, G = [], [], []
        for a, g, w in zip(acts, grads, wgrads):
            xa = bkfac.cols_tensor(MLP_N, a.shape[1], torch.float32, dev)
            xa.copy_(a)
            xg = bkfac.cols_tensor(MLP_N, g.shape[1], torch.float32, dev)
            xg.copy_(g)
            gw = bkfac.grad_tensor(w.shape[0], w.shape[1], torch.float32, dev)
            gw.copy_(w)
            XA.append(xa)
            XG.append(xg)
            G.append(gw)
        out.append((XA, XG, G))
    return out


def run_mlp(args, world, rank, local):
    """The MLP step as the headline (`--workload mlp`).  With N ranks the 8 layers are
    partitioned by the layer-cost model (shard.assign_layers); each rank updates its
    layers' factors and preconditions their gradients, then the ranks all-gather the
    steps (one collective per step).  value = factor updates of the whole MLP per second
    (strong scaling: the total work is fixed)."""
    import torch

    from paper_2210_08494_gb300 import bkfac, shard, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    bkfac.load()
    bkfac.bkfac_status()
    L = len(MLP_WIDTHS) - 1
    parts = shard.assign_layers([shard.layer_cost(MLP_WIDTHS[l], MLP_WIDTHS[l + 1], MLP_R, MLP_N)
                                 for l in range(L)], world)
    mine = parts[rank]
    pool = mlp_inputs(torch, bkfac, synth, dev, 4)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lam = [LAM] * len(mine)
    tune_cache = os.path.join(ROOT, "paper_2210_08494_gb300", "_build", "tune_cache.txt")

    def make_layers(dtype):
        return [(bkfac.Factor(MLP_WIDTHS[l] + 1, min(MLP_R, MLP_WIDTHS[l] + 1), dtype, device=dev),
                 bkfac.Factor(MLP_WIDTHS[l + 1], min(MLP_R, MLP_WIDTHS[l + 1]), dtype, device=dev))
                for l in mine]

    S_all = [bkfac.grad_tensor(x.shape[0], x.shape[1], torch.float32, dev) for x in pool[0][2]]
    results = {}
    # plain FP32 per-layer path: per-factor calls in sequence on one stream
    layers = make_layers(bkfac.F32)
    for a, g in layers:
        bkfac.bkfac_tune(a, MLP_N, tune_cache)
        bkfac.bkfac_tune(g, MLP_N, tune_cache)

    def plain_step(t):
        XA, XG, G = pool[t % len(pool)]
        for (a, g), l in zip(layers, mine):
            for f, X in ((a, XA[l]), (g, XG[l])):
                if f.r_cur == 0:
                    bkfac.bkfac_init(f, X)
                else:
                    bkfac.bkfac_update(f, X, RHO)
            bkfac.bkfac_apply(a, g, LAM, LAM, G[l], S_all[l])
        if world > 1:
            shard.exchange_steps(S_all, parts, rank)

    stream = torch.cuda.current_stream()
    if not args.mlp_only_mixed:
        plain_step(0)
        # the products' tile shapes and K splits, tuned on the step's own shapes (untimed)
        tune_products(bkfac, torch, lambda: plain_step(1), tune_cache)
        for t in range(2, args.warmup + 1):
            plain_step(t)
    torch.cuda.synchronize()

    def timed(fn, steps, s, clk_holder=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for t in range(steps):
            flush.zero_()
            evs[t][0].record(s)
            fn(t)
            evs[t][1].record(s)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return shard.max_over_ranks(float(sum(a.elapsed_time(b) for a, b in evs)), device=dev) / steps

    with ClockSampler(local) as clk:
        ms_plain = timed(lambda t: plain_step(args.warmup + 1 + t), args.steps if not args.mlp_only_mixed else 0,
                         stream) if not args.mlp_only_mixed else float("nan")
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"plain MLP step: {bkfac.strerror(st)}")
    results["plain_f32"] = {"ms_per_step": ms_plain, "value": 2 * L * 1000.0 / ms_plain}

    # batched paths: one graph per step over this rank's layers, fresh inputs copied in
    paths = (("batched_f32_graph", bkfac.F32), ("batched_mixed_bf16_graph", bkfac.MIXED_BF16))
    if args.mlp_only_mixed:
        paths = paths[1:]
    for name, dtype in paths:
        layers_b = make_layers(dtype)
        batch = bkfac.Batch(layers_b, MLP_N, dtype, tune_cache=tune_cache)
        XA0, XG0, G0 = pool[0]
        xa = [bkfac.cols_tensor(MLP_N, XA0[l].shape[1], torch.float32, dev) for l in mine]
        xg = [bkfac.cols_tensor(MLP_N, XG0[l].shape[1], torch.float32, dev) for l in mine]
        gb = [bkfac.grad_tensor(G0[l].shape[0], G0[l].shape[1], torch.float32, dev) for l in mine]
        Sb = [S_all[l] for l in mine]

        def load(t):
            XA, XG, G = pool[t % len(pool)]
            for dst, src in zip(xa + xg + gb, [XA[l] for l in mine] + [XG[l] for l in mine] + [G[l] for l in mine]):
                dst.copy_(src)

        s2 = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s2):
            load(0)
            batch.update(xa, xg, RHO)
            load(1)

            def eager_step():
                batch.update(xa, xg, RHO)
                batch.apply(gb, Sb, lam, lam)

            tune_products(bkfac, torch, eager_step, tune_cache)
            load(2)
            batch.step_graph(xa, xg, RHO, gb, Sb, lam, lam, capture=True)
            for t in range(args.warmup):
                load(3 + t)
                batch.step_graph()
        s2.synchronize()
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} warm-up: {bkfac.strerror(st)}")

        def gstep(t):
            batch.step_graph()
            if world > 1:
                shard.exchange_steps(S_all, parts, rank)

        with torch.cuda.stream(s2):
            ms = timed(gstep, args.steps, s2)
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} timed region: {bkfac.strerror(st)}")
        results[name] = {"ms_per_step": ms, "value": 2 * L * 1000.0 / ms}
        batch.close()

    best = results["batched_mixed_bf16_graph"]
    line = {
        "metric": METRIC, "value": best["value"], "unit": "factor-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"], "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "bf16-operands/f32-accum",
        "data": "synthetic",
        "config": {"workload": MLP_WORKLOAD, "path": "batched mixed BF16, CUDA graph",
                   "inputs": "resident in HBM; L2 flushed between timed steps",
                   "parallelism": (f"layers partitioned over {world} ranks {parts}, all-gather of the steps"
                                   if world > 1 else "single GPU")},
        "preconditioned_grads_per_s": L * 1000.0 / best["ms_per_step"],
        "paths": results, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_gpu(args, world, rank, local):
    import torch

    from paper_2210_08494_gb300 import bkfac, shard, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    bkfac.load()
    bkfac.bkfac_status()
    # an N-layer stack of identical wide layers partitioned over the ranks by the layer-cost
    # model (one layer per rank); after each step the ranks all-gather the layers' steps
    parts = shard.assign_layers([shard.layer_cost(D_A - 1, D_G, R, N)] * world, world)
    layer = parts[rank][0]
    seedA, seedG = synth.factor_seed(2, layer, "A"), synth.factor_seed(2, layer, "G")
    fA = bkfac.Factor(D_A, R, bkfac.F32, device=dev)
    fG = bkfac.Factor(D_G, R, bkfac.F32, device=dev)

    def dev_cols(Xt, f):
        t = bkfac.cols_tensor(Xt.shape[0], Xt.shape[1], torch.float32, dev)
        t.copy_(torch.from_numpy(Xt))
        return t

    XA = [dev_cols(synth.powerlaw_batch(D_A, N, ALPHA, seedA, t), fA) for t in range(POOL_X)]
    XG = [dev_cols(synth.powerlaw_batch(D_G, N, ALPHA, seedG, t), fG) for t in range(POOL_X)]
    gen = torch.Generator(device=dev).manual_seed(seedA + 500)
    Gs = []
    for _ in range(POOL_G):
        g = bkfac.grad_tensor(D_G, D_A, torch.float32, dev, zero=False)
        g.normal_(generator=gen)
        Gs.append(g)
    S_all = [bkfac.grad_tensor(D_G, D_A, torch.float32, dev) for _ in range(world)]
    S = S_all[layer]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    # autotune the eigensolve launch shapes once (untimed; cached per machine)
    tune_cache = os.path.join(ROOT, "paper_2210_08494_gb300", "_build", "tune_cache.txt")
    for f in (fA, fG):
        bkfac.bkfac_tune(f, N, tune_cache)
    bkfac.bkfac_init(fA, XA[0])
    bkfac.bkfac_init(fG, XG[0])
    stream = torch.cuda.current_stream()

    def step(t):
        bkfac.bkfac_update(fA, XA[1 + t % (POOL_X - 1)], RHO)
        bkfac.bkfac_update(fG, XG[1 + t % (POOL_X - 1)], RHO)
        bkfac.bkfac_apply(fA, fG, LAM, LAM, Gs[t % POOL_G], S)
        if world > 1:
            shard.exchange_steps(S_all, parts, rank)  # every rank receives every layer's step

    # the products' tile shapes and K splits, tuned on the step's own shapes (untimed)
    tune_products(bkfac, torch, lambda: step(0), tune_cache)
    for t in range(1, args.warmup):
        step(t)
    torch.cuda.synchronize()
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"device status after warm-up: {bkfac.strerror(st)}")

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    _, launches0 = bkfac.bkfac_trace_read()
    bkfac.bkfac_trace_enable(True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for t in range(args.steps):
            flush.zero_()
            evs[t][0].record(stream)
            step(args.warmup + t)
            evs[t][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    trace, launches1 = bkfac.bkfac_trace_read()
    bkfac.bkfac_trace_enable(False)
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"device status after timed region: {bkfac.strerror(st)}")
    ms_total = shard.max_over_ranks(float(sum(a.elapsed_time(b) for a, b in evs)), device=dev)
    ms_step = ms_total / args.steps
    steps_per_s = 1000.0 / ms_step
    value = 2.0 * steps_per_s * world
    gpu_launches = launches1 - launches0

    # ---- roofline of the dominant phase (CUDA events around each phase, same stream)
    sweeps = int(fA.ws(N)[bkfac.bkfac_debug_offsets(fA, N)[7]:][:4].view(torch.int32).item())
    peaks, peak_src = measured_peaks()
    dom = max(trace.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_cnt) = dom
    work = algorithmic_work(dom_name, dom_ms, dom_cnt, sweeps)
    roof = None
    if work is not None and dom_cnt:
        per_launch_ms = dom_ms / dom_cnt
        if work["bound"] == "hbm":
            ach = work["bytes"] / (per_launch_ms * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_src}
        else:
            ach = work["flops"] / (per_launch_ms * 1e-3) / 1e12
            if work["bound"] == "alu":
                pk = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x FMA x max SM clock
                src = "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"
            else:
                pk = 1.25
                src = "nominal FP64 1.25 TFLOP/s"
            roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": DRAM_BYTES_PER_LAUNCH.get(dom_name), "peak_source": src}
        roof["kernel"] = dom_name
        roof["launch_ms"] = per_launch_ms

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed
    # region: every step copies its batches and gradient in and its preconditioned step out.
    # The copies run on a second stream with two device buffer sets, so that step t + 1's
    # inputs arrive and step t's result leaves while step t computes (how a training loop
    # feeds the library); the timed region spans the first input copy to the last output
    # copy.
    e2e = None
    if not args.no_e2e:
        ldA, ldG, ldg = fA.U.stride(0), fG.U.stride(0), Gs[0].stride(0)
        hXA = torch.empty(N, ldA, dtype=torch.float32, pin_memory=True)
        hXG = torch.empty(N, ldG, dtype=torch.float32, pin_memory=True)
        hG = torch.empty(D_G, ldg, dtype=torch.float32, pin_memory=True)
        hXA[:, :D_A].copy_(XA[1])
        hXG[:, :D_G].copy_(XG[1])
        hG[:, :D_A].copy_(Gs[0])
        hS = [torch.empty(D_G, ldg, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        bufs = []
        for _ in range(2):
            bXA = torch.zeros(N, ldA, dtype=torch.float32, device=dev)
            bXG = torch.zeros(N, ldG, dtype=torch.float32, device=dev)
            bG = torch.zeros(D_G, ldg, dtype=torch.float32, device=dev)
            bS = torch.zeros(D_G, ldg, dtype=torch.float32, device=dev)
            bufs.append((bXA, bXG, bG, bS))
        cs = torch.cuda.Stream(device=dev)
        ev = lambda: torch.cuda.Event()  # noqa: E731
        h2d_done, comp_done, d2h_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        e2e_steps = max(3, min(args.steps, 10))

        def h2d(i):
            bXA, bXG, bG, _ = bufs[i]
            with torch.cuda.stream(cs):
                bXA.copy_(hXA, non_blocking=True)
                bXG.copy_(hXG, non_blocking=True)
                bG.copy_(hG, non_blocking=True)
            h2d_done[i].record(cs)

        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs.wait_event(e0)
        h2d(0)
        for t in range(e2e_steps):
            i = t % 2
            bXA, bXG, bG, bS = bufs[i]
            stream.wait_event(h2d_done[i])
            if t >= 2:
                stream.wait_event(d2h_done[i])  # bS of step t - 2 has left
            bkfac.bkfac_update(fA, bXA[:, :D_A], RHO)
            bkfac.bkfac_update(fG, bXG[:, :D_G], RHO)
            bkfac.bkfac_apply(fA, fG, LAM, LAM, bG[:, :D_A], bS[:, :D_A])
            comp_done[i].record(stream)
            if t + 1 < e2e_steps:
                if t >= 1:
                    cs.wait_event(comp_done[1 - i])  # step t - 1 has finished reading the other set
                h2d(1 - i)
            cs.wait_event(comp_done[i])
            with torch.cuda.stream(cs):
                hS[i].copy_(bS, non_blocking=True)
            d2h_done[i].record(cs)
        stream.wait_event(d2h_done[(e2e_steps - 1) % 2])
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1) / e2e_steps
        e2e = {"value": 2.0 * 1000.0 / ms_e2e * world, "unit": "factor-updates/s",
               "h2d_bytes_per_step": int((hXA.numel() + hXG.numel() + hG.numel()) * 4),
               "d2h_bytes_per_step": int(hS[0].numel() * 4), "ms_per_step": ms_e2e,
               "copies": "pinned host buffers, a copy stream and two device buffer sets "
                         "(step t+1 in and step t out while step t computes)"}

    # ---- the same plain per-factor step with the FP32 products as 3xTF32 on the tensor cores
    def plain_variant(flags):
        gA = bkfac.Factor(D_A, R, bkfac.F32, device=dev, flags=flags)
        gG = bkfac.Factor(D_G, R, bkfac.F32, device=dev, flags=flags)
        bkfac.bkfac_init(gA, XA[0])
        bkfac.bkfac_init(gG, XG[0])

        def vstep(t):
            bkfac.bkfac_update(gA, XA[1 + t % (POOL_X - 1)], RHO)
            bkfac.bkfac_update(gG, XG[1 + t % (POOL_X - 1)], RHO)
            bkfac.bkfac_apply(gA, gG, LAM, LAM, Gs[t % POOL_G], S)

        for t in range(args.warmup):
            vstep(t)
        ve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for t in range(args.steps):
            flush.zero_()
            ve[t][0].record(stream)
            vstep(args.warmup + t)
            ve[t][1].record(stream)
        torch.cuda.synchronize()
        if bkfac.bkfac_status() != bkfac.OK:
            raise RuntimeError("3xTF32 variant: device status not OK")
        ms = shard.max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ve)), device=dev) / args.steps
        return {"value": 2.0 * 1000.0 / ms * world, "unit": "factor-updates/s", "ms_per_step": ms,
                "path": "plain per-factor calls, FP32 products as 3xTF32 on the tensor cores (BKFAC_FLAG_TF32X3)",
                "parity_bound": 1e-4}

    variants = {} if args.no_batched else {"plain_f32_tf32x3": plain_variant(bkfac.FLAG_TF32X3)}

    # ---- the inverse application alone: Algorithm 1 on the dense gradient vs Algorithm 8 on the
    # thin factors of the same layer (A_f 4097 x 256, G_f 4096 x 256; S = G_f-side x A_f-side / n)
    def time_calls(fn, reps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        torch.cuda.synchronize()
        for t in range(reps):
            flush.zero_()
            ev[t][0].record(stream)
            fn(t)
            ev[t][1].record(stream)
        torch.cuda.synchronize()
        if bkfac.bkfac_status() != bkfac.OK:
            raise RuntimeError("apply timing: device status not OK")
        return shard.max_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)), device=dev) / reps

    PA = bkfac.cols_tensor(N, D_A, torch.float32, dev)
    PG = bkfac.cols_tensor(N, D_G, torch.float32, dev)
    xi = lambda t: 1 + t % (POOL_X - 1)  # noqa: E731
    dense_apply = lambda t: bkfac.bkfac_apply(fA, fG, LAM, LAM, Gs[t % POOL_G], S)  # noqa: E731
    fact_apply = lambda t: bkfac.bkfac_apply_factored(fA, fG, LAM, LAM, XA[xi(t)], XG[xi(t)], PA, PG,  # noqa: E731
                                                      alpha=1.0 / N, S=S)
    thin_apply = lambda t: bkfac.bkfac_apply_factored(fA, fG, LAM, LAM, XA[xi(t)], XG[xi(t)], PA, PG)  # noqa: E731
    for fn in ((dense_apply, fact_apply, thin_apply) if not args.no_batched else ()):
        for t in range(args.warmup):
            fn(t)
    flops_dense = 4.0 * D_G * D_A * (R + R)
    flops_thin = 4.0 * N * (R * D_A + R * D_G)
    flops_fact = flops_thin + 2.0 * D_G * D_A * N
    apply_lines = {}
    for name, fn, flops, nbytes, path in () if args.no_batched else (
            ("dense_alg1", dense_apply, flops_dense, 2 * D_G * D_A * 4,
             "Algorithm 1 on the dense 4096 x 4097 gradient (two passes over G)"),
            ("factored_alg8", fact_apply, flops_fact, (N * (2 * D_A + 2 * D_G) + D_G * D_A) * 4,
             "Algorithm 8 on the thin factors, step S = PG PA^T / n formed"),
            ("factored_alg8_thin", thin_apply, flops_thin, N * (2 * D_A + 2 * D_G) * 4,
             "Algorithm 8, preconditioned thin factors only (no S)")):
        ms = time_calls(fn, max(args.steps, 3))
        apply_lines[name] = {"value": 1000.0 / ms * world, "unit": "preconditioned-grads/s", "ms": ms,
                             "gflop": flops / 1e9, "tflops": flops / (ms * 1e-3) / 1e12,
                             "algorithmic_gbytes": nbytes / 1e9, "path": path, "parity_bound": 1e-4}

    # ---- B-KFAC-C / B-R-KFAC pieces on the A factor (d = 4097): the dense EA factor update,
    # a light correction of 128 modes (phi_crc = 0.5) and an RSVD overwrite (r + 10 test
    # columns, 4 power iterations)
    variants_dense = {}
    if not args.no_batched:
        variants_dense = dense_factor_variants(args, bkfac, torch, np, dev, XA, xi, time_calls, seedA)


    batched = {} if args.no_batched else {
        "f32_graph": run_batched(args, bkfac, synth, torch, dev, seedA, seedG, bkfac.F32, flush),
        "mixed_bf16_graph": run_batched(args, bkfac, synth, torch, dev, seedA, seedG, bkfac.MIXED_BF16, flush),
    }
    for v in batched.values():
        v["value"] *= world

    peaks_ps, peak_srcs = pipe_peaks(torch, dev)
    head_items = (update_work(D_A, R, N, R, "f32", sweeps) + update_work(D_G, R, N, R, "f32", sweeps) +
                  apply_work(D_A, D_G, R, R, "f32"))
    composed = composed_roofline(head_items, ms_step, peaks_ps, peak_srcs)
    for bname, v in batched.items():
        prec = "mixed" if bname.startswith("mixed") else "f32"
        v["roofline"] = composed_roofline(update_work(D_A, R, N, R, prec, sweeps) +
                                          update_work(D_G, R, N, R, prec, sweeps) +
                                          apply_work(D_A, D_G, R, R, prec), v["ms_per_step"], peaks_ps, peak_srcs)

    workloads = {}
    if not args.no_workloads:
        for wname, fn in (("small_fp64", small_fp64_workload), ("uneven_batch", uneven_workload),
                          ("mlp", mlp_workload)):
            workloads[wname] = fn(args, bkfac, synth, torch, dev, flush, peaks_ps, peak_srcs)
            torch.cuda.synchronize()
            torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "factor-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "path": "plain FP32 per-factor calls", "layers_per_gpu": 1,
                       "inputs": "resident in HBM; L2 flushed (256 MB write) between timed steps",
                       "parallelism": (f"{world} identical wide layers, one per rank (layer-cost assignment), "
                                       "all-gather of the preconditioned steps in each timed step"
                                       if world > 1 else "single GPU")},
            "preconditioned_grads_per_s": steps_per_s * world,
            "roofline": roof, "composed_roofline": composed, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in trace.items() if v[1]},
            "jacobi_sweeps": sweeps,
            "batched": batched,
            "variants": variants,
            "apply": apply_lines,
            "dense_factor_variants": variants_dense,
            "workloads": workloads,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def dense_factor_variants(args, bkfac, torch, np, dev, XA, xi, time_calls, seedA):
    """B-KFAC-C / B-R-KFAC pieces on the wide layer's A factor (d = 4097): the dense EA factor
    update, a light correction of 128 modes (phi_crc = 0.5) and an RSVD overwrite (r + 10 test
    columns, 4 power iterations)."""
    out = {}
    Md = bkfac.dense_factor(D_A, bkfac.F32, dev)
    bkfac.bkfac_ea_update(Md, XA[0], RHO, bkfac.F32, first=True)
    gB = bkfac.Factor(D_A, R, bkfac.F32, device=dev)
    bkfac.bkfac_init(gB, XA[0])
    idx_crc = [int(i) for i in np.random.default_rng(seedA + 7).choice(R, R // 2, replace=False)]
    Om = bkfac.cols_tensor(R + 10, D_A, torch.float32, dev)
    Om.normal_(generator=torch.Generator(device=dev).manual_seed(seedA + 8))
    ea_fn = lambda t: bkfac.bkfac_ea_update(Md, XA[xi(t)], RHO, bkfac.F32)  # noqa: E731
    crc_fn = lambda t: bkfac.bkfac_correct(gB, Md, idx_crc)  # noqa: E731
    rsvd_fn = lambda t: bkfac.bkfac_rsvd(gB, Md, Om, 4)  # noqa: E731
    for fn in (ea_fn, crc_fn, rsvd_fn):
        for t in range(2):
            fn(t)
    l_rs = R + 10
    for name, fn, flops, nbytes, path in (
            ("ea_update", ea_fn, 2.0 * D_A * D_A * N, 2.0 * D_A * D_A * 4,
             "dense EA factor M = rho M + (1 - rho)/n X X^T (d = 4097, n = 256, FP32)"),
            ("correct_alg6", crc_fn, 2.0 * D_A * D_A * (R // 2), D_A * D_A * 4.0,
             "light correction of 128 of 256 modes against M (Algorithm 6)"),
            ("rsvd_alg5", rsvd_fn, 2.0 * D_A * D_A * l_rs * 6, 6.0 * D_A * D_A * 4,
             "RSVD overwrite, l = 266 test columns, 4 power iterations (Algorithm 5)")):
        ms = time_calls(fn, max(min(args.steps, 5), 3))
        out[name] = {"ms": ms, "gflop": flops / 1e9, "tflops": flops / (ms * 1e-3) / 1e12,
                     "algorithmic_gbytes": nbytes / 1e9, "path": path, "parity_bound": 1e-4}
    return out


# --------------------------------------------------------------------------- profiler case
# A small self-contained run of one factor's updates (and optionally one layer's inverse
# application) at a chosen shape, for kernel profilers: `python bench.py --profile-case
# --d 4097 --r 256 --n 256 --updates 2 [--apply 4096 --synthetic-state --repeat 3]`.


def run_profile_case(args):
    import torch

    from paper_2210_08494_gb300 import bkfac, synth

    dtypes = {"f32": bkfac.F32, "f64": bkfac.F64, "mixed": bkfac.MIXED_BF16}
    bkfac.load()
    bkfac.bkfac_status()
    dtype = dtypes[args.dtype]
    fl = (bkfac.FLAG_TF32X3 if args.tf32x3 else 0) | (bkfac.FLAG_EIG_FP64 if args.eig_fp64 else 0)
    tdt = torch.float64 if dtype == bkfac.F64 else torch.float32

    def with_updates(d, seed):
        f = bkfac.Factor(d, args.r, dtype, flags=fl)
        xs = []
        for t in range(args.updates + 1):
            x = bkfac.cols_tensor(args.n, d, tdt)
            x.copy_(torch.from_numpy(synth.powerlaw_batch(d, args.n, args.alpha, seed, t)))
            xs.append(x)
        bkfac.bkfac_init(f, xs[0])
        for t in range(1, args.updates + 1):
            bkfac.bkfac_update(f, xs[t], RHO)
        return f

    def with_state(d, seed):
        f = bkfac.Factor(d, args.r, dtype, flags=fl)
        sig = np.arange(1, args.r + 1, dtype=np.float64) ** -1.2
        f.load_state(torch.from_numpy(synth.orthonormal_columns(d, args.r, seed)).to(f.torch_dtype).cuda(),
                     torch.from_numpy(sig).cuda())
        return f

    make = with_state if args.synthetic_state else with_updates
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    fA = make(args.d, 2000)
    end.record()
    if args.apply:
        fG = make(args.apply, 2001)
        G = bkfac.grad_tensor(args.apply, args.d, tdt)
        G.normal_(generator=torch.Generator(device="cuda").manual_seed(7))
        S = bkfac.grad_tensor(args.apply, args.d, tdt)
        bkfac.bkfac_apply(fA, fG, LAM, LAM, G, S)  # first call: one-time set-up
        start.record()
        for _ in range(args.repeat):
            bkfac.bkfac_apply(fA, fG, LAM, LAM, G, S)
        end.record()
    torch.cuda.synchronize()
    st = bkfac.bkfac_status()
    reps = args.repeat if args.apply else 1
    print(f"status {st} ({bkfac.strerror(st)}), {start.elapsed_time(end) / reps:.3f} ms per timed call")
    return 0 if st == bkfac.OK else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bkfac", choices=["bkfac", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the small FP64, uneven-batch and MLP workloads of the default run")
    ap.add_argument("--workload", default="wide-layer", choices=["wide-layer", "mlp"])
    ap.add_argument("--mlp-only-mixed", action="store_true",
                    help="with --workload mlp: time only the batched mixed path (for launch lists)")
    pc = ap.add_argument_group("profiler case (--profile-case)")
    pc.add_argument("--profile-case", action="store_true", help="run one factor's updates for a kernel profiler")
    pc.add_argument("--d", type=int, default=4097)
    pc.add_argument("--r", type=int, default=256)
    pc.add_argument("--n", type=int, default=256)
    pc.add_argument("--updates", type=int, default=1)
    pc.add_argument("--dtype", choices=["f32", "f64", "mixed"], default="f32")
    pc.add_argument("--alpha", type=float, default=1.2)
    pc.add_argument("--apply", type=int, default=0, metavar="D_OUT")
    pc.add_argument("--synthetic-state", action="store_true",
                    help="with --apply: load orthonormal factor states instead of running updates")
    pc.add_argument("--repeat", type=int, default=1, help="with --apply: time this many applications")
    pc.add_argument("--tf32x3", action="store_true", help="FP32 products as 3xTF32 on the tensor cores")
    pc.add_argument("--eig-fp64", action="store_true", help="core eigensolve in FP64")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    args.warmup = max(3, args.warmup) if args.impl == "bkfac" else args.warmup
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "mlp":
        return run_mlp(args, world, rank, local)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
