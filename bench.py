"""Benchmark of the B-KFAC preconditioning hot path on one GB300.

Workload (the one-wide-FC-layer configuration): forward factor A at d = 4097
(4096 inputs + bias), backward factor Gamma at d = 4096, rank r = 256, n = 256
new columns per step, rho = 0.95, lambda = 1e-2, FP32 plain per-factor path.
One step = Brand update of A + Brand update of Gamma + damped inverse
application to a fresh 4096 x 4097 FP32 gradient.  Inputs are seeded
synthetic power-law batches (exponent 1.2) and N(0, 1) gradients, resident in
HBM before the timed region (config["inputs"]).

Metric: factor updates per second (two per step); the preconditioned
gradients per second are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bkfac|reference]
Under torchrun (N > 1) every rank runs the same per-GPU workload on its own
layer (independent replicas, weak scaling); timing is the max over ranks.
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
    """The oracle timed on the host cores on one full step (about 10-30 s)."""
    import oracle
    from paper_2210_08494_gb300 import synth

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    seedA, seedG = synth.factor_seed(2, 0, "A"), synth.factor_seed(2, 0, "G")
    XA = [synth.powerlaw_batch(D_A, N, ALPHA, seedA, t) for t in range(2)]
    XG = [synth.powerlaw_batch(D_G, N, ALPHA, seedG, t) for t in range(2)]
    G = synth.gradient(D_G, D_A, seedA, 0)
    UA, sA, iA = oracle.init(XA[0], R)
    UG, sG, iG = oracle.init(XG[0], R)
    t0 = time.perf_counter()
    UA2, sA2, _ = oracle.update(UA, sA, iA["r_new"], XA[1], RHO, R)
    UG2, sG2, _ = oracle.update(UG, sG, iG["r_new"], XG[1], RHO, R)
    oracle.apply(UA2, sA2, LAM, UG2, sG2, LAM, G)
    dt = time.perf_counter() - t0
    return {"value": 2.0 / dt, "unit": "factor-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"1 full step (2 factor updates at d=4097/4096, r=n=256 + 1 apply to 4096x4097), {dt:.1f} s"}


# --------------------------------------------------------------------------- GPU arm


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of the
# kernel on this workload (the 512-column update eigensolve: 1.137 MB read, 0 written;
# the blocks live in shared memory and registers).  Reset to None when the kernel changes.
DRAM_BYTES_PER_LAUNCH = {"jacobi": 1136640}


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
            "parity_bound": 1e-4 if dtype == bkfac.F32 else 2e-2}


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
    import torch

    from paper_2210_08494_gb300 import bkfac, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bkfac.load()
    bkfac.bkfac_status()
    L = len(MLP_WIDTHS) - 1
    pool = mlp_inputs(torch, bkfac, synth, dev, 4)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    lam = [LAM] * L
    tune_cache = os.path.join(ROOT, "paper_2210_08494_gb300", "_build", "tune_cache.txt")

    def make_layers(dtype):
        return [(bkfac.Factor(MLP_WIDTHS[l] + 1, min(MLP_R, MLP_WIDTHS[l] + 1), dtype, device=dev),
                 bkfac.Factor(MLP_WIDTHS[l + 1], min(MLP_R, MLP_WIDTHS[l + 1]), dtype, device=dev))
                for l in range(L)]

    results = {}
    # plain FP32 per-layer path: per-factor calls in sequence on one stream
    layers = make_layers(bkfac.F32)
    for a, g in layers:
        bkfac.bkfac_tune(a, MLP_N, tune_cache)
        bkfac.bkfac_tune(g, MLP_N, tune_cache)
    S = [bkfac.grad_tensor(x.shape[0], x.shape[1], torch.float32, dev) for x in pool[0][2]]

    def plain_step(t):
        XA, XG, G = pool[t % len(pool)]
        for l, (a, g) in enumerate(layers):
            for f, X in ((a, XA[l]), (g, XG[l])):
                if f.r_cur == 0:
                    bkfac.bkfac_init(f, X)
                else:
                    bkfac.bkfac_update(f, X, RHO)
            bkfac.bkfac_apply(a, g, LAM, LAM, G[l], S[l])

    stream = torch.cuda.current_stream()
    for t in range(args.warmup + 1):
        plain_step(t)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for t in range(args.steps):
            flush.zero_()
            evs[t][0].record(stream)
            plain_step(args.warmup + 1 + t)
            evs[t][1].record(stream)
        torch.cuda.synchronize()
    st = bkfac.bkfac_status()
    if st != bkfac.OK:
        raise RuntimeError(f"plain MLP step: {bkfac.strerror(st)}")
    ms_plain = float(sum(a.elapsed_time(b) for a, b in evs)) / args.steps
    results["plain_f32"] = {"ms_per_step": ms_plain, "value": 2 * L * 1000.0 / ms_plain}

    # batched paths: one graph per step, fresh inputs copied into the graph's buffers
    for name, dtype in (("batched_f32_graph", bkfac.F32), ("batched_mixed_bf16_graph", bkfac.MIXED_BF16)):
        layers_b = make_layers(dtype)
        batch = bkfac.Batch(layers_b, MLP_N, dtype, tune_cache=tune_cache)
        XA0, XG0, G0 = pool[0]
        xa = [bkfac.cols_tensor(MLP_N, x.shape[1], torch.float32, dev) for x in XA0]
        xg = [bkfac.cols_tensor(MLP_N, x.shape[1], torch.float32, dev) for x in XG0]
        gb = [bkfac.grad_tensor(x.shape[0], x.shape[1], torch.float32, dev) for x in G0]
        Sb = [bkfac.grad_tensor(x.shape[0], x.shape[1], torch.float32, dev) for x in G0]

        def load(t):
            XA, XG, G = pool[t % len(pool)]
            for dst, src in zip(xa + xg + gb, XA + XG + G):
                dst.copy_(src)

        s2 = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(s2):
            for t in range(2):
                load(t)
                batch.update(xa, xg, RHO)
            load(2)
            batch.step_graph(xa, xg, RHO, gb, Sb, lam, lam, capture=True)
            for t in range(args.warmup):
                load(3 + t)
                batch.step_graph()
        s2.synchronize()
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} warm-up: {bkfac.strerror(st)}")
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with torch.cuda.stream(s2):
            for t in range(args.steps):
                load(t)
                flush.zero_()
                evs[t][0].record(s2)
                batch.step_graph()
                evs[t][1].record(s2)
        s2.synchronize()
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"{name} timed region: {bkfac.strerror(st)}")
        ms = float(sum(a.elapsed_time(b) for a, b in evs)) / args.steps
        results[name] = {"ms_per_step": ms, "value": 2 * L * 1000.0 / ms}
        batch.close()

    best = results["batched_mixed_bf16_graph"]
    line = {
        "metric": METRIC, "value": best["value"] * world, "unit": "factor-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16-operands/f32-accum", "data": "synthetic",
        "config": {"workload": MLP_WORKLOAD, "path": "batched mixed BF16, CUDA graph",
                   "inputs": "resident in HBM; L2 flushed between timed steps"},
        "preconditioned_grads_per_s": L * 1000.0 / best["ms_per_step"] * world,
        "paths": results, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
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
    layer = rank  # each rank preconditions its own layer (independent replicas)
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
    S = bkfac.grad_tensor(D_G, D_A, torch.float32, dev)
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

    for t in range(args.warmup):
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
                       "parallelism": f"replicas x{world}"},
            "preconditioned_grads_per_s": steps_per_s * world,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in trace.items() if v[1]},
            "jacobi_sweeps": sweeps,
            "batched": batched,
            "variants": variants,
            "apply": apply_lines,
            "dense_factor_variants": variants_dense,
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bkfac", choices=["bkfac", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--workload", default="wide-layer", choices=["wide-layer", "mlp"])
    args = ap.parse_args()
    args.warmup = max(3, args.warmup) if args.impl == "bkfac" else args.warmup
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "mlp":
        return run_mlp(args, world, rank, local)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
