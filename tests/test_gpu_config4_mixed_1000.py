"""Mixed precision over 1000 steps on the 16-layer uneven batch (the shapes of
tests/test_gpu_uneven_batch.py: (d_in + bias, d_out) cycling through (513, 1024),
(1025, 2048), (2049, 4096), (4097, 4096), (4097, 10), r cycling through 64, 128,
256, n = 128, rho = 0.95) against the FP64 oracle.

Two variants run in lockstep on the same inputs, each re-orthonormalising every
U every 10 steps (bkfac_batch_reorth: FP64-accurate Gram, FP64 Cholesky):
* "fp64-core": BF16-operand tall-skinny products with FP32 accumulation, the
  CholeskyQR factorisations in FP64 (BKFAC_FLAG_CHOL_FP64) and the core
  eigensolve in FP64 (BKFAC_FLAG_EIG_FP64);
* "default": the same products, CholeskyQR factorisations and core eigensolve
  in FP32 (the mixed path's default).

Every 10 steps, layer 0's two factors (A at d = 513, Gamma at d = 1024, r = 64)
are compared with a free-running FP64 oracle trajectory from the same first
batch (trajectory mode; the oracle runs in a spawned child process beside the
GPU loop): reconstruction error of U diag(sigma) U^T, the largest principal
angle between the leading r/4 eigenvector subspaces, and the error of the damped
inverse application (lambda = 1e-2) to a fixed gradient.  Bound: 2e-2, the
mixed path's multi-step bound -- a one-step error of at most about u_bf16 that
the EA decay forgets over ~1/(1 - rho) = 20 steps, so independent step errors
add up to about sqrt(20) u_bf16 = 1.7e-2.  At the end, one step of the fp64-core
variant is checked on four sampled factors (the largest included) in one-step
mode with the one-step bound 1e-2.
"""
import time

import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests import oracle_worker
from tests.parity_util import judge_step, lowrank_rel_err, max_sin_theta, rel

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

SHAPES = [(513, 1024), (1025, 2048), (2049, 4096), (4097, 4096), (4097, 10)]
RANKS = [64, 128, 256]
NL, N, RHO, ALPHA, LAM = 16, 128, 0.95, 1.2, 1e-2
STEPS, EVERY = 1000, 10
TRAJ_TOL, STEP_TOL = 2e-2, 1e-2
VARIANTS = {"fp64-core": bkfac.FLAG_EIG_FP64 | bkfac.FLAG_CHOL_FP64, "default": 0}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def layer_shape(l):
    dA, dG = SHAPES[l % len(SHAPES)]
    return dA, dG, RANKS[l % len(RANKS)]


def test_config4_mixed_1000_steps_against_fp64_oracle(oracle):
    import os

    threads = max(1, (os.cpu_count() or 2) // 2)
    r0 = layer_shape(0)[2]
    # oracle trajectories of layer 0's A and Gamma, beside the GPU loop
    workers = [oracle_worker.Worker(r0, RHO, EVERY, threads) for _ in range(2)]
    dev = torch.device("cuda")
    gens = [(synth.DevicePowerlaw(layer_shape(l)[0], ALPHA, 4000 + 10 * l, dev),
             synth.DevicePowerlaw(layer_shape(l)[1], ALPHA, 4001 + 10 * l, dev)) for l in range(NL)]
    XA = [bkfac.cols_tensor(N, layer_shape(l)[0], torch.float32) for l in range(NL)]
    XG = [bkfac.cols_tensor(N, layer_shape(l)[1], torch.float32) for l in range(NL)]
    gg = torch.Generator(device=dev).manual_seed(4900)
    G = []
    for l in range(NL):
        dA, dG, _ = layer_shape(l)
        g = bkfac.grad_tensor(dG, dA, torch.float32)
        g.copy_(torch.randn(dG, dA, generator=gg, device=dev))
        G.append(g)
    G0 = G[0].double().cpu().numpy()
    runs = {}
    for name, flags in VARIANTS.items():
        layers = [(bkfac.Factor(layer_shape(l)[0], min(layer_shape(l)[2], layer_shape(l)[0]), bkfac.MIXED_BF16,
                                flags=flags),
                   bkfac.Factor(layer_shape(l)[1], min(layer_shape(l)[2], layer_shape(l)[1]), bkfac.MIXED_BF16,
                                flags=flags)) for l in range(NL)]
        batch = bkfac.Batch(layers, N, bkfac.MIXED_BF16)
        S = [bkfac.grad_tensor(g.shape[0], g.shape[1], torch.float32) for g in G]
        runs[name] = {"layers": layers, "batch": batch, "S": S, "snaps": {}, "ms": 0.0}
    stream = torch.cuda.Stream()
    try:
        for t in range(STEPS):
            with torch.cuda.stream(stream):
                for l in range(NL):
                    gens[l][0].draw(XA[l], N, t)
                    gens[l][1].draw(XG[l], N, t)
            stream.synchronize()
            for w, wk in enumerate(workers):
                X = (XA if w == 0 else XG)[0]
                wk.send(t, X[:, : layer_shape(0)[w]].double().cpu().numpy())
            last = t + 1 == STEPS
            for name, run in runs.items():
                b = run["batch"]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    if last and name == "fp64-core":
                        # one-step mode at the end: keep the states the last step starts from
                        b.sync_descriptors()
                        run["before"] = {(l, w): tuple(x.double().cpu().numpy() for x in run["layers"][l][w].state())
                                         for l, w in ((3, 0), (3, 1), (2, 1), (4, 0))}
                    b.update(XA, XG, RHO)
                    if (t + 1) % EVERY == 0:
                        b.reorth()
                    e1.record(stream)
                stream.synchronize()
                run["ms"] += e0.elapsed_time(e1)
                if (t + 1) % EVERY == 0:
                    with torch.cuda.stream(stream):
                        b.apply(G, run["S"], [LAM] * NL, [LAM] * NL)
                    stream.synchronize()
                    st = bkfac.bkfac_status()
                    assert st == bkfac.OK, (name, t, bkfac.strerror(st))
                    b.sync_descriptors()
                    a, g = run["layers"][0]
                    run["snaps"][t] = tuple(x.double().cpu().numpy() for f in (a, g) for x in f.state()) + (
                        run["S"][0].double().cpu().numpy(),)
        results = [wk.finish() for wk in workers]
    finally:
        for wk in workers:
            wk.kill()
    ref = {t: (UA, sA, UG, sG) for (t, UA, sA), (_, UG, sG) in zip(results[0], results[1])}
    k4 = max(1, r0 // 4)
    for name, run in runs.items():
        worst = {"recon": 0.0, "angle": 0.0, "apply": 0.0}
        lines = []
        for t in sorted(run["snaps"]):
            UA, sA, UG, sG, Sg = run["snaps"][t]
            UAo, sAo, UGo, sGo = ref[t]
            er = max(lowrank_rel_err(UA, sA, UAo, sAo), lowrank_rel_err(UG, sG, UGo, sGo))
            ang = max(max_sin_theta(UA, UAo, k4), max_sin_theta(UG, UGo, k4))
            So = oracle.apply(UAo, sAo, LAM, UGo, sGo, LAM, G0)
            ea = rel(Sg, So)
            worst["recon"] = max(worst["recon"], er)
            worst["angle"] = max(worst["angle"], ang)
            worst["apply"] = max(worst["apply"], ea)
            if (t + 1) % 100 == 0:
                lines.append(f"  step {t + 1}: reconstruction {er:.2e} sin(angle) {ang:.2e} apply {ea:.2e}")
        ups = 2 * NL * STEPS / (run["ms"] / 1000.0)
        print(f"{name}: worst over {STEPS} steps: reconstruction {worst['recon']:.2e}, "
              f"sin(angle, top {k4}) {worst['angle']:.2e}, inverse application {worst['apply']:.2e}; "
              f"{ups:.0f} factor-updates/s (update + reorth every {EVERY}, {run['ms'] / STEPS:.2f} ms per step)")
        print("\n".join(lines))
        assert worst["recon"] < TRAJ_TOL and worst["apply"] < TRAJ_TOL, (name, worst)
    # one-step mode on the last step of the fp64-core variant
    run = runs["fp64-core"]
    for (l, w), (U0, s0) in run["before"].items():
        f = run["layers"][l][w]
        X = (XA if w == 0 else XG)[l][:, : f.d].double().cpu().numpy()
        upd = oracle.update_dense if f.r + N >= f.d else oracle.update
        kin = U0.shape[0]
        Uo, so, info = upd(U0, s0, kin, X, RHO, min(kin + N, f.d))
        k = min(f.r, info["r_new"])
        U, s = f.state()
        m = judge_step(U.double().cpu().numpy(), s.cpu().numpy(), Uo[: info["r_new"]], so[: info["r_new"]], k,
                       bkfac.MIXED_BF16, STEP_TOL)
        print(f"fp64-core last step, layer {l} {'AG'[w]} d={f.d}: sigma {m['sigma']:.2e} "
              f"reconstruction {m['recon']:.2e}")
    for run in runs.values():
        run["batch"].close()
