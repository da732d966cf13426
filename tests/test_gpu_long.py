"""Longer GPU runs through the batch API.

* Mixed BF16 path over many steps with re-orthonormalisation every 10 steps:
  the free-running trajectory stays within the mixed path's stated bound of the
  FP64 oracle's trajectory, and U^T U returns to I after each reorth.
* Checkpoint / resume: the factor state is (U, sigma, r_cur, step); saving it
  after k steps and resuming in a fresh factor reproduces the uninterrupted run
  bit for bit (the kernels are deterministic: fixed reduction orders, no
  atomics in the numerics).
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import lowrank_rel_err, orth_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


LAYERS = [(513, 256, 64), (257, 128, 32)]  # (d_in + bias, d_out, r)
N, RHO, ALPHA = 64, 0.95, 1.2


def batch_inputs(step):
    XA, XG = [], []
    for l, (dA, dG, r) in enumerate(LAYERS):
        a = bkfac.cols_tensor(N, dA, torch.float32)
        a.copy_(torch.from_numpy(synth.powerlaw_batch(dA, N, ALPHA, synth.factor_seed(4, l, "A"), step)))
        g = bkfac.cols_tensor(N, dG, torch.float32)
        g.copy_(torch.from_numpy(synth.powerlaw_batch(dG, N, ALPHA, synth.factor_seed(4, l, "G"), step)))
        XA.append(a)
        XG.append(g)
    return XA, XG


def test_mixed_trajectory_with_reorth_tracks_fp64_oracle(oracle):
    steps = 60
    layers = [(bkfac.Factor(dA, r, bkfac.MIXED_BF16), bkfac.Factor(dG, r, bkfac.MIXED_BF16)) for dA, dG, r in LAYERS]
    batch = bkfac.Batch(layers, N, bkfac.MIXED_BF16)
    ref = {}  # oracle state per factor: (U, sigma, k)
    worst = 0.0
    for t in range(steps):
        XA, XG = batch_inputs(t)
        batch.update(XA, XG, RHO)
        for l, (dA, dG, r) in enumerate(LAYERS):
            for w, X in ((0, XA[l]), (1, XG[l])):
                Xn = X.double().cpu().numpy()
                if (l, w) not in ref:
                    Uo, so, info = oracle.init(Xn, r)
                else:
                    U0, s0, k0 = ref[(l, w)]
                    Uo, so, info = oracle.update(U0, s0, k0, Xn, RHO, r)
                k = info["r_new"]
                ref[(l, w)] = (Uo[:k], so[:k], k)
        if (t + 1) % 10 == 0:
            batch.reorth()
            batch.sync_descriptors()
            assert bkfac.bkfac_status() == bkfac.OK
            for l in range(len(LAYERS)):
                for w in (0, 1):
                    f = layers[l][w]
                    U, s = f.state()
                    Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
                    Uo, so, k = ref[(l, w)]
                    err = lowrank_rel_err(Ug, sg, Uo, so)
                    worst = max(worst, err)
                    assert err < 2e-2, (t, l, w, err)
                    assert orth_err(Ug) < 1e-4, (t, l, w, orth_err(Ug))
    print(f"mixed BF16 trajectory, {steps} steps, reorth every 10: worst reconstruction error {worst:.3e}")
    batch.close()


def test_checkpoint_resume_is_bit_exact():
    d, r, n = 700, 48, 40
    runs = []
    X = []
    for t in range(8):
        x = bkfac.cols_tensor(n, d, torch.float32)
        x.copy_(torch.from_numpy(synth.powerlaw_batch(d, n, ALPHA, 77, t)))
        X.append(x)
    # uninterrupted
    f = bkfac.Factor(d, r, bkfac.F32)
    bkfac.bkfac_init(f, X[0])
    for t in range(1, 8):
        bkfac.bkfac_update(f, X[t], RHO)
    full_U, full_s = (v.clone() for v in f.state())
    # interrupted after 4 steps: save (U, sigma, r_cur, step), resume in a fresh factor
    g = bkfac.Factor(d, r, bkfac.F32)
    bkfac.bkfac_init(g, X[0])
    for t in range(1, 4):
        bkfac.bkfac_update(g, X[t], RHO)
    U_ck, s_ck = (v.clone().cpu() for v in g.state())
    step_ck = g.step
    del g
    h = bkfac.Factor(d, r, bkfac.F32)
    h.load_state(U_ck.cuda(), s_ck.cuda(), step=step_ck)
    for t in range(4, 8):
        bkfac.bkfac_update(h, X[t], RHO)
    assert bkfac.bkfac_status() == bkfac.OK
    Uh, sh = h.state()
    assert h.step == f.step
    assert torch.equal(Uh, full_U) and torch.equal(sh, full_s)
