"""Mixed-precision path over a long run: 1000 batched steps (BF16 tall-skinny
products on the tensor cores, FP32 accumulation, FP64 CholeskyQR) with FP64
re-orthonormalisation of every U each 10 steps, tracked against the FP64
oracle running the same 1000 steps.

Reported every 100 steps and checked against the mixed path's bound (2e-2):
* reconstruction error of U diag(sigma) U^T (relative Frobenius),
* error of the damped inverse application to a fixed gradient,
* the largest principal angle between the leading r/4 eigenvector subspaces
  (reported; those modes are separated from the rest by wide spectral gaps).
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import lowrank_rel_err, rel

pytestmark = pytest.mark.gpu

LAYERS = [(257, 128, 32), (129, 64, 16)]  # (d_in + bias, d_out, r)
N, RHO, ALPHA, LAM, STEPS = 64, 0.95, 1.3, 1e-2, 1000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def max_angle(Ua, Ub, k):
    """Largest principal angle (radians) between the spans of the first k rows."""
    s = np.linalg.svd(np.asarray(Ua[:k]) @ np.asarray(Ub[:k]).T, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def test_mixed_1000_steps_against_fp64_oracle(oracle):
    layers = [(bkfac.Factor(dA, r, bkfac.MIXED_BF16), bkfac.Factor(dG, r, bkfac.MIXED_BF16)) for dA, dG, r in LAYERS]
    batch = bkfac.Batch(layers, N, bkfac.MIXED_BF16)
    grads = [synth.gradient(dG, dA, 6000 + l, 0) for l, (dA, dG, r) in enumerate(LAYERS)]
    G = []
    for l, (dA, dG, r) in enumerate(LAYERS):
        g = bkfac.grad_tensor(dG, dA, torch.float32)
        g.copy_(torch.from_numpy(grads[l]))
        G.append(g)
    S = [bkfac.grad_tensor(g.shape[0], g.shape[1], torch.float32) for g in G]
    XA = [bkfac.cols_tensor(N, dA, torch.float32) for dA, _, _ in LAYERS]
    XG = [bkfac.cols_tensor(N, dG, torch.float32) for _, dG, _ in LAYERS]
    ref = {}
    worst = {"recon": 0.0, "apply": 0.0}
    for t in range(STEPS):
        for l, (dA, dG, r) in enumerate(LAYERS):
            XA[l].copy_(torch.from_numpy(synth.powerlaw_batch(dA, N, ALPHA, synth.factor_seed(5, l, "A"), t)))
            XG[l].copy_(torch.from_numpy(synth.powerlaw_batch(dG, N, ALPHA, synth.factor_seed(5, l, "G"), t)))
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
        if (t + 1) % 100 == 0:
            batch.apply(G, S, [LAM] * len(LAYERS), [LAM] * len(LAYERS))
            batch.sync_descriptors()
            assert bkfac.bkfac_status() == bkfac.OK
            line = [f"step {t + 1}:"]
            for l, (dA, dG, r) in enumerate(LAYERS):
                states = []
                for w in (0, 1):
                    U, s = layers[l][w].state()
                    Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
                    Uo, so, k = ref[(l, w)]
                    er = lowrank_rel_err(Ug, sg, Uo, so)
                    ang = max_angle(Ug, Uo, max(1, r // 4))
                    worst["recon"] = max(worst["recon"], er)
                    assert er < 2e-2, (t, l, w, er)
                    line.append(f"L{l}{'AG'[w]} recon {er:.2e} angle {ang:.2e}")
                    states.append((Uo, so))
                (UA, sA), (UG, sG) = states
                So = oracle.apply(UA, sA, LAM, UG, sG, LAM, grads[l])
                ea = rel(S[l].double().cpu().numpy(), So)
                worst["apply"] = max(worst["apply"], ea)
                assert ea < 2e-2, (t, l, ea)
                line.append(f"L{l} apply {ea:.2e}")
            print(" ".join(line))
    print(f"worst over {STEPS} steps: reconstruction {worst['recon']:.2e}, inverse application {worst['apply']:.2e}")
    batch.close()
