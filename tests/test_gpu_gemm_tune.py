"""GPU: the GEMM autotuner (bkfac_gemm_tune_begin / _end).

The FP32 products an update and an apply launch are noted, each noted shape is
timed over its candidates (64 x 64 or 128 x 128 tiles, K splits within the
call's partial buffer) on synthetic operands, and the fastest is kept in the
process-wide table and the cache file.  Later calls of those shapes run with the
tuned choices; a choice changes only the order of the K sums, so the tuned path
is held to the same parity against the FP64 oracle as the default one: 1e-4 on
the FP32 path for the update (one-step mode, tests.parity_util.judge_step) and
for the damped inverse application.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import rel
from tests.test_gpu_update import check_status, gpu_state, one_step_parity, to_dev

pytestmark = pytest.mark.gpu

D_A, D_G, R, N, RHO, LAM = 1025, 512, 64, 128, 0.95, 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def step_and_apply(fA, fG, t):
    for f, seed in ((fA, 31), (fG, 32)):
        bkfac.bkfac_update(f, to_dev(synth.powerlaw_batch(f.d, N, 1.2, seed, t), f), RHO)
    G = bkfac.grad_tensor(D_G, D_A, torch.float32)
    G.copy_(torch.from_numpy(synth.gradient(D_G, D_A, 33, t)))
    S = bkfac.grad_tensor(D_G, D_A, torch.float32)
    bkfac.bkfac_apply(fA, fG, LAM, LAM, G, S)
    check_status()
    return G, S


def test_gemm_tuning_notes_shapes_and_keeps_parity(oracle, tmp_path):
    cache = str(tmp_path / "tune.txt")
    fA = bkfac.Factor(D_A, R, bkfac.F32)
    fG = bkfac.Factor(D_G, R, bkfac.F32)
    for f, seed in ((fA, 31), (fG, 32)):
        bkfac.bkfac_init(f, to_dev(synth.powerlaw_batch(f.d, N, 1.2, seed, 0), f))
    bkfac.bkfac_gemm_tune_begin()
    step_and_apply(fA, fG, 1)
    bkfac.bkfac_gemm_tune_end(cache)
    lines = [ln.split() for ln in open(cache) if ln.startswith("M ")]
    assert lines, "no product shape was tuned"
    for ln in lines:
        M, Nn, K0, K1, bits, kern, sp = (int(x) for x in ln[1:8])
        assert M > 0 and Nn > 0 and K0 + K1 >= 0 and kern in (1, 2) and 1 <= sp <= 32, ln
        assert float(ln[8]) > 0.0
    shapes = {(int(ln[1]), int(ln[2]), int(ln[3])) for ln in lines}
    print(f"{len(lines)} product shapes tuned: " + ", ".join(
        f"{ln[1]}x{ln[2]} K={ln[3]}+{ln[4]}: {'64x64' if ln[6] == '1' else '128x128'} tiles, {ln[7]} splits"
        for ln in lines))
    # the update's projection U^T X (r x n over K = d) is among them
    assert any(M == R and Nn == N and K0 == D_A for M, Nn, K0 in shapes)
    # tuned calls: the next step and apply against the oracle, from the GPU's state
    before = [gpu_state(f) for f in (fA, fG)]
    G, S = step_and_apply(fA, fG, 2)
    post = []
    for f, seed, (U0, s0) in zip((fA, fG), (31, 32), before):
        X = synth.powerlaw_batch(f.d, N, 1.2, seed, 2)
        Uo, so, info = oracle.update(U0, s0, U0.shape[0], X.astype(np.float32).astype(np.float64), RHO,
                                     min(U0.shape[0] + N, f.d))
        k = min(R, info["r_new"])
        U, s = gpu_state(f)
        Lg = U[:k].T * s[:k] @ U[:k]
        Lo = Uo[:k].T * so[:k] @ Uo[:k]
        e = rel(Lg, Lo)
        print(f"tuned update d={f.d}: reconstruction {e:.2e}")
        assert e < 1e-4
        post.append((U[:k], s[:k]))
    (UA, sA), (UG, sG) = post
    So = oracle.apply(UA, sA, LAM, UG, sG, LAM, G.double().cpu().numpy())
    ea = rel(S.double().cpu().numpy(), So)
    print(f"tuned apply: {ea:.2e}")
    assert ea < 1e-4


def test_gemm_tuning_one_step_parity_after_tuning(oracle):
    # the default one-step parity case of the FP32 path, run after the table holds choices
    one_step_parity(oracle, 600, 48, 40, bkfac.F32, alpha=1.2, steps=3)
