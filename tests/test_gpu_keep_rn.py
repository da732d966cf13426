"""Truncation just before the next update (Algorithm 4's order, BKFAC_FLAG_KEEP_RN):
after an update the factor keeps the rank-(r + n) representation and the inverse
applications use it; the next update starts from its leading r modes.  Checked
against the FP64 oracle run with the same order (truncate the input to r, keep
min(r + n, ...) output modes)."""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import lowrank_rel_err, rel

pytestmark = pytest.mark.gpu

TOL = {bkfac.F64: 1e-10, bkfac.F32: 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def to_dev(Xt, f):
    t = bkfac.cols_tensor(Xt.shape[0], Xt.shape[1], f.torch_dtype)
    t.copy_(torch.from_numpy(Xt))
    return t


def run_side(oracle, d, r, n, dtype, seed, steps, rho=0.95):
    """One factor updated `steps` times with the rank-(r + n) representation kept; one-step
    parity (the oracle restarts from the GPU state each step)."""
    f = bkfac.Factor(d, r, dtype, flags=bkfac.FLAG_KEEP_RN, r_extra=n)
    X0 = synth.powerlaw_batch(d, n, 1.3, seed, 0)
    X0 = torch.from_numpy(X0).to(f.torch_dtype).double().numpy()
    bkfac.bkfac_init(f, to_dev(X0, f))
    Uo, so, info = oracle.init(X0, r + n)
    assert f.r_cur == info["r_new"] == min(n, d)
    worst = 0.0
    for t in range(1, steps + 1):
        U, s = f.state()
        Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
        k = min(f.r_cur, r)  # truncation to r just before the update
        X = torch.from_numpy(synth.powerlaw_batch(d, n, 1.3, seed, t)).to(f.torch_dtype).double().numpy()
        bkfac.bkfac_update(f, to_dev(X, f), rho)
        Uo, so, info = oracle.update(Ug[:k], sg[:k], k, X, rho, r + n)
        assert f.r_cur == info["r_new"] == min(k + n, r + n, d)
        Un, sn = f.state()
        err = lowrank_rel_err(Un.double().cpu().numpy(), sn.cpu().numpy(), Uo[:f.r_cur], so[:f.r_cur])
        worst = max(worst, err)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    assert worst < TOL[dtype], worst
    return f, worst


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_keep_rn_updates_and_apply(oracle, dtype):
    r, n = 24, 8
    fA, eA = run_side(oracle, 300, r, n, dtype, 7100, steps=5)
    fG, eG = run_side(oracle, 140, r, n, dtype, 7101, steps=5)
    assert fA.r_cur == r + n and fG.r_cur == r + n
    # the apply uses all r + n modes
    Gn = synth.gradient(140, 300, 7102, 0)
    G = bkfac.grad_tensor(140, 300, fA.torch_dtype)
    G.copy_(torch.from_numpy(Gn))
    S = bkfac.grad_tensor(140, 300, fA.torch_dtype)
    bkfac.bkfac_apply(fA, fG, 0.05, 0.05, G, S)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    (UA, sA), (UG, sG) = fA.state(), fG.state()
    So = oracle.apply(UA.double().cpu().numpy(), sA.cpu().numpy(), 0.05, UG.double().cpu().numpy(),
                      sG.cpu().numpy(), 0.05, G.double().cpu().numpy())
    ea = rel(S.double().cpu().numpy(), So)
    print(f"keep r+n dtype {dtype}: update {max(eA, eG):.2e}, apply with r+n modes {ea:.2e}")
    assert ea < TOL[dtype]


def test_keep_rn_reorth(oracle):
    """Re-orthonormalisation works on all r + n held modes."""
    f, _ = run_side(oracle, 200, 16, 8, bkfac.F32, 7103, steps=3)
    U, s = f.state()
    Ub, sb = U.double().cpu().numpy(), s.cpu().numpy()
    bkfac.bkfac_reorth(f)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    Ur, sr = f.state()
    assert f.r_cur == 24
    assert lowrank_rel_err(Ur.double().cpu().numpy(), sr.cpu().numpy(), Ub, sb) < 1e-5
