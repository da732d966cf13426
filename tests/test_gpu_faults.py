"""Device-side failure detection through the C ABI, in forms that fault, trap or
hang no GPU: every failure is made by the inputs or by a host-set limit, the
kernel records the error code in the status word and returns, and the next
call on the same context succeeds.

* BKFAC_ENOCONV: the eigensolve's sweep cap, set from the host to one sweep,
  is reached (the Brand core of a 600-row FP32 factor needs several sweeps);
* BKFAC_ETIMEOUT: the bounded mbarrier wait that guards the eigensolve's block
  exchange, given a short limit, waits on a barrier phase that nothing
  completes;
* BKFAC_ECHOL: the light correction of B-KFAC-C (Algorithm 6) is handed a
  dense factor M that is not positive semidefinite (M = -I), so the Cholesky
  factorisation of its projection U_s^T M U_s meets negative pivots.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import lowrank_rel_err, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield
    bkfac.bkfac_set_sweep_cap(0)


def to_dev(Xt, dtype):
    t = bkfac.cols_tensor(Xt.shape[0], Xt.shape[1], bkfac._TORCH_DTYPE[dtype])
    t.copy_(torch.from_numpy(Xt))
    return t


def clean_update_matches_oracle(oracle, seed):
    """A fresh factor's init and update: status OK and the oracle's result."""
    d, r, n = 400, 32, 24
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, n, 1.2, seed, 0)
    bkfac.bkfac_init(f, to_dev(X0, bkfac.F32))
    U, s = f.state()
    Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
    X = synth.powerlaw_batch(d, n, 1.2, seed, 1)
    Xd = to_dev(X, bkfac.F32)
    bkfac.bkfac_update(f, Xd, 0.95)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], Xd.double().cpu().numpy(), 0.95, r)
    U2, s2 = f.state()
    k = f.r_cur
    assert rel(s2.cpu().numpy(), so[:k]) < 1e-4
    assert lowrank_rel_err(U2.double().cpu().numpy(), s2.cpu().numpy(), Uo[:k], so[:k]) < 1e-4


def test_sweep_cap_reports_noconv_then_recovers(oracle):
    d, r, n = 600, 48, 40
    f = bkfac.Factor(d, r, bkfac.F32)
    bkfac.bkfac_init(f, to_dev(synth.powerlaw_batch(d, n, 1.2, 8100, 0), bkfac.F32))
    assert bkfac.bkfac_status() == bkfac.OK
    prev = bkfac.bkfac_set_sweep_cap(1)
    try:
        bkfac.bkfac_update(f, to_dev(synth.powerlaw_batch(d, n, 1.2, 8100, 1), bkfac.F32), 0.95)
        st = bkfac.bkfac_status()
    finally:
        bkfac.bkfac_set_sweep_cap(prev)
    assert st == bkfac.ENOCONV, bkfac.strerror(st)
    # the capped eigensolve still returned finite columns
    U, s = f.state()
    assert torch.isfinite(U).all() and torch.isfinite(s).all()
    assert bkfac.bkfac_status() == bkfac.OK  # cleared by the read
    clean_update_matches_oracle(oracle, 8101)


def test_sweep_cap_rejects_negative():
    with pytest.raises(bkfac.BkfacError) as e:
        bkfac.bkfac_set_sweep_cap(-3)
    assert e.value.code == bkfac.EINVAL


def test_bounded_wait_times_out_then_recovers(oracle):
    # 2^20 cycles: about half a millisecond at the GB300's clock
    bkfac.bkfac_selftest_wait_timeout(1 << 20)
    st = bkfac.bkfac_status()
    assert st == bkfac.ETIMEOUT, bkfac.strerror(st)
    assert bkfac.bkfac_status() == bkfac.OK
    clean_update_matches_oracle(oracle, 8102)
    with pytest.raises(bkfac.BkfacError) as e:
        bkfac.bkfac_selftest_wait_timeout(0)
    assert e.value.code == bkfac.EINVAL


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_indefinite_dense_factor_reports_echol_then_recovers(oracle, dtype):
    d, r, n = 200, 24, 8
    f = bkfac.Factor(d, r, dtype)
    M = bkfac.dense_factor(d, dtype)
    for t in range(4):
        X = to_dev(synth.powerlaw_batch(d, n, 1.1, 8110, t), dtype)
        if t == 0:
            bkfac.bkfac_init(f, X)
        else:
            bkfac.bkfac_update(f, X, 0.95)
        bkfac.bkfac_ea_update(M, X, 0.95, dtype, first=(t == 0))
    assert bkfac.bkfac_status() == bkfac.OK
    idx = [0, 5, 11, 3]
    bad = bkfac.dense_factor(d, dtype)
    bad[:, :d].copy_(-torch.eye(d, dtype=bad.dtype, device=bad.device))
    bkfac.bkfac_correct(f, bad, idx)
    st = bkfac.bkfac_status()
    assert st == bkfac.ECHOL, bkfac.strerror(st)
    assert bkfac.bkfac_status() == bkfac.OK
    # a p.s.d. dense factor on a fresh copy of the state: no error, the oracle's result
    g = bkfac.Factor(d, r, dtype)
    for t in range(4):
        X = to_dev(synth.powerlaw_batch(d, n, 1.1, 8110, t), dtype)
        if t == 0:
            bkfac.bkfac_init(g, X)
        else:
            bkfac.bkfac_update(g, X, 0.95)
    U, s = g.state()
    Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
    bkfac.bkfac_correct(g, M, idx)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    Uo, so = oracle.correct(Ug, sg, M.double().cpu().numpy().T.copy()[:, :d], idx)
    U2, s2 = g.state()
    tol = 1e-10 if dtype == bkfac.F64 else 1e-4
    assert lowrank_rel_err(U2.double().cpu().numpy(), s2.cpu().numpy(), Uo, so) < tol
