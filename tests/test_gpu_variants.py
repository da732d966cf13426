"""GPU parity of the B-R-KFAC / B-KFAC-C pieces through the C ABI, against the
FP64 CPU oracle: the dense EA factor (Eq. (5)), the light correction
(Algorithm 6) and the RSVD overwrite (Algorithm 5)."""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import lowrank_rel_err, orth_err, rel

pytestmark = pytest.mark.gpu

TOL = {bkfac.F64: 1e-10, bkfac.F32: 1e-4, bkfac.MIXED_BF16: 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def check_status():
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)


def to_dev(Xt, dtype):
    t = bkfac.cols_tensor(Xt.shape[0], Xt.shape[1], bkfac._TORCH_DTYPE[dtype])
    t.copy_(torch.from_numpy(Xt))
    return t


def dense_np(M):
    return M.double().cpu().numpy().T.copy()  # (d, ld) rows = columns of the column-major M


def build(d, r, n, dtype, seed, steps, rho=0.95, alpha=1.1):
    """A factor after `steps` updates and the dense EA factor of the same batches."""
    f = bkfac.Factor(d, r, dtype)
    M = bkfac.dense_factor(d, dtype)
    for t in range(steps + 1):
        X = to_dev(synth.powerlaw_batch(d, n, alpha, seed, t), dtype)
        if t == 0:
            bkfac.bkfac_init(f, X)
        else:
            bkfac.bkfac_update(f, X, rho)
        bkfac.bkfac_ea_update(M, X, rho, dtype, first=(t == 0))
    check_status()
    return f, M


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32, bkfac.MIXED_BF16])
def test_ea_update(oracle, dtype):
    d, n, rho = 300, 16, 0.9
    M = bkfac.dense_factor(d, dtype)
    Mo = None
    for t in range(4):
        X = to_dev(synth.powerlaw_batch(d, n, 1.2, 7200, t), dtype)
        bkfac.bkfac_ea_update(M, X, rho, dtype, first=(t == 0))
        Mo = oracle.ea_update(Mo, X.double().cpu().numpy(), rho, first=(t == 0))
    check_status()
    err = rel(dense_np(M)[:, :d], Mo)
    print(f"EA factor dtype {dtype}: {err:.2e}")
    assert err < TOL[dtype]


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_correct(oracle, dtype):
    d, r, n = 200, 24, 8
    f, M = build(d, r, n, dtype, 7210, steps=6)
    U, s = f.state()
    Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
    Mn = dense_np(M)[:, :d]
    idx = [3, 17, 0, 9, 21, 12, 6]
    bkfac.bkfac_correct(f, M, idx)
    check_status()
    Uo, so = oracle.correct(Ug, sg, Mn, idx)
    U2, s2 = f.state()
    Uc, sc = U2.double().cpu().numpy(), s2.cpu().numpy()
    err = lowrank_rel_err(Uc, sc, Uo, so)
    print(f"correction dtype {dtype}: {err:.2e}, orth {orth_err(Uc):.1e}")
    assert err < TOL[dtype]
    assert np.all(np.diff(sc) <= 0)
    assert np.abs(sc - so).max() <= TOL[dtype] * so.max()


def test_correct_rejects_bad_indices():
    f, M = build(64, 8, 4, bkfac.F64, 7211, steps=2)
    for idx in ([1, 1], [0, 8], [-1]):
        with pytest.raises(bkfac.BkfacError):
            bkfac.bkfac_correct(f, M, idx)


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_rsvd(oracle, dtype):
    d, r, n, l, q = 300, 20, 16, 28, 2
    f, M = build(d, r, n, dtype, 7220, steps=8)
    Om = np.random.default_rng(7221).standard_normal((l, d))
    bkfac.bkfac_rsvd(f, M, to_dev(Om, dtype), q)
    check_status()
    Mn = dense_np(M)[:, :d]
    Uo, so = oracle.rsvd(Mn, torch.from_numpy(Om).to(f.torch_dtype).double().numpy(), r, q)
    U, s = f.state()
    assert f.r_cur == r
    err = lowrank_rel_err(U.double().cpu().numpy(), s.cpu().numpy(), Uo, so)
    print(f"RSVD dtype {dtype}: {err:.2e}")
    assert err < TOL[dtype]


def test_wide_layer_correct_and_rsvd(oracle):
    """The wide layer's A factor (d = 4097, r = 256, n = 256, FP32): a correction of
    128 modes (phi_crc = 0.5) and an RSVD overwrite with 10 extra test columns and 4
    power iterations (the paper's settings), against the oracle."""
    d, r, n = 4097, 256, 256
    f, M = build(d, r, n, bkfac.F32, 7230, steps=2, alpha=1.2)
    Mn = dense_np(M)[:, :d]
    U, s = f.state()
    Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
    idx = list(np.random.default_rng(7231).choice(r, 128, replace=False))
    bkfac.bkfac_correct(f, M, idx)
    check_status()
    Uo, so = oracle.correct(Ug, sg, Mn, idx)
    U2, s2 = f.state()
    err = lowrank_rel_err(U2.double().cpu().numpy(), s2.cpu().numpy(), Uo, so)
    print(f"wide-layer correction (128 modes): {err:.2e}")
    assert err < 1e-4
    Om = np.random.default_rng(7232).standard_normal((r + 10, d))
    bkfac.bkfac_rsvd(f, M, to_dev(Om, bkfac.F32), 4)
    check_status()
    Uo, so = oracle.rsvd(Mn, torch.from_numpy(Om).float().double().numpy(), r, 4)
    U3, s3 = f.state()
    err = lowrank_rel_err(U3.double().cpu().numpy(), s3.cpu().numpy(), Uo, so)
    print(f"wide-layer RSVD overwrite (r = 256, l = 266, q = 4): {err:.2e}")
    assert err < 1e-4
