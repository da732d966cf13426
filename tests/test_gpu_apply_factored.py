"""GPU parity of the linear inverse application on the thin gradient factors
(Algorithm 8) through the C ABI, against the FP64 CPU oracle."""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import rel
from tests.test_gpu_apply import TOL, make_factor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def run_factored(oracle, dA, rA, kA, dG, rG, kG, n, dtype, lamA=0.1, lamG=0.05, flags=0, inplace=False,
                 form_step=True, seed=11, alpha=None):
    fA, UA, sA = make_factor(dA, rA, kA, dtype, seed)
    fG, UG, sG = make_factor(dG, rG, kG, dtype, seed + 1)
    alpha = 1.0 / n if alpha is None else alpha
    tdt = fA.torch_dtype
    XA = bkfac.cols_tensor(n, dA, tdt)
    XA.copy_(torch.from_numpy(synth.powerlaw_batch(dA, n, 1.2, seed + 2, 0)))
    XG = bkfac.cols_tensor(n, dG, tdt)
    XG.copy_(torch.from_numpy(synth.powerlaw_batch(dG, n, 1.2, seed + 3, 0)))
    XAr, XGr = XA.double().cpu().numpy(), XG.double().cpu().numpy()
    PA = XA if inplace else bkfac.cols_tensor(n, dA, tdt)
    PG = XG if inplace else bkfac.cols_tensor(n, dG, tdt)
    S = bkfac.grad_tensor(dG, dA, tdt) if form_step else None
    bkfac.bkfac_apply_factored(fA, fG, lamA, lamG, XA, XG, PA, PG, alpha=alpha, S=S, flags=flags)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    PAo, PGo, So = oracle.apply_factored(UA, sA, lamA, UG, sG, lamG, XAr, XGr, alpha=alpha, form_step=form_step,
                                         continuation=bool(flags & bkfac.SPECTRUM_CONTINUATION),
                                         relative=bool(flags & bkfac.DAMPING_RELATIVE))
    errs = [rel(PA.double().cpu().numpy(), PAo), rel(PG.double().cpu().numpy(), PGo)]
    if form_step:
        errs.append(rel(S.double().cpu().numpy(), So))
    assert max(errs) < TOL[dtype], errs
    return errs


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32, bkfac.MIXED_BF16])
def test_factored_ragged_shapes(oracle, dtype):
    errs = run_factored(oracle, 301, 24, 24, 130, 16, 16, 37, dtype)
    print(f"factored apply dtype {dtype}: PA {errs[0]:.2e} PG {errs[1]:.2e} S {errs[2]:.2e}")


def test_factored_in_place_without_step(oracle):
    run_factored(oracle, 200, 12, 12, 90, 8, 8, 20, bkfac.F32, inplace=True, form_step=False)


def test_factored_spectrum_continuation(oracle):
    run_factored(oracle, 150, 10, 10, 80, 6, 6, 9, bkfac.F64, flags=bkfac.SPECTRUM_CONTINUATION)


def test_factored_relative_damping(oracle):
    run_factored(oracle, 150, 10, 10, 80, 6, 6, 9, bkfac.F32, lamA=0.1, lamG=0.02,
                 flags=bkfac.DAMPING_RELATIVE | bkfac.SPECTRUM_CONTINUATION)


@pytest.mark.parametrize("kA,kG", [(0, 5), (7, 0), (3, 5)])
def test_factored_partial_ranks(oracle, kA, kG):
    run_factored(oracle, 100, 9, kA, 60, 7, kG, 13, bkfac.F64)


def test_factored_complete_basis(oracle):
    """A 10-wide output layer whose Gamma basis is complete (r_cur = d = 10)."""
    run_factored(oracle, 129, 16, 16, 10, 10, 10, 24, bkfac.F32, lamA=1e-2, lamG=1e-2)


def test_factored_single_column(oracle):
    run_factored(oracle, 64, 8, 8, 40, 4, 4, 1, bkfac.F64, alpha=1.0)


def test_factored_wide_layer_full_size(oracle):
    """One wide FC layer: A_f 4097 x 256, G_f 4096 x 256, r = 256, lambda = 1e-2, S formed."""
    errs = run_factored(oracle, 4097, 256, 256, 4096, 256, 256, 256, bkfac.F32, lamA=1e-2, lamG=1e-2)
    print(f"wide-layer factored apply: PA {errs[0]:.2e} PG {errs[1]:.2e} S {errs[2]:.2e}")


def test_factored_equals_dense_apply_on_formed_gradient():
    """Algorithm 8 and Algorithm 1 on the GPU agree on G = alpha G_f A_f^T (FP64)."""
    dA, dG, n = 257, 129, 31
    fA, _, _ = make_factor(dA, 20, 20, bkfac.F64, 21)
    fG, _, _ = make_factor(dG, 12, 12, bkfac.F64, 22)
    XA = bkfac.cols_tensor(n, dA, torch.float64)
    XA.copy_(torch.from_numpy(synth.powerlaw_batch(dA, n, 1.2, 23, 0)))
    XG = bkfac.cols_tensor(n, dG, torch.float64)
    XG.copy_(torch.from_numpy(synth.powerlaw_batch(dG, n, 1.2, 24, 0)))
    PA = bkfac.cols_tensor(n, dA, torch.float64)
    PG = bkfac.cols_tensor(n, dG, torch.float64)
    S1 = bkfac.grad_tensor(dG, dA, torch.float64)
    bkfac.bkfac_apply_factored(fA, fG, 0.1, 0.2, XA, XG, PA, PG, alpha=1.0 / n, S=S1)
    G = bkfac.grad_tensor(dG, dA, torch.float64)
    G.copy_(XG.t() @ XA / n)
    S2 = bkfac.grad_tensor(dG, dA, torch.float64)
    bkfac.bkfac_apply(fA, fG, 0.1, 0.2, G, S2)
    assert bkfac.bkfac_status() == bkfac.OK
    assert rel(S1.cpu().numpy(), S2.cpu().numpy()) < 1e-12
