"""GPU parity of the damped inverse application (Algorithm 1, K-FAC identity
of Eq. (4)) through the C ABI, against the FP64 CPU oracle."""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import rel

pytestmark = pytest.mark.gpu

TOL = {bkfac.F64: 1e-10, bkfac.F32: 1e-4, bkfac.MIXED_BF16: 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def make_factor(d, r, k, dtype, seed, flags=0):
    f = bkfac.Factor(d, r, dtype, flags=flags)
    if k:
        Ut = synth.orthonormal_columns(d, k, seed)
        sig = np.sort(2.0 * np.exp(-np.linspace(0, 5, k)))[::-1].copy()
        f.load_state(torch.from_numpy(Ut).to(f.torch_dtype).cuda(), torch.from_numpy(sig).cuda())
    U, s = f.state()
    return f, U.double().cpu().numpy(), s.cpu().numpy()


def run_apply(oracle, dA, rA, kA, dG, rG, kG, dtype, lamA=0.1, lamG=0.05, flags=0, inplace=False, seed=1,
              fflags=0):
    fA, UA, sA = make_factor(dA, rA, kA, dtype, seed, fflags)
    fG, UG, sG = make_factor(dG, rG, kG, dtype, seed + 1, fflags)
    Gn = synth.gradient(dG, dA, seed + 2, 0)
    G = bkfac.grad_tensor(dG, dA, fA.torch_dtype)
    G.copy_(torch.from_numpy(Gn))
    Gr = G.double().cpu().numpy()
    S = G if inplace else bkfac.grad_tensor(dG, dA, fA.torch_dtype)
    bkfac.bkfac_apply(fA, fG, lamA, lamG, G, S, flags=flags)
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    So = oracle.apply(UA, sA, lamA, UG, sG, lamG, Gr, continuation=bool(flags & bkfac.SPECTRUM_CONTINUATION),
                      relative=bool(flags & bkfac.DAMPING_RELATIVE))
    err = rel(S.double().cpu().numpy(), So)
    assert err < TOL[dtype], err
    return err


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32, bkfac.MIXED_BF16])
def test_apply_ragged_shapes(oracle, dtype):
    err = run_apply(oracle, 301, 24, 24, 130, 16, 16, dtype)
    print(f"apply dtype {dtype}: {err:.2e}")


def test_apply_small_layer_f64(oracle):
    run_apply(oracle, 512, 64, 64, 256, 64, 64, bkfac.F64, lamA=0.1, lamG=0.1)


def test_apply_spectrum_continuation(oracle):
    run_apply(oracle, 200, 12, 12, 90, 8, 8, bkfac.F64, flags=bkfac.SPECTRUM_CONTINUATION)


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_apply_relative_damping(oracle, dtype):
    """lambda = phi * largest eigenvalue (the experiments' schedule), also with continuation."""
    run_apply(oracle, 220, 14, 14, 96, 9, 9, dtype, lamA=0.1, lamG=0.05, flags=bkfac.DAMPING_RELATIVE)
    run_apply(oracle, 220, 14, 14, 96, 9, 9, dtype, lamA=0.1, lamG=0.05,
              flags=bkfac.DAMPING_RELATIVE | bkfac.SPECTRUM_CONTINUATION)


def test_apply_relative_damping_needs_modes():
    fA, _, _ = make_factor(50, 4, 0, bkfac.F64, 3)
    fG, _, _ = make_factor(30, 4, 4, bkfac.F64, 4)
    G = bkfac.grad_tensor(30, 50, torch.float64)
    with pytest.raises(bkfac.BkfacError):
        bkfac.bkfac_apply(fA, fG, 0.1, 0.1, G, G, flags=bkfac.DAMPING_RELATIVE)


def test_apply_in_place(oracle):
    run_apply(oracle, 160, 10, 10, 70, 6, 6, bkfac.F32, inplace=True)


@pytest.mark.parametrize("kA,kG", [(0, 5), (7, 0), (0, 0), (3, 5)])
def test_apply_partial_ranks(oracle, kA, kG):
    """r_cur below r (and empty factors: S = G / (lamA lamG))."""
    run_apply(oracle, 100, 9, kA, 60, 7, kG, bkfac.F64)


def test_apply_wide_layer_full_size(oracle):
    """One wide FC layer: G 4096 x 4097 FP32 with r_A = r_G = 256, lambda = 1e-2."""
    err = run_apply(oracle, 4097, 256, 256, 4096, 256, 256, bkfac.F32, lamA=1e-2, lamG=1e-2)
    print(f"wide-layer apply relative error {err:.2e}")


def test_apply_wide_layer_tf32x3(oracle):
    """The wide layer's apply with 3xTF32 tensor-core passes."""
    err = run_apply(oracle, 4097, 256, 256, 4096, 256, 256, bkfac.F32, lamA=1e-2, lamG=1e-2, fflags=bkfac.FLAG_TF32X3)
    print(f"wide-layer 3xTF32 apply relative error {err:.2e}")


@pytest.mark.parametrize("dA,kA,dG,kG", [(301, 24, 130, 16), (1000, 64, 777, 48), (129, 0, 200, 10), (257, 9, 70, 0),
                                          (96, 0, 40, 0), (600, 200, 450, 130)])
def test_apply_mixed_shapes(oracle, dA, kA, dG, kG):
    """The mixed path's apply (BF16 operands rounded once into K-major copies, products on
    the TMA-fed tensor cores): ragged tiles along every dimension, empty factors, ranks
    above one tile; relative Frobenius and element-wise against the oracle."""
    err = run_apply(oracle, dA, max(kA, 1), kA, dG, max(kG, 1), kG, bkfac.MIXED_BF16, seed=11)
    print(f"mixed apply {dG} x {dA} (kA {kA}, kG {kG}): {err:.2e}")


def test_apply_mixed_in_place(oracle):
    run_apply(oracle, 333, 20, 20, 190, 12, 12, bkfac.MIXED_BF16, inplace=True, seed=13)


def test_apply_wide_layer_mixed(oracle):
    """The wide layer (G 4096 x 4097, r = 256 on both sides) on the mixed path, element by element."""
    fA, UA, sA = make_factor(4097, 256, 256, bkfac.MIXED_BF16, 21)
    fG, UG, sG = make_factor(4096, 256, 256, bkfac.MIXED_BF16, 22)
    Gn = synth.gradient(4096, 4097, 23, 0)
    G = bkfac.grad_tensor(4096, 4097, torch.float32)
    G.copy_(torch.from_numpy(Gn))
    S = bkfac.grad_tensor(4096, 4097, torch.float32)
    bkfac.bkfac_apply(fA, fG, 1e-2, 1e-2, G, S)
    assert bkfac.bkfac_status() == bkfac.OK
    So = oracle.apply(UA, sA, 1e-2, UG, sG, 1e-2, G.double().cpu().numpy())
    Sg = S.double().cpu().numpy()
    err = rel(Sg, So)
    em = float(np.abs(Sg - So).max() / np.abs(So).max())
    print(f"wide-layer mixed apply: {err:.2e} (element-wise {em:.2e})")
    assert err < 1e-2 and em < 1e-2
