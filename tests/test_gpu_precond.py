"""GPU parity of the Brand update when the eigensolve runs on the Cholesky factor
of the core matrix (FP32 eigensolves of cores with at least 128 columns).

The core matrix K = L L^T is factored in FP32 as K = G G^T on a 16-CTA cluster
(32 x 32 blocks, a ragged last block when N is not a multiple of 32) and the
one-sided Jacobi orthogonalises the columns of G instead of those of L: same
left singular vectors and singular values, fewer sweeps.  The oracle computes
the same update with a dense FP64 eigendecomposition of K, so these tests pin
the preconditioned path to the definition (tolerances as for the other FP32 and
mixed-precision update tests), including rank-deficient cores whose pivots are
dropped.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import NEAR_TIE, lowrank_rel_err, orth_err, rel, truncation_gap
from tests.test_gpu_update import check_status, gpu_state, one_step_parity, rounded, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def orth_bound(N, steps):
    """Orthonormality of U after init + `steps` updates with no re-orthonormalisation in
    between: each step adds at most the eigensolve's stopping tolerance on the pair
    cosines, max(4 sqrt(N), 32) u (u = 2^-24), and about as much again for the rounding
    of U' = [U Q] V and of CholeskyQR2."""
    return (steps + 1) * 2.0 * max(4.0 * np.sqrt(N), 32.0) * 2.0 ** -24


def sweeps_of(f, n):
    off = bkfac.bkfac_debug_offsets(f, n)[7]
    return int(f.ws(n)[off:off + 4].view(torch.int32).item())


@pytest.mark.parametrize("d,r,n", [(700, 100, 73), (900, 128, 31), (1100, 200, 129)])
def test_preconditioned_update_f32(oracle, d, r, n):
    """N = 173, 159, 329: several 32-column blocks and a ragged tail on the 4 x 4 CTA grid."""
    _, worst = one_step_parity(oracle, d, r, n, bkfac.F32, alpha=1.2, steps=3, orth=orth_bound(r + n, 3))
    print(f"N = {r + n}: worst relative error {worst:.3e}")


def test_preconditioned_update_mixed(oracle):
    _, worst = one_step_parity(oracle, 1200, 160, 96, bkfac.MIXED_BF16, alpha=1.2, steps=3)
    print(f"mixed N = 256: worst relative error {worst:.3e}")


def test_preconditioned_wide_core_fewer_sweeps(oracle):
    """The wide-layer core (r = n = 256, N = 512): parity, and the eigensolve on G
    converges in fewer sweeps than the 11-12 that L takes on these spectra."""
    f, worst = one_step_parity(oracle, 2049, 256, 256, bkfac.F32, alpha=1.2, steps=3, orth=orth_bound(512, 3))
    sw = sweeps_of(f, 256)
    print(f"N = 512: worst relative error {worst:.3e}, {sw} sweeps")
    assert 1 <= sw <= 10


def test_preconditioned_duplicate_columns(oracle):
    """Repeated batch columns: the residual's CholeskyQR drops their pivots, L has zero
    rows, K = L L^T is singular and its factorisation drops the same pivots."""
    d, r, n = 800, 120, 64
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, 2 * r, 1.2, 8, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    check_status()
    Ug, sg = gpu_state(f)
    X = synth.powerlaw_batch(d, n, 1.2, 8, 1)
    X[40:] = X[:24]
    bkfac.bkfac_update(f, to_dev(X, f), 0.95)
    check_status()
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], rounded(X, f), 0.95, r)
    U2, s2 = gpu_state(f)
    k = f.r_cur
    assert k == info["r_new"]
    assert rel(s2, so[:k]) < 1e-4
    assert lowrank_rel_err(U2, s2, Uo[:k], so[:k]) < 1e-4
    assert orth_err(U2[s2 > 0]) < orth_bound(120 + 64, 1)


def test_preconditioned_batch_in_span(oracle):
    """X = U C: the residual vanishes, K has rank r_cur; the span is kept."""
    d, r, n = 600, 100, 48
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, 2 * r, 1.3, 9, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    check_status()
    Ug, sg = gpu_state(f)
    C = np.random.default_rng(9).standard_normal((n, Ug.shape[0])) * np.sqrt(sg)[None, :]
    X = C @ Ug
    bkfac.bkfac_update(f, to_dev(X, f), 0.9)
    check_status()
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], rounded(X, f), 0.9, r)
    U2, s2 = gpu_state(f)
    k = f.r_cur
    assert rel(s2, so[:k]) < 1e-4
    assert lowrank_rel_err(U2, s2, Uo[:k], so[:k]) < 1e-4
    # the new basis stays in the old span
    assert np.abs(U2 - (U2 @ Ug.T) @ Ug).max() < 1e-4


def test_preconditioned_trajectory_stays_close(oracle):
    """Free-running trajectory (both sides from the same first batch) over 6 steps.
    Trajectory parity: the FP32 path's 1e-4 applies to the final state when no step
    met a near tie at the truncation index (relative gap below 1e3 u_32), where the
    r-th mode is not determined by FP32 rounding and the trajectories may keep
    different r-th modes; the oracle keeps every mode of each step to see the gap."""
    d, r, n = 1024, 128, 64
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, 2 * r, 1.2, 12, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    check_status()
    Uo, so, info = oracle.init(rounded(X0, f), 2 * r)
    min_gap = truncation_gap(so[: info["r_new"]], r)
    Uo, so = Uo[:r], so[:r]
    for t in range(1, 7):
        X = synth.powerlaw_batch(d, n, 1.2, 12, t)
        bkfac.bkfac_update(f, to_dev(X, f), 0.95)
        check_status()
        Uo, so, info = oracle.update(Uo, so, Uo.shape[0], rounded(X, f), 0.95, r + n)
        min_gap = min(min_gap, truncation_gap(so[: info["r_new"]], r))
        Uo, so = Uo[:r], so[:r]
    U2, s2 = gpu_state(f)
    es, er = rel(s2, so), lowrank_rel_err(U2, s2, Uo, so)
    print(f"FP32 trajectory after 6 steps: sigma {es:.2e} reconstruction {er:.2e} (min truncation gap {min_gap:.2e})")
    assert min_gap > NEAR_TIE[bkfac.F32]
    assert es < 1e-4 and er < 1e-4


@pytest.mark.parametrize("eps", [1e-5, 5e-4, 8e-4, 1.1e-3, 1.4e-3, 1.8e-3, 2.5e-3, 3e-3])
def test_fp32_choleskyqr_nearly_dependent_columns(oracle, eps):
    """Batch columns that repeat others up to a relative perturbation eps: the residual
    is ill-conditioned (kappa ~ 1/eps).  The FP32 and mixed paths factor its FP64 Gram
    in FP32 and drop pivot j when its Schur complement is within 4 sqrt(n) u_32 of its
    diagonal, i.e. for a direction independent of the others by less than
    sqrt(4 sqrt(64) u_32) ~ 1.4e-3 of its residual norm here: at eps = 1e-5 the repeated
    directions are dropped (their energy, ~eps^2 of a column's, is far below the
    tolerance); at eps = 3e-3 they are kept and the second CholeskyQR pass restores
    orthonormality; the values in between straddle the point where the kept-or-dropped
    decision flips, where parity must hold either way."""
    d, r, n = 900, 96, 64
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, 2 * r, 1.2, 21, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    check_status()
    Ug, sg = gpu_state(f)
    X = synth.powerlaw_batch(d, n, 1.2, 21, 1)
    rng = np.random.default_rng(21)
    for j in range(40, n):
        src = X[j - 40]
        X[j] = src + eps * np.linalg.norm(src) * rng.standard_normal(d) / np.sqrt(d)
    bkfac.bkfac_update(f, to_dev(X, f), 0.95)
    check_status()
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], rounded(X, f), 0.95, r)
    U2, s2 = gpu_state(f)
    k = f.r_cur
    assert rel(s2, so[:k]) < 1e-4
    assert lowrank_rel_err(U2, s2, Uo[:k], so[:k]) < 1e-4
    assert orth_err(U2[s2 > 0]) < orth_bound(r + n, 1)
