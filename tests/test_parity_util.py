"""CPU checks of the parity judge the GPU tests use (tests/parity_util.py):
it must accept the oracle's own result and reject each kind of mistake its
parts are there to catch, including ones the relative Frobenius error alone
lets through."""
import numpy as np
import pytest

from paper_2210_08494_gb300 import synth
from tests.parity_util import MODE_TOL, NEAR_TIE, gapped_prefix, judge_step, rel, truncation_gap

F64, F32, MIXED = 0, 1, 2


@pytest.fixture(scope="module")
def step(oracle):
    """An untruncated Brand step of a d = 300, r = 24 factor (FP64 oracle)."""
    d, r, n = 300, 24, 20
    X0 = synth.powerlaw_batch(d, n, 1.2, 77, 0)
    U, s, info = oracle.init(X0, r)
    k = info["r_new"]
    X = synth.powerlaw_batch(d, n, 1.2, 77, 1)
    Uo, so, info = oracle.update(U[:k], s[:k], k, X, 0.95, k + n)
    return Uo[: info["r_new"]], so[: info["r_new"]], r


def test_accepts_the_oracles_own_result(step):
    Uo, so, r = step
    for dt, tol in ((F64, 1e-10), (F32, 1e-4), (MIXED, 1e-2)):
        m = judge_step(Uo[:r], so[:r], Uo, so, r, dt, tol, orth_tol=1e-12)
        assert m["sigma"] == 0.0 and m["recon"] < 1e-13


def test_rejects_a_tail_eigenvalue_error_the_frobenius_norm_misses(step):
    Uo, so, r = step
    s = so[:r].copy()
    s[r - 1] += 2 * MODE_TOL[F32] * so[0]  # the r-th eigenvalue off by twice MODE_TOL of sigma_1
    assert rel(s, so[:r]) < 1e-4  # relative Frobenius alone would pass it
    with pytest.raises(AssertionError, match="per-mode"):
        judge_step(Uo[:r], s, Uo, so, r, F32, 1e-4)


def test_rejects_swapped_eigenvectors(step):
    Uo, so, r = step
    U = Uo[:r].copy()
    U[[0, 1]] = U[[1, 0]]  # the two leading eigenvectors exchanged, eigenvalues kept
    with pytest.raises(AssertionError, match="subspace"):
        judge_step(U, so[:r], Uo, so, r, F32, 1e-4)


def test_rejects_a_rotated_basis_vector(step):
    Uo, so, r = step
    U = Uo[:r].copy()
    c, s_ = np.cos(1e-2), np.sin(1e-2)
    U[2] = c * Uo[2] - s_ * Uo[r]  # mode 3 leaks into a truncated direction
    with pytest.raises(AssertionError):
        judge_step(U, so[:r], Uo, so, r, F32, 1e-4)


def test_near_tie_judges_the_leading_modes(step):
    Uo, so, r = step
    s = so.copy()
    s[r] = s[r - 1] * (1.0 - 0.5 * NEAR_TIE[F32])  # the (r+1)-th eigenvalue within the near-tie band
    assert truncation_gap(s, r) < NEAR_TIE[F32]
    U = Uo.copy()
    U[[r - 1, r]] = U[[r, r - 1]]  # the tied r-th mode taken from the other side of the tie
    k0 = gapped_prefix(s, r, NEAR_TIE[F32])
    assert 0 < k0 < r
    m = judge_step(U[:r], s[:r], Uo, s, r, F32, 1e-4)
    assert m["tie"]
    s2 = s.copy()
    s2[r] = s2[r - 1] * 0.9  # a clear gap: the same swap now fails
    with pytest.raises(AssertionError):
        judge_step(U[:r], s2[:r], Uo, s2, r, F32, 1e-4)
