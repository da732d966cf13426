"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: closed forms
derived by hand, the secular equation of a rank-one update, numpy/LAPACK
``eigh``/``solve`` on small dense matrices, algebraic identities (QR, the core
identity of Eq. (7)), and the propositions of the paper (3.1, 3.2, 4.1, 4.2).
The paper prints no worked numeric example.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2210_08494_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def dense(Ut, sigma):
    """U diag(sigma) U^T from the (k, d) row-per-column layout."""
    Ut = np.asarray(Ut)
    return (Ut.T * np.asarray(sigma)[None, :]) @ Ut


def sym_eig_desc(K):
    w, v = np.linalg.eigh(K)
    return w[::-1], v[:, ::-1]


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_state(d, k, seed, spread=3.0):
    Ut = synth.orthonormal_columns(d, k, seed)
    sigma = np.sort(np.exp(-spread * np.linspace(0, 1, k)) * 2.0)[::-1].copy()
    return Ut, sigma


# --------------------------------------------------------------------------- closed forms


def test_closed_form_rank_one_golden(oracle):
    g = json.load(open(os.path.join(HERE, "golden", "closed_form_rank1.json")))
    Ut = np.array(g["U_cols"])
    Xt = np.array(g["X_cols"])
    Uo, so, info = oracle.update(Ut, np.array(g["sigma"]), g["k"], Xt, g["rho"], g["r"])
    exp = [eval(e, {"sqrt": math.sqrt}) for e in g["sigma_expected_exprs"]]
    assert np.allclose(exp, g["sigma_expected"], rtol=0, atol=1e-15)
    assert np.allclose(so, exp, rtol=1e-14, atol=1e-15)
    for j, lam in enumerate(exp):
        v = np.array([1.0 / 3.0, lam - 7.0 / 3.0, 0.0])
        v /= np.linalg.norm(v)
        assert abs(abs(Uo[j] @ v) - 1.0) < 1e-13


def secular(lam, a, z, c):
    return 1.0 + c * np.sum(z * z / (a - lam))


def test_rank_one_secular_equation(oracle):
    """A rank-one update of a diagonal: every new eigenvalue solves the secular
    equation 1 + c sum z_i^2 / (a_i - lam) = 0 (Golub 1973); brute-force roots
    by bisection in each interlacing interval, no LAPACK involved."""
    d, k = 40, 6
    rho = 0.9
    a_full = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    Ut = np.eye(d)[:k]  # U = [e_1 .. e_k]
    z = np.zeros(d)
    z[:k] = [0.3, -0.7, 0.2, 0.5, -0.1, 0.4]
    z[k] = 0.6  # a component outside span(U)
    Xt = z[None, :].copy()
    Uo, so, info = oracle.update(Ut, a_full, k, Xt, rho, k + 1)
    c = 1.0 - rho
    a = np.concatenate([rho * a_full, [0.0]])
    zz = z[: k + 1]
    # interlacing: roots in (a_(i+1), a_i) and (a_0, a_0 + c|z|^2)
    order = np.argsort(-a)
    a_s, z_s = a[order], zz[order]
    bounds = [a_s[0] + c * zz @ zz] + list(a_s)
    roots = []
    for i in range(k + 1):
        lo, hi = bounds[i + 1], bounds[i]
        flo, fhi = lo + 1e-15 * max(1, abs(lo)), hi - 1e-15 * max(1, abs(hi))
        for _ in range(200):
            mid = 0.5 * (flo + fhi)
            if secular(mid, a_s, z_s, c) > 0:
                fhi = mid  # f increases through the pole structure; f>0 right of the root
            else:
                flo = mid
        roots.append(0.5 * (flo + fhi))
    assert np.allclose(so, roots, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------- Jacobi


@pytest.mark.parametrize("N", [1, 2, 5, 17, 48])
def test_jacobi_vs_lapack(oracle, N):
    rng = np.random.default_rng(N)
    B = rng.standard_normal((N, N))
    A = B + B.T
    lam, V, sweeps = oracle.jacobi_eig(A)
    w, _ = sym_eig_desc(A)
    assert np.allclose(lam, w, rtol=0, atol=1e-13 * np.abs(w).max())
    assert np.linalg.norm(A @ V - V * lam[None, :]) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(V.T @ V - np.eye(N)) <= 1e-13 * max(N, 1)
    assert np.all(np.diff(lam) <= 0)


def test_jacobi_known_spectrum_with_repeats(oracle):
    N = 30
    Q = synth.orthogonal_basis(N, 7)
    lam_true = np.array([4.0] * 3 + [2.0] * 5 + list(np.linspace(1.5, 0.01, 17)) + [0.0] * 5)
    A = (Q * lam_true[None, :]) @ Q.T
    lam, V, _ = oracle.jacobi_eig(A)
    assert np.allclose(lam, np.sort(lam_true)[::-1], atol=1e-13)
    assert np.linalg.norm(A @ V - V * lam[None, :]) <= 1e-13 * np.linalg.norm(A)


# --------------------------------------------------------------------------- QR with pivoting


def test_qrcp_identities(oracle):
    d, n = 60, 12
    Pt = synth.gaussian_columns(d, n, 3)
    Qt, R, m = oracle.qrcp(Pt, 1e-12)
    assert m == n
    assert np.linalg.norm(Qt @ Qt.T - np.eye(n)) < 1e-13
    assert rel(R.T @ Qt, Pt) < 1e-14  # P = Q R
    assert rel(R.T @ R, Pt @ Pt.T) < 1e-13  # Gram invariant
    # R is a column permutation of an upper-triangular matrix with diag >= 0
    nz = [int(np.nonzero(np.abs(R[:, j]) > 0)[0].max()) for j in range(n)]
    assert sorted(nz) == list(range(n))
    assert np.all([R[nz[j], j] > 0 for j in range(n)])


def test_qrcp_rank_deficient(oracle):
    d, n = 50, 8
    base = synth.gaussian_columns(d, 5, 4)
    Pt = np.concatenate([base, base[:2] * 2.0 - base[3:4], base[4:5] * 0.5], axis=0)
    Qt, R, m = oracle.qrcp(Pt, 1e-10)
    assert m == 5
    assert np.all(Qt[m:] == 0) and np.all(R[m:] == 0)
    assert np.linalg.norm(Qt[:m] @ Qt[:m].T - np.eye(m)) < 1e-13
    assert rel(R.T @ Qt, Pt) < 1e-13


# --------------------------------------------------------------------------- Brand steps


def brand_inputs(d=64, k=10, n=6, seed=11):
    Ut, sigma = random_state(d, k, seed)
    Xt = synth.powerlaw_batch(d, n, 1.5, seed, 1)
    return Ut, sigma, Xt


def test_project_invariants(oracle):
    Ut, sigma, Xt = brand_inputs()
    M, Pt = oracle.project(Ut, Xt)
    assert np.abs(Ut @ Pt.T).max() < 1e-14 * np.abs(Xt).max() * 10  # U^T P = 0
    assert rel(M.T @ Ut + Pt, Xt) < 1e-15  # X = U M + P


def test_core_identity_eq7(oracle):
    """[U Q] M_S [U Q]^T reproduces rho U S U^T + c X X^T (Eq. (7) with the
    substitutions of Sec. 3.1), and eig(M_S) are the nonzero eigenvalues of it."""
    rho = 0.95
    Ut, sigma, Xt = brand_inputs()
    n = Xt.shape[0]
    c = (1 - rho) / n
    M, Pt = oracle.project(Ut, Xt)
    Qt, R, m = oracle.qrcp(Pt, 1e-12)
    MS = oracle.core(sigma, rho, c, M, R)
    B = np.concatenate([Ut, Qt], axis=0).T  # d x (k+n)
    K = rho * dense(Ut, sigma) + c * Xt.T @ Xt
    assert rel(B @ MS @ B.T, K) < 1e-14
    assert np.allclose(MS, MS.T, atol=0)
    w = np.linalg.eigvalsh(MS)[::-1]
    wk = sym_eig_desc(K)[0][: len(w)]
    assert np.allclose(w, wk, atol=1e-14 * wk[0])


# --------------------------------------------------------------------------- full update


@pytest.mark.parametrize("d,k,n,r", [(64, 10, 6, 16), (64, 10, 6, 20), (33, 5, 4, 9)])
def test_update_exact_without_truncation(oracle, d, k, n, r):
    """Brand's update is exact (Sec. 2.3): with r >= k + n nothing is truncated,
    U' S' U'^T equals rho U S U^T + c X X^T and S' its eigenvalues."""
    rho = 0.95
    Ut, sigma = random_state(d, k, d + k)
    Xt = synth.powerlaw_batch(d, n, 1.5, d + n, 2)
    Uo, so, info = oracle.update(Ut, sigma, k, Xt, rho, r)
    K = rho * dense(Ut, sigma) + (1 - rho) / n * Xt.T @ Xt
    assert info["r_new"] == min(r, k + n)
    rn = info["r_new"]
    assert rel(dense(Uo[:rn], so[:rn]), K) < 1e-13
    w = sym_eig_desc(K)[0]
    assert np.allclose(so[:rn], w[:rn], atol=1e-13 * w[0])
    assert np.linalg.norm(Uo[:rn] @ Uo[:rn].T - np.eye(rn)) < 1e-13
    assert np.all(Uo[rn:] == 0) and np.all(so[rn:] == 0)


def test_update_truncation_error_is_discarded_spectrum(oracle):
    """Truncation to rank r (Sec. 3.1): the error K - U'S'U'^T is p.s.d. with
    exactly the discarded eigenvalues, so ||.||_F^2 = sum of their squares and
    ||.||_2 = lambda_(r+1)."""
    d, k, n, r, rho = 80, 12, 8, 12, 0.9
    Ut, sigma = random_state(d, k, 5)
    Xt = synth.powerlaw_batch(d, n, 1.2, 6, 0)
    Uo, so, info = oracle.update(Ut, sigma, k, Xt, rho, r)
    K = rho * dense(Ut, sigma) + (1 - rho) / n * Xt.T @ Xt
    E = K - dense(Uo, so)
    w = sym_eig_desc(K)[0]
    assert np.allclose(so, w[:r], atol=1e-13 * w[0])
    assert abs(np.linalg.norm(E) ** 2 - np.sum(w[r:] ** 2)) < 1e-12 * w[0] ** 2
    ew = np.linalg.eigvalsh(E)
    assert ew.min() > -1e-13 * w[0]
    assert abs(ew.max() - w[r]) < 1e-13 * w[0]


def test_rho_zero_is_top_r_evd(oracle):
    d, k, n, r = 50, 5, 9, 6
    Ut, sigma = random_state(d, k, 9)
    Xt = synth.powerlaw_batch(d, n, 1.5, 10, 0)
    Uo, so, _ = oracle.update(Ut, sigma, k, Xt, 0.0, r)
    w, v = sym_eig_desc(Xt.T @ Xt / n)
    assert np.allclose(so, w[:r], atol=1e-13 * w[0])
    P_o = Uo.T @ Uo
    P_ref = v[:, :r] @ v[:, :r].T
    assert np.linalg.norm(P_o - P_ref) < 1e-10  # eigen-gaps are O(1e-2) here


def test_init_is_exact_evd_and_keeps_rank_n(oracle):
    """kappa(0) = 1 in Eq. (5): the first state is the EVD of X X^T / n; with
    n < r the rank stays n (reading: no arbitrary null vectors)."""
    d, n, r = 40, 5, 8
    Xt = synth.powerlaw_batch(d, n, 1.5, 12, 0)
    Uo, so, info = oracle.init(Xt, r)
    assert info["r_new"] == n
    w = sym_eig_desc(Xt.T @ Xt / n)[0]
    assert np.allclose(so[:n], w[:n], atol=1e-13 * w[0])
    assert rel(dense(Uo[:n], so[:n]), Xt.T @ Xt / n) < 1e-13


def test_update_in_span_keeps_span(oracle):
    """X = U C: the residual P vanishes, the QR has rank 0 and the update is a
    rotation inside span(U) (Sec. 2.3, Q_A R_A = (I - U U^T) A = 0)."""
    d, k, n, rho = 60, 8, 5, 0.95
    Ut, sigma = random_state(d, k, 13)
    C = np.random.default_rng(1).standard_normal((n, k))
    Xt = C @ Ut
    Uo, so, info = oracle.update(Ut, sigma, k, Xt, rho, k)
    assert info["rank_p"] == 0
    proj_out = Uo - (Uo @ Ut.T) @ Ut
    assert np.abs(proj_out).max() < 1e-13
    K = rho * dense(Ut, sigma) + (1 - rho) / n * Xt.T @ Xt
    assert rel(dense(Uo, so), K) < 1e-13


def test_dense_update_vs_lapack(oracle):
    d, k, n, r, rho = 10, 10, 32, 10, 0.95
    Xt0 = synth.powerlaw_batch(d, n, 1.2, 14, 0)
    U0, s0, info0 = oracle.init(Xt0, r, dense=True)
    assert info0["r_new"] == r
    assert rel(dense(U0, s0), Xt0.T @ Xt0 / n) < 1e-13
    Xt = synth.powerlaw_batch(d, n, 1.2, 14, 1)
    Uo, so, info = oracle.update_dense(U0, s0, k, Xt, rho, r)
    K = rho * dense(U0, s0) + (1 - rho) / n * Xt.T @ Xt
    assert rel(dense(Uo, so), K) < 1e-13
    assert np.allclose(so, sym_eig_desc(K)[0], atol=1e-14 * so[0])


def test_dense_matches_brand_when_both_apply(oracle):
    d, k, n, r, rho = 30, 6, 5, 8, 0.9
    Ut, sigma = random_state(d, k, 15)
    Xt = synth.powerlaw_batch(d, n, 1.5, 16, 0)
    Ub, sb, _ = oracle.update(Ut, sigma, k, Xt, rho, r)
    Ud, sd, _ = oracle.update_dense(Ut, sigma, k, Xt, rho, r)
    assert np.allclose(sb, sd, atol=1e-14 * sb[0])
    assert rel(dense(Ub, sb), dense(Ud, sd)) < 1e-12


# --------------------------------------------------------------------------- trajectory (Props 3.1-4.2)


def test_trajectory_propositions(oracle):
    """Along a B-KFAC trajectory with the dense EA factor M_k of Eq. (8):
    * Props. 3.2 / 4.1: M_k - B_k and M_k - M~_B,k are p.s.d. (B-KFAC only under-estimates);
    * Prop. 3.1: ||M_k - B_k|| >= ||M_k - top_r(M_k)|| and
      ||M_k - M~_B,k|| >= ||M_k - top_(r+n)(M_k)|| (Frobenius and spectral);
    * Prop. 4.1: M_k - B_k = sum_i rho^(k-i) (M~_B,i - B_i) (EA of truncation errors);
    * Prop. 4.2: ||M~_B,i - B_i||_F <= (1 - rho) ||X_i X_i^T / n||_F.
    """
    d, n, r, rho, steps = 48, 4, 6, 0.9, 25
    Xs = [synth.powerlaw_batch(d, n, 1.5, 17, t) for t in range(steps)]
    Mk = Xs[0].T @ Xs[0] / n
    U, s, info = oracle.init(Xs[0], r)
    k = info["r_new"]
    trunc_errs = [Mk - dense(U[:k], s[:k])]  # i = 0: M~_B,0 = M_0
    for t in range(1, steps):
        X = Xs[t]
        inc = X.T @ X / n
        Mk = rho * Mk + (1 - rho) * inc
        B_prev = dense(U[:k], s[:k])
        Mtil = rho * B_prev + (1 - rho) * inc
        U, s, info = oracle.update(U, s, k, X, rho, r)
        k = info["r_new"]
        Bk = dense(U[:k], s[:k])
        scale = np.linalg.norm(Mk)
        assert np.linalg.eigvalsh(Mk - Bk).min() > -1e-12 * scale
        assert np.linalg.eigvalsh(Mk - Mtil).min() > -1e-12 * scale
        w, v = sym_eig_desc(Mk)
        top_r = (v[:, :r] * w[:r]) @ v[:, :r].T
        top_rn = (v[:, : r + n] * w[: r + n]) @ v[:, : r + n].T
        for ordn in ("fro", 2):
            assert np.linalg.norm(Mk - Bk, ordn) >= np.linalg.norm(Mk - top_r, ordn) - 1e-12 * scale
            assert np.linalg.norm(Mk - Mtil, ordn) >= np.linalg.norm(Mk - top_rn, ordn) - 1e-12 * scale
        te = Mtil - Bk
        assert np.linalg.norm(te) <= (1 - rho) * np.linalg.norm(inc) * (1 + 1e-12)
        trunc_errs.append(te)
        ea = sum(rho ** (t - i) * trunc_errs[i] for i in range(t + 1))
        assert np.linalg.norm((Mk - Bk) - ea) < 1e-12 * scale


# --------------------------------------------------------------------------- reorth


def test_reorth_restores_orthonormality(oracle):
    d, k = 70, 9
    Ut, sigma = random_state(d, k, 18)
    noisy = Ut + 1e-3 * np.random.default_rng(2).standard_normal(Ut.shape)
    Uo, so = oracle.reorth(noisy, sigma)
    assert np.linalg.norm(Uo @ Uo.T - np.eye(k)) < 1e-13
    assert rel(dense(Uo, so), dense(noisy, sigma)) < 1e-13
    Uo2, so2 = oracle.reorth(Ut, sigma)
    assert np.allclose(so2, sigma, atol=1e-14)


# --------------------------------------------------------------------------- apply


def low_rank_factor(d, k, seed):
    Ut, sigma = random_state(d, k, seed)
    return Ut, sigma


@pytest.mark.parametrize("dA,kA,dG,kG", [(24, 5, 17, 4), (40, 0, 12, 3), (9, 9, 30, 0)])
def test_apply_vs_dense_solve(oracle, dA, kA, dG, kG):
    """S = (Gamma + lG I)^-1 G (A + lA I)^-1 with A = U_A S_A U_A^T etc.
    (K-FAC identity, Eq. (4)), checked against LAPACK solves."""
    UA, sA = low_rank_factor(dA, kA, 19) if kA else (np.zeros((0, dA)), np.zeros(0))
    UG, sG = low_rank_factor(dG, kG, 20) if kG else (np.zeros((0, dG)), np.zeros(0))
    G = synth.gradient(dG, dA, 21, 0)
    lA, lG = 0.1, 0.03
    S = oracle.apply(UA, sA, lA, UG, sG, lG, G)
    Arep = dense(UA, sA) if kA else np.zeros((dA, dA))
    Grep = dense(UG, sG) if kG else np.zeros((dG, dG))
    ref = np.linalg.solve(Grep + lG * np.eye(dG), G) @ np.linalg.inv(Arep + lA * np.eye(dA))
    assert rel(S, ref) < 1e-12


def test_apply_large_damping_limit(oracle):
    dA, dG = 20, 15
    UA, sA = low_rank_factor(dA, 4, 22)
    UG, sG = low_rank_factor(dG, 3, 23)
    G = synth.gradient(dG, dA, 24, 0)
    lam = 1e7
    S = oracle.apply(UA, sA, lam, UG, sG, lam, G)
    assert rel(S * lam * lam, G) < 1e-6


def test_apply_spectrum_continuation(oracle):
    """Sec. 3.5.1: lam <- lam + min(sigma), sigma <- sigma - min(sigma); the
    represented matrix becomes U (S - m) U^T + (lam + m) I."""
    dA, dG = 22, 14
    UA, sA = low_rank_factor(dA, 5, 25)
    UG, sG = low_rank_factor(dG, 4, 26)
    G = synth.gradient(dG, dA, 27, 0)
    lA, lG = 0.05, 0.2
    S = oracle.apply(UA, sA, lA, UG, sG, lG, G, continuation=True)
    mA, mG = sA.min(), sG.min()
    Arep = dense(UA, sA - mA) + (lA + mA) * np.eye(dA)
    Grep = dense(UG, sG - mG) + (lG + mG) * np.eye(dG)
    ref = np.linalg.solve(Grep, G) @ np.linalg.inv(Arep)
    assert rel(S, ref) < 1e-12


@pytest.mark.parametrize("dA,kA,dG,kG,n", [(24, 5, 17, 4, 6), (40, 0, 12, 3, 3), (9, 9, 30, 0, 5), (15, 4, 11, 2, 1)])
def test_apply_factored_vs_dense_solve(oracle, dA, kA, dG, kG, n):
    """Algorithm 8: PA = (A + lA I)^-1 A_f and PG = (Gamma + lG I)^-1 G_f on the thin
    factors, checked column by column against LAPACK solves with the dense
    represented factors; S = alpha PG PA^T."""
    UA, sA = low_rank_factor(dA, kA, 31) if kA else (np.zeros((0, dA)), np.zeros(0))
    UG, sG = low_rank_factor(dG, kG, 32) if kG else (np.zeros((0, dG)), np.zeros(0))
    XA = synth.powerlaw_batch(dA, n, 1.2, 33, 0)
    XG = synth.powerlaw_batch(dG, n, 1.2, 34, 0)
    lA, lG, alpha = 0.07, 0.02, 1.0 / n
    PA, PG, S = oracle.apply_factored(UA, sA, lA, UG, sG, lG, XA, XG, alpha=alpha)
    Arep = (dense(UA, sA) if kA else np.zeros((dA, dA))) + lA * np.eye(dA)
    Grep = (dense(UG, sG) if kG else np.zeros((dG, dG))) + lG * np.eye(dG)
    refA = np.linalg.solve(Arep, XA.T).T
    refG = np.linalg.solve(Grep, XG.T).T
    assert rel(PA, refA) < 1e-12 and rel(PG, refG) < 1e-12
    assert rel(S, alpha * refG.T @ refA) < 1e-12


def test_apply_factored_equals_dense_apply(oracle):
    """Algorithm 8 and Algorithm 1 are the same operator on G = alpha G_f A_f^T:
    (Gamma + lG)^-1 (G_f A_f^T) (A + lA)^-1 = [(Gamma + lG)^-1 G_f] [(A + lA)^-1 A_f]^T
    (both damped factors are symmetric), with and without spectrum continuation."""
    dA, dG, n = 33, 21, 7
    UA, sA = low_rank_factor(dA, 6, 35)
    UG, sG = low_rank_factor(dG, 5, 36)
    XA = synth.powerlaw_batch(dA, n, 1.5, 37, 0)
    XG = synth.powerlaw_batch(dG, n, 1.5, 38, 0)
    alpha = 2.0 / n
    for cont in (False, True):
        _, _, S = oracle.apply_factored(UA, sA, 0.05, UG, sG, 0.3, XA, XG, alpha=alpha, continuation=cont)
        Sd = oracle.apply(UA, sA, 0.05, UG, sG, 0.3, alpha * XG.T @ XA, continuation=cont)
        assert rel(S, Sd) < 1e-12


def test_apply_factored_without_step(oracle):
    dA, dG, n = 12, 10, 3
    UA, sA = low_rank_factor(dA, 3, 39)
    UG, sG = low_rank_factor(dG, 2, 40)
    XA = synth.powerlaw_batch(dA, n, 1.2, 41, 0)
    XG = synth.powerlaw_batch(dG, n, 1.2, 42, 0)
    PA, PG, S = oracle.apply_factored(UA, sA, 0.1, UG, sG, 0.1, XA, XG, form_step=False)
    PA2, PG2, _ = oracle.apply_factored(UA, sA, 0.1, UG, sG, 0.1, XA, XG)
    assert S is None and np.array_equal(PA, PA2) and np.array_equal(PG, PG2)


def test_apply_relative_damping(oracle):
    """Damping relative to the largest eigenvalue (the schedule of the experiments,
    lambda = lambda_max * phi): checked against LAPACK's largest eigenvalue of the
    dense represented factors and dense solves, alone and with spectrum continuation,
    for Algorithm 1 and Algorithm 8."""
    dA, dG, n = 26, 18, 4
    UA, sA = low_rank_factor(dA, 6, 43)
    UG, sG = low_rank_factor(dG, 5, 44)
    G = synth.gradient(dG, dA, 45, 0)
    XA = synth.powerlaw_batch(dA, n, 1.2, 46, 0)
    XG = synth.powerlaw_batch(dG, n, 1.2, 47, 0)
    phiA, phiG = 0.1, 0.05
    lmA = np.linalg.eigvalsh(dense(UA, sA)).max()
    lmG = np.linalg.eigvalsh(dense(UG, sG)).max()
    for cont in (False, True):
        mA, mG = (sA.min(), sG.min()) if cont else (0.0, 0.0)
        Arep = dense(UA, sA - mA) + (phiA * lmA + mA) * np.eye(dA)
        Grep = dense(UG, sG - mG) + (phiG * lmG + mG) * np.eye(dG)
        S = oracle.apply(UA, sA, phiA, UG, sG, phiG, G, continuation=cont, relative=True)
        assert rel(S, np.linalg.solve(Grep, G) @ np.linalg.inv(Arep)) < 1e-12
        PA, PG, _ = oracle.apply_factored(UA, sA, phiA, UG, sG, phiG, XA, XG, form_step=False, continuation=cont,
                                          relative=True)
        assert rel(PA, np.linalg.solve(Arep, XA.T).T) < 1e-12
        assert rel(PG, np.linalg.solve(Grep, XG.T).T) < 1e-12


# --------------------------------------------------------------------------- dense EA factor, Algorithms 5-6


def test_ea_update_is_the_weighted_sum(oracle):
    """Eq. (5): after batches X_0..X_T the EA factor is sum_j w_j X_j X_j^T / n with
    w_0 = rho^T (kappa(0) = 1) and w_j = rho^(T-j) (1 - rho); checked as Y Y^T of the
    weighted concatenation Y = [sqrt(w_j / n) X_j]."""
    d, n, rho, T = 23, 5, 0.9, 4
    M = None
    Ys = []
    for t in range(T + 1):
        X = synth.powerlaw_batch(d, n, 1.2, 51, t)
        M = oracle.ea_update(M, X, rho, first=(t == 0))
        w = rho ** T if t == 0 else rho ** (T - t) * (1 - rho)
        Ys.append(np.sqrt(w / n) * X)
    Y = np.concatenate(Ys, axis=0)
    assert rel(M, Y.T @ Y) < 1e-13


def test_ea_update_matches_untruncated_brand(oracle):
    """Without truncation the Brand representation is the EA factor itself (Sec. 2.3):
    two independent pipelines agree."""
    d, n, rho = 40, 4, 0.95
    X = synth.powerlaw_batch(d, n, 1.3, 52, 0)
    M = oracle.ea_update(None, X, rho, first=True)
    Ut, s, info = oracle.init(X, d)
    k = info["r_new"]
    for t in range(1, 5):
        X = synth.powerlaw_batch(d, n, 1.3, 52, t)
        M = oracle.ea_update(M, X, rho)
        Ut, s, info = oracle.update(Ut[:k], s[:k], k, X, rho, d)
        k = info["r_new"]
    assert rel(dense(Ut[:k], s[:k]), M) < 1e-12


def _truncated_state(oracle, d, r, n, rho, seed, steps):
    X = synth.powerlaw_batch(d, n, 1.1, seed, 0)
    M = oracle.ea_update(None, X, rho, first=True)
    Ut, s, info = oracle.init(X, r)
    k = info["r_new"]
    for t in range(1, steps + 1):
        X = synth.powerlaw_batch(d, n, 1.1, seed, t)
        M = oracle.ea_update(M, X, rho)
        Ut, s, info = oracle.update(Ut[:k], s[:k], k, X, rho, r)
        k = info["r_new"]
    return Ut[:k], s[:k], M


def test_correct_properties(oracle):
    """Algorithm 6: after the correction the representation agrees with M on the chosen
    subspace (U_s^T (M - M~) U_s = 0), the Frobenius error does not grow (the paper's
    footnote), U stays orthonormal, the corrected values are the LAPACK eigenvalues of
    U_s^T M U_s, and the modes come back sorted."""
    d, r, n, rho = 60, 12, 6, 0.9
    Ut, s, M = _truncated_state(oracle, d, r, n, rho, 53, 6)
    idx = [11, 2, 7, 5, 9, 0]
    Us = Ut[idx]
    Uc, sc = oracle.correct(Ut, s, M, idx)
    assert np.abs(Uc @ Uc.T - np.eye(len(sc))).max() < 1e-12
    E_new = M - dense(Uc, sc)
    assert np.linalg.norm(Us @ E_new @ Us.T) < 1e-12 * np.linalg.norm(M)
    assert np.linalg.norm(E_new) <= np.linalg.norm(M - dense(Ut, s)) * (1 + 1e-12)
    lam = np.linalg.eigvalsh(Us @ M @ Us.T)
    for v in lam:
        assert np.min(np.abs(sc - v)) < 1e-12 * np.abs(lam).max()
    assert np.all(np.diff(sc) <= 0)


def test_correct_is_identity_on_an_exact_representation(oracle):
    """When M is exactly U diag(sigma) U^T plus a part orthogonal to span(U), the
    correction changes nothing (up to the order and sign of eigenvectors)."""
    d, k = 30, 7
    Ut, s = random_state(d, k, 54)
    Vt = synth.orthonormal_columns(d, k + 3, 54)[k:]  # orthogonal to span(U)
    M = dense(Ut, s) + dense(Vt, np.array([0.3, 0.2, 0.1]))
    Uc, sc = oracle.correct(Ut, s, M, [1, 4, 6])
    assert rel(dense(Uc, sc), dense(Ut, s)) < 1e-12


def test_rsvd_exact_on_low_rank(oracle):
    """Algorithm 5's RSVD recovers a rank-r0 <= r factor exactly (range finder spans it)."""
    d, r0, r, l = 50, 6, 8, 12
    Ut, s = random_state(d, r0, 55)
    M = dense(Ut, s)
    Om = np.random.default_rng(56).standard_normal((l, d))
    U, sig = oracle.rsvd(M, Om, r, q=1)
    assert rel(dense(U, sig), M) < 1e-12
    assert np.abs(sig[:r0] - np.sort(s)[::-1]).max() < 1e-12 * s.max()


def test_rsvd_gapped_spectrum(oracle):
    """With a wide gap after r the RSVD's top-r subspace matches LAPACK's."""
    d, r, l = 64, 5, 10
    rng = np.random.default_rng(57)
    Q = synth.orthonormal_columns(d, d, 57)
    lam = np.concatenate([np.linspace(10, 5, r), 1e-4 * rng.random(d - r)])
    M = (Q.T * lam) @ Q
    U, sig = oracle.rsvd(M, rng.standard_normal((l, d)), r, q=3)
    w, V = np.linalg.eigh(M)
    Vt = V[:, ::-1][:, :r].T
    svals = np.linalg.svd(U @ Vt.T, compute_uv=False)
    assert 1 - svals.min() < 1e-12
    assert np.abs(sig - w[::-1][:r]).max() < 1e-10


# --------------------------------------------------------------------------- planted mistakes


def test_pins_catch_a_planted_mistake(oracle):
    """A wrong scaling of the new term (c = 1 - rho instead of (1 - rho)/n, a
    plausible mistake) must fail the exactness pin: run the oracle with n-times
    duplicated columns scaled so the *wrong* formula would be indistinguishable
    only if the pin were blind to c."""
    d, k, n, r, rho = 40, 6, 5, 11, 0.9
    Ut, sigma = random_state(d, k, 28)
    Xt = synth.powerlaw_batch(d, n, 1.5, 29, 0)
    Uo, so, _ = oracle.update(Ut, sigma, k, Xt, rho, r)
    K_right = rho * dense(Ut, sigma) + (1 - rho) / n * Xt.T @ Xt
    K_wrong = rho * dense(Ut, sigma) + (1 - rho) * Xt.T @ Xt
    assert rel(dense(Uo, so), K_right) < 1e-13
    assert rel(dense(Uo, so), K_wrong) > 1e-2


@pytest.mark.parametrize("case", ["steady", "init", "deficient"])
def test_update_eigh_equals_update(oracle, case):
    """The long-trajectory variant (LAPACK eigh for the core) is the same update:
    eigenvalues and the represented matrix agree with the Jacobi oracle to FP64
    rounding, including a rank-deficient residual and the first step."""
    d, r, n = 300, 24, 20
    rng = np.random.default_rng(31)
    X0 = synth.powerlaw_batch(d, 32, 1.3, 77, 0)
    U, s, info = oracle.init(X0, r)
    k = info["r_new"]
    X = synth.powerlaw_batch(d, n, 1.3, 77, 1)
    if case == "init":
        U, s, k = np.zeros((1, d)), np.zeros(1), 0
    if case == "deficient":
        X[10:] = X[:10]
        X[3] = (rng.standard_normal(k) * np.sqrt(np.maximum(s[:k], 0.0))) @ U[:k]  # inside span(U)
    Ua, sa, ia = oracle.update(U[:max(k, 1)], s[:max(k, 1)], k, X, 0.95, r)
    Ub, sb, ib = oracle.update_eigh(U[:max(k, 1)], s[:max(k, 1)], k, X, 0.95, r)
    assert ia["r_new"] == ib["r_new"] and ia["rank_p"] == ib["rank_p"]
    kk = ia["r_new"]
    assert np.abs(sa - sb).max() <= 1e-13 * sa[0]
    Ka = (Ua[:kk].T * sa[:kk]) @ Ua[:kk]
    Kb = (Ub[:kk].T * sb[:kk]) @ Ub[:kk]
    assert np.linalg.norm(Ka - Kb) <= 1e-12 * np.linalg.norm(Ka)
