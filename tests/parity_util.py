"""Comparison metrics shared by the GPU parity tests (numpy, float64).

Low-rank matrices are compared without forming d x d products: both live in
span([U1, U2]), so with an orthonormal basis Q of that span,
||U1 S1 U1^T - U2 S2 U2^T||_F = ||Q^T (...) Q||_F exactly (no cancellation).
"""
import numpy as np


def lowrank_rel_err(U1t, s1, U2t, s2):
    """Relative Frobenius distance of U1 diag(s1) U1^T to U2 diag(s2) U2^T (reference)."""
    U1 = np.asarray(U1t, dtype=np.float64).T
    U2 = np.asarray(U2t, dtype=np.float64).T
    s1 = np.asarray(s1, dtype=np.float64)
    s2 = np.asarray(s2, dtype=np.float64)
    Q, _ = np.linalg.qr(np.concatenate([U1, U2], axis=1))
    A = Q.T @ U1
    B = Q.T @ U2
    E = (A * s1[None, :]) @ A.T - (B * s2[None, :]) @ B.T
    R = (B * s2[None, :]) @ B.T
    nr = np.linalg.norm(R)
    return float(np.linalg.norm(E) / (nr if nr > 0 else 1.0))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def orth_err(Ut):
    U = np.asarray(Ut, dtype=np.float64)
    k = U.shape[0]
    return float(np.abs(U @ U.T - np.eye(k)).max()) if k else 0.0


def truncation_gap(lam, r):
    """Relative gap at the truncation index: (lam_r - lam_{r+1}) / lam_r (1-based r)."""
    lam = np.asarray(lam, dtype=np.float64)
    if r >= len(lam) or lam[r - 1] <= 0:
        return np.inf
    return float((lam[r - 1] - lam[r]) / lam[r - 1])


# Unit roundoff of each path's eigensolve input, for the near-tie reading at the
# truncation index: the FP64 and FP32 paths take 1e3 u (eigenvalues closer than that
# may swap order under the path's rounding); the mixed path's core carries the BF16
# rounding of its tall-skinny products, so ties are flagged within 10 u_bf16.
NEAR_TIE = {0: 1e3 * 2.0 ** -53, 1: 1e3 * 2.0 ** -24, 2: 10 * 2.0 ** -8}

# Per-mode eigenvalue bound relative to the largest eigenvalue (Weyl: every sorted
# eigenvalue moves by at most the 2-norm of the perturbation, which each path's
# rounding bounds by about N u |K| with N = r + n <= 512 columns): FP64 1e-12,
# FP32 2e-5 (N u_32 = 3e-5), mixed 8e-3 (2 u_bf16, the BF16 operands of the core).
MODE_TOL = {0: 1e-12, 1: 2e-5, 2: 8e-3}


def mixed_apply_bound(G, S_ref, lamA, lamG, c=2.0):
    """Stated bound of a mixed-precision inverse application: S = G / (lamA lamG) +
    W1 U_A^T + U_G W2 adds terms of size |G| / (lamA lamG) that cancel in the span of the
    factors, each carrying the BF16 rounding (u = 2^-8) of its operands, so the error is
    about c u |G|_F / (lamA lamG), c = 2 -- relative to |S| that is c u when G has most of its
    energy outside the factors' spans (|S| ~ |G| / (lamA lamG)), and grows by the damped
    condition sigma / lambda when G lies in them (as a layer's own gradient does).
    Returns the relative Frobenius bound (at least 1e-2)."""
    G = np.asarray(G, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    scale = np.linalg.norm(G) / (lamA * lamG) / max(np.linalg.norm(S_ref), 1e-300)
    return max(1e-2, c * 2.0 ** -8 * scale)


def gapped_prefix(lam, r, thr):
    """Largest k < r whose relative gap (lam_k - lam_{k+1}) / lam_k is at least thr (0 if none)."""
    lam = np.asarray(lam, dtype=np.float64)
    for k in range(min(r, len(lam)) - 1, 0, -1):
        if lam[k - 1] > 0 and (lam[k - 1] - lam[k]) / lam[k - 1] >= thr:
            return k
    return 0


def max_sin_theta(U1t, U2t, k):
    """sin of the largest principal angle between the spans of the first k rows: the
    2-norm of the part of A = U1[:k] outside span(B = U2[:k]), A - (A B^T) B (B
    orthonormalised first).  Unlike sqrt(1 - cos^2) it stays accurate for tiny angles
    and is blind to rows of A that are a little off unit norm."""
    if k <= 0:
        return 0.0
    A = np.asarray(U1t, dtype=np.float64)[:k]
    B = np.asarray(U2t, dtype=np.float64)[:k]
    Qb, _ = np.linalg.qr(B.T)  # d x k orthonormal basis of span(B)
    Qa, _ = np.linalg.qr(A.T)
    R = Qa - Qb @ (Qb.T @ Qa)
    return float(np.linalg.norm(R, 2))


def judge_step(Ug, sg, Uo_full, so_full, k, dtype, tol, orth_tol=None):
    """Compares one GPU step (k modes Ug (k, d), sg) with the oracle's untruncated
    result (Uo_full (N, d), so_full (N,) descending) under the parity readings:

    * sigma: relative Frobenius error < tol, and every mode within MODE_TOL of the
      largest eigenvalue (Weyl's bound holds for sorted eigenvalues, ties or not);
    * subspaces: at every index j <= k whose relative gap exceeds 1e-3, the sine
      of the largest angle between the top-j subspaces is within the Davis-Kahan
      bound 10 MODE_TOL sigma_1 / (sigma_j - sigma_{j+1});
    * reconstruction U diag(sigma) U^T: relative Frobenius error < tol -- unless the
      oracle's gap at the truncation index is a near tie (below NEAR_TIE), where the
      k-th mode is not determined by the path's precision: then the reconstruction
      is judged on the leading modes up to the last index whose gap clears NEAR_TIE.

    Returns a dict of the measured quantities."""
    so = np.asarray(so_full, dtype=np.float64)
    Uo = np.asarray(Uo_full, dtype=np.float64)
    sg = np.asarray(sg, dtype=np.float64)[:k]
    Ug = np.asarray(Ug, dtype=np.float64)[:k]
    out = {}
    bad = []
    es = rel(sg, so[:k])
    out["sigma"] = es
    if not es < tol:
        bad.append(("sigma", es))
    s1 = max(so[0], 1e-300) if len(so) else 1.0
    mode = float(np.abs(sg - so[:k]).max() / s1) if k else 0.0
    out["mode"] = mode
    if not mode < MODE_TOL[dtype]:
        bad.append(("per-mode sigma", mode))
    worst_angle = 0.0
    gapped = [j for j in range(1, k + 1)
              if so[j - 1] > 0 and (so[j - 1] - (so[j] if j < len(so) else 0.0)) / so[j - 1] > 1e-3]
    if len(gapped) > 32:  # 32 evenly spaced gapped indices, the last one included
        gapped = [gapped[i] for i in np.linspace(0, len(gapped) - 1, 32).round().astype(int)]
    for j in gapped:
        nxt = so[j] if j < len(so) else 0.0
        bound = min(1.0, 10.0 * MODE_TOL[dtype] * s1 / (so[j - 1] - nxt))
        st = max_sin_theta(Ug, Uo, j)
        worst_angle = max(worst_angle, st / bound)
        if not st <= bound:
            bad.append(("subspace", j, st, bound))
    out["angle_frac"] = worst_angle
    tie = truncation_gap(so, k) < NEAR_TIE[dtype] if k < len(so) else False
    out["tie"] = bool(tie)
    if tie:
        k0 = gapped_prefix(so, k, NEAR_TIE[dtype])
        er = lowrank_rel_err(Ug[:k0], sg[:k0], Uo[:k0], so[:k0]) if k0 else 0.0
    else:
        er = lowrank_rel_err(Ug, sg, Uo[:k], so[:k])
    out["recon"] = er
    if not er < tol:
        bad.append(("reconstruction", er, "near tie" if tie else ""))
    if orth_tol is not None:
        pos = sg > 0
        oe = orth_err(Ug[pos])
        out["orth"] = oe
        if not oe < orth_tol:
            bad.append(("orthonormality", oe))
    assert not bad, (bad, out)
    return out
