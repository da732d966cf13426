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
