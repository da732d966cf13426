"""Error study of the B-KFAC variants on synthetic data (the numerical
investigation of Sec. 5): how far each low-rank inverse representation is from
the exact damped inverse of the EA K-factors, step by step.

    python -m paper_2210_08494_gb300.error_study --steps 60 --out error_study.json

One FC layer (A: d_in + 1 = 513, Gamma: 256), n = 32 new columns per step,
rho = 0.95, rank r = 64, damping relative to the largest eigenvalue
(phi = 0.1) with spectrum continuation, as in the paper's experiments.  The
inputs follow the power-law recipe of ``synth.powerlaw_batch`` with a basis
that drifts a little every step (a product of small random rotations), so the
factors keep changing.  The algorithms, all through the library's C ABI on
the GPU:

  b-kfac     a Brand update every step (Algorithm 4);
  b-r-kfac   the same, the representation overwritten by an RSVD of the dense
             EA factor every T_heavy steps (Algorithm 5);
  b-kfac-c   the same, with a light correction of phi_crc = 0.5 of the modes
             every T_heavy steps (Algorithms 6-7);
  r-kfac     an RSVD of the dense EA factor every T_heavy steps, nothing in
             between (the representation goes stale);
  k-fac      the exact inverse every T_heavy steps, nothing in between.

Reference: the exact damped inverse of the dense EA factors at every step
(FP64 eigendecomposition on the host).  Metrics (Sec. 5.1): (1) and (2) the
relative Frobenius error of A^-1 and Gamma^-1, (3) the relative error of the
preconditioned step s = Gamma^-1 G A^-1 for the step's gradient
G = G_f A_f^T / n (formed by Algorithm 8 from the thin factors), (4) 1 - cos of
the angle between s and the reference step.  The random draws (correction
modes, RSVD test matrices) are seeded.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import bkfac, synth

ALGOS = ("b-kfac", "b-r-kfac", "b-kfac-c", "r-kfac", "k-fac")


def damped_inverse(U, s, phi, d):
    """(U diag(s) U^T + lam I)^-1 with lam = phi max(s) and spectrum continuation:
    lam' = lam + min(s), s' = s - min(s) (dense, FP64)."""
    lam = phi * s.max()
    m = s.min()
    lp = lam + m
    c = 1.0 / (s - m + lp) - 1.0 / lp
    return np.eye(d) / lp + (U.T * c) @ U


def exact_inverse(M, phi):
    w = np.linalg.eigvalsh(M)
    lam = phi * w.max()
    return np.linalg.inv(M + lam * np.eye(M.shape[0]))


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


class Drift:
    """Orthogonal basis that drifts by a small random rotation every step."""

    def __init__(self, d, seed, eps=0.02):
        self.Q = synth.orthogonal_basis(d, seed).copy()
        self.rng = np.random.default_rng(seed + 1)
        self.eps = eps

    def batch(self, n, alpha, seed, t):
        d = self.Q.shape[0]
        z = np.random.default_rng([seed, t]).standard_normal((n, d))
        x = (z * (np.arange(1, d + 1) ** (-alpha / 2.0))) @ self.Q.T
        q, rr = np.linalg.qr(np.eye(d) + self.eps * self.rng.standard_normal((d, d)))
        self.Q = self.Q @ (q * np.sign(np.diag(rr)))
        return np.ascontiguousarray(x)


def run(steps=60, heavy=10, dA=513, dG=256, r=64, n=32, rho=0.95, phi=0.1, alpha=1.2, seed=9000,
        dtype=bkfac.F32, verbose=True):
    bkfac.load()
    bkfac.bkfac_status()
    tdt = bkfac._TORCH_DTYPE[dtype]
    sides = {"A": Drift(dA, seed), "G": Drift(dG, seed + 10)}
    dims = {"A": dA, "G": dG}
    Mdev = {w: bkfac.dense_factor(dims[w], dtype) for w in "AG"}
    fac = {a: {w: bkfac.Factor(dims[w], r, dtype) for w in "AG"} for a in ALGOS if a != "k-fac"}
    kfac_inv = {}
    rng = np.random.default_rng(seed + 20)
    flags = bkfac.SPECTRUM_CONTINUATION | bkfac.DAMPING_RELATIVE
    hist = {a: [] for a in ALGOS}
    corr_checks = []
    for t in range(steps + 1):
        X = {}
        for w in "AG":
            Xt = sides[w].batch(n, alpha, seed + (0 if w == "A" else 1), t)
            X[w] = bkfac.cols_tensor(n, dims[w], tdt)
            X[w].copy_(torch.from_numpy(Xt))
            bkfac.bkfac_ea_update(Mdev[w], X[w], rho, dtype, first=(t == 0))
        Mh = {w: Mdev[w].double().cpu().numpy().T.copy() for w in "AG"}
        refinv = {w: exact_inverse(Mh[w], phi) for w in "AG"}
        heavy_step = t % heavy == 0
        for a, fw in fac.items():
            for w in "AG":
                f = fw[w]
                if a == "r-kfac":
                    if heavy_step:
                        Om = bkfac.cols_tensor(r + 10, dims[w], tdt)
                        Om.copy_(torch.from_numpy(rng.standard_normal((r + 10, dims[w]))))
                        bkfac.bkfac_rsvd(f, Mdev[w], Om, 4)
                    continue
                if t == 0:
                    bkfac.bkfac_init(f, X[w])
                else:
                    bkfac.bkfac_update(f, X[w], rho)
                if heavy_step and t > 0 and a == "b-r-kfac":
                    Om = bkfac.cols_tensor(r + 10, dims[w], tdt)
                    Om.copy_(torch.from_numpy(rng.standard_normal((r + 10, dims[w]))))
                    bkfac.bkfac_rsvd(f, Mdev[w], Om, 4)
                if heavy_step and t > 0 and a == "b-kfac-c":
                    U0, s0 = (v.double().cpu().numpy() for v in f.state())
                    before = np.linalg.norm(Mh[w] - (U0.T * s0) @ U0)
                    idx = rng.choice(f.r_cur, f.r_cur // 2, replace=False)
                    bkfac.bkfac_correct(f, Mdev[w], idx)
                    U1, s1 = (v.double().cpu().numpy() for v in f.state())
                    corr_checks.append((before, np.linalg.norm(Mh[w] - (U1.T * s1) @ U1)))
        if heavy_step:
            kfac_inv = dict(refinv)
        st = bkfac.bkfac_status()
        if st != bkfac.OK:
            raise RuntimeError(f"device status {bkfac.strerror(st)} at step {t}")
        # the step's gradient from its thin factors and the reference step
        G = (X["G"].double().cpu().numpy().T @ X["A"].double().cpu().numpy()) / n
        s_ref = refinv["G"] @ G @ refinv["A"]
        for a in ALGOS:
            if a == "k-fac":
                invA, invG = kfac_inv["A"], kfac_inv["G"]
                s = invG @ G @ invA
            else:
                fA, fG = fac[a]["A"], fac[a]["G"]
                UA, sA = (v.double().cpu().numpy() for v in fA.state())
                UG, sG = (v.double().cpu().numpy() for v in fG.state())
                invA, invG = damped_inverse(UA, sA, phi, dA), damped_inverse(UG, sG, phi, dG)
                PA = bkfac.cols_tensor(n, dA, tdt)
                PG = bkfac.cols_tensor(n, dG, tdt)
                S = bkfac.grad_tensor(dG, dA, tdt)
                bkfac.bkfac_apply_factored(fA, fG, phi, phi, X["A"], X["G"], PA, PG, alpha=1.0 / n, S=S, flags=flags)
                s = S.double().cpu().numpy()
            cosang = float(np.sum(s * s_ref) / (np.linalg.norm(s) * np.linalg.norm(s_ref)))
            hist[a].append([rel(invA, refinv["A"]), rel(invG, refinv["G"]), rel(s, s_ref), 1.0 - cosang])
        if verbose and t % heavy == 0:
            print(f"step {t}: " + "  ".join(f"{a} {hist[a][-1][2]:.2e}" for a in ALGOS), flush=True)
    names = ["err_Ainv", "err_Ginv", "err_step", "one_minus_cos"]
    summary = {a: {nm: float(np.mean([h[i] for h in hist[a][1:]])) for i, nm in enumerate(names)} for a in ALGOS}
    return {"summary": summary, "history": {a: hist[a] for a in ALGOS}, "correction_checks": corr_checks,
            "config": {"steps": steps, "heavy_every": heavy, "dA": dA, "dG": dG, "r": r, "n": n, "rho": rho,
                       "phi": phi, "alpha": alpha, "dtype": int(dtype)}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--heavy", type=int, default=10)
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    res = run(steps=args.steps, heavy=args.heavy)
    print("mean over the steps (metrics 1-4 of Sec. 5.1):")
    print(f"{'algorithm':10s} {'A^-1':>10s} {'Gamma^-1':>10s} {'step':>10s} {'1-cos':>10s}")
    for a, m in res["summary"].items():
        print(f"{a:10s} {m['err_Ainv']:10.3e} {m['err_Ginv']:10.3e} {m['err_step']:10.3e} {m['one_minus_cos']:10.3e}")
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
