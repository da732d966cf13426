"""Error study of the B-KFAC variants on synthetic data (the numerical
investigation of Sec. 5): how far each low-rank inverse representation is from
the exact damped inverse of the EA K-factors, step by step.

    python -m paper_2210_08494_gb300.error_study --steps 60 --out error_study.json
    python -m paper_2210_08494_gb300.error_study --mlp --steps 20
    python -m paper_2210_08494_gb300.error_study --mlp --width 4096 --depth 8 --n 256 --r 220 --steps 10

Two sources of K-factor statistics:

* one FC layer (A: d_in + 1 = 513, Gamma: 256), n = 32 new columns per step,
  power-law inputs (``synth.powerlaw_batch`` recipe) in a basis that drifts a
  little every step (a product of small random rotations), so the factors
  keep changing;
* ``--mlp``: every layer of a ReLU MLP (the preconditioning workload's
  architecture: width 4096, 8 layers, 10 outputs, minibatch 256, r = 220 at
  full size; a narrower copy by default) trained by plain SGD on N(0, 1) inputs
  and uniform labels, so its activations and back-propagated gradients drift
  the way training moves them.  A_l = [a_l; 1] and G_l = n dLoss/dz_l.

rho = 0.95, damping relative to the largest eigenvalue (phi = 0.1) with
spectrum continuation, as in the paper's experiments.  The algorithms, all
through the library's C ABI on the GPU:

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
the angle between s and the reference step; with several layers each metric is
the mean over the layers.  The random draws (correction modes, RSVD test
matrices) are seeded.  With ``keep_last`` the run returns the last step's
dense EA factors, gradients, states and steps, so that a test can recompute
the metrics of that step independently.
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


class DriftLayer:
    """One FC layer whose input and output statistics come from drifting bases."""

    def __init__(self, dA, dG, n, alpha, seed):
        self.dims = [(dA, dG)]
        self.n, self.alpha, self.seed = n, alpha, seed
        self.sides = (Drift(dA, seed), Drift(dG, seed + 10))

    def step(self, t):
        return [(self.sides[0].batch(self.n, self.alpha, self.seed, t),
                 self.sides[1].batch(self.n, self.alpha, self.seed + 1, t))]


class TrainingMLP:
    """A ReLU MLP trained by plain SGD on N(0, 1) inputs and uniform labels
    (cross-entropy, mean reduction): each step returns every layer's activations
    with the bias ones column (n, d_l + 1) and pre-activation gradients scaled by n
    (n, d_{l+1}), then takes the SGD step, so the statistics drift with training."""

    def __init__(self, widths, n, seed, lr=0.05, device="cuda"):
        g = torch.Generator(device="cpu").manual_seed(int(seed))
        self.W = [(torch.randn(widths[l + 1], widths[l], generator=g, dtype=torch.float64)
                   * np.sqrt(2.0 / widths[l])).float().to(device) for l in range(len(widths) - 1)]
        self.b = [torch.zeros(widths[l + 1], device=device) for l in range(len(widths) - 1)]
        self.dims = [(widths[l] + 1, widths[l + 1]) for l in range(len(widths) - 1)]
        self.widths, self.n, self.seed, self.lr, self.device = widths, n, seed, lr, device

    def step(self, t):
        gx = torch.Generator(device="cpu").manual_seed(int(self.seed) * 100003 + int(t) + 1)
        x = torch.randn(self.n, self.widths[0], generator=gx).to(self.device)
        y = torch.randint(0, self.widths[-1], (self.n,), generator=gx).to(self.device)
        Ws = [w.clone().requires_grad_(True) for w in self.W]
        bs = [b.clone().requires_grad_(True) for b in self.b]
        acts, zs, h = [], [], x
        for l, (w, b) in enumerate(zip(Ws, bs)):
            acts.append(h.detach())
            z = h @ w.T + b
            z.retain_grad()
            zs.append(z)
            h = torch.relu(z) if l + 1 < len(Ws) else z
        torch.nn.functional.cross_entropy(h, y).backward()
        ones = torch.ones(self.n, 1, device=self.device)
        out = [(torch.cat([a, ones], 1).double().cpu().numpy(), (z.grad * self.n).double().cpu().numpy())
               for a, z in zip(acts, zs)]
        with torch.no_grad():
            for l in range(len(self.W)):
                self.W[l] -= self.lr * Ws[l].grad
                self.b[l] -= self.lr * bs[l].grad
        return out


def study(source, steps=60, heavy=10, r=64, rho=0.95, phi=0.1, seed=9000, dtype=bkfac.F32, verbose=True,
          keep_last=False):
    """Runs the five algorithms on the layers of `source` (DriftLayer or TrainingMLP)."""
    bkfac.load()
    bkfac.bkfac_status()
    tdt = bkfac._TORCH_DTYPE[dtype]
    dims = source.dims
    L = len(dims)
    n = source.n
    Mdev = [[bkfac.dense_factor(d, dtype) for d in dims[l]] for l in range(L)]
    fac = {a: [[bkfac.Factor(d, min(r, d), dtype) for d in dims[l]] for l in range(L)] for a in ALGOS if a != "k-fac"}
    kfac_inv = [None] * L
    rng = np.random.default_rng(seed + 20)
    flags = bkfac.SPECTRUM_CONTINUATION | bkfac.DAMPING_RELATIVE
    hist = {a: [] for a in ALGOS}
    corr_checks = []
    last = None
    for t in range(steps + 1):
        batches = source.step(t)
        heavy_step = t % heavy == 0
        per_algo = {a: [] for a in ALGOS}
        last = {"layers": []} if keep_last and t == steps else None
        for l in range(L):
            X, Mh = [], []
            for w in range(2):
                d = dims[l][w]
                Xt = bkfac.cols_tensor(n, d, tdt)
                Xt.copy_(torch.from_numpy(batches[l][w]))
                X.append(Xt)
                bkfac.bkfac_ea_update(Mdev[l][w], Xt, rho, dtype, first=(t == 0))
                Mh.append(Mdev[l][w].double().cpu().numpy().T.copy()[:, :d])
            refinv = [exact_inverse(Mh[w], phi) for w in range(2)]
            for a, fl in fac.items():
                for w in range(2):
                    f, d = fl[l][w], dims[l][w]
                    lt = min(f.r + 10, d)  # RSVD test columns: r + 10 oversampling, at most d
                    if a == "r-kfac":
                        if heavy_step:
                            Om = bkfac.cols_tensor(lt, d, tdt)
                            Om.copy_(torch.from_numpy(rng.standard_normal((lt, d))))
                            bkfac.bkfac_rsvd(f, Mdev[l][w], Om, 4)
                        continue
                    if t == 0:
                        bkfac.bkfac_init(f, X[w])
                    else:
                        bkfac.bkfac_update(f, X[w], rho)
                    if heavy_step and t > 0 and a == "b-r-kfac":
                        Om = bkfac.cols_tensor(lt, d, tdt)
                        Om.copy_(torch.from_numpy(rng.standard_normal((lt, d))))
                        bkfac.bkfac_rsvd(f, Mdev[l][w], Om, 4)
                    if heavy_step and t > 0 and a == "b-kfac-c" and f.r_cur >= 2:
                        U0, s0 = (v.double().cpu().numpy() for v in f.state())
                        before = np.linalg.norm(Mh[w] - (U0.T * s0) @ U0)
                        idx = rng.choice(f.r_cur, f.r_cur // 2, replace=False)
                        bkfac.bkfac_correct(f, Mdev[l][w], idx)
                        U1, s1 = (v.double().cpu().numpy() for v in f.state())
                        corr_checks.append((before, np.linalg.norm(Mh[w] - (U1.T * s1) @ U1)))
            if heavy_step:
                kfac_inv[l] = list(refinv)
            st = bkfac.bkfac_status()
            if st != bkfac.OK:
                raise RuntimeError(f"device status {bkfac.strerror(st)} at step {t}")
            # the step's gradient from its thin factors and the reference step
            XA, XG = (x.double().cpu().numpy() for x in X)
            dA, dG = dims[l]
            G = (XG[:, :dG].T @ XA[:, :dA]) / n
            s_ref = refinv[1] @ G @ refinv[0]
            rec = {"MA": Mh[0], "MG": Mh[1], "XA": XA[:, :dA], "XG": XG[:, :dG], "algos": {}} if last is not None \
                else None
            for a in ALGOS:
                if a == "k-fac":
                    invA, invG = kfac_inv[l]
                    s = invG @ G @ invA
                else:
                    fA, fG = fac[a][l]
                    UA, sA = (v.double().cpu().numpy() for v in fA.state())
                    UG, sG = (v.double().cpu().numpy() for v in fG.state())
                    invA, invG = damped_inverse(UA, sA, phi, dA), damped_inverse(UG, sG, phi, dG)
                    PA = bkfac.cols_tensor(n, dA, tdt)
                    PG = bkfac.cols_tensor(n, dG, tdt)
                    S = bkfac.grad_tensor(dG, dA, tdt)
                    bkfac.bkfac_apply_factored(fA, fG, phi, phi, X[0], X[1], PA, PG, alpha=1.0 / n, S=S,
                                               flags=flags)
                    s = S.double().cpu().numpy()
                    if rec is not None:
                        rec["algos"][a] = {"UA": UA, "sA": sA, "UG": UG, "sG": sG, "s": s}
                cosang = float(np.sum(s * s_ref) / (np.linalg.norm(s) * np.linalg.norm(s_ref)))
                per_algo[a].append([rel(invA, refinv[0]), rel(invG, refinv[1]), rel(s, s_ref), 1.0 - cosang])
            if rec is not None:
                last["layers"].append(rec)
        for a in ALGOS:
            hist[a].append([float(np.mean([m[i] for m in per_algo[a]])) for i in range(4)])
            if last is not None:
                last.setdefault("per_layer", {})[a] = per_algo[a]
        if verbose and t % heavy == 0:
            print(f"step {t}: " + "  ".join(f"{a} {hist[a][-1][2]:.2e}" for a in ALGOS), flush=True)
    names = ["err_Ainv", "err_Ginv", "err_step", "one_minus_cos"]
    summary = {a: {nm: float(np.mean([h[i] for h in hist[a][1:]])) for i, nm in enumerate(names)} for a in ALGOS}
    res = {"summary": summary, "history": {a: hist[a] for a in ALGOS}, "correction_checks": corr_checks,
           "config": {"steps": steps, "heavy_every": heavy, "dims": dims, "r": r, "n": n, "rho": rho, "phi": phi,
                      "dtype": int(dtype)}}
    if keep_last:
        res["last"] = last
    return res


def run(steps=60, heavy=10, dA=513, dG=256, r=64, n=32, rho=0.95, phi=0.1, alpha=1.2, seed=9000,
        dtype=bkfac.F32, verbose=True, keep_last=False):
    """The single-layer study on drifting power-law statistics."""
    return study(DriftLayer(dA, dG, n, alpha, seed), steps, heavy, r, rho, phi, seed, dtype, verbose, keep_last)


def run_mlp(steps=20, heavy=10, width=512, depth=4, outputs=10, n=128, r=64, rho=0.95, phi=0.1, lr=0.05,
            seed=5000, dtype=bkfac.F32, verbose=True, keep_last=False):
    """The study on every layer of a training ReLU MLP (width x depth, `outputs` classes)."""
    widths = [width] * depth + [outputs]
    return study(TrainingMLP(widths, n, seed, lr), steps, heavy, r, rho, phi, seed, dtype, verbose, keep_last)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--heavy", type=int, default=10)
    ap.add_argument("--mlp", action="store_true", help="the layers of a training ReLU MLP")
    ap.add_argument("--width", type=int, default=512)
    ap.add_argument("--depth", type=int, default=4)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--r", type=int, default=64)
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    if args.mlp:
        res = run_mlp(steps=args.steps, heavy=args.heavy, width=args.width, depth=args.depth, n=args.n, r=args.r)
    else:
        res = run(steps=args.steps, heavy=args.heavy)
    print("mean over the steps (metrics 1-4 of Sec. 5.1):")
    print(f"{'algorithm':10s} {'A^-1':>10s} {'Gamma^-1':>10s} {'step':>10s} {'1-cos':>10s}")
    for a, m in res["summary"].items():
        print(f"{a:10s} {m['err_Ainv']:10.3e} {m['err_Ginv']:10.3e} {m['err_step']:10.3e} {m['one_minus_cos']:10.3e}")
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({k: v for k, v in res.items() if k != "last"}, fh)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
