"""Seeded synthetic inputs shaped like wide-FC K-FAC workloads.

This module only draws random numbers; it holds none of the method's
arithmetic.  It is the one module that both the oracle-side tests and the CUDA
path consume, so parity tests feed identical arrays to both.

Recipe (stands in for the CIFAR10 / VGG16_bn FC-layer statistics of the
paper's Sec. 6, which are not available here):

* ``powerlaw_batch``: X = Q_d diag(k^(-alpha/2)) Z, k = 1..d, Z ~ N(0, 1) of
  size d x n, so that E[X X^T / n] = Q_d diag(k^-alpha) Q_d^T -- the decaying
  K-factor spectrum the paper relies on (Sec. 3.1, Sec. 3.5.1).  Q_d is a
  seeded random orthogonal matrix (QR of a Gaussian d x d matrix with
  diag(R) > 0), generated once per (d, seed) and cached.
* ``gradient``: a d_out x d_in N(0, 1) gradient matrix.
* ``mlp_batches``: activations and back-propagated pre-activation gradients of
  a random-init ReLU MLP on N(0, 1) inputs (bias row of ones appended to the
  activations; gradients scaled by n so that G G^T / n is the empirical Fisher
  factor).

Seeds: ``seed = 1000 * config + 10 * layer + {0: A, 1: Gamma}``; step t draws
from the stream SeedSequence([seed, t]).

Layout: a d x n column-major batch is returned as a C-contiguous (n, d) array,
the same memory as a torch (n, d) tensor.
"""
from __future__ import annotations

import functools

import numpy as np


def factor_seed(config: int, layer: int, which: str) -> int:
    return 1000 * int(config) + 10 * int(layer) + (0 if which in ("A", "a") else 1)


def _rng(seed: int, step: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(step)])))


@functools.lru_cache(maxsize=8)
def orthogonal_basis(d: int, seed: int) -> np.ndarray:
    """Seeded random orthogonal d x d matrix (float64), cached per (d, seed)."""
    g = _rng(seed, 1 << 30).standard_normal((d, d))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    q *= s[None, :]
    q.setflags(write=False)
    return q


def powerlaw_scales(d: int, alpha: float) -> np.ndarray:
    k = np.arange(1, d + 1, dtype=np.float64)
    return k ** (-alpha / 2.0)


def powerlaw_batch(d: int, n: int, alpha: float, seed: int, step: int) -> np.ndarray:
    """One batch X (d x n) returned as a C-contiguous (n, d) float64 array."""
    q = orthogonal_basis(d, seed)
    z = _rng(seed, step).standard_normal((n, d))
    return np.ascontiguousarray((z * powerlaw_scales(d, alpha)[None, :]) @ q.T)


def gaussian_columns(d: int, n: int, seed: int, step: int = 0) -> np.ndarray:
    """n i.i.d. N(0, 1) columns of length d, as a C-contiguous (n, d) array."""
    return np.ascontiguousarray(_rng(seed, step).standard_normal((n, d)))


def gradient(d_out: int, d_in: int, seed: int, step: int) -> np.ndarray:
    """A d_out x d_in N(0, 1) gradient matrix (row-major, float64)."""
    return np.ascontiguousarray(_rng(seed + 500, step).standard_normal((d_out, d_in)))


def with_bias_row(Xt: np.ndarray) -> np.ndarray:
    """Append the K-FAC bias coordinate (a row of ones) to a (n, d) batch -> (n, d + 1)."""
    n = Xt.shape[0]
    return np.ascontiguousarray(np.concatenate([Xt, np.ones((n, 1), dtype=Xt.dtype)], axis=1))


def orthonormal_columns(d: int, k: int, seed: int) -> np.ndarray:
    """k orthonormal columns of length d, as a (k, d) array (first k columns of Q_d)."""
    return np.ascontiguousarray(orthogonal_basis(d, seed)[:, :k].T)


def mlp_batches(widths, n: int, seed_w: int, seed_x: int, step: int, device="cpu", dtype=None):
    """Activations and pre-activation gradients of a random-init ReLU MLP.

    widths: [d_0, d_1, ..., d_L] (layer l maps d_l -> d_{l+1}); Kaiming-normal
    weights (seed_w), N(0, 1) inputs and uniform labels (seed_x, step),
    cross-entropy loss with mean reduction.  Returns (acts, grads, weight_grads)
    where acts[l] is (n, d_l + 1) with the bias ones column appended,
    grads[l] is (n, d_{l+1}) = n * dLoss/dz_l, and weight_grads[l] is the
    (d_{l+1}, d_l + 1) gradient [dW | db] of the loss.
    """
    import torch

    dtype = dtype or torch.float32
    gw = torch.Generator(device="cpu").manual_seed(int(seed_w))
    weights, biases = [], []
    for l in range(len(widths) - 1):
        w = torch.randn(widths[l + 1], widths[l], generator=gw, dtype=torch.float64) * np.sqrt(2.0 / widths[l])
        weights.append(w.to(device=device, dtype=dtype).requires_grad_(True))
        biases.append(torch.zeros(widths[l + 1], device=device, dtype=dtype, requires_grad=True))
    gx = torch.Generator(device="cpu").manual_seed(int(seed_x) * 100003 + int(step))
    x = torch.randn(n, widths[0], generator=gx, dtype=torch.float64).to(device=device, dtype=dtype)
    y = torch.randint(0, widths[-1], (n,), generator=gx).to(device)
    acts, zs = [], []
    h = x
    for l, (w, b) in enumerate(zip(weights, biases)):
        acts.append(h.detach())
        z = h @ w.T + b
        z.retain_grad()
        zs.append(z)
        h = torch.relu(z) if l + 1 < len(weights) else z
    loss = torch.nn.functional.cross_entropy(h, y)
    loss.backward()
    ones = torch.ones(n, 1, device=device, dtype=dtype)
    acts_b = [torch.cat([a, ones], dim=1).contiguous() for a in acts]
    grads = [(z.grad * n).detach().contiguous() for z in zs]
    wgrads = [torch.cat([w.grad, b.grad[:, None]], dim=1).detach().contiguous() for w, b in zip(weights, biases)]
    return acts_b, grads, wgrads


class DevicePowerlaw:
    """The powerlaw_batch recipe drawn on a CUDA device, for runs too long for host
    generation (hundreds of steps at d = 4097).  Q_d comes from a QR of a seeded
    Gaussian on the device (a different draw from orthogonal_basis), Z ~ N(0, 1) from
    torch's generator seeded with (seed, step); X = Q_d diag(k^(-alpha/2)) Z is
    formed in FP32 and written into a caller buffer (an (n, ld) column tensor)."""

    def __init__(self, d: int, alpha: float, seed: int, device):
        import torch

        self.d, self.seed, self.device = int(d), int(seed), device
        g = torch.Generator(device=device).manual_seed(int(seed) * 7919 + 17)
        a = torch.randn(self.d, self.d, generator=g, device=device, dtype=torch.float64)
        q, r = torch.linalg.qr(a)
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        q = q * s[None, :]
        sc = torch.from_numpy(powerlaw_scales(self.d, alpha)).to(device)
        self.qs_t = (q * sc[None, :]).T.contiguous().float()  # rows: scaled basis vectors
        self.gen = torch.Generator(device=device)

    def draw(self, out, n: int, step: int):
        """Writes batch `step` (n columns) into out[:n, :d] (float32)."""
        import torch

        self.gen.manual_seed(self.seed * 1000003 + int(step))
        z = torch.randn(n, self.d, generator=self.gen, device=self.device, dtype=torch.float32)
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            out[:n, : self.d].copy_(z @ self.qs_t)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
        return out
