"""Run one factor's Brand updates (and optionally one layer's inverse
application) on the GPU at a chosen shape: the small, self-contained workload
for kernel profilers.

    python -m paper_2210_08494_gb300.profile_case --d 4097 --r 256 --n 256 --updates 1
    python -m paper_2210_08494_gb300.profile_case --d 4097 --r 256 --n 256 --apply 4096

Inputs follow the synthetic power-law recipe of ``synth.powerlaw_batch``; the
first batch initialises the factor (exact EVD, Eq. (5) with kappa(0) = 1),
each further batch is one update (Algorithm 4 via Algorithm 3).  With
``--apply d_out`` a Gamma factor of size d_out is built the same way and the
damped inverse application (Algorithm 1) runs on a d_out x d FP32 gradient.
Prints the device status and the elapsed time of the last call.
"""
from __future__ import annotations

import argparse

import torch

from . import bkfac, synth

DTYPES = {"f32": bkfac.F32, "f64": bkfac.F64, "mixed": bkfac.MIXED_BF16}


def factor_with_updates(d, r, n, dtype, updates, seed, alpha, flags=0):
    f = bkfac.Factor(d, r, dtype, flags=flags)
    tdt = torch.float64 if dtype == bkfac.F64 else torch.float32
    xs = []
    for t in range(updates + 1):
        x = bkfac.cols_tensor(n, d, tdt)
        x.copy_(torch.from_numpy(synth.powerlaw_batch(d, n, alpha, seed, t)))
        xs.append(x)
    bkfac.bkfac_init(f, xs[0])
    for t in range(1, updates + 1):
        bkfac.bkfac_update(f, xs[t], 0.95)
    return f


def factor_with_state(d, r, dtype, seed, flags=0):
    """A factor holding r orthonormal columns and a power-law spectrum (no updates)."""
    import numpy as np

    f = bkfac.Factor(d, r, dtype, flags=flags)
    Ut = synth.orthonormal_columns(d, r, seed)
    sig = np.arange(1, r + 1, dtype=np.float64) ** -1.2
    f.load_state(torch.from_numpy(Ut).to(f.torch_dtype).cuda(), torch.from_numpy(sig).cuda())
    return f


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--d", type=int, default=4097)
    ap.add_argument("--r", type=int, default=256)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--updates", type=int, default=1)
    ap.add_argument("--dtype", choices=sorted(DTYPES), default="f32")
    ap.add_argument("--alpha", type=float, default=1.2)
    ap.add_argument("--apply", type=int, default=0, metavar="D_OUT")
    ap.add_argument("--synthetic-state", action="store_true",
                    help="with --apply: load orthonormal factor states instead of running updates")
    ap.add_argument("--repeat", type=int, default=1, help="with --apply: time this many applications")
    ap.add_argument("--tf32x3", action="store_true", help="FP32 products as 3xTF32 on the tensor cores")
    args = ap.parse_args(argv)
    bkfac.load()
    bkfac.bkfac_status()
    dtype = DTYPES[args.dtype]
    fl = bkfac.FLAG_TF32X3 if args.tf32x3 else 0
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    if args.synthetic_state:
        fA = factor_with_state(args.d, args.r, dtype, 2000, fl)
    else:
        fA = factor_with_updates(args.d, args.r, args.n, dtype, args.updates, 2000, args.alpha, fl)
    end.record()
    if args.apply:
        if args.synthetic_state:
            fG = factor_with_state(args.apply, args.r, dtype, 2001, fl)
        else:
            fG = factor_with_updates(args.apply, args.r, args.n, dtype, args.updates, 2001, args.alpha, fl)
        tdt = torch.float64 if dtype == bkfac.F64 else torch.float32
        G = bkfac.grad_tensor(args.apply, args.d, tdt)
        G.normal_(generator=torch.Generator(device="cuda").manual_seed(7))
        S = bkfac.grad_tensor(args.apply, args.d, tdt)
        bkfac.bkfac_apply(fA, fG, 1e-2, 1e-2, G, S)  # first call: one-time set-up
        start.record()
        for _ in range(args.repeat):
            bkfac.bkfac_apply(fA, fG, 1e-2, 1e-2, G, S)
        end.record()
    torch.cuda.synchronize()
    st = bkfac.bkfac_status()
    reps = args.repeat if args.apply else 1
    print(f"status {st} ({bkfac.strerror(st)}), {start.elapsed_time(end) / reps:.3f} ms per timed call")
    return 0 if st == bkfac.OK else 1


if __name__ == "__main__":
    raise SystemExit(main())
