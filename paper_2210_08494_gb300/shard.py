"""Host-side logic for running the hot path on several GPUs of one node.

The preconditioning work partitions into independent layers: a layer's two
factor updates and its apply need nothing from other layers.  So ranks take
whole layers, and the one data exchange of a step comes after the work: every
rank needs every layer's preconditioned gradient S_l for its weight update, so
the ranks all-gather the steps of their layers (exchange_steps).  Timing takes
the max of the elapsed times over ranks.

The per-layer cost model follows the update's work: d (r + n)^2 for the
tall-skinny products plus a (r + n)^3 term for the core eigensolve, for each
of the layer's two factors (d_in + 1 and d_out).
"""
from __future__ import annotations


def layer_cost(d_in: int, d_out: int, r: int, n: int, core_weight: float = 30.0) -> float:
    cost = 0.0
    for d in (d_in + 1, d_out):
        rr = min(r, d)
        N = rr + n
        cost += d * N * N + core_weight * N ** 3
    return cost


def assign_layers(costs, world: int):
    """Greedy longest-processing-time assignment of layers to ranks.

    Returns a list of `world` lists of layer indices (each layer exactly once;
    ties broken by index, so every rank computes the same assignment)."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        out[r].append(i)
        loads[r] += costs[i]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over the ranks of the default process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def owners(parts):
    """Layer index -> owning rank for an assignment from assign_layers."""
    own = {}
    for r, p in enumerate(parts):
        for l in p:
            own[l] = r
    return own


def exchange_steps(S, parts, rank: int):
    """All-gather of the preconditioned gradients: rank `rank` has written S[l] for its
    layers parts[rank]; afterwards every rank holds every S[l] (written in place).

    One collective per step: each rank packs its layers' steps, in layer order, into one
    flat buffer of the largest rank's size, the buffers are all-gathered, and each rank
    unpacks the other ranks' layers.  S[l] may be a strided 2-D view (padded rows)."""
    import torch
    import torch.distributed as dist

    world = len(parts)
    if world == 1:
        return
    sizes = [sum(S[l].numel() for l in p) for p in parts]
    m = max(sizes)
    ref = S[parts[rank][0]] if parts[rank] else S[0]
    buf = torch.zeros(m, dtype=ref.dtype, device=ref.device)
    off = 0
    for l in parts[rank]:
        k = S[l].numel()
        buf[off:off + k].view(S[l].shape).copy_(S[l])
        off += k
    out = torch.empty(world * m, dtype=ref.dtype, device=ref.device)
    dist.all_gather_into_tensor(out, buf)
    for r, p in enumerate(parts):
        if r == rank:
            continue
        off = r * m
        for l in p:
            k = S[l].numel()
            S[l].copy_(out[off:off + k].view(S[l].shape))
            off += k
