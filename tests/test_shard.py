"""Multi-rank host logic on CPU: world_size 2 over gloo (127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2210_08494_gb300 import shard


def test_assignment_covers_each_layer_once_and_balances():
    widths = [4096] * 8 + [10]
    costs = [shard.layer_cost(widths[l], widths[l + 1], 220, 256) for l in range(8)]
    for world in (1, 2, 3, 4, 8):
        parts = shard.assign_layers(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(8))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= min(loads) + max(costs) + 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [shard.layer_cost(4096, 4096, 256, 256)] * 3 + [shard.layer_cost(4096, 10, 256, 256)]
    parts = shard.assign_layers(costs, world)
    mine = parts[rank]
    elapsed = 10.0 + rank  # each rank's own (fake) timing
    t = shard.max_over_ranks(elapsed)
    dist.barrier()
    q.put((rank, mine, t))
    dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    assert res[0][2] == res[1][2] == 11.0  # max over ranks
    assert sorted(res[0][1] + res[1][1]) == [0, 1, 2, 3]  # every layer once, no overlap


def _exchange_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    widths = [64] * 4 + [10]
    costs = [shard.layer_cost(widths[l], widths[l + 1], 16, 8) for l in range(4)]
    parts = shard.assign_layers(costs, world)
    # padded-row steps like the library's gradients: (d_out, d_in + 1) views of (d_out, ld)
    S, base = [], []
    for l in range(4):
        full = torch.full((widths[l + 1], widths[l] + 8), -1.0)
        base.append(full)
        S.append(full[:, : widths[l] + 1])
    for l in parts[rank]:
        S[l].copy_(torch.arange(S[l].numel(), dtype=torch.float32).view(S[l].shape) + 1000.0 * l)
    shard.exchange_steps(S, parts, rank)
    ok = all(torch.equal(S[l], torch.arange(S[l].numel(), dtype=torch.float32).view(S[l].shape) + 1000.0 * l)
             for l in range(4))
    pads = all(bool((base[l][:, widths[l] + 1:] == -1.0).all()) for l in range(4))
    q.put((rank, ok, pads, parts))
    dist.destroy_process_group()


def test_step_exchange_over_gloo():
    """Each of two ranks preconditions its own layers; after the all-gather both hold
    every layer's step, and the rows' padding is left alone."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=60) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok, pads, parts in res:
        assert ok and pads, rank
        assert sorted(parts[0] + parts[1]) == [0, 1, 2, 3] and parts[0] and parts[1]
