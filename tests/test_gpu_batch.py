"""GPU tests of the batched calls (bkfac_batch_*): every factor of every FC
layer updated, then every layer preconditioned, with uneven d, r and a
dense-path factor (d = 10, the 10-way output layer's Gamma).

* Batched results equal the per-factor calls bit for bit (same kernels, same
  launch shapes, no order-dependent reductions), so the batch adds no error.
* A graph replay of a captured step equals the same step run eagerly, bit for
  bit.
* One batched step matches the FP64 oracle within the path's tolerance.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import lowrank_rel_err, rel

pytestmark = pytest.mark.gpu

# (d_in + bias, d_out, r)
LAYERS = [(129, 64, 16), (257, 10, 24), (65, 300, 8)]
N = 32


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def make_layers(dtype):
    return [(bkfac.Factor(dA, min(r, dA), dtype), bkfac.Factor(dG, min(r, dG), dtype)) for dA, dG, r in LAYERS]


def batches(dtype, step):
    tdt = torch.float64 if dtype == bkfac.F64 else torch.float32
    XA, XG, G = [], [], []
    for l, (dA, dG, r) in enumerate(LAYERS):
        a = bkfac.cols_tensor(N, dA, tdt)
        a.copy_(torch.from_numpy(synth.powerlaw_batch(dA, N, 1.5, synth.factor_seed(3, l, "A"), step)))
        g = bkfac.cols_tensor(N, dG, tdt)
        g.copy_(torch.from_numpy(synth.powerlaw_batch(dG, N, 1.5, synth.factor_seed(3, l, "G"), step)))
        gr = bkfac.grad_tensor(dG, dA, tdt)
        gr.copy_(torch.from_numpy(synth.gradient(dG, dA, synth.factor_seed(3, l, "A"), step)))
        XA.append(a)
        XG.append(g)
        G.append(gr)
    return XA, XG, G


def state_copy(layers):
    return [(a.U.clone(), a.sigma.clone(), g.U.clone(), g.sigma.clone()) for a, g in layers]


def out_like(G):
    return [bkfac.grad_tensor(g.shape[0], g.shape[1], g.dtype) for g in G]


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_batch_equals_per_factor_calls(dtype):
    lam = [0.1, 0.05, 0.2]
    ref = make_layers(dtype)
    bat_layers = make_layers(dtype)
    batch = bkfac.Batch(bat_layers, N, dtype)
    for step in range(3):
        XA, XG, G = batches(dtype, step)
        S_ref, S_bat = out_like(G), out_like(G)
        for l, (a, g) in enumerate(ref):
            for f, X in ((a, XA[l]), (g, XG[l])):
                (bkfac.bkfac_init(f, X) if f.r_cur == 0 else bkfac.bkfac_update(f, X, 0.95))
            bkfac.bkfac_apply(a, g, lam[l], lam[l] * 0.5, G[l], S_ref[l])
        batch.update(XA, XG, 0.95)
        batch.apply(G, S_bat, lam, [x * 0.5 for x in lam])
        st = bkfac.bkfac_status()
        assert st == bkfac.OK, bkfac.strerror(st)
        for l in range(len(LAYERS)):
            assert torch.equal(S_ref[l], S_bat[l]), (step, l)
            assert torch.equal(ref[l][0].U, bat_layers[l][0].U) and torch.equal(ref[l][1].sigma, bat_layers[l][1].sigma)
    batch.sync_descriptors()
    assert [f.r_cur for ab in bat_layers for f in ab] == [f.r_cur for ab in ref for f in ab]
    batch.close()


def test_graph_replay_equals_eager_step():
    dtype = bkfac.F32
    lam = [0.1, 0.05, 0.2]
    eager, graphed = make_layers(dtype), make_layers(dtype)
    be, bg = bkfac.Batch(eager, N, dtype), bkfac.Batch(graphed, N, dtype)
    XA, XG, G = batches(dtype, 0)
    # reach the steady rank (r_cur == r) before capturing
    for b in (be, bg):
        for _ in range(3):
            b.update(XA, XG, 0.95)
    XA, XG, G = batches(dtype, 1)
    Se, Sg = out_like(G), out_like(G)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for t in range(3):
            be.update(XA, XG, 0.95)
            be.apply(G, Se, lam, lam)
            if t == 0:
                bg.step_graph(XA, XG, 0.95, G, Sg, lam, lam, capture=True)
            else:
                bg.step_graph()
    stream.synchronize()
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    for l in range(len(LAYERS)):
        assert torch.equal(Se[l], Sg[l])
        assert torch.equal(eager[l][0].U, graphed[l][0].U)
    bg.sync_descriptors()
    be.sync_descriptors()
    assert graphed[0][0].step == eager[0][0].step
    be.close()
    bg.close()


def test_batch_one_step_matches_oracle(oracle):
    dtype = bkfac.F64
    layers = make_layers(dtype)
    batch = bkfac.Batch(layers, N, dtype)
    XA0, XG0, _ = batches(dtype, 0)
    batch.update(XA0, XG0, 0.95)
    batch.sync_descriptors()
    states = state_copy(layers)
    ranks = [(a.r_cur, g.r_cur) for a, g in layers]
    XA, XG, G = batches(dtype, 1)
    batch.update(XA, XG, 0.95)
    batch.sync_descriptors()
    for l, (dA, dG, r) in enumerate(LAYERS):
        for w, (X, d) in enumerate(((XA[l], dA), (XG[l], dG))):
            f = layers[l][w]
            U0, s0 = states[l][2 * w], states[l][2 * w + 1]
            k0 = ranks[l][w]
            upd = oracle.update_dense if f.r + N >= d else oracle.update
            Uo, so, info = upd(U0[:k0].cpu().numpy(), s0[:k0].cpu().numpy(), k0, X.cpu().numpy(), 0.95, f.r)
            k = info["r_new"]
            Ug, sg = f.state()
            assert rel(sg.cpu().numpy(), so[:k]) < 1e-10
            assert lowrank_rel_err(Ug.cpu().numpy(), sg.cpu().numpy(), Uo[:k], so[:k]) < 1e-10
    assert bkfac.bkfac_status() == bkfac.OK
    batch.close()


def test_autotune_writes_cache_and_keeps_parity(oracle, tmp_path):
    """bkfac_tune times the eigensolve's launch candidates and records the
    fastest; the update computes the same decomposition under the tuned shape."""
    cache = str(tmp_path / "tune.txt")
    d, r, n = 600, 48, 40
    f = bkfac.Factor(d, r, bkfac.F32)
    bkfac.bkfac_tune(f, n, cache)
    lines = open(cache).read().split()
    assert len(lines) >= 6 and int(lines[0]) in (r + n,) and int(lines[1]) == r + n
    X0 = synth.powerlaw_batch(d, n, 1.2, 41, 0)
    X1 = synth.powerlaw_batch(d, n, 1.2, 41, 1)
    xs = []
    for X in (X0, X1):
        t = bkfac.cols_tensor(n, d, torch.float32)
        t.copy_(torch.from_numpy(X))
        xs.append(t)
    bkfac.bkfac_init(f, xs[0])
    U0, s0 = (v.clone() for v in f.state())
    bkfac.bkfac_update(f, xs[1], 0.95)
    assert bkfac.bkfac_status() == bkfac.OK
    Uo, so, info = oracle.update(U0.double().cpu().numpy(), s0.cpu().numpy(), U0.shape[0],
                                 xs[1].double().cpu().numpy(), 0.95, r)
    Ug, sg = f.state()
    assert rel(sg.cpu().numpy(), so[: f.r_cur]) < 1e-4
    assert lowrank_rel_err(Ug.double().cpu().numpy(), sg.cpu().numpy(), Uo[: f.r_cur], so[: f.r_cur]) < 1e-4
