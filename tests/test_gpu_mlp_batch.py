"""GPU parity of the batched step on the full synthetic preconditioning
workload: an 8-layer ReLU MLP of width 4096 (input 4096, output 10), minibatch
n = 256, r = 220, rho = 0.95, lambda = 1e-2 -- the shapes the benchmark's MLP
arm times: seven layers with A at d = 4097 and Gamma at d = 4096 (Brand cores of
N = r + n = 476, a core size whose padding and register blocking differ from
the 512 of the wide layer), and the output layer whose Gamma (d = 10) takes the
dense path.  Activations and per-sample pre-activation gradients come from the
seeded random-init MLP on N(0, 1) inputs (synth.mlp_batches).

Every factor and every layer is checked after one captured-graph replay: the
oracle repeats the step from the GPU's state on the same batches
(tests.parity_util.judge_step) and applies the damped inverses of the updated
states to each layer's weight gradient, compared in relative Frobenius norm and
element by element.  Tolerances: 1e-4 for FP32, 1e-2 for one mixed BF16 update;
the mixed inverse application is held to its stated bound
(tests.parity_util.mixed_apply_bound), which grows with the damped condition
sigma / lambda of the factors because an MLP layer's gradient lies largely in
their spans.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import judge_step, mixed_apply_bound, rel

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

WIDTHS = [4096] * 8 + [10]
R, N, RHO, LAM = 220, 256, 0.95, 1e-2
TOL = {bkfac.F32: 1e-4, bkfac.MIXED_BF16: 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


@pytest.fixture(scope="module")
def batches():
    """Four steps of (activations, gradients, weight gradients) on the device."""
    dev = torch.device("cuda")
    out = []
    for t in range(4):
        acts, grads, wgrads = synth.mlp_batches(WIDTHS, N, 5000, 5001, t, device=dev)
        out.append((acts, grads, wgrads))
    return out


@pytest.mark.parametrize("dtype", [bkfac.F32, bkfac.MIXED_BF16])
def test_mlp_batch_graph_step_matches_oracle(oracle, batches, dtype):
    L = len(WIDTHS) - 1
    layers = [(bkfac.Factor(WIDTHS[l] + 1, min(R, WIDTHS[l] + 1), dtype),
               bkfac.Factor(WIDTHS[l + 1], min(R, WIDTHS[l + 1]), dtype)) for l in range(L)]
    batch = bkfac.Batch(layers, N, dtype)
    acts0, grads0, w0 = batches[0]
    XA = [bkfac.cols_tensor(N, a.shape[1], torch.float32) for a in acts0]
    XG = [bkfac.cols_tensor(N, g.shape[1], torch.float32) for g in grads0]
    G = [bkfac.grad_tensor(w.shape[0], w.shape[1], torch.float32) for w in w0]
    S = [bkfac.grad_tensor(w.shape[0], w.shape[1], torch.float32) for w in w0]
    lam = [LAM] * L

    def load(t):
        acts, grads, wg = batches[t]
        for l in range(L):
            XA[l].copy_(acts[l])
            XG[l].copy_(grads[l])
            G[l].copy_(wg[l])

    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for t in range(2):
            load(t)
            batch.update(XA, XG, RHO)
        load(2)
        batch.step_graph(XA, XG, RHO, G, S, lam, lam, capture=True)
    stream.synchronize()
    assert bkfac.bkfac_status() == bkfac.OK
    batch.sync_descriptors()
    before = {}
    for l in range(L):
        for w in (0, 1):
            U, s = layers[l][w].state()
            before[(l, w)] = (U.double().cpu().numpy(), s.cpu().numpy())
    with torch.cuda.stream(stream):
        load(3)
        batch.step_graph()
    stream.synchronize()
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)
    batch.sync_descriptors()
    tol = TOL[dtype]
    report, failures = [], []
    for l in range(L):
        post = []
        for w in (0, 1):
            f = layers[l][w]
            d = f.d
            U0, s0 = before[(l, w)]
            X = (XA if w == 0 else XG)[l][:, :d].double().cpu().numpy()  # the values the GPU received
            upd = oracle.update_dense if f.r + N >= d else oracle.update
            kin = U0.shape[0]
            Uo, so, info = upd(U0, s0, kin, X, RHO, min(kin + N, d))
            k = min(f.r, info["r_new"])
            assert f.r_cur == k
            U, s = f.state()
            Ug, sg = U.double().cpu().numpy(), s.cpu().numpy()
            try:
                m = judge_step(Ug, sg, Uo[: info["r_new"]], so[: info["r_new"]], k, dtype, tol,
                               orth_tol=1e-4 if dtype == bkfac.F32 else 2e-2)
                report.append("layer %d %s d=%d r=%d: sigma %.2e per-mode %.2e reconstruction %.2e%s"
                              % (l, "AG"[w], d, f.r, m["sigma"], m["mode"], m["recon"],
                                 " (near tie)" if m["tie"] else ""))
            except AssertionError as e:
                failures.append(f"layer {l} {'AG'[w]}: {e}")
            post.append((Ug[:k], sg[:k]))
        (UA, sA), (UG, sG) = post
        Gn = G[l].double().cpu().numpy()
        So = oracle.apply(UA, sA, LAM, UG, sG, LAM, Gn)
        Sg = S[l].double().cpu().numpy()
        ea = rel(Sg, So)
        em = float(np.abs(Sg - So).max() / np.abs(So).max())
        # mixed: the stated bound grows with sigma / lambda when the layer's gradient lies in
        # the span of its factors (tests.parity_util.mixed_apply_bound); element-wise within
        # ten times the Frobenius bound
        ta = tol if dtype == bkfac.F32 else mixed_apply_bound(Gn, So, LAM, LAM)
        report.append("layer %d apply %d x %d gradient: %.2e (elementwise %.2e, bound %.1e)"
                      % (l, Gn.shape[0], Gn.shape[1], ea, em, ta))
        if not (ea < ta and em < 10 * ta):
            failures.append(f"layer {l} apply: {ea:.2e} / elementwise {em:.2e} (bound {ta:.1e})")
    print("\n".join(report))
    batch.close()
    assert not failures, failures
