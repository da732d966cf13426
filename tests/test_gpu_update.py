"""GPU parity of the B-KFAC update (Algorithm 4 via Algorithm 3) and of the
re-orthonormalisation, through the C ABI, against the FP64 CPU oracle.

One-step parity: before each step the oracle starts from the GPU's state
(exact values up-cast to float64) and both sides consume the same seeded
batch (rounded to the path's dtype), so each step's tolerance applies to that
step alone.  Trajectory parity: both run free from the same first batch.

Tolerances (relative Frobenius): 1e-10 for the FP64 path, 1e-4 for the FP32
path, 1e-2 for one step of the mixed BF16 path (operand rounding u_bf16 = 2^-8
in each tall-skinny product, FP32 accumulation: a one-step result moves by a
few tenths of u_bf16 to about u_bf16; 1e-2 is 2.5 u_bf16).  Each step is
judged by tests.parity_util.judge_step: relative sigma and reconstruction
errors, every eigenvalue within the path's Weyl bound, the top-j subspaces at
gapped indices within their Davis-Kahan bound, and the near-tie reading at the
truncation index.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth
from tests.parity_util import judge_step, lowrank_rel_err, orth_err, rel, truncation_gap

pytestmark = pytest.mark.gpu

TOL = {bkfac.F64: 1e-10, bkfac.F32: 1e-4, bkfac.MIXED_BF16: 1e-2}
ORTH = {bkfac.F64: 1e-12, bkfac.F32: 2e-5, bkfac.MIXED_BF16: 2e-2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    bkfac.load()
    bkfac.bkfac_status()
    yield


def to_dev(Xt, f):
    """(n, d) float64 numpy batch -> (n, d) device view with padded rows, f's dtype."""
    n, d = Xt.shape
    t = bkfac.cols_tensor(n, d, f.torch_dtype)
    t.copy_(torch.from_numpy(Xt))
    return t


def rounded(Xt, f):
    """The exact values the GPU receives, as float64."""
    return torch.from_numpy(Xt).to(f.torch_dtype).double().numpy()


def gpu_state(f):
    U, s = f.state()
    return U.double().cpu().numpy(), s.cpu().numpy()


def check_status():
    st = bkfac.bkfac_status()
    assert st == bkfac.OK, bkfac.strerror(st)


def one_step_parity(oracle, d, r, n, dtype, rho=0.95, steps=4, alpha=1.5, seed=1, flags=0, orth=None, tol=None):
    """Init, then `steps` updates; before each update the oracle starts from the GPU's
    state.  The oracle keeps every mode (no truncation) so that the truncation gap and
    the per-mode bounds can be judged; returns (factor, worst relative error)."""
    f = bkfac.Factor(d, r, dtype, flags=flags)
    dense = r + n >= d
    tol = TOL[dtype] if tol is None else tol
    orth_tol = ORTH[dtype] if orth is None else orth
    X0 = synth.powerlaw_batch(d, n, alpha, seed, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    check_status()
    Uo, so, info = oracle.init(rounded(X0, f), min(n, d), dense=dense)
    Ug, sg = gpu_state(f)
    k = min(r, info["r_new"])
    assert f.r_cur == k
    m = judge_step(Ug, sg, Uo[:info["r_new"]], so[:info["r_new"]], k, dtype, tol)
    worst, ties, mode = max(m["sigma"], m["recon"]), int(m["tie"]), m["mode"]
    for t in range(1, steps + 1):
        Ug, sg = gpu_state(f)
        X = synth.powerlaw_batch(d, n, alpha, seed, t)
        bkfac.bkfac_update(f, to_dev(X, f), rho)
        check_status()
        upd = oracle.update_dense if dense else oracle.update
        kin = Ug.shape[0]
        full = min(kin + n, d)
        Uo, so, info = upd(Ug, sg, kin, rounded(X, f), rho, full)
        k = min(r, info["r_new"])
        assert f.r_cur == k
        U2, s2 = gpu_state(f)
        m = judge_step(U2, s2, Uo[:info["r_new"]], so[:info["r_new"]], k, dtype, tol, orth_tol=orth_tol)
        worst = max(worst, m["sigma"], m["recon"])
        ties += int(m["tie"])
        mode = max(mode, m["mode"])
    print(f"d={d} r={r} n={n} dtype={dtype}: worst {worst:.2e}, per-mode {mode:.2e}, near ties {ties}")
    return f, worst


@pytest.mark.parametrize("d,r,n", [(300, 24, 20), (65, 7, 3), (512, 64, 32)])
def test_update_f64_one_step(oracle, d, r, n):
    one_step_parity(oracle, d, r, n, bkfac.F64, steps=5)


@pytest.mark.parametrize("d,r,n", [(600, 48, 40), (257, 16, 33)])
def test_update_f32_one_step(oracle, d, r, n):
    one_step_parity(oracle, d, r, n, bkfac.F32, alpha=1.2, steps=4)


def test_update_f32_with_fp64_eigensolve(oracle):
    one_step_parity(oracle, 400, 32, 24, bkfac.F32, alpha=1.2, steps=3, flags=bkfac.FLAG_EIG_FP64)


def test_update_f32_tf32x3_one_step(oracle):
    """F32 factor with its tall-skinny products as 3xTF32 on the tensor cores."""
    # U' = [U Q] V carries the products' ~1e-5 relative error: orthonormality to the
    # path's tolerance rather than the SIMT FP32 level
    _, worst = one_step_parity(oracle, 600, 48, 40, bkfac.F32, alpha=1.2, steps=3, flags=bkfac.FLAG_TF32X3,
                               orth=1e-4)
    print(f"3xTF32 one-step worst relative error {worst:.3e}")


def test_update_mixed_one_step(oracle):
    _, worst = one_step_parity(oracle, 700, 40, 48, bkfac.MIXED_BF16, alpha=1.2, steps=3)
    print(f"mixed one-step worst relative error {worst:.3e}")


@pytest.mark.parametrize("d,r,n,dtype", [(300, 24, 1, bkfac.F32), (300, 1, 16, bkfac.F32), (64, 1, 1, bkfac.F64),
                                          (129, 2, 3, bkfac.F64)])
def test_update_edge_ranks(oracle, d, r, n, dtype):
    """Degenerate shapes: a single new column per step, a rank-one factor."""
    one_step_parity(oracle, d, r, n, dtype, steps=3)


def test_update_largest_core(oracle):
    """The largest Brand core the FP32 eigensolve holds: N = r + n = 768 (1024-row
    padded columns, two 24-column blocks per CTA in 192 KB of shared memory, two
    columns per warp per register block, 16-CTA cluster)."""
    _, worst = one_step_parity(oracle, 2048, 384, 384, bkfac.F32, alpha=1.2, steps=1)
    print(f"N = 768 core: worst relative error {worst:.3e}")


def test_shapes_beyond_the_eigensolve_are_rejected():
    """N = 1024 with FP32 (two 32-column blocks of 1024 rows exceed the shared
    memory) and N = 640 with FP64 (more than 512 rows): no workspace size, and
    the update itself returns BKFAC_EINVAL before any launch."""
    for d, r, n, dtype in ((2048, 384, 640, bkfac.F32), (2048, 320, 320, bkfac.F64)):
        f = bkfac.Factor(d, r, dtype)
        assert bkfac.bkfac_workspace_size(f, n) == 0
        f.load_state(torch.from_numpy(synth.orthonormal_columns(d, r, 5)).to(f.torch_dtype).cuda(),
                     torch.ones(r, dtype=torch.float64).cuda())
        X = bkfac.cols_tensor(n, d, f.torch_dtype)
        with pytest.raises(bkfac.BkfacError) as e:
            bkfac.bkfac_update(f, X, 0.95, ws=bkfac.workspace(1 << 20))
        assert e.value.code == bkfac.EINVAL
    assert bkfac.bkfac_status() == bkfac.OK


@pytest.mark.parametrize("dtype", [bkfac.F64, bkfac.F32])
def test_dense_path_small_factor(oracle, dtype):
    """r + n >= d (the 10-way output layer's Gamma): explicit K, exact EVD."""
    one_step_parity(oracle, 10, 10, 32, dtype, steps=3)


def test_dense_path_wider(oracle):
    one_step_parity(oracle, 90, 64, 40, bkfac.F64, steps=2)


@pytest.mark.parametrize("d,r,n", [(10, 10, 256), (10, 10, 255), (12, 12, 500)])
def test_dense_path_wide_batch(oracle, d, r, n):
    """A 10-wide output layer's Gamma with a whole minibatch of columns: the
    eigensolve's column padding is at its largest (cluster of 16, block width
    rounded up to the register-blocking width)."""
    one_step_parity(oracle, d, r, n, bkfac.F32, steps=2)


def test_init_keeps_rank_n_when_n_below_r(oracle):
    f, _ = one_step_parity(oracle, 200, 30, 8, bkfac.F64, steps=3)
    assert f.r_cur == 30


def test_trajectory_f64_small_factor(oracle):
    """Small FP64 workload: A factor d=512, Gamma factor d=256, r=64, n=32,
    rho=0.95, alpha=1.5, both free-running for 50 steps on each side from the
    first batch's exact EVD; then (Gamma + 0.1 I)^-1 G (A + 0.1 I)^-1 for a
    256 x 512 N(0, 1) gradient, compared with the oracle's application on its
    own trajectory."""
    r, n, rho, steps = 64, 32, 0.95, 50
    sides = []
    for d, seed in ((512, 1000), (256, 1001)):
        f = bkfac.Factor(d, r, bkfac.F64)
        X0 = synth.powerlaw_batch(d, n, 1.5, seed, 0)
        bkfac.bkfac_init(f, to_dev(X0, f))
        Uo, so, info = oracle.init(X0, r)
        k = info["r_new"]
        min_gap = np.inf
        for t in range(1, steps + 1):
            X = synth.powerlaw_batch(d, n, 1.5, seed, t)
            bkfac.bkfac_update(f, to_dev(X, f), rho)
            Uo, so, info = oracle.update(Uo[:k], so[:k], k, X, rho, r)
            k = info["r_new"]
            min_gap = min(min_gap, truncation_gap(so, min(r, len(so) - 1)))
        check_status()
        Ug, sg = gpu_state(f)
        err = lowrank_rel_err(Ug, sg, Uo[:k], so[:k])
        print(f"d={d}: trajectory error after {steps} steps {err:.3e} (min truncation gap {min_gap:.2e})")
        # no step came within the FP64 near-tie threshold (1e3 u) of swapping the r-th mode
        assert min_gap > 1e3 * 2.0 ** -53
        assert err < 1e-10
        sides.append((f, Uo[:k], so[:k]))
    (fA, UA, sA), (fG, UG, sG) = sides
    Gn = synth.gradient(256, 512, 1002, 0)
    G = bkfac.grad_tensor(256, 512, torch.float64)
    G.copy_(torch.from_numpy(Gn))
    S = bkfac.grad_tensor(256, 512, torch.float64)
    bkfac.bkfac_apply(fA, fG, 0.1, 0.1, G, S)
    check_status()
    So = oracle.apply(UA, sA, 0.1, UG, sG, 0.1, Gn)
    ea = rel(S.cpu().numpy(), So)
    print(f"apply after {steps} steps: relative error {ea:.3e}")
    assert ea < 1e-10


def test_update_in_span_drops_residual(oracle):
    """X = U C: the residual vanishes, its pivots are dropped, the span is kept."""
    d, r, n = 256, 16, 8
    f = bkfac.Factor(d, r, bkfac.F64)
    X0 = synth.powerlaw_batch(d, 32, 1.5, 3, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    Ug, sg = gpu_state(f)
    C = np.random.default_rng(0).standard_normal((n, Ug.shape[0]))
    X = C @ Ug
    bkfac.bkfac_update(f, to_dev(X, f), 0.9)
    check_status()
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], X, 0.9, r)
    U2, s2 = gpu_state(f)
    assert lowrank_rel_err(U2, s2, Uo[: f.r_cur], so[: f.r_cur]) < 1e-10
    assert np.abs(U2 - (U2 @ Ug.T) @ Ug).max() < 1e-10


def test_update_duplicate_columns(oracle):
    d, r, n = 300, 20, 12
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, n, 1.2, 4, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    Ug, sg = gpu_state(f)
    X = synth.powerlaw_batch(d, n, 1.2, 4, 1)
    X[6:] = X[:6]
    bkfac.bkfac_update(f, to_dev(X, f), 0.95)
    check_status()
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], rounded(X, f), 0.95, r)
    U2, s2 = gpu_state(f)
    k = f.r_cur
    assert rel(s2, so[:k]) < 1e-4
    assert lowrank_rel_err(U2, s2, Uo[:k], so[:k]) < 1e-4


@pytest.mark.parametrize("dtype", [bkfac.F32, bkfac.MIXED_BF16])
def test_reorth_restores_orthonormality(oracle, dtype):
    d, r = 500, 40
    f = bkfac.Factor(d, r, dtype)
    Ut = synth.orthonormal_columns(d, r, 5)
    noisy = Ut + 1e-3 * np.random.default_rng(1).standard_normal(Ut.shape)
    sig = np.sort(np.exp(-np.linspace(0, 4, r)))[::-1].copy()
    f.load_state(torch.from_numpy(noisy).to(f.torch_dtype).cuda(), torch.from_numpy(sig).cuda())
    Uin, sin = gpu_state(f)
    bkfac.bkfac_reorth(f)
    check_status()
    Uo, so = oracle.reorth(Uin, sin)
    U2, s2 = gpu_state(f)
    assert orth_err(U2) < 2e-5
    assert rel(s2, so) < 1e-4
    assert lowrank_rel_err(U2, s2, Uo, so) < 1e-4


def test_nonfinite_input_sets_status():
    d, r, n = 128, 8, 8
    f = bkfac.Factor(d, r, bkfac.F32)
    X = synth.powerlaw_batch(d, n, 1.5, 6, 0)
    X[2, 5] = np.nan
    bkfac.bkfac_init(f, to_dev(X, f))
    assert bkfac.bkfac_status() == bkfac.ENONFINITE
    assert bkfac.bkfac_status() == bkfac.OK  # cleared by the read


def test_invalid_arguments_are_rejected_before_launch():
    f = bkfac.Factor(64, 8, bkfac.F32)
    X = bkfac.cols_tensor(4, 64, torch.float32)
    with pytest.raises(bkfac.BkfacError) as e:
        bkfac.bkfac_update(f, X, 0.95)  # r_cur == 0: init first
    assert e.value.code == bkfac.EINVAL
    with pytest.raises(bkfac.BkfacError) as e:
        bkfac.bkfac_init(f, X, ws=bkfac.workspace(64))
    assert e.value.code == bkfac.EWORKSPACE
    with pytest.raises(bkfac.BkfacError) as e:
        bkfac.bkfac_init(f, torch.zeros(4, 63, device="cuda"))  # ld 63 floats is not 16-byte aligned
    assert e.value.code == bkfac.EINVAL
    assert bkfac.bkfac_status() == bkfac.OK


def test_wide_layer_full_size_one_step(oracle):
    """One wide FC layer's A factor (d = 4097, r = n = 256, FP32, rho = 0.95, alpha =
    1.2), in the launch configuration the benchmark times: init on the GPU,
    then one update compared with the oracle started from the GPU state."""
    d, r, n, rho = 4097, 256, 256, 0.95
    f = bkfac.Factor(d, r, bkfac.F32)
    X0 = synth.powerlaw_batch(d, n, 1.2, 2000, 0)
    bkfac.bkfac_init(f, to_dev(X0, f))
    check_status()
    Ug, sg = gpu_state(f)
    X = synth.powerlaw_batch(d, n, 1.2, 2000, 1)
    bkfac.bkfac_update(f, to_dev(X, f), rho)
    check_status()
    Uo, so, info = oracle.update(Ug, sg, Ug.shape[0], rounded(X, f), rho, r)
    U2, s2 = gpu_state(f)
    es, er = rel(s2, so), lowrank_rel_err(U2, s2, Uo, so)
    print(f"wide-layer one-step: sigma {es:.2e} reconstruction {er:.2e} orth {orth_err(U2):.2e}")
    assert es < 1e-4 and er < 1e-4
    assert orth_err(U2) < 1e-4
