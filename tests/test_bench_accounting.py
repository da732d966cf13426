"""The benchmark's roofline arithmetic (host logic, no GPU): the composed step
bound takes, per phase, the longer of its work at its pipe's peak and its bytes
at the HBM peak, and sums over the phases; the per-phase work lists switch to
the dense path when r + n >= d and hold the preconditioning Cholesky only for
FP32 eigensolves of 128 columns or more."""
import math

import bench

PEAKS = {"fp32": 1e13, "fp64": 1e12, "bf16": 1e15, "hbm": 6.8e12}


def test_composed_bound_takes_the_longer_side_of_each_phase():
    items = [("compute", 1e12, 0.0, "fp32"),          # 0.1 s of FP32 work
             ("stream", 0.0, 6.8e9, "hbm"),           # 1 ms of HBM traffic
             ("both", 1e9, 6.8e10, "bf16")]           # 1 us of BF16 work, 10 ms of traffic
    r = bench.composed_roofline(items, 222.0, PEAKS, {})
    assert math.isclose(r["bound_ms"], 100.0 + 1.0 + 10.0, rel_tol=1e-12)
    assert math.isclose(r["frac"], 111.0 / 222.0, rel_tol=1e-12)
    assert math.isclose(r["bound_ms_by_pipe"]["fp32"], 100.0, rel_tol=1e-12)
    assert math.isclose(r["bound_ms_by_pipe"]["hbm"], 11.0, rel_tol=1e-12)
    assert "bf16" not in r["bound_ms_by_pipe"]


def test_update_work_paths_and_precondition():
    dense = bench.update_work(d=300, k=100, n=256, r=100, prec="f32", sweeps=8)
    assert [it[0] for it in dense] == ["dense_jacobi"]
    brand = dict((it[0], it) for it in bench.update_work(d=4097, k=256, n=256, r=256, prec="f32", sweeps=8))
    assert "precond" in brand and brand["jacobi"][3] == "fp32"
    # eigensolve work grows with the sweeps, the products with d
    more = dict((it[0], it) for it in bench.update_work(d=4097, k=256, n=256, r=256, prec="f32", sweeps=9))
    assert math.isclose(more["jacobi"][1] / brand["jacobi"][1], 9 / 8)
    wide = dict((it[0], it) for it in bench.update_work(d=8194, k=256, n=256, r=256, prec="f32", sweeps=8))
    assert math.isclose(wide["proj"][1] / brand["proj"][1], 2.0)
    # an FP64 eigensolve has no preconditioning Cholesky, and the mixed products run on BF16
    f64eig = dict((it[0], it) for it in bench.update_work(4097, 256, 256, 256, "mixed", 8, eig64=True))
    assert "precond" not in f64eig and f64eig["jacobi"][3] == "fp64" and f64eig["proj"][3] == "bf16"
    small = dict((it[0], it) for it in bench.update_work(d=600, k=40, n=32, r=40, prec="f32", sweeps=8))
    assert "precond" not in small  # N = 72 < 128


def test_apply_work_two_passes():
    p1, p2 = bench.apply_work(4097, 4096, 256, 256, "f32")
    assert p1[0] == "apply_pass1" and p2[0] == "apply_pass2"
    assert p1[1] == p2[1] == 2.0 * 4096 * 4097 * 512
    assert p2[2] == 2 * p1[2] == 2 * 4 * 4096 * 4097
