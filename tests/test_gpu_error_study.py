"""The error study of the B-KFAC variants (Sec. 5) on the GPU.

* The single-layer study on drifting power-law statistics runs end to end, its
  metrics are well formed, and the light correction never increases the
  Frobenius error of the representation (the footnote to Algorithm 6).
* The study on every layer of a training ReLU MLP (the preconditioning
  workload's architecture, narrowed so the dense references stay small) is
  pinned to the FP64 oracle at its last step: the oracle's two-sided Jacobi
  eigendecomposition of each dense EA factor gives the exact damped inverse,
  its direct inverse application (Algorithm 1 with the complete basis) the
  reference step, and metrics 3 and 4 of Sec. 5.1 recomputed from those match
  the study's own values for every layer and every algorithm that keeps a
  representation.
"""
import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, error_study

pytestmark = pytest.mark.gpu


def test_error_study_short_run():
    assert torch.cuda.is_available()
    res = error_study.run(steps=20, heavy=5, dA=129, dG=96, r=24, n=16, verbose=False)
    for a, hist in res["history"].items():
        h = np.asarray(hist)
        assert np.all(np.isfinite(h)), a
        assert np.all(h[:, 3] >= -1e-6) and np.all(h[:, 3] <= 2.0), a
    # k-fac holds the exact inverse at its refresh steps
    kf = np.asarray(res["history"]["k-fac"])
    assert kf[0][0] < 1e-12 and kf[5][0] < 1e-12
    for before, after in res["correction_checks"]:
        assert after <= before * (1 + 1e-3)
    s = res["summary"]
    print({a: round(v["err_step"], 4) for a, v in s.items()})


def test_mlp_error_study_pinned_to_oracle(oracle):
    assert torch.cuda.is_available()
    phi = 0.1
    res = error_study.run_mlp(steps=8, heavy=4, width=96, depth=3, outputs=10, n=32, r=16, phi=phi,
                              verbose=False, keep_last=True)
    last = res["last"]
    n = res["config"]["n"]
    worst = 0.0
    for l, rec in enumerate(last["layers"]):
        lamA, VA, _ = oracle.jacobi_eig(rec["MA"])
        lamG, VG, _ = oracle.jacobi_eig(rec["MG"])
        # the exact damped inverse from the oracle's eigendecomposition against the study's reference
        exact_A = (VA / (lamA + phi * lamA.max())) @ VA.T
        assert np.linalg.norm(exact_A - error_study.exact_inverse(rec["MA"], phi)) <= 1e-10 * np.linalg.norm(exact_A)
        G = rec["XG"].T @ rec["XA"] / n
        s_ref = oracle.apply(VA.T.copy(), lamA, phi, VG.T.copy(), lamG, phi, G, relative=True)
        for a, st in rec["algos"].items():
            s = st["s"]
            m3 = float(np.linalg.norm(s - s_ref) / np.linalg.norm(s_ref))
            m4 = 1.0 - float(np.sum(s * s_ref) / (np.linalg.norm(s) * np.linalg.norm(s_ref)))
            got = last["per_layer"][a][l]
            assert abs(got[2] - m3) <= 1e-9 + 1e-7 * m3, (l, a, got[2], m3)
            assert abs(got[3] - m4) <= 1e-9 + 1e-6 * abs(m4), (l, a, got[3], m4)
            worst = max(worst, abs(got[2] - m3))
    for before, after in res["correction_checks"]:
        # the footnote's claim holds in exact arithmetic; FP32 rounding adds noise at
        # about u_32 of a column norm once the representation is already this close
        assert after <= before * (1 + 1e-3) + 1e-6, (before, after)
    h = np.asarray(res["history"]["b-kfac"])
    assert np.all(np.isfinite(h))
    print(f"MLP study: last-step metric 3 vs the oracle's reference, largest difference {worst:.2e}; means",
          {a: round(v["err_step"], 4) for a, v in res["summary"].items()})
