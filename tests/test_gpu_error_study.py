"""The error study of the B-KFAC variants (Sec. 5) runs end to end on the GPU,
its metrics are well formed, and the light correction never increases the
Frobenius error of the representation (the paper's footnote to Algorithm 6)."""
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
