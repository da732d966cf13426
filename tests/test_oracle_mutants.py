"""The oracle's pins are not blind: plant plausible mistakes in a copy of the
oracle's C source (on the CPU), rebuild it, and check that the pin suite fails
for every mutant while passing for the unmodified source."""
import inspect
import os
import tempfile

import pytest

import oracle as oracle_mod
from tests import test_oracle_pins as pins

MUTANTS = [
    ("core scaling sqrt(c) -> c (Eq. (7) substitution)", "double sc = sqrt(c);", "double sc = c;"),
    ("EA decay rho dropped from the core", "Dg[i] = rho * sigma[i];", "Dg[i] = sigma[i];"),
    ("Jacobi rotation sign", "AT(A, lda, i, p) = c * aip - s * aiq;", "AT(A, lda, i, p) = c * aip + s * aiq;"),
    ("Householder vector sign", "v[s] = v0;", "v[s] = -v0;"),
    ("residual sign P = X + U M", "P[(size_t)i + (size_t)j * d] = s - um;", "P[(size_t)i + (size_t)j * d] = s + um;"),
    ("transposed V in the rotation [U Q] V",
     "Q[(size_t)i + (size_t)l * d] * V[(size_t)(k + l) + (size_t)j * N]",
     "Q[(size_t)i + (size_t)l * d] * V[(size_t)j + (size_t)(k + l) * N]"),
    ("apply: g * lam instead of g / lam", "t[j] = g[j] / lA;", "t[j] = g[j] * lA;"),
    ("apply: damped coefficient misses -1/lam",
     "coef[i] = 1.0 / ((sigma[i] - shift) + l) - 1.0 / l;", "coef[i] = 1.0 / ((sigma[i] - shift) + l);"),
    ("eigenvalues sorted ascending", "(best < 0 || lam[i] > lam[best])", "(best < 0 || lam[i] < lam[best])"),
    ("linear apply: damped column misses its x / lam term", "for (int i = 0; i < d; ++i) p[i] = x[i] / l;",
     "for (int i = 0; i < d; ++i) p[i] = 0.0;"),
    ("linear apply: the step's scale alpha dropped", "srow[j] = alpha * acc;", "srow[j] = acc;"),
    ("relative damping scaled by the smallest eigenvalue", "if (sigma[i] > top) top = sigma[i];",
     "if (sigma[i] < top) top = sigma[i];"),
    ("EA factor: (1 - rho) dropped from the new term", "const double c = first ? 1.0 / n : (1.0 - rho) / n;",
     "const double c = first ? 1.0 / n : 1.0 / n;"),
    ("correction: projects M^2 instead of M", "mat_tn(n_crc, n_crc, d, Us, d, MU, d, Ms, n_crc);",
     "mat_tn(n_crc, n_crc, d, MU, d, MU, d, Ms, n_crc);"),
    ("correction: modes not re-sorted", "rc = sort_modes(d, k, U, ldu, sigma);", "rc = BKO_OK;"),
    ("RSVD: core Q^T Q instead of Q^T M Q", "mat_tn(l, l, d, Q, d, Y, d, B, l);", "mat_tn(l, l, d, Q, d, Q, d, B, l);"),
    ("dense path: rho applied to X X^T instead of U S U^T",
     "K[(size_t)i + (size_t)j * d] = s + c * t;", "K[(size_t)i + (size_t)j * d] = s / rho + rho * c * t;"),
]


def _pin_calls():
    calls = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_") or name == "test_pins_catch_a_planted_mistake":
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if not params:
            calls.append((name, fn, {}))
            continue
        argnames = [a.strip() for a in params[0].args[0].split(",")]
        for vals in params[0].args[1]:
            vals = vals if isinstance(vals, tuple) else (vals,)
            calls.append((f"{name}{vals}", fn, dict(zip(argnames, vals))))
    return calls


def _failures(lib_path):
    failed = []
    with oracle_mod.use_library(lib_path):
        for name, fn, kw in _pin_calls():
            try:
                fn(oracle_mod, **kw)
            except Exception:  # an assertion, a non-convergence or an error code
                failed.append(name)
    return failed


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


def test_unmodified_source_passes(workdir):
    lib = oracle_mod.build_variant(oracle_mod.source(), os.path.join(workdir, "orig.so"))
    assert _failures(lib) == []


@pytest.mark.parametrize("idx", range(len(MUTANTS)))
def test_mutant_is_caught(workdir, idx):
    what, old, new = MUTANTS[idx]
    src = oracle_mod.source()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
    lib = oracle_mod.build_variant(src.replace(old, new), os.path.join(workdir, f"mut{idx}.so"))
    failed = _failures(lib)
    assert failed, f"no pin caught the planted mistake: {what}"
