"""The autotuner's cache file (host logic, no GPU): eigensolve lines ("rows cols
prec b dsm ms"), grouped-eigensolve lines ("G rows cols prec count b dsm ms")
and product lines ("M M N K0 K1 layout kernel splits ms") are read into the
process-wide tables and written back; malformed or out-of-range lines are
dropped.  Ending a GEMM tuning session with no product noted makes no device
call, so the round trip runs on the CPU.  The shapes used here occur in no
other test (the tables are process-wide)."""
import pytest

from paper_2210_08494_gb300 import bkfac

VALID = [
    "997 997 1 16 1 3.2500",
    "G 995 995 1 7 8 0 4.7500",
    "M 123 45 67 0 4 2 3 0.0270",
    "M 321 54 76 8 3 1 1 0.0130",
]
INVALID = [
    "M 123 45 67 0 4 3 1 0.1000",    # kernel must be 1 or 2
    "M 123 45 67 0 4 1 0 0.1000",    # at least one split
    "M 0 45 67 0 4 1 1 0.1000",      # empty output
    "G 995 995 1 0 8 0 1.0000",      # a group has at least one problem
    "997 997 1 33 1 1.0000",         # block width at most 32
    "997 997 2 16 1 1.0000",         # precision 0 or 1
    "not a line",
]


def test_tune_cache_round_trip(tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("\n".join(VALID + INVALID) + "\n")
    bkfac.bkfac_gemm_tune_begin()
    bkfac.bkfac_gemm_tune_end(str(path))  # reads the file, tunes nothing new, writes the tables back
    out = [ln.strip() for ln in path.read_text().splitlines() if ln.strip()]
    for ln in VALID:
        assert ln in out, (ln, out)
    for ln in INVALID:
        assert ln not in out, (ln, out)
    # each line once, whatever else the tables hold
    assert len(out) == len(set(out))


def test_tune_cache_missing_file_is_created(tmp_path):
    path = tmp_path / "fresh.txt"
    bkfac.bkfac_gemm_tune_begin()
    bkfac.bkfac_gemm_tune_end(str(path))
    assert path.exists()
