"""The C-ABI library loads and exports every function include/bkfac.h declares
(no GPU needed: loading the shared library does not touch the device)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bkfac.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bkfac_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_documented_calls():
    names = declared_functions()
    for n in ("bkfac_init", "bkfac_update", "bkfac_apply", "bkfac_reorth", "bkfac_status", "bkfac_strerror",
              "bkfac_workspace_size", "bkfac_batch_create", "bkfac_batch_update", "bkfac_batch_apply",
              "bkfac_batch_step_graph", "bkfac_batch_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2210_08494_gb300 import bkfac

    lib = bkfac.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_host_side_calls_without_gpu():
    """Calls that never touch the device: version, strerror, workspace sizing,
    argument validation (an invalid call returns EINVAL before any launch)."""
    import ctypes

    from paper_2210_08494_gb300 import bkfac

    lib = bkfac.load()
    assert lib.bkfac_version() >= 100
    assert lib.bkfac_strerror(bkfac.EINVAL).decode() == "invalid argument"
    f = bkfac.bkfac_factor(4097, 256, 0, bkfac.F32, 0x10000, 4128, 0x20000, 0, 0, 0)
    ws = lib.bkfac_workspace_size(ctypes.byref(f), 256, bkfac.OP_UPDATE)
    assert ws > 4097 * 256 * 4 * 3
    assert lib.bkfac_workspace_size(ctypes.byref(f), 0, bkfac.OP_UPDATE) == 0
    bad = bkfac.bkfac_factor(10, 11, 0, bkfac.F32, 0x10000, 12, 0x20000, 0, 0, 0)  # r > d
    assert lib.bkfac_workspace_size(ctypes.byref(bad), 4, bkfac.OP_UPDATE) == 0
    misaligned = bkfac.bkfac_factor(10, 4, 0, bkfac.F32, 0x10000, 10, 0x20000, 0, 0, 0)  # ld*4 % 16 != 0
    assert lib.bkfac_workspace_size(ctypes.byref(misaligned), 4, bkfac.OP_UPDATE) == 0
    # update with r_cur == 0 is refused before anything is enqueued
    rc = lib.bkfac_update(ctypes.byref(f), ctypes.c_void_p(0x30000), 4128, 256, 0.95, ctypes.c_void_p(0x40000),
                          ws, None)
    assert rc == bkfac.EINVAL
