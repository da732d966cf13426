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


def test_factored_apply_host_checks_without_gpu():
    """Workspace sizing and argument validation of the linear inverse application
    (Algorithm 8); invalid calls return EINVAL before anything is enqueued."""
    import ctypes

    from paper_2210_08494_gb300 import bkfac

    lib = bkfac.load()
    fA = bkfac.bkfac_factor(4097, 256, 256, bkfac.F32, 0x10000, 4128, 0x20000, 0, 0, 0)
    fG = bkfac.bkfac_factor(4096, 256, 256, bkfac.F32, 0x10000, 4096, 0x20000, 0, 0, 0)
    ws = lib.bkfac_apply_factored_workspace_size(ctypes.byref(fA), ctypes.byref(fG), 256)
    assert ws >= 2 * 256 * 256 * 4
    assert lib.bkfac_apply_factored_workspace_size(ctypes.byref(fA), ctypes.byref(fG), 0) == 0
    P = ctypes.c_void_p
    args = dict(XA=P(0x30000), ldxa=4128, XG=P(0x50000), ldxg=4096, n=256, PA=P(0x70000), ldpa=4128,
                PG=P(0x90000), ldpg=4096)

    def call(**kw):
        a = dict(args, **kw)
        return lib.bkfac_apply_factored(ctypes.byref(fA), ctypes.byref(fG), 1e-2, 1e-2, a["XA"], a["ldxa"], a["XG"],
                                        a["ldxg"], a["n"], a["PA"], a["ldpa"], a["PG"], a["ldpg"], 1.0, None, 0, 0,
                                        P(0x100000), ws, None)

    assert call(XA=P(0x30004)) == bkfac.EINVAL        # misaligned base
    assert call(ldxa=4097) == bkfac.EINVAL            # leading dimension not 16-byte aligned
    assert call(ldpg=4000) == bkfac.EINVAL            # ld < d
    assert call(n=0) == bkfac.EINVAL
    assert call(PA=P(0x30000), ldpa=4160) == bkfac.EINVAL  # in place with another ld
