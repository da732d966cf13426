"""bkfac_apply_noalloc -- the damped inverse application for callers that
cannot allocate device memory -- against bkfac_apply with a caller workspace.

The entry point keeps its scratch in a fixed device array inside the library
instead of taking a workspace, so that code which cannot call cudaMalloc
(inside a graph capture that forbids synchronising calls, or under a framework
that owns all device memory) can still precondition a gradient.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2210_08494_gb300 import bkfac, synth

pytestmark = pytest.mark.gpu

TOL = {bkfac.F64: 1e-10, bkfac.F32: 1e-4}


def _factor(d, r, dtype, seed):
    f = bkfac.Factor(d, r, dtype)
    Ut = synth.orthonormal_columns(d, r, seed)
    sig = np.sort(2.0 * np.exp(-np.linspace(0, 5, r)))[::-1].copy()
    f.load_state(torch.from_numpy(Ut).to(f.torch_dtype).cuda(), torch.from_numpy(sig).cuda())
    return f


def _noalloc(lib, fA, fG, lamA, lamG, G, S, flags=0):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bkfac_apply_noalloc(ctypes.byref(fA.desc), ctypes.byref(fG.desc), ctypes.c_double(lamA),
                                   ctypes.c_double(lamG), ctypes.c_void_p(G.data_ptr()), G.stride(0),
                                   ctypes.c_void_p(S.data_ptr()), S.stride(0), flags, stream)


@pytest.mark.parametrize("dtype,dA,rA,dG,rG", [(bkfac.F32, 4097, 256, 4096, 256), (bkfac.F64, 513, 64, 300, 48)])
def test_noalloc_matches_workspace_apply_twice(dtype, dA, rA, dG, rG):
    assert torch.cuda.is_available()
    lib = bkfac.load()
    bkfac.bkfac_status()
    fA = _factor(dA, rA, dtype, 31)
    fG = _factor(dG, rG, dtype, 32)
    assert bkfac.bkfac_apply_workspace_size(fA, fG) <= 32 * 1024 * 1024
    for call, (seed, flags) in enumerate(((33, 0), (34, bkfac.SPECTRUM_CONTINUATION))):
        G = bkfac.grad_tensor(dG, dA, fA.torch_dtype)
        G.copy_(torch.from_numpy(synth.gradient(dG, dA, seed, call)))
        S_ref = bkfac.grad_tensor(dG, dA, fA.torch_dtype)
        S_new = bkfac.grad_tensor(dG, dA, fA.torch_dtype)
        bkfac.bkfac_apply(fA, fG, 1e-2, 3e-2, G, S_ref, flags=flags)
        rc = _noalloc(lib, fA, fG, 1e-2, 3e-2, G, S_new, flags)
        assert rc == bkfac.OK, bkfac.strerror(rc)
        st = bkfac.bkfac_status()
        assert st == bkfac.OK, bkfac.strerror(st)
        ref = S_ref.double()
        err = float(torch.linalg.norm(S_new.double() - ref) / torch.linalg.norm(ref))
        assert err < TOL[dtype], (call, err)


def test_noalloc_rejects_pairs_beyond_its_scratch():
    lib = bkfac.load()
    fA = bkfac.Factor(8192, 1024, bkfac.F32)
    fG = bkfac.Factor(8192, 1024, bkfac.F32)
    assert bkfac.bkfac_apply_workspace_size(fA, fG) > 32 * 1024 * 1024
    G = bkfac.grad_tensor(4, 4, torch.float32)
    rc = _noalloc(lib, fA, fG, 1e-2, 1e-2, G, G)
    assert rc == bkfac.EWORKSPACE
    assert bkfac.bkfac_status() == bkfac.OK
