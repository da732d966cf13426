"""Thin ctypes binding of libbkfac (include/bkfac.h).

Argument marshalling only: every step of the B-KFAC update and apply runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  If
the library is missing or a GPU is absent the calls raise -- there is no CPU
fallback.

Layout helpers: a d x m column-major matrix with leading dimension ld is a
torch tensor of shape (m, d) whose row stride is ld (``cols_tensor``); the
library requires ld * element_size to be a multiple of 16 bytes and a 16-byte
aligned base.  Gradients are (d_out, d_in) tensors with a padded row stride
(``grad_tensor``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

F64, F32, MIXED_BF16 = 0, 1, 2
OK, EINVAL, ENOTAPPLICABLE, ECHOL, ENOCONV, ENONFINITE, ETIMEOUT, ECUDA, EWORKSPACE, ENOMEM = range(10)
FLAG_EIG_FP64 = 1
FLAG_TF32X3 = 2
FLAG_KEEP_RN = 4
FLAG_CHOL_FP64 = 8
SPECTRUM_CONTINUATION = 1
DAMPING_RELATIVE = 2
OP_UPDATE, OP_REORTH = 0, 1

_TORCH_DTYPE = {F64: torch.float64, F32: torch.float32, MIXED_BF16: torch.float32}


class bkfac_factor(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("r", ctypes.c_int32), ("r_cur", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64), ("sigma", ctypes.c_void_p),
                ("step", ctypes.c_int64), ("flags", ctypes.c_uint32), ("r_extra", ctypes.c_int32)]


class bkfac_layer_desc(ctypes.Structure):
    _fields_ = [("A", bkfac_factor), ("G", bkfac_factor)]


class BkfacError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} (code {code})")
        self.code = code


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbkfac.so (building it first when missing).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libbkfac not built at {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        P, I, I64, D, S, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t, ctypes.c_uint32
        FP = ctypes.POINTER(bkfac_factor)
        sig = {
            "bkfac_version": ([], I),
            "bkfac_strerror": ([I], ctypes.c_char_p),
            "bkfac_status": ([P], I),
            "bkfac_workspace_size": ([FP, I, I], S),
            "bkfac_apply_workspace_size": ([FP, FP], S),
            "bkfac_init": ([FP, P, I64, I, P, S, P], I),
            "bkfac_update": ([FP, P, I64, I, D, P, S, P], I),
            "bkfac_reorth": ([FP, P, S, P], I),
            "bkfac_apply": ([FP, FP, D, D, P, I64, P, I64, U32, P, S, P], I),
            "bkfac_apply_noalloc": ([FP, FP, D, D, P, I64, P, I64, U32, P], I),
            "bkfac_apply_factored_workspace_size": ([FP, FP, I], S),
            "bkfac_ea_update": ([I, I, P, I64, P, I64, I, D, I, P], I),
            "bkfac_correct_workspace_size": ([FP, I], S),
            "bkfac_correct": ([FP, P, I64, ctypes.POINTER(ctypes.c_int32), I, P, S, P], I),
            "bkfac_rsvd_workspace_size": ([FP, I], S),
            "bkfac_rsvd": ([FP, P, I64, P, I64, I, I, P, S, P], I),
            "bkfac_apply_factored": ([FP, FP, D, D, P, I64, P, I64, I, P, I64, P, I64, D, P, I64, U32, P, S, P], I),
            "bkfac_debug_offsets": ([FP, I, ctypes.POINTER(ctypes.c_int64)], I),
            "bkfac_batch_create": ([ctypes.POINTER(bkfac_layer_desc), I, I, I, ctypes.c_char_p], P),
            "bkfac_batch_get_factor": ([P, I, I, FP], I),
            "bkfac_batch_update": ([P, ctypes.POINTER(P), ctypes.POINTER(I64), ctypes.POINTER(P),
                                    ctypes.POINTER(I64), D, P], I),
            "bkfac_batch_apply": ([P, ctypes.POINTER(P), ctypes.POINTER(I64), ctypes.POINTER(P),
                                   ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D), U32, P], I),
            "bkfac_batch_step_graph": ([P, ctypes.POINTER(P), ctypes.POINTER(I64), ctypes.POINTER(P),
                                        ctypes.POINTER(I64), D, ctypes.POINTER(P), ctypes.POINTER(I64),
                                        ctypes.POINTER(P), ctypes.POINTER(I64), ctypes.POINTER(D),
                                        ctypes.POINTER(D), U32, I, P], I),
            "bkfac_batch_destroy": ([P], None),
            "bkfac_batch_reorth": ([P, P], I),
            "bkfac_trace_enable": ([I], I),
            "bkfac_tune": ([FP, I, ctypes.c_char_p], I),
            "bkfac_gemm_tune_begin": ([], I),
            "bkfac_gemm_tune_end": ([ctypes.c_char_p], I),
            "bkfac_trace_read": ([ctypes.POINTER(D), ctypes.POINTER(I64), I, ctypes.POINTER(I64)], I),
            "bkfac_trace_phase_name": ([I], ctypes.c_char_p),
            "bkfac_set_sweep_cap": ([I], I),
            "bkfac_selftest_wait_timeout": ([I64, P], I),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols():
    """Names of the bkfac_* functions the loaded library exports (for the ABI tests)."""
    lib = load()
    names = []
    for n in ("bkfac_version", "bkfac_strerror", "bkfac_status", "bkfac_workspace_size",
              "bkfac_apply_workspace_size", "bkfac_init", "bkfac_update", "bkfac_reorth", "bkfac_apply",
              "bkfac_debug_offsets", "bkfac_batch_create", "bkfac_batch_get_factor", "bkfac_batch_update",
              "bkfac_batch_apply", "bkfac_batch_step_graph", "bkfac_batch_destroy", "bkfac_trace_enable",
              "bkfac_trace_read", "bkfac_trace_phase_name", "bkfac_apply_noalloc", "bkfac_tune", "bkfac_batch_reorth",
              "bkfac_apply_factored_workspace_size", "bkfac_apply_factored", "bkfac_ea_update",
              "bkfac_correct_workspace_size", "bkfac_correct", "bkfac_rsvd_workspace_size", "bkfac_rsvd",
              "bkfac_set_sweep_cap", "bkfac_selftest_wait_timeout", "bkfac_gemm_tune_begin",
              "bkfac_gemm_tune_end"):
        if hasattr(lib, n):
            names.append(n)
    return names


def strerror(code: int) -> str:
    try:
        return load().bkfac_strerror(int(code)).decode()
    except Exception:  # library not loadable: still give a readable message
        return f"error {code}"


def _check(rc: int, what: str):
    if rc != OK:
        raise BkfacError(rc, what)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _cols_ld(t: torch.Tensor) -> int:
    """Leading dimension of a (m, d) tensor viewed as a d x m column-major matrix."""
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D tensor with unit stride along its last dimension")
    return t.stride(0) if t.shape[0] > 1 else max(t.stride(0), t.shape[1])


def padded_ld(d: int, dtype: torch.dtype) -> int:
    """Smallest leading dimension >= d that keeps rows 16-byte aligned."""
    per = 16 // torch.tensor([], dtype=dtype).element_size()
    return (d + per - 1) // per * per


def cols_tensor(m: int, d: int, dtype, device="cuda", ld: int | None = None, zero: bool = True) -> torch.Tensor:
    """A (m, d) view of an (m, ld) buffer: m columns of length d, 16-byte aligned rows."""
    ld = ld or padded_ld(d, dtype)
    buf = (torch.zeros if zero else torch.empty)((max(m, 1), ld), dtype=dtype, device=device)
    return buf[:m, :d]


grad_tensor = cols_tensor  # (d_out, d_in) row-major gradient with padded rows


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A 256-byte aligned device byte buffer of at least nbytes."""
    t = torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)
    off = (-t.data_ptr()) % 256
    return t[off:off + max(int(nbytes), 1)]


class Factor:
    """Device state of one K-factor: U (d x r column-major, stored as an (r, ldu)
    tensor), sigma (r doubles) and the C descriptor the library updates."""

    def __init__(self, d: int, r: int, dtype: int = F32, device="cuda", flags: int = 0, r_extra: int = 0):
        self.d, self.r, self.dtype = int(d), int(r), int(dtype)
        self.r_extra = int(r_extra) if (int(flags) & FLAG_KEEP_RN) else 0
        tdt = _TORCH_DTYPE[self.dtype]
        self.U = cols_tensor(self.r + self.r_extra, self.d, tdt, device)
        self.sigma = torch.zeros(self.r + self.r_extra, dtype=torch.float64, device=device)
        self.desc = bkfac_factor(self.d, self.r, 0, self.dtype, self.U.data_ptr(), _cols_ld(self.U),
                                 self.sigma.data_ptr(), 0, int(flags), self.r_extra)
        self._ws = {}

    @property
    def r_cur(self) -> int:
        return int(self.desc.r_cur)

    @property
    def step(self) -> int:
        return int(self.desc.step)

    @property
    def torch_dtype(self):
        return _TORCH_DTYPE[self.dtype]

    def ws(self, n: int, op: int = OP_UPDATE) -> torch.Tensor:
        key = (op, n)
        if key not in self._ws:
            nb = bkfac_workspace_size(self, n, op)
            if nb == 0:
                raise BkfacError(EINVAL, "bkfac_workspace_size")
            self._ws[key] = workspace(nb, self.U.device)
        return self._ws[key]

    def state(self):
        """(U[:, :r_cur] as an (r_cur, d) tensor, sigma[:r_cur])."""
        k = self.r_cur
        return self.U[:k], self.sigma[:k]

    def load_state(self, Ut: torch.Tensor, sigma: torch.Tensor, step: int = 1):
        """Overwrite the state with k = len(sigma) modes (e.g. to resume or to seed a test)."""
        k = int(sigma.shape[0])
        self.U.zero_()
        self.sigma.zero_()
        self.U[:k].copy_(Ut[:k])
        self.sigma[:k].copy_(sigma)
        self.desc.r_cur = k
        self.desc.step = int(step)


# --------------------------------------------------------------------------- C ABI wrappers


def bkfac_version() -> int:
    return int(load().bkfac_version())


def bkfac_status(stream=None) -> int:
    return int(load().bkfac_status(_stream(stream)))


def bkfac_set_sweep_cap(cap: int) -> int:
    """Sets the Jacobi sweep cap of later eigensolves (0 = default); returns the previous cap."""
    prev = int(load().bkfac_set_sweep_cap(int(cap)))
    if prev < 0:
        raise BkfacError(-prev, "bkfac_set_sweep_cap")
    return prev


def bkfac_selftest_wait_timeout(limit_cycles: int, stream=None):
    """Runs the bounded-wait self-test (a wait that must time out); check bkfac_status()."""
    _check(load().bkfac_selftest_wait_timeout(int(limit_cycles), _stream(stream)), "bkfac_selftest_wait_timeout")


def bkfac_workspace_size(f: Factor, n: int, op: int = OP_UPDATE) -> int:
    return int(load().bkfac_workspace_size(ctypes.byref(f.desc), int(n), int(op)))


def bkfac_apply_workspace_size(fA: Factor, fG: Factor) -> int:
    return int(load().bkfac_apply_workspace_size(ctypes.byref(fA.desc), ctypes.byref(fG.desc)))


def bkfac_init(f: Factor, X: torch.Tensor, ws: torch.Tensor | None = None, stream=None):
    """X: (n, d) tensor view (n columns of length d) of f's dtype on the device."""
    n = X.shape[0]
    ws = f.ws(n) if ws is None else ws
    _check(load().bkfac_init(ctypes.byref(f.desc), _ptr(X), _cols_ld(X), n, _ptr(ws), ws.numel(), _stream(stream)),
           "bkfac_init")


def bkfac_update(f: Factor, X: torch.Tensor, rho: float, ws: torch.Tensor | None = None, stream=None):
    n = X.shape[0]
    ws = f.ws(n) if ws is None else ws
    _check(load().bkfac_update(ctypes.byref(f.desc), _ptr(X), _cols_ld(X), n, float(rho), _ptr(ws), ws.numel(),
                               _stream(stream)), "bkfac_update")


def bkfac_reorth(f: Factor, ws: torch.Tensor | None = None, stream=None):
    ws = f.ws(0, OP_REORTH) if ws is None else ws
    _check(load().bkfac_reorth(ctypes.byref(f.desc), _ptr(ws), ws.numel(), _stream(stream)), "bkfac_reorth")


def bkfac_apply(fA: Factor, fG: Factor, lamA: float, lamG: float, G: torch.Tensor, S: torch.Tensor,
                flags: int = 0, ws: torch.Tensor | None = None, stream=None):
    """G, S: (d_out, d_in) tensors with unit column stride (S may be G)."""
    if ws is None:
        key = ("apply", id(fG))
        if key not in fA._ws:
            fA._ws[key] = workspace(bkfac_apply_workspace_size(fA, fG), fA.U.device)
        ws = fA._ws[key]
    _check(load().bkfac_apply(ctypes.byref(fA.desc), ctypes.byref(fG.desc), float(lamA), float(lamG), _ptr(G),
                              G.stride(0), _ptr(S), S.stride(0), int(flags), _ptr(ws), ws.numel(), _stream(stream)),
           "bkfac_apply")


def bkfac_apply_factored(fA: Factor, fG: Factor, lamA: float, lamG: float, XA: torch.Tensor, XG: torch.Tensor,
                         PA: torch.Tensor, PG: torch.Tensor, alpha: float = 1.0, S: torch.Tensor | None = None,
                         flags: int = 0, ws: torch.Tensor | None = None, stream=None):
    """Linear inverse application (Algorithm 8) on the thin gradient factors.

    XA: (n, d_in) and XG: (n, d_out) column tensors (cols_tensor layout), PA / PG the
    outputs in the same layouts (may be XA / XG); S: (d_out, d_in) or None."""
    n = XA.shape[0]
    if ws is None:
        key = ("factored", id(fG), n)
        if key not in fA._ws:
            fA._ws[key] = workspace(load().bkfac_apply_factored_workspace_size(ctypes.byref(fA.desc),
                                                                               ctypes.byref(fG.desc), n), fA.U.device)
        ws = fA._ws[key]
    _check(load().bkfac_apply_factored(
        ctypes.byref(fA.desc), ctypes.byref(fG.desc), float(lamA), float(lamG), _ptr(XA), _cols_ld(XA), _ptr(XG),
        _cols_ld(XG), n, _ptr(PA), _cols_ld(PA), _ptr(PG), _cols_ld(PG), float(alpha),
        _ptr(S) if S is not None else None, S.stride(0) if S is not None else 0, int(flags), _ptr(ws), ws.numel(),
        _stream(stream)), "bkfac_apply_factored")


def dense_factor(d: int, dtype: int = F32, device="cuda") -> torch.Tensor:
    """A zeroed d x d dense EA factor (column-major = a (d, ld) row-major tensor)."""
    return cols_tensor(d, d, _TORCH_DTYPE[int(dtype)], device)


def bkfac_ea_update(M: torch.Tensor, X: torch.Tensor, rho: float, dtype: int, first: bool = False, stream=None):
    """Dense EA factor M (d x d) <- rho M + (1 - rho)/n X X^T (X: (n, d) columns)."""
    n, d = X.shape
    _check(load().bkfac_ea_update(d, int(dtype), _ptr(M), _cols_ld(M), _ptr(X), _cols_ld(X), n, float(rho),
                                  1 if first else 0, _stream(stream)), "bkfac_ea_update")


def bkfac_correct(f: Factor, M: torch.Tensor, idx, ws: torch.Tensor | None = None, stream=None):
    """Light correction (Algorithm 6) of f along the modes idx against the dense factor M."""
    ix = (ctypes.c_int32 * len(idx))(*[int(i) for i in idx])
    if ws is None:
        key = ("correct", len(idx))
        if key not in f._ws:
            nb = load().bkfac_correct_workspace_size(ctypes.byref(f.desc), len(idx))
            if nb == 0:
                raise BkfacError(EINVAL, "bkfac_correct_workspace_size")
            f._ws[key] = workspace(nb, f.U.device)
        ws = f._ws[key]
    _check(load().bkfac_correct(ctypes.byref(f.desc), _ptr(M), _cols_ld(M), ix, len(idx), _ptr(ws), ws.numel(),
                                _stream(stream)), "bkfac_correct")


def bkfac_rsvd(f: Factor, M: torch.Tensor, Omega: torch.Tensor, q: int, ws: torch.Tensor | None = None, stream=None):
    """RSVD overwrite (Algorithm 5) of f from the dense factor M; Omega: (l, d) test columns."""
    l = Omega.shape[0]
    if ws is None:
        key = ("rsvd", l)
        if key not in f._ws:
            nb = load().bkfac_rsvd_workspace_size(ctypes.byref(f.desc), l)
            if nb == 0:
                raise BkfacError(EINVAL, "bkfac_rsvd_workspace_size")
            f._ws[key] = workspace(nb, f.U.device)
        ws = f._ws[key]
    _check(load().bkfac_rsvd(ctypes.byref(f.desc), _ptr(M), _cols_ld(M), _ptr(Omega), _cols_ld(Omega), l, int(q),
                             _ptr(ws), ws.numel(), _stream(stream)), "bkfac_rsvd")


def bkfac_debug_offsets(f: Factor, n: int):
    out = (ctypes.c_int64 * 8)()
    _check(load().bkfac_debug_offsets(ctypes.byref(f.desc), int(n), out), "bkfac_debug_offsets")
    return list(out)


def bkfac_trace_enable(on: bool = True):
    _check(load().bkfac_trace_enable(1 if on else 0), "bkfac_trace_enable")


def bkfac_trace_read():
    """Per-phase totals since tracing was enabled: {name: (ms, count)}, plus the
    library's kernel-launch counter."""
    lib = load()
    nmax = 64
    ms = (ctypes.c_double * nmax)()
    cnt = (ctypes.c_int64 * nmax)()
    launches = ctypes.c_int64(0)
    nph = lib.bkfac_trace_read(ms, cnt, nmax, ctypes.byref(launches))
    if nph < 0:
        raise BkfacError(-nph, "bkfac_trace_read")
    out = {lib.bkfac_trace_phase_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(nph)}
    return out, int(launches.value)


def bkfac_launch_count() -> int:
    return bkfac_trace_read()[1]


# --------------------------------------------------------------------------- batch


def _arr(ctype, vals):
    return (ctype * len(vals))(*vals)


class Batch:
    """All factors of all FC layers (bkfac_batch_*): grouped update / apply and
    one-graph replay of a full step.  layers: list of (Factor A, Factor G); the
    batch works on copies of their descriptors and owns its own workspace."""

    def __init__(self, layers, n: int, dtype: int = F32, tune_cache: str | None = None):
        self.layers = layers
        self.n = int(n)
        self.dtype = int(dtype)
        descs = (bkfac_layer_desc * len(layers))(*[bkfac_layer_desc(a.desc, g.desc) for a, g in layers])
        h = load().bkfac_batch_create(descs, len(layers), self.n, self.dtype,
                                      tune_cache.encode() if tune_cache else None)
        if not h:
            raise BkfacError(EINVAL, "bkfac_batch_create")
        self.h = ctypes.c_void_p(h)
        self._graph_args = None

    def factor(self, layer: int, which: int) -> bkfac_factor:
        out = bkfac_factor()
        _check(load().bkfac_batch_get_factor(self.h, layer, which, ctypes.byref(out)), "bkfac_batch_get_factor")
        return out

    def sync_descriptors(self):
        """Copy the batch's r_cur / step back into the layers' Factor objects."""
        for l, (a, g) in enumerate(self.layers):
            for w, f in ((0, a), (1, g)):
                d = self.factor(l, w)
                f.desc.r_cur, f.desc.step = d.r_cur, d.step

    def update(self, XA, XG, rho: float, stream=None):
        P = ctypes.c_void_p
        _check(load().bkfac_batch_update(self.h, _arr(P, [x.data_ptr() for x in XA]),
                                         _arr(ctypes.c_int64, [_cols_ld(x) for x in XA]),
                                         _arr(P, [x.data_ptr() for x in XG]),
                                         _arr(ctypes.c_int64, [_cols_ld(x) for x in XG]), float(rho),
                                         _stream(stream)), "bkfac_batch_update")

    def apply(self, G, S, lamA, lamG, flags: int = 0, stream=None):
        P = ctypes.c_void_p
        _check(load().bkfac_batch_apply(self.h, _arr(P, [g.data_ptr() for g in G]),
                                        _arr(ctypes.c_int64, [g.stride(0) for g in G]),
                                        _arr(P, [s.data_ptr() for s in S]),
                                        _arr(ctypes.c_int64, [s.stride(0) for s in S]),
                                        _arr(ctypes.c_double, list(lamA)), _arr(ctypes.c_double, list(lamG)),
                                        int(flags), _stream(stream)), "bkfac_batch_apply")

    def step_graph(self, XA=None, XG=None, rho=0.95, G=None, S=None, lamA=None, lamG=None, flags: int = 0,
                   capture: bool = False, stream=None):
        """capture=True: capture one full step (update then apply) with these
        tensors and replay it once; capture=False: replay the captured graph."""
        P = ctypes.c_void_p
        lib = load()
        if capture:
            args = (_arr(P, [x.data_ptr() for x in XA]), _arr(ctypes.c_int64, [_cols_ld(x) for x in XA]),
                    _arr(P, [x.data_ptr() for x in XG]), _arr(ctypes.c_int64, [_cols_ld(x) for x in XG]),
                    float(rho), _arr(P, [g.data_ptr() for g in G]), _arr(ctypes.c_int64, [g.stride(0) for g in G]),
                    _arr(P, [s.data_ptr() for s in S]), _arr(ctypes.c_int64, [s.stride(0) for s in S]),
                    _arr(ctypes.c_double, list(lamA)), _arr(ctypes.c_double, list(lamG)))
            self._graph_args = args
            _check(lib.bkfac_batch_step_graph(self.h, *args, int(flags), 1, _stream(stream)), "bkfac_batch_step_graph")
        else:
            _check(lib.bkfac_batch_step_graph(self.h, None, None, None, None, 0.0, None, None, None, None, None,
                                              None, int(flags), 0, _stream(stream)), "bkfac_batch_step_graph")

    def reorth(self, stream=None):
        _check(load().bkfac_batch_reorth(self.h, _stream(stream)), "bkfac_batch_reorth")

    def close(self):
        if getattr(self, "h", None):
            load().bkfac_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bkfac_tune(f: Factor, n: int, cache_path: str | None = None):
    """Autotune the eigensolve launch shape of f at batch width n (see include/bkfac.h)."""
    _check(load().bkfac_tune(ctypes.byref(f.desc), int(n), cache_path.encode() if cache_path else None), "bkfac_tune")


def bkfac_gemm_tune_begin():
    """Start noting the FP32 product shapes the library launches (see include/bkfac.h)."""
    _check(load().bkfac_gemm_tune_begin(), "bkfac_gemm_tune_begin")


def bkfac_gemm_tune_end(cache_path: str | None = None):
    """Stop noting; time the candidates of every noted shape and keep the fastest."""
    _check(load().bkfac_gemm_tune_end(cache_path.encode() if cache_path else None), "bkfac_gemm_tune_end")
