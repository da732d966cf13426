"""Plain FP64 CPU oracle for the B-KFAC hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library's product path never calls
it: there is no CPU fallback.  The oracle shares no code with the CUDA library;
both sides receive the same arrays from the seeded input generator.

The arithmetic lives in ``bkfac_oracle.c`` (plain loops, IEEE double,
``-ffp-contract=off``).  This module compiles it with gcc on first use and
wraps it with ctypes.  Conventions of the wrappers (numpy, float64):

* a d x k column-major matrix (U, X, Q, P) is passed as a C-contiguous array of
  shape (k, d), i.e. one row per column -- the same memory as a torch (k, d)
  tensor;
* the gradient G and the step S are C-contiguous (d_G, d_A) arrays (torch
  ``weight.grad`` layout);
* small square matrices (M, R, M_S, V) come back as numpy arrays in the natural
  (row, column) orientation.

Paper: "Brand New K-FACs" (arXiv 2210.08494).  The functions follow Sec. 3.1
(Algorithm 4, B-KFAC), Sec. 2.3 (Algorithm 3, symmetric Brand update, and the
core of Eq. (7)), Algorithm 1 (damped inverse application, Eq. (4)) and
Algorithm 8 (the inverse application on the thin gradient factors), and the
dense EA factor with Algorithms 5 and 6 (the RSVD overwrite of B-R-KFAC and
the light correction of B-KFAC-C).

Parity status: pinned by ``tests/test_oracle_pins.py`` (closed forms, LAPACK
cross-checks on small inputs, Propositions 3.1/3.2/4.1/4.2).  The paper prints
no worked numeric example, so nothing here is pinned to a printed value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bkfac_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbkfac_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOCONV, ENOMEM = 0, 1, 4, 9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
    lib.bko_jacobi_eig.argtypes = [I, dp, L, dp, dp, L, I, ip]
    lib.bko_qrcp.argtypes = [I, I, dp, L, D, dp, L, dp, L, ip]
    lib.bko_project.argtypes = [I, I, dp, L, I, dp, L, dp, dp]
    lib.bko_core.argtypes = [I, I, dp, D, D, dp, dp, L, dp, L]
    upd = [I, I, I, dp, L, dp, I, dp, L, D, dp, L, dp, ip]
    lib.bko_update.argtypes = upd
    lib.bko_update_dense.argtypes = upd
    lib.bko_reorth.argtypes = [I, I, dp, L, dp, dp, L, dp]
    lib.bko_apply.argtypes = [I, I, dp, L, dp, D, I, I, dp, L, dp, D, dp, L, dp, L, I]
    lib.bko_apply_factored.argtypes = [I, I, dp, L, dp, D, I, I, dp, L, dp, D, I, dp, L, dp, L, dp, L, dp, L, D,
                                       dp, L, I]
    lib.bko_ea_update.argtypes = [I, dp, L, I, dp, L, D, I]
    lib.bko_correct.argtypes = [I, I, dp, L, dp, dp, L, I, ip]
    lib.bko_rsvd.argtypes = [I, I, I, dp, L, dp, L, I, dp, L, dp]
    for f in (lib.bko_jacobi_eig, lib.bko_qrcp, lib.bko_project, lib.bko_core, lib.bko_update,
              lib.bko_update_dense, lib.bko_reorth, lib.bko_apply, lib.bko_apply_factored, lib.bko_ea_update,
              lib.bko_correct, lib.bko_rsvd):
        f.restype = ctypes.c_int
    return lib


_override = None


def _load():
    global _lib
    if _override is not None:
        return _override
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager: route the wrappers through another compiled copy of the
    oracle (the mutation tests build deliberately broken copies)."""

    def __init__(self, path: str):
        self.lib = _bind(ctypes.CDLL(path))

    def __enter__(self):
        global _override
        self._prev, _override = _override, self.lib
        return self

    def __exit__(self, *exc):
        global _override
        _override = self._prev
        return False


def build_variant(source_text: str, out_path: str) -> str:
    """Compile a variant of the oracle source (same flags) to out_path."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", out_path, src, "-lm"], check=True)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what} failed with code {rc}")


def jacobi_eig(A: np.ndarray, max_sweeps: int = 100):
    """Two-sided cyclic Jacobi: returns (lambda descending, V with V[:, i] the eigenvectors, sweeps)."""
    A = _f64(A)
    N = A.shape[0]
    W = np.array(A.T, dtype=np.float64, order="C")  # column-major storage of A
    lam = np.zeros(max(N, 1))
    V = np.zeros((max(N, 1), max(N, 1)))
    sw = ctypes.c_int(0)
    _check(_load().bko_jacobi_eig(N, _p(W), N, _p(lam), _p(V), N, max_sweeps, ctypes.byref(sw)), "jacobi_eig")
    return lam[:N], V[:N, :N].T.copy(), sw.value  # V stored column-major -> transpose to (row, col)


def qrcp(Pt: np.ndarray, tol: float):
    """Householder QR with column pivoting of the d x n matrix given as (n, d).

    Returns (Qt (n, d) -- rows are the columns of Q, Rt (n x n, natural orientation), rank).
    """
    Pt = _f64(Pt)
    n, d = Pt.shape
    Qt = np.zeros((n, d))
    R = np.zeros((n, n))
    m = ctypes.c_int(0)
    _check(_load().bko_qrcp(d, n, _p(Pt), d, tol, _p(Qt), d, _p(R), n, ctypes.byref(m)), "qrcp")
    return Qt, R.T.copy(), m.value


def project(Ut: np.ndarray, Xt: np.ndarray):
    """M = U^T X (k x n, natural orientation) and P = X - U M returned as Pt (n, d)."""
    Ut, Xt = _f64(Ut), _f64(Xt)
    k = Ut.shape[0]
    n, d = Xt.shape
    M = np.zeros((n, max(k, 1)))
    Pt = np.zeros((n, d))
    _check(_load().bko_project(d, k, _p(Ut) if k else _p(np.zeros(1)), d, n, _p(Xt), d, _p(M), _p(Pt)), "project")
    return M[:, :k].T.copy(), Pt


def core(sigma: np.ndarray, rho: float, c: float, M: np.ndarray, R: np.ndarray):
    """The Brand core M_S of Eq. (7) with the B-KFAC substitutions (natural orientation)."""
    sigma = _f64(sigma)
    k = sigma.shape[0]
    n = R.shape[0]
    Mc = np.array(_f64(M).reshape(k, n).T, order="C") if k else np.zeros((n, 1))  # column-major k x n
    Rc = np.array(_f64(R).T, order="C")
    N = k + n
    MS = np.zeros((N, N))
    _check(_load().bko_core(k, n, _p(sigma) if k else _p(np.zeros(1)), rho, c, _p(Mc), _p(Rc), n, _p(MS), N),
           "core")
    return MS.T.copy()


def _update(fn, Ut, sigma, k, Xt, rho, r):
    Xt = _f64(Xt)
    n, d = Xt.shape
    Uin = np.zeros((max(k, 1), d)) if k == 0 else _f64(Ut)[:k]
    sin = np.zeros(max(k, 1)) if k == 0 else _f64(sigma)[:k]
    Uo = np.zeros((r, d))
    so = np.zeros(r)
    diag = (ctypes.c_int * 4)()
    _check(fn(d, r, k, _p(Uin), d, _p(sin), n, _p(Xt), d, float(rho), _p(Uo), d, _p(so), diag), "update")
    return Uo, so, {"r_new": diag[0], "rank_p": diag[1], "sweeps": diag[2], "N": diag[3]}


def update(Ut, sigma, k: int, Xt, rho: float, r: int):
    """One B-KFAC update (Algorithm 4 via Algorithm 3).

    Ut: (>=k, d) rows = columns of U; sigma: (>=k,); Xt: (n, d).  Returns
    (Ut' (r, d), sigma' (r,), info) with zero rows / values past info['r_new'].
    """
    return _update(_load().bko_update, Ut, sigma, k, Xt, rho, r)


def update_eigh(Ut, sigma, k: int, Xt, rho: float, r: int):
    """The update of ``update`` with LAPACK's symmetric eigensolver (numpy ``eigh``) in
    place of the two-sided Jacobi for the core's eigendecomposition (step 4 of the
    Brand update); projection, pivoted Householder QR, the core of Eq. (7) and the
    rotation are the oracle's own steps.  For long trajectories, where the Jacobi's
    cost dominates; pinned to ``update`` in tests/test_oracle_pins.py."""
    Xt = _f64(Xt)
    n, d = Xt.shape
    Uk = _f64(Ut)[:k] if k else np.zeros((0, d))
    sk = _f64(sigma)[:k]
    M, Pt = project(Uk, Xt)
    tol = 1e-12 * float(np.sqrt(np.max(np.sum(Xt * Xt, axis=1))))
    Qt, R, m = qrcp(Pt, tol)
    MS = core(sk, rho, (1.0 - rho) / n, M, R)
    w, V = np.linalg.eigh(MS)
    order = np.argsort(-w, kind="stable")  # descending, ties: lower index first
    w, V = w[order], V[:, order]
    N = k + n
    r_new = min(r, N)
    Uo = np.zeros((r, d))
    so = np.zeros(r)
    Uo[:r_new] = V[:, :r_new].T @ np.concatenate([Uk, Qt], axis=0)
    so[:r_new] = w[:r_new]
    return Uo, so, {"r_new": r_new, "rank_p": m, "sweeps": 0, "N": N}


def update_dense(Ut, sigma, k: int, Xt, rho: float, r: int):
    """Dense update (r + n >= d): explicit K and its top-r eigenpairs."""
    return _update(_load().bko_update_dense, Ut, sigma, k, Xt, rho, r)


def init(Xt, r: int, dense: bool = False):
    """Initial state from the first batch (kappa(0) = 1): top-r EVD of X X^T / n."""
    d = _f64(Xt).shape[1]
    return (update_dense if dense else update)(np.zeros((1, d)), np.zeros(1), 0, Xt, 0.0, r)


def reorth(Ut, sigma):
    """Top eigenpairs of U diag(sigma) U^T within span(U) (U given as (k, d))."""
    Ut, sigma = _f64(Ut), _f64(sigma)
    k, d = Ut.shape
    Uo = np.zeros((k, d))
    so = np.zeros(k)
    _check(_load().bko_reorth(d, k, _p(Ut), d, _p(sigma), _p(Uo), d, _p(so)), "reorth")
    return Uo, so


def apply(UAt, sigA, lamA: float, UGt, sigG, lamG: float, G, continuation: bool = False,
          relative: bool = False):
    """S = (Gamma + lamG I)^-1 G (A + lamA I)^-1 with the low-rank factors (Algorithm 1).

    UAt: (kA, dA), UGt: (kG, dG), G: (dG, dA) row-major.  Returns S (dG, dA).
    relative: lamA / lamG are multiples of each factor's largest eigenvalue.
    """
    UAt, UGt, G = _f64(UAt), _f64(UGt), _f64(G)
    sigA, sigG = _f64(sigA), _f64(sigG)
    kA, dA = UAt.shape
    kG, dG = UGt.shape
    assert G.shape == (dG, dA)
    S = np.zeros((dG, dA))
    one = np.zeros(1)
    _check(_load().bko_apply(dA, kA, _p(UAt) if kA else _p(np.zeros(dA)), dA, _p(sigA) if kA else _p(one),
                             float(lamA), dG, kG, _p(UGt) if kG else _p(np.zeros(dG)), dG,
                             _p(sigG) if kG else _p(one), float(lamG), _p(G), dA, _p(S), dA,
                             (1 if continuation else 0) | (2 if relative else 0)), "apply")
    return S


def apply_factored(UAt, sigA, lamA: float, UGt, sigG, lamG: float, XAt, XGt, alpha: float = 1.0,
                   form_step: bool = True, continuation: bool = False, relative: bool = False):
    """Linear inverse application (Algorithm 8) on the thin gradient factors.

    XAt: (n, dA) -- the input columns A_f, one row per column; XGt: (n, dG) -- the
    back-propagated columns G_f.  Returns (PAt, PGt, S): PA = (A + lamA I)^-1 A_f and
    PG = (Gamma + lamG I)^-1 G_f in the same (n, d) layout, and the step
    S = alpha * PG PA^T as a (dG, dA) row-major array (None unless form_step).
    """
    UAt, UGt, XAt, XGt = _f64(UAt), _f64(UGt), _f64(XAt), _f64(XGt)
    sigA, sigG = _f64(sigA), _f64(sigG)
    kA, dA = UAt.shape
    kG, dG = UGt.shape
    n = XAt.shape[0]
    assert XAt.shape == (n, dA) and XGt.shape == (n, dG)
    PA = np.zeros((max(n, 1), dA))
    PG = np.zeros((max(n, 1), dG))
    S = np.zeros((dG, dA)) if form_step else None
    one = np.zeros(1)
    XA = XAt if n else np.zeros((1, dA))
    XG = XGt if n else np.zeros((1, dG))
    _check(_load().bko_apply_factored(
        dA, kA, _p(UAt) if kA else _p(np.zeros(dA)), dA, _p(sigA) if kA else _p(one), float(lamA),
        dG, kG, _p(UGt) if kG else _p(np.zeros(dG)), dG, _p(sigG) if kG else _p(one), float(lamG),
        n, _p(XA), dA, _p(XG), dG, _p(PA), dA, _p(PG), dG, float(alpha),
        _p(S) if form_step else None, dA, (1 if continuation else 0) | (2 if relative else 0)), "apply_factored")
    return PA[:n], PG[:n], S


def ea_update(M, Xt, rho: float, first: bool = False):
    """Dense EA K-factor (Eq. (5)): returns rho M + (1 - rho)/n X X^T, or X X^T / n when
    first.  M: (d, d) symmetric; Xt: (n, d) -- the batch, one row per column."""
    Xt = _f64(Xt)
    n, d = Xt.shape
    Mo = np.array(M, dtype=np.float64, order="F", copy=True) if M is not None else np.zeros((d, d), order="F")
    _check(_load().bko_ea_update(d, _p(Mo), d, n, _p(Xt), d, float(rho), 1 if first else 0), "ea_update")
    return np.ascontiguousarray(Mo)


def correct(Ut, sigma, M, idx):
    """Light correction (Algorithm 6) of the representation (Ut (k, d), sigma) against the
    dense factor M along the modes idx; returns (Ut, sigma) re-sorted by decreasing sigma."""
    Ut = np.array(_f64(Ut), copy=True)
    sigma = np.array(_f64(sigma), copy=True)
    k, d = Ut.shape
    Mf = np.asfortranarray(_f64(M))
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    _check(_load().bko_correct(d, k, _p(Ut) if k else _p(np.zeros(d)), d, _p(sigma) if k else _p(np.zeros(1)),
                               _p(Mf), d, len(ix), ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "correct")
    return Ut, sigma


def rsvd(M, Omega_t, r: int, q: int):
    """RSVD overwrite (Algorithm 5): the top-r eigenpairs of the dense factor M estimated from
    the test matrix Omega (given as (l, d), one row per column) with q power iterations.
    Returns (Ut (r, d), sigma (r))."""
    Om = _f64(Omega_t)
    l, d = Om.shape
    Mf = np.asfortranarray(_f64(M))
    Ut = np.zeros((r, d))
    sigma = np.zeros(r)
    _check(_load().bko_rsvd(d, r, l, _p(Mf), d, _p(Om), d, int(q), _p(Ut), d, _p(sigma)), "rsvd")
    return Ut, sigma


def set_threads(n: int) -> None:
    """Set the OpenMP thread count used by the oracle's parallel loops."""
    lib = _load()
    try:
        omp = ctypes.CDLL("libgomp.so.1")
        omp.omp_set_num_threads(int(n))
    except OSError:
        os.environ["OMP_NUM_THREADS"] = str(int(n))
    del lib


def max_threads() -> int:
    _load()
    try:
        omp = ctypes.CDLL("libgomp.so.1")
        omp.omp_get_max_threads.restype = ctypes.c_int
        return int(omp.omp_get_max_threads())
    except OSError:
        return int(os.environ.get("OMP_NUM_THREADS", "1"))
