"""FP64 CPU oracle of the cooperative conjugate gradient method (cCG).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
CUDA solver never imports, links or calls it, and it imports nothing from the
CUDA solver.

The arithmetic lives in ``ccg_oracle.c`` (plain loops, no BLAS/LAPACK): it
runs Algorithm 2 of the paper (cCG) with the rank-deficiency deflation of
Algorithm 3 (mcCG) and the stopping rule of Algorithm 4, in FP64.  This module
only builds that file with gcc and marshals numpy arrays through ctypes.

Pins (tests/test_oracle_pins.py) tie it to things other than itself: a direct
LAPACK solve, textbook Hestenes-Stiefel CG at p = 1 (Algorithm 1), the
properties of Theorem 2 (orthogonality, A-conjugacy, subspace optimality),
finite termination (Theorem 3), the residual recurrence, the CG error bound of
Theorem 1, the p = 2 closed forms (Eq. 3 and Eq. 7) and the deflation cases of
Algorithm 3.  Published SplitMix64 outputs pin the initial-block generator,
and exact rational sums pin the compensated (Dot2) Gram products
(tests/test_oracle_gram_exact.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccg_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libccg_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_INVALID", -2: "ERR_NOT_SPD",
          -3: "ERR_NUMERICAL", -4: "ERR_OOM"}


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("agent", ctypes.c_int),
        ("p_final", ctypes.c_int),
        ("replacements", ctypes.c_int),
        ("drops", ctypes.c_int),
        ("relres_true", ctypes.c_double),
        ("relres_recur", ctypes.c_double),
    ]


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                            _IP, _DP, _DP, _DP, _DP, _DP, _DP)


def build(force: bool = False) -> str:
    """Compile ccg_oracle.c into a shared library with gcc (OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_ccg.restype = ctypes.c_int
            lib.oracle_ccg.argtypes = [
                ctypes.c_int64, _DP, ctypes.c_int64, _DP, _DP, ctypes.c_int,
                ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP, _DP, _IP,
                ctypes.POINTER(OracleStats), TRACE_FN, ctypes.c_void_p]
            lib.oracle_block_product.restype = None
            lib.oracle_block_product.argtypes = [ctypes.c_int64, _DP, ctypes.c_int64, _DP,
                                                 ctypes.c_int, _DP, ctypes.c_int]
            lib.oracle_splitmix64_at.restype = ctypes.c_uint64
            lib.oracle_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_initial_block.restype = None
            lib.oracle_initial_block.argtypes = [
                ctypes.c_int64, ctypes.c_int, _DP, ctypes.c_double,
                ctypes.c_uint64, _DP]
            lib.oracle_true_relres.restype = ctypes.c_double
            lib.oracle_true_relres.argtypes = [ctypes.c_int64, _DP, ctypes.c_int64,
                                               _DP, _DP, ctypes.c_int]
            lib.oracle_gram.restype = None
            lib.oracle_gram.argtypes = [ctypes.c_int64, ctypes.c_int, _DP, _DP, _DP]
            lib.oracle_max_threads.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def splitmix64_at(seed: int, counter: int) -> int:
    return int(_load().oracle_splitmix64_at(seed & (2**64 - 1), counter & (2**64 - 1)))


def initial_block(n: int, p: int, x0=None, spread: float = 1.0, seed: int = 0) -> np.ndarray:
    """X_0 built from one x0: column 0 = x0, column j >= 1 = x0 + spread*u_j."""
    X0 = np.empty((n, p), dtype=np.float64)
    x0a = _f64(x0) if x0 is not None else None
    _load().oracle_initial_block(n, p, _dp(x0a) if x0a is not None else None,
                                 float(spread), seed & (2**64 - 1), _dp(X0))
    return X0


def gram(U, V) -> np.ndarray:
    """G = U^T V for n x q blocks (q <= 32), each entry a Dot2 sum: the
    inner products the solver takes for M, G, H and the residue norms."""
    U = _f64(U); V = _f64(V)
    if U.ndim != 2 or U.shape != V.shape or not 1 <= U.shape[1] <= 32:
        raise ValueError("U and V must be n x q with the same shape, q <= 32")
    n, q = U.shape
    G = np.empty((q, q), dtype=np.float64)
    _load().oracle_gram(n, q, _dp(U), _dp(V), _dp(G))
    return G


# summation orders of the block product: ascending, descending, blocks of 64,
# 64 interleaved sums, compensated (Dot2)
PRODUCT_ORDERS = (0, 1, 2, 3, 4)


def block_product(A, V, order: int = 0) -> np.ndarray:
    """W = A V with each entry a plain FP64 sum in the given order (the block
    product of the solver, exposed for its pins)."""
    A = _f64(A); V = _f64(V)
    n, q = V.shape
    if A.shape[0] != n or A.shape[1] < n or not 1 <= q <= 32 or order not in PRODUCT_ORDERS:
        raise ValueError("A must be n x (>= n), V n x q with q <= 32, order in 0..4")
    W = np.empty((n, q), dtype=np.float64)
    _load().oracle_block_product(n, _dp(A), A.shape[1], _dp(V), q, _dp(W), int(order))
    return W


def true_relres(A, b, x, nthreads: int = 1) -> float:
    A = _f64(A); b = _f64(b); x = _f64(x)
    n = b.shape[0]
    return float(_load().oracle_true_relres(n, _dp(A), A.shape[1], _dp(b), _dp(x), nthreads))


def ccg(A, b, X0, tol: float, maxit: int, rank_tol: float = 1e-12,
        residual_replacement: bool = True, nthreads: int = 1, trace: bool = False,
        explicit_residual: bool = False, product_order: int = 0):
    """Run the oracle cCG/mcCG on A x = b from the initial block X0 (n x p).

    Returns a dict with x, X (final active block), agents (original indices of
    its columns), status, iterations, agent, p_final, relres_true,
    relres_recur, replacements, drops and, if trace, a list of per-iteration
    states (k, agents, X, R, D, W, alpha, beta) copied out of the callback.
    product_order picks the summation order of the block product A D (see
    block_product); 0, ascending, is the default.
    """
    if product_order not in PRODUCT_ORDERS:
        raise ValueError("product_order must be one of 0, 1, 2, 3, 4")
    A = _f64(A)
    b = _f64(b)
    X0 = _f64(X0)
    n = b.shape[0]
    if X0.ndim == 1:
        X0 = X0.reshape(n, 1)
    p = X0.shape[1]
    lda = A.shape[1] if A.ndim == 2 else n
    x = np.zeros(n, dtype=np.float64)
    Xf = np.zeros((n, p), dtype=np.float64)
    agents = np.full(p, -1, dtype=np.int32)
    st = OracleStats()
    states = []

    def _cb(ctx, k, pk, agent, X, R, D, W, alpha, beta):
        def blk(ptr):
            if not ptr:
                return None
            return np.ctypeslib.as_array(ptr, shape=(n, pk)).copy()

        def sq(ptr):
            if not ptr:
                return None
            return np.ctypeslib.as_array(ptr, shape=(pk, pk)).copy()
        states.append(dict(k=k, agents=np.ctypeslib.as_array(agent, shape=(pk,)).copy(),
                           X=blk(X), R=blk(R), D=blk(D), W=blk(W),
                           alpha=sq(alpha), beta=sq(beta)))

    cb = TRACE_FN(_cb) if trace else TRACE_FN()
    rc = _load().oracle_ccg(n, _dp(A), lda, _dp(b), _dp(X0), p, float(tol), int(maxit),
                            float(rank_tol), int(bool(residual_replacement)),
                            int(bool(explicit_residual)), int(product_order), int(nthreads),
                            _dp(x), _dp(Xf), agents.ctypes.data_as(_IP), ctypes.byref(st),
                            cb, None)
    pf = st.p_final
    out = dict(status=int(rc), status_name=STATUS.get(int(rc), str(rc)), x=x,
               X=Xf.reshape(-1)[: n * pf].reshape(n, pf) if pf > 0 else Xf[:, :0],
               agents=agents[:pf].copy(), iterations=st.iterations, agent=st.agent,
               p_final=pf, relres_true=st.relres_true, relres_recur=st.relres_recur,
               replacements=st.replacements, drops=st.drops)
    if trace:
        out["trace"] = states
    return out
