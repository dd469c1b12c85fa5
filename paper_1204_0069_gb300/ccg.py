"""ctypes binding of the C ABI in ``include/ccg.h`` (libccg.so).

Argument marshalling only: every step of a solve runs in the CUDA kernels of
the library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they
must be C-contiguous float64.  There is no fallback: if ``libccg.so`` has not
been built, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libccg.so")

STATUS = {0: "CCG_OK", 1: "CCG_NOT_CONVERGED", -1: "CCG_ERR_INVALID", -2: "CCG_ERR_NOT_SPD",
          -3: "CCG_ERR_NUMERICAL", -4: "CCG_ERR_OOM", -5: "CCG_ERR_TIMEOUT", -6: "CCG_ERR_CUDA"}
OK, NOT_CONVERGED = 0, 1
EXPORTED = ["ccg_config_init", "ccg_create", "ccg_destroy", "ccg_solve", "ccg_solve_block",
            "ccg_block_product", "ccg_selftest_barrier_timeout", "ccg_status_string",
            "ccg_version", "ccg_lowp_create", "ccg_lowp_block_product", "ccg_lowp_bytes",
            "ccg_lowp_destroy", "ccg_solve_noalloc", "ccg_solve_mixed", "ccg_solve_batched",
            "ccg_server_config_init", "ccg_server_create", "ccg_server_submit", "ccg_server_poll",
            "ccg_server_stats", "ccg_server_destroy", "ccg_batch_tuning"]
FP64, FP32_IR, BF16_IR, FP8_IR, FP64_SLICED = 0, 1, 2, 3, 4
MIXED_AUTO, MIXED_REFINE, MIXED_PRECOND = 0, 1, 2
NOALLOC_MAX_NP = 131072
LOWP_BF16, LOWP_FP8_E4M3, LOWP_FP32, LOWP_FP64_SLICED = 0, 1, 2, 3


class Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("precision", ctypes.c_int), ("rank_tol", ctypes.c_double),
                ("x0_spread", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("residual_replacement", ctypes.c_int),
                ("barrier_timeout_ms", ctypes.c_double), ("max_ctas", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("explicit_residual", ctypes.c_int), ("batch_autotune", ctypes.c_int),
                ("mixed_method", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("cheb_ratio", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("workers", ctypes.c_int), ("precision", ctypes.c_int),
                ("budget_bytes", ctypes.c_double), ("ctas_per_worker", ctypes.c_int),
                ("slots", ctypes.c_int), ("max_n", ctypes.c_int64), ("max_p", ctypes.c_int)]


class ServerResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("outer_steps", ctypes.c_int), ("worker", ctypes.c_int), ("ctas", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("in_flight", ctypes.c_int), ("peak_in_flight", ctypes.c_int),
                ("ctas_per_worker", ctypes.c_int), ("reserved_bytes", ctypes.c_double),
                ("peak_reserved_bytes", ctypes.c_double), ("now_ms", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("agent", ctypes.c_int), ("p_final", ctypes.c_int),
                ("replacements", ctypes.c_int), ("drops", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("relres_recur", ctypes.c_double),
                ("device_ms", ctypes.c_float), ("ctas", ctypes.c_int),
                ("outer_steps", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS.get(self.status, str(self.status))
        return d


_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64


def lib():
    """Load libccg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libccg.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.ccg_config_init.argtypes = [ctypes.POINTER(Config)]
        L.ccg_config_init.restype = None
        L.ccg_create.argtypes = [ctypes.POINTER(_VP), ctypes.POINTER(Config)]
        L.ccg_destroy.argtypes = [_VP]
        L.ccg_solve.argtypes = [_VP, _I64, _VP, _I64, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, _VP, ctypes.POINTER(Result)]
        L.ccg_solve_block.argtypes = [_VP, _I64, _VP, _I64, _VP, _VP, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, _VP, _VP,
                                      ctypes.POINTER(Result)]
        L.ccg_block_product.argtypes = [_VP, _I64, _VP, _I64, _VP, _VP, ctypes.c_int, _VP, _VP,
                                        _VP, ctypes.POINTER(ctypes.c_float)]
        L.ccg_selftest_barrier_timeout.argtypes = [_VP, ctypes.c_double]
        L.ccg_status_string.argtypes = [ctypes.c_int]
        L.ccg_status_string.restype = ctypes.c_char_p
        L.ccg_version.argtypes = []
        L.ccg_version.restype = ctypes.c_char_p
        L.ccg_lowp_create.argtypes = [_VP, ctypes.c_int, _I64, _VP, _I64, ctypes.POINTER(_VP)]
        L.ccg_lowp_block_product.argtypes = [_VP, _VP, _VP, ctypes.c_int, _VP,
                                             ctypes.POINTER(ctypes.c_float)]
        L.ccg_lowp_bytes.argtypes = [_VP]
        L.ccg_lowp_bytes.restype = ctypes.c_int64
        L.ccg_lowp_destroy.argtypes = [_VP]
        L.ccg_solve_noalloc.argtypes = [ctypes.c_int, _VP, _I64, _VP, _I64, _VP, _VP, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, _VP, ctypes.POINTER(Result)]
        L.ccg_solve_noalloc.restype = ctypes.c_int
        L.ccg_solve_mixed.argtypes = [_VP, _VP, _I64, _VP, _I64, _VP, _VP, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, _VP, ctypes.POINTER(Result)]
        L.ccg_solve_mixed.restype = ctypes.c_int
        L.ccg_solve_batched.argtypes = [_VP, _I64, _VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.POINTER(Result)]
        L.ccg_solve_batched.restype = ctypes.c_int
        L.ccg_batch_tuning.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int]
        L.ccg_batch_tuning.restype = ctypes.c_int
        L.ccg_server_config_init.argtypes = [ctypes.POINTER(ServerConfig)]
        L.ccg_server_config_init.restype = None
        L.ccg_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_VP)]
        L.ccg_server_submit.argtypes = [_VP, ctypes.c_int64, _I64, _VP, _I64, _VP, _VP,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.ccg_server_poll.argtypes = [_VP, ctypes.POINTER(ServerResult), ctypes.c_int, ctypes.c_int]
        L.ccg_server_stats.argtypes = [_VP, ctypes.POINTER(ServerStats)]
        L.ccg_server_destroy.argtypes = [_VP]
        for name in ["ccg_server_create", "ccg_server_submit", "ccg_server_poll",
                     "ccg_server_stats", "ccg_server_destroy", "ccg_batch_tuning"]:
            getattr(L, name).restype = ctypes.c_int
        for name in ["ccg_create", "ccg_destroy", "ccg_solve", "ccg_solve_block",
                     "ccg_block_product", "ccg_selftest_barrier_timeout", "ccg_lowp_create",
                     "ccg_lowp_block_product", "ccg_lowp_destroy"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    """Data pointer of a contiguous float64 torch tensor / numpy array (or None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float64")
        return a.ctypes.data
    import torch  # local: torch is only needed for tensor arguments
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _current_stream(device: int):
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return None


@dataclass
class SolveResult:
    status: int
    status_name: str
    iterations: int
    agent: int
    p_final: int
    replacements: int
    drops: int
    relres_true: float
    relres_recur: float
    device_ms: float
    ctas: int
    outer_steps: int


class Solver:
    """A solver handle (``ccg_create``) bound to one device and stream."""

    def __init__(self, device: int = 0, stream=None, rank_tol: float = 1e-12,
                 x0_spread: float = 1.0, seed: int = 0, residual_replacement: bool = True,
                 barrier_timeout_ms: float = 10000.0, max_ctas: int = 0, precision: int = 0,
                 inner_tol: float = 0.0, max_outer: int = 0, explicit_residual: bool = False,
                 batch_autotune: bool = True, mixed_method: int = 0, cheb_degree: int = 0,
                 cheb_ratio: float = 0.0):
        L = lib()
        cfg = Config()
        L.ccg_config_init(ctypes.byref(cfg))
        cfg.device = device
        cfg.stream = stream if stream is not None else _current_stream(device)
        cfg.rank_tol = rank_tol
        cfg.x0_spread = x0_spread
        cfg.seed = seed & (2**64 - 1)
        cfg.residual_replacement = int(bool(residual_replacement))
        cfg.barrier_timeout_ms = barrier_timeout_ms
        cfg.max_ctas = max_ctas
        cfg.precision = precision
        cfg.inner_tol = inner_tol
        cfg.max_outer = max_outer
        cfg.explicit_residual = int(bool(explicit_residual))
        cfg.batch_autotune = int(bool(batch_autotune))
        cfg.mixed_method = int(mixed_method)
        cfg.cheb_degree = int(cheb_degree)
        cfg.cheb_ratio = float(cheb_ratio)
        h = _VP()
        rc = L.ccg_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != 0:
            raise RuntimeError(f"ccg_create failed: {STATUS.get(rc, rc)}")
        self._h = h
        self._lib = L

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ccg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _res(r: Result) -> SolveResult:
        d = r.as_dict()
        return SolveResult(**{k: d[k] for k in SolveResult.__dataclass_fields__})

    def solve(self, A, b, x_out, p: int, tol: float, maxit: int, x0=None, lda=None) -> SolveResult:
        n = int(b.shape[0])
        lda = int(A.shape[1]) if lda is None else lda
        r = Result()
        self._lib.ccg_solve(self._h, n, _ptr(A), lda, _ptr(b), _ptr(x0), int(p), float(tol),
                            int(maxit), _ptr(x_out), ctypes.byref(r))
        return self._res(r)

    def solve_block(self, A, b, X0, x_out, tol: float, maxit: int, X_out=None,
                    lda=None) -> SolveResult:
        n = int(b.shape[0])
        p = int(X0.shape[1])
        lda = int(A.shape[1]) if lda is None else lda
        r = Result()
        self._lib.ccg_solve_block(self._h, n, _ptr(A), lda, _ptr(b), _ptr(X0), p, float(tol),
                                  int(maxit), _ptr(x_out), _ptr(X_out), ctypes.byref(r))
        return self._res(r)

    def block_product(self, A, V, W, U=None, want_grams: bool = True, lda=None):
        """W = A V and (M = V'W symmetrised, G = U'V) as numpy q x q arrays."""
        n = int(V.shape[0])
        q = int(V.shape[1])
        lda = int(A.shape[1]) if lda is None else lda
        M = np.zeros((q, q)) if want_grams else None
        G = np.zeros((q, q)) if (want_grams and U is not None) else None
        ms = ctypes.c_float(0.0)
        rc = self._lib.ccg_block_product(self._h, n, _ptr(A), lda, _ptr(V), _ptr(U), q, _ptr(W),
                                         _ptr(M), _ptr(G), ctypes.byref(ms))
        return rc, M, G, ms.value

    def solve_mixed(self, lpA: "LowpMatrix", A, b, x_out, p: int, tol: float, maxit: int,
                    x0=None, lda=None) -> SolveResult:
        """ccg_solve_mixed: FP64 refinement around inner solves on lpA."""
        n = int(b.shape[0])
        lda = int(A.shape[1]) if lda is None else lda
        r = Result()
        self._lib.ccg_solve_mixed(self._h, lpA._m, n, _ptr(A), lda, _ptr(b), _ptr(x0), int(p),
                                  float(tol), int(maxit), _ptr(x_out), ctypes.byref(r))
        return self._res(r)

    def solve_batched(self, sizes, A_packed, b_packed, x_packed, p: int, tol: float, maxit: int):
        """ccg_solve_batched over systems packed as described in include/ccg.h
        (see pack_batch).  Returns (summary, status[], iterations[], relres[])."""
        cnt = len(sizes)
        nn = np.ascontiguousarray(sizes, dtype=np.int64)
        st = np.zeros(cnt, dtype=np.int32)
        it = np.zeros(cnt, dtype=np.int32)
        rr = np.zeros(cnt, dtype=np.float64)
        r = Result()
        self._lib.ccg_solve_batched(self._h, cnt, nn.ctypes.data, _ptr(A_packed), _ptr(b_packed),
                                    int(p), float(tol), int(maxit), _ptr(x_packed),
                                    st.ctypes.data, it.ctypes.data, rr.ctypes.data, ctypes.byref(r))
        return self._res(r), st, it, rr

    def batch_tuning(self, p: int, precision: int = 0, variants=None):
        """ccg_batch_tuning: returns the A-pass variant table of the batched
        solver for (p, precision) (-1 = bucket not tuned yet), or sets it."""
        arr = (ctypes.c_int * 8)()
        if variants is not None:
            for k, v in enumerate(variants):
                arr[k] = int(v)
        rc = self._lib.ccg_batch_tuning(self._h, int(p), int(precision), arr,
                                        0 if variants is None else 1)
        if rc != 0:
            raise RuntimeError(f"ccg_batch_tuning failed: {STATUS.get(rc, rc)}")
        return list(arr)

    def lowp_matrix(self, A, fmt: int, lda=None) -> "LowpMatrix":
        """Quantised copy of A (ccg_lowp_create) on this handle's device."""
        n = int(A.shape[0])
        lda = int(A.shape[1]) if lda is None else lda
        m = _VP()
        rc = self._lib.ccg_lowp_create(self._h, int(fmt), n, _ptr(A), lda, ctypes.byref(m))
        if rc != 0:
            raise RuntimeError(f"ccg_lowp_create failed: {STATUS.get(rc, rc)}")
        return LowpMatrix(self, m)

    def selftest_barrier_timeout(self, timeout_ms: float) -> int:
        return int(self._lib.ccg_selftest_barrier_timeout(self._h, float(timeout_ms)))


class LowpMatrix:
    """A quantised matrix (ccg_lowp_matrix); freed by close()."""

    def __init__(self, solver: Solver, handle):
        self._solver = solver
        self._m = handle

    def nbytes(self) -> int:
        return int(self._solver._lib.ccg_lowp_bytes(self._m))

    def block_product(self, V, W):
        """W = A_lp V (ccg_lowp_block_product); returns (status, device_ms)."""
        ms = ctypes.c_float(0.0)
        rc = self._solver._lib.ccg_lowp_block_product(self._solver._h, self._m, _ptr(V),
                                                      int(V.shape[1]), _ptr(W), ctypes.byref(ms))
        return int(rc), ms.value

    def close(self):
        if getattr(self, "_m", None):
            self._solver._lib.ccg_lowp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop (ccg_server_create): submit requests, poll results.
    Worker threads by default; slots > 0 serves every request from one
    persistent kernel (continuous batching)."""

    def __init__(self, device: int = 0, workers: int = 8, precision: int = 0,
                 budget_bytes: float = 150e9, ctas_per_worker: int = 0, slots: int = 0,
                 max_n: int = 0, max_p: int = 0):
        """slots > 0: one persistent serving kernel with that many slots
        (continuous batching, CCG_FP64); otherwise `workers` worker threads."""
        L = lib()
        c = ServerConfig()
        L.ccg_server_config_init(ctypes.byref(c))
        c.device, c.workers, c.precision = device, workers, precision
        c.budget_bytes, c.ctas_per_worker = budget_bytes, ctas_per_worker
        c.slots = slots
        if max_n:
            c.max_n = max_n
        if max_p:
            c.max_p = max_p
        h = _VP()
        rc = L.ccg_server_create(ctypes.byref(c), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"ccg_server_create failed: {STATUS.get(rc, rc)}")
        self._h, self._lib = h, L

    def submit(self, rid: int, A, b, x_out, p: int, tol: float, maxit: int, lda=None) -> int:
        n = int(b.shape[0])
        lda = int(A.shape[1]) if lda is None else lda
        return int(self._lib.ccg_server_submit(self._h, int(rid), n, _ptr(A), lda, _ptr(b),
                                               _ptr(x_out), int(p), float(tol), int(maxit)))

    def poll(self, max_results: int = 64, wait_ms: int = 0):
        buf = (ServerResult * max_results)()
        k = self._lib.ccg_server_poll(self._h, buf, max_results, int(wait_ms))
        return [{f: getattr(buf[i], f) for f, _ in ServerResult._fields_} for i in range(max(k, 0))]

    def stats(self):
        st = ServerStats()
        self._lib.ccg_server_stats(self._h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ccg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_offsets(sizes):
    """Element offsets of the packed batch layout of ccg_solve_batched: A_i at
    sum_{j<i} n_j ld_j (ld_j = n_j rounded up to even), b_i / x_i at
    sum_{j<i} n_j.  Returns (a_off, v_off, a_total, v_total)."""
    a_off, v_off = [], []
    a = v = 0
    for nn in sizes:
        a_off.append(a)
        v_off.append(v)
        a += nn * (nn + (nn & 1))
        v += nn
    return a_off, v_off, a, v


def solve_noalloc(A, b, x_out, p: int, tol: float, maxit: int, x0=None, device: int = 0,
                  stream=None, lda=None) -> SolveResult:
    """ccg_solve_noalloc: a solve that allocates nothing (device tensors only;
    its scratch is a fixed device array, so calls must not overlap)."""
    n = int(b.shape[0])
    lda = int(A.shape[1]) if lda is None else lda
    r = Result()
    lib().ccg_solve_noalloc(int(device), stream, n, _ptr(A), lda, _ptr(b), _ptr(x0), int(p),
                            float(tol), int(maxit), _ptr(x_out), ctypes.byref(r))
    return Solver._res(r)


def status_string(code: int) -> str:
    return lib().ccg_status_string(int(code)).decode()


def version() -> str:
    return lib().ccg_version().decode()
