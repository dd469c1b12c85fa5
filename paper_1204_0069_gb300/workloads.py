"""Seeded synthetic SPD systems used by the tests and the benchmark.

This module only draws inputs; it holds none of the solver's arithmetic and is
shared, as the sole common dependency, by the CUDA-path tests and the oracle
tests.  Every generator is deterministic in its seed (numpy ``default_rng``),
draws in the order documented, and returns C-contiguous float64 arrays.

Families:
  * ``gram_shift``: A = G G^T / n + shift I with G n x n i.i.d. N(0, 1), then
    b ~ N(0, 1) from the same stream (spectrum inside [shift, shift + 4]).
  * ``exp_kernel``: points z_i uniform in [0, 1]^3, A_ij = exp(-|z_i - z_j| / l)
    + nugget * delta_ij (an exponential / Matern-1/2 covariance), then
    b ~ N(0, 1) from the same stream.
  * ``haar_spectrum``: the paper's experimental family (Sec. 5): A = U L U^T
    with L diagonal uniform in [1, kappa] and U Haar-orthogonal (QR of a
    Gaussian matrix with the sign fix of Mezzadri, 2007); b and X_0 entries
    uniform in [-10, 10].
"""
from __future__ import annotations

import numpy as np


def gram_shift(n: int, seed: int = 0, shift: float = 0.5):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    A = G @ G.T / n
    A[np.diag_indices(n)] += shift
    A = 0.5 * (A + A.T)  # exact symmetry of the stored matrix
    b = rng.standard_normal(n)
    return np.ascontiguousarray(A), np.ascontiguousarray(b)


def exp_kernel(n: int, seed: int = 1, length: float = 0.2, nugget: float = 1e-2,
               dim: int = 3):
    rng = np.random.default_rng(seed)
    z = rng.random((n, dim))
    A = np.empty((n, n), dtype=np.float64)
    chunk = max(1, (1 << 24) // max(n, 1))
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        diff = z[i0:i1, None, :] - z[None, :, :]
        dist = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
        np.exp(-dist / length, out=A[i0:i1])
    A[np.diag_indices(n)] += nugget
    b = rng.standard_normal(n)
    return A, np.ascontiguousarray(b)


def haar_spectrum(n: int, seed: int = 5, kappa: float = 1e6, p: int = 3):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, n))
    Q, Rq = np.linalg.qr(Z)
    Q = Q * np.sign(np.diag(Rq))[None, :]
    lam = rng.uniform(1.0, kappa, size=n)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.uniform(-10.0, 10.0, size=n)
    X0 = rng.uniform(-10.0, 10.0, size=(n, p))
    return np.ascontiguousarray(A), b, np.ascontiguousarray(X0)


def random_spd(n: int, seed: int, cond: float = 100.0):
    """Small SPD matrix with a prescribed 2-norm condition number (for tests)."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    return np.ascontiguousarray(A), b


def random_block(n: int, p: int, seed: int, scale: float = 1.0):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(scale * rng.standard_normal((n, p)))
