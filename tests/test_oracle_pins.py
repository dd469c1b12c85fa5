"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test names the passage of the paper (arXiv:1204.0069) or the textbook
fact it checks.  Together they are chosen so that a plausible slip in the
oracle -- a dropped term, a wrong sign, a transposed stepsize, a wrong index
in a Gram product, an absolute instead of relative stop test -- fails at
least one of them:

  * direct solve (LAPACK)                      -> final answer
  * p = 1 equals textbook Hestenes-Stiefel CG  -> Algorithm 1 / "CG is p = 1"
  * Theorem 2: residue blocks orthogonal, direction blocks A-orthogonal
  * Theorem 2: column j of X_{k+1} minimises f on X_0 e_j + span[D_0..D_k]
  * Theorem 3: finite termination in floor(n/p) (+ at most p-1) steps
  * residual recurrence R_{k+1} = R_k + A D_k alpha_k^T equals A X - b 1^T
  * Theorem 1 CG error bound, and every agent at least as good as CG
  * p = 2 closed forms of alpha (Eq. 3) and beta (Eq. 7)
  * Algorithm 3 deflation: dependent agents are removed, result unchanged
  * published SplitMix64 outputs for the initial block
"""
import os

import numpy as np
import pytest

from paper_1204_0069_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def textbook_cg(A, b, x0, iters):
    """Hestenes-Stiefel CG written in the usual b - A x convention.

    Independent of the paper's sign convention and of the oracle's block
    formulas: scalar steps alpha = r.r / d.Ad, beta = r'.r' / r.r.
    Returns the iterates x_0 .. x_iters (stops early on exact convergence).
    """
    x = x0.astype(np.float64).copy()
    r = b - A @ x
    d = r.copy()
    out = [x.copy()]
    rr = r @ r
    for _ in range(iters):
        if rr == 0.0:
            break
        Ad = A @ d
        a = rr / (d @ Ad)
        x = x + a * d
        r = r - a * Ad
        rr_new = r @ r
        d = r + (rr_new / rr) * d
        rr = rr_new
        out.append(x.copy())
    return out


def a_norm(A, v):
    return float(np.sqrt(max(v @ (A @ v), 0.0)))


# --------------------------------------------------------------------------
# Initial block generator
# --------------------------------------------------------------------------

def test_splitmix64_published_outputs(oracle_mod):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if ln.strip() and not ln.startswith("#")]
    for c, hexval in rows:
        assert oracle_mod.splitmix64_at(0, int(c)) == int(hexval, 16)


def test_initial_block_layout(oracle_mod):
    n, p = 50, 5
    x0 = np.linspace(-1, 1, n)
    X0 = oracle_mod.initial_block(n, p, x0, spread=2.0, seed=7)
    assert np.array_equal(X0[:, 0], x0)
    dev = X0[:, 1:] - x0[:, None]
    assert np.all(dev >= -2.0) and np.all(dev < 2.0)
    # entry (i, j) comes from counter j*n + i: check one against the generator
    i, j = 13, 3
    u = (oracle_mod.splitmix64_at(7, j * n + i) >> 11) * 2.0 ** -53
    assert X0[i, j] == x0[i] + 2.0 * (2.0 * u - 1.0)
    assert np.linalg.matrix_rank(X0 - x0[:, None] @ np.ones((1, p))) == p - 1


# --------------------------------------------------------------------------
# Final answer: direct solve (the unique minimiser x* = A^{-1} b, Sec. 2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,p,cond", [(8, 1, 10.0), (30, 3, 1e3), (64, 4, 1e3),
                                      (64, 5, 1e2), (33, 8, 1e2)])
def test_direct_solve(oracle_mod, n, p, cond):
    A, b = wl.random_spd(n, seed=n + p, cond=cond)
    X0 = wl.random_block(n, p, seed=1)
    r = oracle_mod.ccg(A, b, X0, tol=1e-13, maxit=10 * n)
    assert r["status"] == 0, r["status_name"]
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(r["x"] - xs) / np.linalg.norm(xs) <= 1e-10
    assert r["relres_true"] <= 1e-13


def test_relative_stop_test_is_scale_invariant(oracle_mod):
    """Stop rule min_j ||R e_j|| <= tol ||b|| (Algorithm 4, read as relative):
    scaling b and X_0 together scales every residue and leaves the iteration
    count unchanged; an absolute test would not.  A power-of-two scale makes
    every rounding scale with it, so the result scales bitwise."""
    A, b = wl.random_spd(40, seed=3, cond=50.0)
    X0 = wl.random_block(40, 3, seed=4)
    s = 2.0 ** 20
    r1 = oracle_mod.ccg(A, b, X0, tol=1e-9, maxit=400)
    r2 = oracle_mod.ccg(A, s * b, s * X0, tol=1e-9, maxit=400)
    assert r1["iterations"] == r2["iterations"]
    assert np.array_equal(r2["x"], s * r1["x"])


# --------------------------------------------------------------------------
# p = 1 is CG (Algorithm 1; "CG is the case p = 1", Sec. 3.2)
# --------------------------------------------------------------------------

def test_p1_equals_textbook_cg(oracle_mod):
    n = 48
    A, b = wl.random_spd(n, seed=11, cond=200.0)
    x0 = wl.random_block(n, 1, seed=12)[:, 0]
    r = oracle_mod.ccg(A, b, x0[:, None], tol=1e-10, maxit=500, trace=True,
                       residual_replacement=False)
    # Two algebraically equal CG recurrences drift apart at the rate rounding
    # errors are amplified (Greenbaum 1997); compare the early iterates, where
    # the drift is still at the 1e-14 level.
    xs_cg = textbook_cg(A, b, x0, 14)
    for st in r["trace"][1:15]:
        k = st["k"]
        xk = st["X"][:, 0]
        assert np.linalg.norm(xk - xs_cg[k]) <= 1e-12 * np.linalg.norm(xs_cg[k]), k
    # same iteration count to the same relative tolerance
    x = x0.copy()
    it = 0
    for it, xc in enumerate(textbook_cg(A, b, x0, 500)):
        if np.linalg.norm(A @ xc - b) <= 1e-10 * np.linalg.norm(b):
            break
    assert abs(r["iterations"] - it) <= 1


# --------------------------------------------------------------------------
# Theorem 2: orthogonality and A-conjugacy; subspace optimality
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [2, 3, 4])
def test_theorem2_orthogonality(oracle_mod, p):
    n = 60
    A, b = wl.random_spd(n, seed=21 + p, cond=20.0)
    X0 = wl.random_block(n, p, seed=22)
    r = oracle_mod.ccg(A, b, X0, tol=1e-14, maxit=6, trace=True,
                       residual_replacement=False)
    tr = r["trace"]
    assert len(tr) == 7
    Rs = [s["R"] for s in tr]
    Ds = [s["D"] for s in tr]
    for i in range(len(tr)):
        for j in range(i):
            # R_i^T R_j = 0 (columnwise cosines)
            C = Rs[i].T @ Rs[j]
            nrm = np.outer(np.linalg.norm(Rs[i], axis=0), np.linalg.norm(Rs[j], axis=0))
            assert np.max(np.abs(C) / nrm) <= 1e-9, (i, j)
            # D_i^T A D_j = 0
            Ca = Ds[i].T @ A @ Ds[j]
            na = np.outer(np.sqrt(np.einsum("ij,ij->j", Ds[i], A @ Ds[i])),
                          np.sqrt(np.einsum("ij,ij->j", Ds[j], A @ Ds[j])))
            assert np.max(np.abs(Ca) / na) <= 1e-9, (i, j)
    # local relations at every step: D_k^T R_{k+1} = 0 (alpha, Eq. 35) and
    # D_{k+1}^T A D_k = 0 (beta)
    for k in range(len(tr) - 1):
        Dk, Rk1, Dk1 = Ds[k], Rs[k + 1], Ds[k + 1]
        c1 = np.abs(Dk.T @ Rk1) / np.outer(np.linalg.norm(Dk, axis=0),
                                           np.linalg.norm(Rk1, axis=0))
        assert c1.max() <= 1e-10
        c2 = np.abs(Dk1.T @ A @ Dk)
        c2 /= np.outer(np.sqrt(np.einsum("ij,ij->j", Dk1, A @ Dk1)),
                       np.sqrt(np.einsum("ij,ij->j", Dk, A @ Dk)))
        assert c2.max() <= 1e-10


@pytest.mark.parametrize("p", [2, 3])
def test_theorem2_subspace_optimality(oracle_mod, p):
    """Column j of X_{k+1} minimises f(x) = x'Ax/2 - b'x on
    X_0 e_j + span[D_0 .. D_k]: solved here by brute force (projected normal
    equations with numpy)."""
    n = 36
    A, b = wl.random_spd(n, seed=31 + p, cond=30.0)
    X0 = wl.random_block(n, p, seed=32)
    r = oracle_mod.ccg(A, b, X0, tol=1e-14, maxit=5, trace=True,
                       residual_replacement=False)
    tr = r["trace"]
    for k in range(len(tr) - 1):
        V = np.concatenate([tr[i]["D"] for i in range(k + 1)], axis=1)
        Q, _ = np.linalg.qr(V)
        for j in range(p):
            rhs = Q.T @ (b - A @ X0[:, j])
            y = np.linalg.solve(Q.T @ A @ Q, rhs)
            xbest = X0[:, j] + Q @ y
            got = tr[k + 1]["X"][:, j]
            assert np.linalg.norm(got - xbest) <= 1e-9 * max(1.0, np.linalg.norm(xbest)), (k, j)


# --------------------------------------------------------------------------
# Theorem 3 / Theorem 4: finite termination
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,p", [(12, 1), (12, 2), (12, 3), (12, 4), (12, 6), (13, 4), (14, 3)])
def test_finite_termination(oracle_mod, n, p):
    A, b = wl.random_spd(n, seed=40 + n + p, cond=10.0)
    X0 = wl.random_block(n, p, seed=41)
    r = oracle_mod.ccg(A, b, X0, tol=1e-9, maxit=4 * n, residual_replacement=False)
    assert r["status"] == 0
    kstar = n // p
    # floor(n/p) cooperative steps, then at most n - p*floor(n/p) <= p-1 more
    assert r["iterations"] <= kstar + (n - p * kstar)
    assert r["iterations"] <= n  # Theorem 4


def test_rank_nonincreasing_and_bounded(oracle_mod):
    n, p = 40, 6
    A, b = wl.random_spd(n, seed=50, cond=100.0)
    X0 = wl.random_block(n, p, seed=51)
    r = oracle_mod.ccg(A, b, X0, tol=1e-12, maxit=10 * n, trace=True)
    pks = [s["X"].shape[1] for s in r["trace"]]
    assert all(pks[i + 1] <= pks[i] for i in range(len(pks) - 1))
    assert r["iterations"] <= n
    assert r["status"] == 0


# --------------------------------------------------------------------------
# Residual recurrence (proof of Theorem 2): R_{k+1} = A X_{k+1} - b 1^T
# --------------------------------------------------------------------------

def test_residual_recurrence(oracle_mod):
    n, p = 50, 4
    A, b = wl.random_spd(n, seed=60, cond=100.0)
    X0 = wl.random_block(n, p, seed=61)
    r = oracle_mod.ccg(A, b, X0, tol=1e-12, maxit=200, trace=True,
                       residual_replacement=False)
    nA = np.linalg.norm(A, 2)
    for st in r["trace"]:
        X, R = st["X"], st["R"]
        expl = A @ X - b[:, None]
        drift = np.linalg.norm(R - expl) / (nA * np.linalg.norm(X) + np.sqrt(X.shape[1]) * np.linalg.norm(b))
        assert drift <= 1e-12, st["k"]


# --------------------------------------------------------------------------
# Monotonicity and the CG error bound (Theorem 1, Eq. speed2)
# --------------------------------------------------------------------------

def test_monotone_objective(oracle_mod):
    n, p = 50, 4
    A, b = wl.random_spd(n, seed=70, cond=500.0)
    X0 = wl.random_block(n, p, seed=71)
    r = oracle_mod.ccg(A, b, X0, tol=1e-12, maxit=200, trace=True,
                       residual_replacement=False)
    f = lambda x: 0.5 * x @ (A @ x) - b @ x
    xs = np.linalg.solve(A, b)
    tr = r["trace"]
    for k in range(len(tr) - 1):
        for j in range(tr[k + 1]["X"].shape[1]):
            a = tr[k]["X"][:, j]
            c = tr[k + 1]["X"][:, j]
            assert f(c) <= f(a) + 1e-12 * abs(f(a))
            assert a_norm(A, c - xs) <= a_norm(A, a - xs) * (1 + 1e-9) + 1e-13


def test_cg_error_bound_and_agents_beat_cg(oracle_mod):
    n, p = 80, 4
    cond = 400.0
    A, b = wl.random_spd(n, seed=80, cond=cond)
    X0 = wl.random_block(n, p, seed=81)
    xs = np.linalg.solve(A, b)
    rate = (np.sqrt(cond) - 1) / (np.sqrt(cond) + 1)
    # p = 1: the Theorem 1 bound
    r1 = oracle_mod.ccg(A, b, X0[:, :1], tol=1e-13, maxit=400, trace=True,
                        residual_replacement=False)
    e0 = a_norm(A, X0[:, 0] - xs)
    for st in r1["trace"]:
        assert a_norm(A, st["X"][:, 0] - xs) <= 2 * rate ** st["k"] * e0 * (1 + 1e-9) + 1e-12
    # p > 1: agent j minimises over a block Krylov space containing the
    # single-vector one, so it is never worse than CG started from X_0 e_j
    rp = oracle_mod.ccg(A, b, X0, tol=1e-13, maxit=400, trace=True,
                        residual_replacement=False)
    cgs = [textbook_cg(A, b, X0[:, j], 60) for j in range(p)]
    for st in rp["trace"][:40]:
        k = st["k"]
        for c, j in enumerate(st["agents"]):
            if k < len(cgs[j]):
                ecg = a_norm(A, cgs[j][k] - xs)
                assert a_norm(A, st["X"][:, c] - xs) <= ecg * (1 + 1e-6) + 1e-10 * e0


# --------------------------------------------------------------------------
# p = 2 closed forms (Sec. 3.1, Eq. 3 and Eq. 7) with explicit 2x2 inverses
# --------------------------------------------------------------------------

def inv2(m):
    det = m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0]
    return np.array([[m[1, 1], -m[0, 1]], [-m[1, 0], m[0, 0]]]) / det


def test_p2_closed_forms(oracle_mod):
    n = 30
    A, b = wl.random_spd(n, seed=90, cond=50.0)
    X0 = wl.random_block(n, 2, seed=91)
    r = oracle_mod.ccg(A, b, X0, tol=1e-14, maxit=4, trace=True,
                       residual_replacement=False)
    tr = r["trace"]
    for k in range(len(tr) - 1):
        Rk, Dk = tr[k]["R"], tr[k]["D"]
        Rk1 = tr[k + 1]["R"]
        d, dp = Dk[:, 0], Dk[:, 1]
        r_, rp = Rk[:, 0], Rk[:, 1]
        # Eq. 3:  alpha = - (r r')^T (d d') ((d d')^T A (d d'))^{-1}
        Mi = inv2(np.array([[d @ A @ d, d @ A @ dp], [dp @ A @ d, dp @ A @ dp]]))
        RtD = np.array([[r_ @ d, r_ @ dp], [rp @ d, rp @ dp]])
        alpha = -RtD @ Mi
        # Eq. 7 (with the residues of step k+1): beta = -(r r')^T A (d d') M^{-1}
        r1, r1p = Rk1[:, 0], Rk1[:, 1]
        RtAD = np.array([[r1 @ A @ d, r1 @ A @ dp], [r1p @ A @ d, r1p @ A @ dp]])
        beta = -RtAD @ Mi
        np.testing.assert_allclose(tr[k + 1]["alpha"], alpha, rtol=1e-9, atol=1e-12 * np.abs(alpha).max())
        np.testing.assert_allclose(tr[k + 1]["beta"], beta, rtol=1e-9, atol=1e-12 * np.abs(beta).max())
        # and the updates X_{k+1} = X_k + D alpha^T, D_{k+1} = R_{k+1} + D beta^T
        np.testing.assert_allclose(tr[k + 1]["X"], tr[k]["X"] + Dk @ alpha.T, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(tr[k + 1]["D"], Rk1 + Dk @ beta.T, rtol=1e-10, atol=1e-12)


# --------------------------------------------------------------------------
# Algorithm 3 (mcCG): rank-deficient initial blocks
# --------------------------------------------------------------------------

def test_identical_agents_collapse_to_cg(oracle_mod):
    n = 40
    A, b = wl.random_spd(n, seed=100, cond=80.0)
    x0 = wl.random_block(n, 1, seed=101)
    X0 = np.repeat(x0, 4, axis=1)
    r4 = oracle_mod.ccg(A, b, X0, tol=1e-10, maxit=400)
    r1 = oracle_mod.ccg(A, b, x0, tol=1e-10, maxit=400)
    assert r4["p_final"] == 1 and r4["drops"] == 3
    assert r4["iterations"] == r1["iterations"]
    assert np.array_equal(r4["x"], r1["x"])


def test_affinely_dependent_agent_is_dropped(oracle_mod):
    n = 40
    A, b = wl.random_spd(n, seed=110, cond=80.0)
    X2 = wl.random_block(n, 2, seed=111)
    # agent 2 = midpoint of agents 0 and 1  =>  R_0 e_2 = (R_0 e_0 + R_0 e_1)/2
    X3 = np.concatenate([X2, 0.5 * (X2[:, :1] + X2[:, 1:2])], axis=1)
    r3 = oracle_mod.ccg(A, b, X3, tol=1e-10, maxit=400)
    r2 = oracle_mod.ccg(A, b, X2, tol=1e-10, maxit=400)
    assert r3["p_final"] == 2 and r3["drops"] == 1
    assert list(r3["agents"]) == [0, 1]
    assert r3["iterations"] == r2["iterations"]
    assert np.array_equal(r3["x"], r2["x"])


def test_rank_test_threshold_on_the_scaled_pivot(oracle_mod):
    """Algorithm 3 drops an agent whose direction is numerically dependent on
    the agents before it.  Reading of the rank test: Cholesky of the
    unit-diagonal scaling S M S of M = D'AD, S = diag(M)^(-1/2), in agent
    order; agent j is dropped when the squared pivot l_jj^2 (the squared
    A-sine between d_j and the span of the earlier directions) is below
    rank_tol.  The pivot is computed here with LAPACK, and rank_tol is put a
    decade on either side of it; the blocks are scaled far from unit norm, so
    an unscaled pivot, an unsquared one or the wrong agent order changes the
    decision."""
    n = 30
    A, b = wl.random_spd(n, seed=120, cond=20.0)
    Xab = 50.0 * wl.random_block(n, 2, seed=121)
    w = wl.random_block(n, 1, seed=122)
    X0 = np.concatenate([Xab, Xab[:, :1] + 2e-2 * w], axis=1)
    D0 = A @ X0 - b[:, None]
    M = D0.T @ A @ D0
    s = 1.0 / np.sqrt(np.diag(M))
    L = np.linalg.cholesky(M * s[:, None] * s[None, :])
    piv = np.diag(L) ** 2
    assert piv[0] == pytest.approx(1.0) and piv[1] > 1e-2
    assert 1e-9 < piv[2] < 1e-4          # agent 2 nearly repeats agent 0
    assert np.diag(M)[2] > 1e3            # far from unit scale
    kept = oracle_mod.ccg(A, b, X0, tol=1e-14, maxit=1, rank_tol=piv[2] / 10)
    assert kept["p_final"] == 3 and kept["drops"] == 0
    dropped = oracle_mod.ccg(A, b, X0, tol=1e-14, maxit=1, rank_tol=piv[2] * 10)
    assert dropped["p_final"] == 2 and dropped["drops"] == 1
    assert list(dropped["agents"]) == [0, 1]
    # the same three starts in another order: the later of the two near
    # copies is the one dropped
    Xr = X0[:, [2, 1, 0]]
    again = oracle_mod.ccg(A, b, Xr, tol=1e-14, maxit=1, rank_tol=piv[2] * 10)
    assert again["drops"] == 1 and list(again["agents"]) == [0, 1]


# --------------------------------------------------------------------------
# Edge cases and errors
# --------------------------------------------------------------------------

def test_zero_rhs_returns_zero(oracle_mod):
    A, _ = wl.random_spd(10, seed=1)
    r = oracle_mod.ccg(A, np.zeros(10), wl.random_block(10, 3, seed=2), 1e-10, 100)
    assert r["status"] == 0 and r["iterations"] == 0 and not r["x"].any()


def test_exact_start_needs_no_iteration(oracle_mod):
    A, b = wl.random_spd(10, seed=3, cond=5.0)
    xs = np.linalg.solve(A, b)
    X0 = np.stack([xs, xs + 1.0], axis=1)
    r = oracle_mod.ccg(A, b, X0, 1e-8, 100)
    assert r["status"] == 0 and r["iterations"] == 0 and r["agent"] == 0


def test_maxit_zero_and_not_converged(oracle_mod):
    A, b = wl.random_spd(20, seed=4, cond=50.0)
    r = oracle_mod.ccg(A, b, wl.random_block(20, 2, seed=5), 1e-10, 0)
    assert r["status"] == 1 and r["iterations"] == 0
    r = oracle_mod.ccg(A, b, wl.random_block(20, 2, seed=5), 1e-14, 3)
    assert r["status"] == 1 and r["iterations"] == 3


def test_invalid_arguments(oracle_mod):
    A, b = wl.random_spd(10, seed=6)
    assert oracle_mod.ccg(A, b, wl.random_block(10, 2, seed=1), -1.0, 10)["status"] == -1
    assert oracle_mod.ccg(A[:4, :4], b[:4], wl.random_block(4, 5, seed=1), 1e-8, 10)["status"] == -1


def test_indefinite_matrix_detected(oracle_mod):
    n = 20
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(-3.0, 5.0, n)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    r = oracle_mod.ccg(A, b, wl.random_block(n, 3, seed=8), 1e-10, 200)
    assert r["status"] == -2


def test_nan_input_detected(oracle_mod):
    A, b = wl.random_spd(10, seed=9)
    b[3] = np.nan
    assert oracle_mod.ccg(A, b, wl.random_block(10, 2, seed=1), 1e-8, 10)["status"] == -3


def test_true_relres_helper_matches_numpy(oracle_mod):
    """The oracle's exit check ||b - A x|| / ||b|| (Algorithm 4's stop test
    verified on the true residual) against numpy's norm of b - A @ x."""
    A, b = wl.random_spd(37, seed=17, cond=30.0)
    x = wl.random_block(37, 1, seed=18)[:, 0]
    ref = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(oracle_mod.true_relres(A, b, x) - ref) <= 1e-14 * ref


# --------------------------------------------------------------------------
# Explicit residual: Algorithm 2 as printed forms R_{k+1} = A X_{k+1} - b 1^T
# (a second product with A per iteration, as Algorithm 4 does); the proof of
# Theorem 2 shows it equals the recurrence in exact arithmetic.
# --------------------------------------------------------------------------

def textbook_cg_recomputed(A, b, x0, iters):
    """Textbook CG whose residual is recomputed as b - A x at every step."""
    x = x0.astype(np.float64).copy()
    r = b - A @ x
    d = r.copy()
    out = [x.copy()]
    rr = r @ r
    for _ in range(iters):
        if rr == 0.0:
            break
        Ad = A @ d
        a = rr / (d @ Ad)
        x = x + a * d
        r = b - A @ x
        rr_new = r @ r
        d = r + (rr_new / rr) * d
        rr = rr_new
        out.append(x.copy())
    return out


def test_explicit_residual_p1_equals_textbook_cg(oracle_mod):
    n = 64
    A, b = wl.random_spd(n, seed=21, cond=30.0)
    x0 = wl.random_block(n, 1, seed=22)[:, 0]
    r = oracle_mod.ccg(A, b, x0[:, None], tol=1e-10, maxit=500, trace=True,
                       residual_replacement=False, explicit_residual=True)
    xs_cg = textbook_cg_recomputed(A, b, x0, 14)
    for st in r["trace"][1:15]:
        k = st["k"]
        assert np.linalg.norm(st["X"][:, 0] - xs_cg[k]) <= 1e-12 * np.linalg.norm(xs_cg[k]), k
    it = 0
    for it, xc in enumerate(textbook_cg_recomputed(A, b, x0, 500)):
        if np.linalg.norm(A @ xc - b) <= 1e-10 * np.linalg.norm(b):
            break
    assert abs(r["iterations"] - it) <= 1


@pytest.mark.parametrize("n,p,cond", [(30, 3, 1e3), (64, 4, 1e3), (33, 8, 1e2)])
def test_explicit_residual_direct_solve(oracle_mod, n, p, cond):
    A, b = wl.random_spd(n, seed=n + 7 * p, cond=cond)
    X0 = wl.random_block(n, p, seed=2)
    r = oracle_mod.ccg(A, b, X0, tol=1e-13, maxit=10 * n, explicit_residual=True)
    assert r["status"] == 0, r["status_name"]
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(r["x"] - xs) / np.linalg.norm(xs) <= 1e-10


def test_explicit_residual_trace_is_the_true_residual(oracle_mod):
    n, p = 40, 3
    A, b = wl.random_spd(n, seed=31, cond=100.0)
    X0 = wl.random_block(n, p, seed=32)
    r = oracle_mod.ccg(A, b, X0, tol=1e-12, maxit=200, trace=True,
                       residual_replacement=False, explicit_residual=True)
    for st in r["trace"]:
        true = A @ st["X"] - b[:, None]
        scale = np.abs(A) @ np.abs(st["X"]) + np.abs(b)[:, None]
        assert np.all(np.abs(st["R"] - true) <= 1e-13 * scale), st["k"]


def test_explicit_and_recurrence_forms_agree_early(oracle_mod):
    n, p = 60, 4
    A, b = wl.random_spd(n, seed=41, cond=100.0)
    X0 = wl.random_block(n, p, seed=42)
    kw = dict(tol=1e-12, maxit=200, trace=True, residual_replacement=False)
    r1 = oracle_mod.ccg(A, b, X0, **kw)
    r2 = oracle_mod.ccg(A, b, X0, explicit_residual=True, **kw)
    for s1, s2 in zip(r1["trace"][1:6], r2["trace"][1:6]):
        assert np.array_equal(s1["agents"], s2["agents"])
        assert np.linalg.norm(s1["X"] - s2["X"]) <= 1e-11 * np.linalg.norm(s1["X"])
    assert abs(r1["iterations"] - r2["iterations"]) <= 2


# --------------------------------------------------------------------------
# Summation order of the block product (a rounding choice the method leaves
# open).  Each order must be exactly the plain sum it names, and all of them
# the same solve up to rounding.
# --------------------------------------------------------------------------

def python_sum(terms, order):
    """The plain FP64 sum of `terms` in the named order, one Python float
    addition at a time (Python floats are IEEE binary64)."""
    n = len(terms)
    if order == 0:
        idx = range(n)
    elif order == 1:
        idx = range(n - 1, -1, -1)
    if order in (0, 1):
        s = 0.0
        for i in idx:
            s += terms[i]
        return s
    if order == 2:
        s = 0.0
        for l0 in range(0, n, 64):
            part = 0.0
            for i in range(l0, min(n, l0 + 64)):
                part += terms[i]
            s += part
        return s
    parts = [0.0] * 64
    for i in range(n):
        parts[i % 64] += terms[i]
    s = 0.0
    for t in parts:
        s += t
    return s


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_block_product_orders_are_the_plain_sums(oracle_mod, order):
    """Each entry of W = A V equals the sequential Python sum of the products
    A_il V_lc (each product rounded once) in the order named, bit for bit."""
    rng = np.random.default_rng(40 + order)
    n, q = 150, 3
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-8, 8, (n, n)))
    V = rng.standard_normal((n, q))
    W = oracle_mod.block_product(A, V, order)
    for i in range(0, n, 7):
        for c in range(q):
            terms = [float(A[i, l] * V[l, c]) for l in range(n)]
            assert W[i, c] == python_sum(terms, order), (i, c)


def test_block_product_orders_within_the_rounding_bound(oracle_mod):
    """|fl(sum) - sum| <= gamma_n sum |a_l v_l| (Higham, Thm. 3.1) in every
    order, against the product in extended precision; the orders differ."""
    rng = np.random.default_rng(44)
    n, q = 1000, 4
    A = rng.standard_normal((n, n))
    V = rng.standard_normal((n, q))
    exact = (A.astype(np.longdouble) @ V.astype(np.longdouble)).astype(np.float64)
    u = 2.0 ** -53
    bound = n * u / (1 - n * u) * (np.abs(A) @ np.abs(V))
    Ws = [oracle_mod.block_product(A, V, o) for o in oracle_mod.PRODUCT_ORDERS]
    for W in Ws:
        assert np.all(np.abs(W - exact) <= bound)
    assert not np.array_equal(Ws[0], Ws[1])


def test_solve_does_not_depend_on_the_product_order_when_well_conditioned(oracle_mod):
    """On a well-conditioned system (kappa = 9) the five orders give the same
    iteration count and answers within a few roundings of each other."""
    A, b = wl.gram_shift(256, seed=0, shift=0.5)
    X0 = oracle_mod.initial_block(256, 4, None, 1.0, 0)
    rs = [oracle_mod.ccg(A, b, X0, 1e-10, 2560, product_order=o)
          for o in oracle_mod.PRODUCT_ORDERS]
    assert len({r["iterations"] for r in rs}) == 1
    for r in rs[1:]:
        assert np.linalg.norm(r["x"] - rs[0]["x"]) <= 1e-13 * np.linalg.norm(rs[0]["x"])


def test_compensated_block_product_is_nearly_exact(oracle_mod):
    """Order 4 (Dot2, Ogita-Rump-Oishi 2005, Prop. 5.5):
    |W - S| <= u |S| + gamma_n^2 sum_l |A_il V_lc|, S the exact sum (rational
    arithmetic), on entries with heavy cancellation."""
    from fractions import Fraction
    rng = np.random.default_rng(46)
    n, q = 120, 2
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-20, 20, (n, n)))
    V = rng.standard_normal((n, q))
    W = oracle_mod.block_product(A, V, 4)
    u = 2.0 ** -53
    g = n * u / (1 - n * u)
    for i in range(0, n, 11):
        for c in range(q):
            S = sum((Fraction(float(A[i, l])) * Fraction(float(V[l, c])) for l in range(n)),
                    Fraction(0))
            mag = sum(abs(float(A[i, l]) * float(V[l, c])) for l in range(n))
            assert abs(Fraction(float(W[i, c])) - S) <= Fraction(u) * abs(S) + Fraction(g * g * mag)
