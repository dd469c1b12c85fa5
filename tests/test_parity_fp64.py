"""GPU parity of the FP64 persistent cCG solver against the FP64 oracle.

Tolerances (from the method's target): true relative residual <= tol (1e-10),
||x - x_oracle|| / ||x_oracle|| <= 1e-8, iteration counts within 2.  Iterates
after a fixed number of steps are compared element by element at 1e-9
relative (both sides run the same formulas; only the summation order of the
block product and of the Gram sums differs).  Integer outputs (iterations
when exact, agent ids, deflation counts) compare exactly where the method
fixes them.
"""
import numpy as np
import pytest
from envelope import oracle_counts, within_envelope

from paper_1204_0069_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_0069_gb300 import build as B
    B.build()
    import oracle
    oracle.build()
    from paper_1204_0069_gb300 import ccg
    s = ccg.Solver(device=0)
    yield dict(torch=torch, ccg=ccg, solver=s, oracle=oracle)
    s.close()


def dev(env, a):
    return env["torch"].from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gpu_solve(env, A, b, p, tol=TOL, maxit=None, x0=None):
    torch = env["torch"]
    n = b.shape[0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    r = env["solver"].solve(dev(env, A), dev(env, b), x, p=p, tol=tol,
                            maxit=maxit if maxit is not None else 20 * n,
                            x0=None if x0 is None else dev(env, x0))
    torch.cuda.synchronize()
    return r, x.cpu().numpy()


def check_against_oracle(env, A, b, p, tol=TOL, maxit=None):
    n = b.shape[0]
    maxit = maxit if maxit is not None else 20 * n
    r, x = gpu_solve(env, A, b, p, tol, maxit)
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, tol, maxit, nthreads=8)
    assert ref["status"] == 0, ref["status_name"]
    assert r.status == 0, r
    assert r.relres_true <= tol
    xt = np.linalg.norm(A @ x - b) / np.linalg.norm(b)
    assert xt <= tol * 1.01, xt  # independent FP64 check of the returned x
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= 1e-8, err
    assert abs(r.iterations - ref["iterations"]) <= 2, (r.iterations, ref["iterations"])
    assert r.p_final == ref["p_final"]
    return r, ref


def test_small_gram_system_n256_p4(env):
    A, b = wl.gram_shift(256, seed=0, shift=0.5)
    check_against_oracle(env, A, b, 4)


@pytest.mark.parametrize("n,p", [(13, 1), (13, 4), (64, 3), (100, 5), (257, 8), (300, 16),
                                 (333, 17), (520, 32), (1000, 2), (1031, 7), (2048, 32)])
def test_random_spd_against_oracle(env, n, p):
    A, b = wl.random_spd(n, seed=n * 7 + p, cond=300.0)
    check_against_oracle(env, A, b, p)


@pytest.mark.parametrize("p", [1, 4, 8])
def test_exp_kernel_n2048(env, p):
    A, b = wl.exp_kernel(2048, seed=1, length=0.2, nugget=1e-2)
    check_against_oracle(env, A, b, p)


@pytest.mark.parametrize("n,p,k", [(200, 4, 1), (200, 4, 3), (333, 7, 5), (1030, 16, 4),
                                   (129, 1, 6)])
def test_iterates_after_k_steps_elementwise(env, n, p, k):
    """X_k after exactly k iterations, element by element (explicit X0)."""
    torch = env["torch"]
    A, b = wl.random_spd(n, seed=n + k, cond=100.0)
    X0 = wl.random_block(n, p, seed=k)
    s = env["ccg"].Solver(device=0, residual_replacement=False)
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    Xo = torch.zeros((n, p), dtype=torch.float64, device="cuda:0")
    r = s.solve_block(dev(env, A), dev(env, b), dev(env, X0), x, tol=1e-300, maxit=k, X_out=Xo)
    s.close()
    ref = env["oracle"].ccg(A, b, X0, 1e-300, k, residual_replacement=False)
    assert r.status == 1 and ref["status"] == 1
    assert r.iterations == k == ref["iterations"]
    Xg = Xo.cpu().numpy()[:, list(ref["agents"])]
    np.testing.assert_allclose(Xg, ref["X"], rtol=1e-9, atol=1e-9 * np.abs(ref["X"]).max())


@pytest.mark.parametrize("n,q", [(1, 1), (7, 3), (63, 4), (129, 5), (1000, 8), (1031, 16),
                                 (777, 17), (640, 32), (4100, 1)])
def test_block_product_and_grams(env, n, q):
    torch = env["torch"]
    rng = np.random.default_rng(n + q)
    A = rng.standard_normal((n, n))
    A = 0.5 * (A + A.T)
    V = rng.standard_normal((n, q))
    U = rng.standard_normal((n, q))
    W = torch.zeros((n, q), dtype=torch.float64, device="cuda:0")
    rc, M, G, _ = env["solver"].block_product(dev(env, A), dev(env, V), W, U=dev(env, U))
    assert rc == 0
    Wr = A @ V
    np.testing.assert_allclose(W.cpu().numpy(), Wr, rtol=0, atol=1e-12 * np.abs(A).sum(1).max() * np.abs(V).max())
    Mr = V.T @ Wr
    Mr = 0.5 * (Mr + Mr.T)
    np.testing.assert_allclose(M, Mr, rtol=1e-11, atol=1e-11 * np.abs(Mr).max())
    np.testing.assert_allclose(G, U.T @ V, rtol=1e-11, atol=1e-11 * np.abs(U.T @ V).max())


def exact_gram(U, V):
    """U' V in exact rational arithmetic (every double is a dyadic rational)."""
    from fractions import Fraction
    Uf = [[Fraction(float(x)) for x in col] for col in U.T]
    Vf = [[Fraction(float(x)) for x in col] for col in V.T]
    return [[sum((a * b for a, b in zip(u, v)), Fraction(0)) for v in Vf] for u in Uf]


@pytest.mark.parametrize("max_ctas", [0, 1])
def test_grams_within_one_rounding_of_exact(env, max_ctas):
    """The Gram sums of Table 1 (M = V'AV, G = U'V) are accumulated exactly
    per lane in a long integer accumulator and combined across lanes and CTAs
    in doubled precision, so every entry is the exact sum rounded once, up to
    2^-90 sum_i |u_i v_i| (plus the FP64 underflow unit).  Inputs: entries
    over 50 decades, a pair of columns made orthogonal (cancellation to the
    rounding level), products in the subnormal range and near 1e176."""
    from fractions import Fraction
    torch, ccg = env["torch"], env["ccg"]
    n, q = 3000, 4
    rng = np.random.default_rng(21)
    U = rng.standard_normal((n, q)) * np.exp(rng.uniform(-30, 30, (n, q)))
    V = rng.standard_normal((n, q)) * np.exp(rng.uniform(-30, 30, (n, q)))
    V[:, 1] -= (U[:, 0] @ V[:, 1]) / (U[:, 0] @ U[:, 0]) * U[:, 0]
    U[:, 2] *= 1e-160
    V[:, 2] *= 1e-160
    U[:, 3] *= 1e150
    A = np.eye(n)
    W = torch.zeros((n, q), dtype=torch.float64, device="cuda:0")
    with ccg.Solver(device=0, max_ctas=max_ctas) as s:
        rc, M, G, _ = s.block_product(dev(env, A), dev(env, V), W, U=dev(env, U))
    assert rc == 0
    assert np.array_equal(W.cpu().numpy(), V)
    tiny = Fraction(2) ** -1074
    for got, X, Y in ((G, U, V), (M, V, V)):
        ex = exact_gram(X, Y)
        mag = np.abs(X).T @ np.abs(Y)
        for a in range(q):
            for c in range(q):
                S = ex[a][c]
                err = abs(Fraction(float(got[a, c])) - S)
                bound = Fraction(2) ** -53 * abs(S) + Fraction(2) ** -90 * Fraction(float(mag[a, c])) * 2 + tiny
                assert err <= bound, (a, c, float(err), float(bound))


def test_block_product_odd_lda_and_host_buffers(env):
    """Unaligned leading dimension (scalar A stream) and host pointers."""
    n, q, lda = 301, 6, 303
    rng = np.random.default_rng(5)
    Afull = rng.standard_normal((n, lda))
    V = rng.standard_normal((n, q))
    W = np.zeros((n, q))
    rc, M, _, _ = env["solver"].block_product(Afull, V, W, lda=lda)
    assert rc == 0
    np.testing.assert_allclose(W, Afull[:, :n] @ V, rtol=0, atol=1e-11)


def test_host_and_device_pointers_agree_bitwise(env):
    torch = env["torch"]
    A, b = wl.random_spd(500, seed=3, cond=200.0)
    r1, x1 = gpu_solve(env, A, b, 6)
    xh = np.zeros(500)
    r2 = env["solver"].solve(A, b, xh, p=6, tol=TOL, maxit=10000)
    assert r1.iterations == r2.iterations
    assert np.array_equal(x1, xh)


def test_runs_are_bitwise_reproducible(env):
    A, b = wl.exp_kernel(1500, seed=4, length=0.3, nugget=1e-2)
    outs = [gpu_solve(env, A, b, 8) for _ in range(3)]
    for r, x in outs[1:]:
        assert r.iterations == outs[0][0].iterations
        assert np.array_equal(x, outs[0][1])


def test_x0_is_used(env):
    A, b = wl.random_spd(200, seed=8, cond=50.0)
    xs = np.linalg.solve(A, b)
    r, x = gpu_solve(env, A, b, 3, x0=xs)
    assert r.status == 0 and r.iterations == 0 and r.agent == 0


def test_zero_rhs(env):
    A, _ = wl.random_spd(50, seed=9)
    r, x = gpu_solve(env, A, np.zeros(50), 4)
    assert r.status == 0 and r.iterations == 0 and not x.any()


def test_maxit_zero_not_converged(env):
    A, b = wl.random_spd(50, seed=10, cond=50.0)
    r, _ = gpu_solve(env, A, b, 2, maxit=0)
    assert r.status == 1 and r.iterations == 0


def test_deflation_identical_agents(env):
    torch = env["torch"]
    n = 120
    A, b = wl.random_spd(n, seed=11, cond=80.0)
    x0 = wl.random_block(n, 1, seed=12)
    X0 = np.repeat(x0, 5, axis=1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    r = env["solver"].solve_block(dev(env, A), dev(env, b), dev(env, X0), x, tol=TOL, maxit=2000)
    ref = env["oracle"].ccg(A, b, X0, TOL, 2000)
    assert r.status == 0 and r.p_final == 1 and r.drops == 4
    assert ref["p_final"] == 1
    assert abs(r.iterations - ref["iterations"]) <= 2
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    r1 = env["solver"].solve_block(dev(env, A), dev(env, b), dev(env, x0), x1, tol=TOL, maxit=2000)
    assert abs(r1.iterations - r.iterations) <= 2


def test_deflation_affine_dependent_agent(env):
    torch = env["torch"]
    n = 150
    A, b = wl.random_spd(n, seed=13, cond=80.0)
    X2 = wl.random_block(n, 2, seed=14)
    X3 = np.concatenate([X2, 0.5 * (X2[:, :1] + X2[:, 1:2])], axis=1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    Xo = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda:0")
    r = env["solver"].solve_block(dev(env, A), dev(env, b), dev(env, X3), x, tol=TOL,
                                  maxit=2000, X_out=Xo)
    assert r.status == 0 and r.p_final == 2 and r.drops == 1
    Xo = Xo.cpu().numpy()
    assert not np.isnan(Xo).any()  # dropped agent's column holds its iterate
    np.testing.assert_allclose(Xo[:, 2], X3[:, 2], rtol=0, atol=0)  # dropped at k = 0


def test_invalid_arguments(env):
    torch = env["torch"]
    A, b = wl.random_spd(10, seed=1)
    x = torch.zeros(10, dtype=torch.float64, device="cuda:0")
    s = env["solver"]
    assert s.solve(dev(env, A), dev(env, b), x, p=11, tol=1e-8, maxit=10).status == -1
    assert s.solve(dev(env, A), dev(env, b), x, p=2, tol=0.0, maxit=10).status == -1
    assert s.solve(dev(env, A), dev(env, b), x, p=2, tol=1e-8, maxit=-1).status == -1
    assert s.solve(dev(env, A), dev(env, b), x, p=2, tol=1e-8, maxit=10, lda=5).status == -1


def test_indefinite_matrix_reports_not_spd(env):
    n = 40
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * np.linspace(-3.0, 5.0, n)) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    r, _ = gpu_solve(env, A, b, 3, maxit=400)
    assert r.status == -2


def test_nan_rhs_reports_numerical(env):
    A, b = wl.random_spd(30, seed=15)
    b[4] = np.nan
    r, _ = gpu_solve(env, A, b, 2)
    assert r.status == -3


def test_barrier_wait_limit_returns_timeout_and_handle_survives(env):
    s = env["solver"]
    assert s.selftest_barrier_timeout(200.0) == -5
    A, b = wl.random_spd(64, seed=16, cond=10.0)
    r, _ = gpu_solve(env, A, b, 2)
    assert r.status == 0


# Residual replacement (exit rule of Algorithm 4 with the recurrence of the
# proof of Thm. 2): the agents start far from the solution (entries ~ 1e5 to
# 1e6 against a solution of order 1), so the recurrence residual R carries
# rounding errors of order u ||A|| ||X_0|| while it keeps decreasing; it meets
# tol well before the true residual b - A x does, the true-residual check
# fails, R is replaced by A X - b 1^T and D by R, and the iteration continues
# to tol.  The oracle fires exactly one replacement on these systems in every
# summation order of its block product.  How many iterations follow the
# replacement is set by the rounding the early iterations left in X, so it
# depends on the accuracy of the product (the compensated product needs 6 to
# 14 fewer than the ascending sum); the count is held to the oracle's
# envelope over its orders (tests/envelope.py).
REPLACEMENT_CASES = [(200, 100.0, 3, 1e6), (500, 100.0, 4, 1e6), (2048, 100.0, 8, 1e5),
                     (1031, 300.0, 7, 1e7)]


@pytest.mark.parametrize("n,cond,p,scale", REPLACEMENT_CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp64_sliced"])
def test_residual_replacement_against_oracle(env, n, cond, p, scale, precision):
    torch, ccg = env["torch"], env["ccg"]
    A, b = wl.random_spd(n, seed=33, cond=cond)
    X0 = wl.random_block(n, p, seed=1, scale=scale)
    ref, counts, status = oracle_counts(env["oracle"], A, b, X0, TOL, 20 * n)
    assert all(st == 0 for st in status), status
    assert ref["replacements"] == 1, ref["replacements"]
    pol = ccg.FP64 if precision == "fp64" else ccg.FP64_SLICED
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    with ccg.Solver(device=0, precision=pol) as s:
        r = s.solve_block(dev(env, A), dev(env, b), dev(env, X0), x, tol=TOL, maxit=20 * n)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    assert r.status == 0, r
    assert r.replacements == 1, r
    assert r.relres_true <= TOL
    assert np.linalg.norm(A @ xg - b) / np.linalg.norm(b) <= TOL * 1.01
    assert np.linalg.norm(xg - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert within_envelope(r.iterations, counts), (r.iterations, counts)


@pytest.mark.parametrize("n,p", [(64, 3), (257, 8), (1031, 7), (2048, 16)])
def test_explicit_residual_against_oracle(env, n, p):
    """Algorithm 2 as printed: R_{k+1} = A X_{k+1} - b 1^T each iteration."""
    torch = env["torch"]
    A, b = wl.random_spd(n, seed=n * 5 + p, cond=300.0)
    x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    with env["ccg"].Solver(device=0, explicit_residual=True) as s:
        r = s.solve(dev(env, A), dev(env, b), x, p=p, tol=TOL, maxit=20 * n)
    torch.cuda.synchronize()
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, TOL, 20 * n, nthreads=8, explicit_residual=True)
    assert ref["status"] == 0 and r.status == 0, (ref["status_name"], r)
    xg = x.cpu().numpy()
    assert np.linalg.norm(A @ xg - b) / np.linalg.norm(b) <= TOL * 1.01
    assert np.linalg.norm(xg - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert abs(r.iterations - ref["iterations"]) <= 2, (r.iterations, ref["iterations"])


def test_explicit_residual_rejected_with_mixed_precision(env):
    with pytest.raises(RuntimeError):
        env["ccg"].Solver(device=0, explicit_residual=True, precision=env["ccg"].FP32_IR)
