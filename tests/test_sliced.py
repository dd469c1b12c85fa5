"""GPU tests of the sliced FP64 path: the block product A D formed on the FP8
tensor cores from an error-free split of A and D into 4-bit integer slices
(Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012), and the FP64 cCG
solve built on it.

Block product bound, from the construction: slicing A's row i to 14 slices
(rounded to nearest) drops at most 2^-57 of 2^e_i <= 2 max_k |A_ik| per entry
(same for D's column j), every slice product is exact in the FP32 accumulator, and the
slices are combined in FP64 (at most ~60 roundings of partial sums bounded by
(|A| |D|)_ij).  So

  |W - A D|_ij <= 2^-56 (max_k |A_ik| sum_k |D_kj| + max_k |D_kj| sum_k |A_ik|)
                 + 64 * 2^-53 (|A| |D|)_ij,

checked against the product in extended precision (numpy longdouble).  The
solve is held to the FP64 parity bar against the FP64 oracle.
"""
import numpy as np
import pytest

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


def exact_product(A, V):
    return (A.astype(np.longdouble) @ V.astype(np.longdouble)).astype(np.float64)


@pytest.mark.parametrize("n,q", [(1, 1), (100, 3), (128, 8), (300, 16), (1031, 5), (2100, 16)])
def test_sliced_block_product_is_fp64_accurate(env, n, q):
    torch = env["torch"]
    rng = np.random.default_rng(7 * n + q)
    # entries over several decades, signs mixed, and a row of zeros
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-6, 6, (n, n)))
    A[n // 2, :] = 0.0
    V = rng.standard_normal((n, q)) * np.exp(rng.uniform(-4, 4, (n, q)))
    m = env["solver"].lowp_matrix(torch.from_numpy(A).cuda(), env["ccg"].LOWP_FP64_SLICED)
    W = torch.zeros((n, q), dtype=torch.float64, device="cuda")
    dV = torch.from_numpy(V).cuda()
    rc, _ = m.block_product(dV, W)
    assert rc == 0
    Wg = W.cpu().numpy()
    ref = exact_product(A, V)
    absA, absV = np.abs(A), np.abs(V)
    bound = (2.0 ** -56 * (absA.max(axis=1)[:, None] * absV.sum(axis=0)[None, :]
                           + absV.max(axis=0)[None, :] * absA.sum(axis=1)[:, None])
             + 64 * 2.0 ** -53 * (absA @ absV))
    err = np.abs(Wg - ref)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    # as accurate as FP64 matrix multiplication on the same data (or better)
    err64 = np.abs(A @ V - ref)
    assert err.max() <= 4.0 * err64.max() + 1e-300
    W2 = torch.zeros_like(W)
    assert m.block_product(dV, W2)[0] == 0
    assert torch.equal(W, W2)  # fixed-order combination: bitwise repeatable
    m.close()


def test_sliced_format_bytes_and_limits(env):
    torch, ccg = env["torch"], env["ccg"]
    n = 300
    A = np.eye(n)
    m = env["solver"].lowp_matrix(A, ccg.LOWP_FP64_SLICED)  # host A staged inside
    assert m.nbytes() == 14 * 384 * 384 + 4 * n  # 14 slices of padded rows, row scales
    V = np.ones((n, 17))
    W = np.zeros((n, 17))
    assert m.block_product(V, W)[0] == -1       # at most 16 operand columns
    m.close()
    with pytest.raises(RuntimeError):
        with ccg.Solver(device=0, precision=ccg.FP64_SLICED, explicit_residual=True):
            pass


def solve_sliced(env, A, b, p, tol=TOL, host=False):
    torch, ccg = env["torch"], env["ccg"]
    n = b.shape[0]
    with ccg.Solver(device=0, precision=ccg.FP64_SLICED) as s:
        if host:
            x = np.zeros(n)
            r = s.solve(np.ascontiguousarray(A), b, x, p=p, tol=tol, maxit=20 * n)
            return r, x
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        r = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), x, p=p, tol=tol,
                    maxit=20 * n)
        torch.cuda.synchronize()
        return r, x.cpu().numpy()


@pytest.mark.parametrize("n,p", [(13, 1), (64, 3), (257, 8), (300, 16), (1031, 7), (2048, 16)])
def test_sliced_solve_matches_oracle(env, n, p):
    A, b = wl.random_spd(n, seed=n * 11 + p, cond=300.0)
    r, x = solve_sliced(env, A, b, p)
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, TOL, 20 * n, nthreads=8)
    assert ref["status"] == 0 and r.status == 0, (ref["status_name"], r)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= TOL * 1.01
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert abs(r.iterations - ref["iterations"]) <= 2, (r.iterations, ref["iterations"])
    assert r.p_final == ref["p_final"]


@pytest.mark.parametrize("p", [1, 8, 16])
def test_sliced_solve_exp_kernel_n2048(env, p):
    """Ill-conditioned kernel matrix (kappa ~ 1e4).  The sliced block product
    is closer to the exact product than the oracle's sequential FP64 sum (whose
    rounding is ~sqrt(n) 2^-53 relative), and at this conditioning the
    iteration count follows such ulp-level differences: the count may differ
    by 3 % of the iterations (at least 2), the answer by nothing beyond the
    FP64 bar."""
    A, b = wl.exp_kernel(2048, seed=4, length=0.2, nugget=1e-2)
    r, x = solve_sliced(env, A, b, p)
    X0 = env["oracle"].initial_block(2048, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, TOL, 20 * 2048, nthreads=8)
    assert r.status == 0 and ref["status"] == 0
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= TOL * 1.01
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert abs(r.iterations - ref["iterations"]) <= max(2, 0.03 * ref["iterations"]), (
        r.iterations, ref["iterations"])


def test_sliced_solve_host_buffers_and_odd_lda(env):
    n, p = 301, 4
    A, b = wl.random_spd(n, seed=5, cond=100.0)
    r1, x1 = solve_sliced(env, A, b, p, host=True)
    r2, x2 = solve_sliced(env, A, b, p)
    assert r1.status == 0 and r2.status == 0
    assert np.array_equal(x1, x2)   # same grid and data: bitwise the same


def test_sliced_rejects_more_than_16_agents(env):
    A, b = wl.random_spd(64, seed=1, cond=10.0)
    r, _ = solve_sliced(env, A, b, 17)
    assert r.status == -1


# ---- edge cases of the full solve on the sliced product ----

def test_sliced_zero_rhs_and_maxit_zero(env):
    A, b = wl.random_spd(50, seed=9)
    r, x = solve_sliced(env, A, np.zeros(50), 4)
    assert r.status == 0 and r.iterations == 0 and not x.any()
    torch, ccg = env["torch"], env["ccg"]
    with ccg.Solver(device=0, precision=ccg.FP64_SLICED) as s:
        x = torch.zeros(50, dtype=torch.float64, device="cuda")
        r = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), x, p=2, tol=TOL,
                    maxit=0)
    assert r.status == 1 and r.iterations == 0


def test_sliced_deflation_of_identical_agents(env):
    torch, ccg = env["torch"], env["ccg"]
    n = 120
    A, b = wl.random_spd(n, seed=11, cond=80.0)
    X0 = np.repeat(wl.random_block(n, 1, seed=12), 5, axis=1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with ccg.Solver(device=0, precision=ccg.FP64_SLICED) as s:
        r = s.solve_block(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(),
                          torch.from_numpy(X0).cuda(), x, tol=TOL, maxit=2000)
    ref = env["oracle"].ccg(A, b, X0, TOL, 2000)
    assert r.status == 0 and r.p_final == 1 and r.drops == 4 and ref["p_final"] == 1
    assert abs(r.iterations - ref["iterations"]) <= 2


def test_sliced_nan_and_indefinite(env):
    A, b = wl.random_spd(30, seed=15)
    b[4] = np.nan
    r, _ = solve_sliced(env, A, b, 2)
    assert r.status == -3
    n = 40
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * np.linspace(-3.0, 5.0, n)) @ Q.T
    A = 0.5 * (A + A.T)
    r, _ = solve_sliced(env, A, rng.standard_normal(n), 3)
    assert r.status == -2


@pytest.mark.parametrize("n,p", [(129, 5), (383, 13), (640, 2)])
def test_sliced_ragged_sizes_and_agent_counts(env, n, p):
    A, b = wl.random_spd(n, seed=3 * n + p, cond=500.0)
    r, x = solve_sliced(env, A, b, p)
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, TOL, 20 * n, nthreads=8)
    assert r.status == 0
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) <= TOL * 1.01
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert abs(r.iterations - ref["iterations"]) <= 2, (r.iterations, ref["iterations"])


def test_sliced_two_ctas_many_row_tiles_each(env):
    """Two CTAs own 1050 rows each (9 row tiles of 128): the fixup walks its
    row tiles in chunks and the Gram partials read the blocks directly (too
    many rows to stage); the answer is held to the same FP64 bar."""
    torch, ccg = env["torch"], env["ccg"]
    n, p = 2100, 4
    A, b = wl.random_spd(n, seed=23, cond=200.0)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with ccg.Solver(device=0, precision=ccg.FP64_SLICED, max_ctas=2) as s:
        r = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), x, p=p, tol=TOL,
                    maxit=20 * n)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, TOL, 20 * n, nthreads=8)
    assert r.status == 0 and ref["status"] == 0
    assert np.linalg.norm(A @ xg - b) / np.linalg.norm(b) <= TOL * 1.01
    assert np.linalg.norm(xg - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
    assert abs(r.iterations - ref["iterations"]) <= 2, (r.iterations, ref["iterations"])

