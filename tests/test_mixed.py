"""GPU tests of the mixed-precision solves, whose low-precision block products
run on the tensor cores (A stored in BF16, FP8 E4M3 or FP32):

* CCG_MIXED_REFINE: FP64 refinement around inner cCG solves on the quantised
  A.  On systems where the quantised matrix is close enough to A for the
  conditioning (kappa * u < 1, u = 2^-9 for BF16, 2^-4 for FP8) it must reach
  the FP64 target: true relative residual <= 1e-10 and
  ||x - x_oracle|| / ||x_oracle|| <= 1e-8 against the FP64 oracle.  Where it
  cannot (ill-conditioned kernel matrices), the solve must say so
  (CCG_NOT_CONVERGED) and report the residual of the x it returns truthfully.
* CCG_MIXED_PRECOND (the default for BF16 and FP8): FP64 cCG whose directions
  come from a Chebyshev polynomial in the quantised A.  Its products with A
  are FP64, so it must reach the same FP64 target whatever kappa * u, on the
  ill-conditioned kernels too.
"""
import numpy as np
import pytest
from envelope import oracle_counts, within_envelope

from paper_1204_0069_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


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
    return dict(torch=torch, ccg=ccg, oracle=oracle)


def solve(env, A, b, p, precision, tol=1e-10, inner_tol=0.0, method=0, **kw):
    torch, ccg = env["torch"], env["ccg"]
    n = b.shape[0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with ccg.Solver(precision=precision, inner_tol=inner_tol, mixed_method=method, **kw) as s:
        r = s.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), x, p=p, tol=tol,
                    maxit=20 * n)
    return r, x.cpu().numpy()


@pytest.mark.parametrize("precision,shift,n,p", [
    (2, 0.5, 1024, 4), (2, 0.5, 1500, 8), (2, 0.5, 777, 16), (2, 0.5, 640, 32),
    (3, 2.0, 1024, 4), (3, 2.0, 900, 8)], ids=["bf16-n1024-p4", "bf16-n1500-p8",
                                               "bf16-n777-p16", "bf16-n640-p32",
                                               "fp8-n1024-p4", "fp8-n900-p8"])
@pytest.mark.parametrize("method", [1, 2], ids=["refine", "precond"])
def test_mixed_reaches_fp64_accuracy(env, precision, shift, n, p, method):
    A, b = wl.gram_shift(n, seed=n + p, shift=shift)
    r, x = solve(env, A, b, p, precision, method=method)
    assert r.status == 0, r
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert relres <= 1e-10 * 1.01, relres
    assert abs(relres - r.relres_true) <= 1e-3 * relres + 1e-16
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, 1e-10, 20 * n, nthreads=8)
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= 1e-8, err
    assert r.outer_steps >= 1 and r.iterations > 0


@pytest.mark.parametrize("n,p", [(2048, 8), (1500, 4), (3000, 16)])
def test_fp32_ir_reaches_fp64_on_ill_conditioned_kernel(env, n, p):
    """Exponential kernel (kappa ~ 1e4): A stored in FP32 with TF32x3 tensor-core
    products is accurate enough (kappa * 2^-21 << 1) for refinement to reach
    the FP64 target."""
    A, b = wl.exp_kernel(n, seed=1, length=0.2, nugget=1e-2)
    r, x = solve(env, A, b, p, 1)
    assert r.status == 0, r
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert relres <= 1e-10 * 1.01, relres
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, 1e-10, 20 * n, nthreads=8)
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= 1e-8, err


def test_mixed_reports_truthfully_when_refinement_stalls(env):
    """Exponential kernel, kappa ~ 1e4: BF16 A is too coarse for plain
    refinement to reach 1e-10; the status and residual must say so."""
    A, b = wl.exp_kernel(1024, seed=1, length=0.2, nugget=1e-2)
    r, x = solve(env, A, b, 8, 2, method=1)
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(relres - r.relres_true) <= 1e-3 * relres
    if r.status == 0:
        assert relres <= 1e-10 * 1.01
    else:
        assert r.status == 1 and relres > 1e-10


def test_prequantised_matrix_reused_across_solves(env):
    torch, ccg = env["torch"], env["ccg"]
    n, p = 1200, 8
    A, b = wl.gram_shift(n, seed=3, shift=0.5)
    dA = torch.from_numpy(A).cuda()
    with ccg.Solver() as s:
        m = s.lowp_matrix(dA, ccg.LOWP_BF16)
        for k in range(2):
            bb = torch.from_numpy(b * (k + 1)).cuda()
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            r = s.solve_mixed(m, dA, bb, x, p=p, tol=1e-10, maxit=20 * n)
            assert r.status == 0
            xs = x.cpu().numpy()
            assert np.linalg.norm(b * (k + 1) - A @ xs) / np.linalg.norm(b * (k + 1)) <= 1.01e-10
        m.close()


# Exponential kernels with kappa * u >> 1 for BF16 and FP8: the quantised A is
# not even positive definite there, so refinement stalls, while the
# preconditioned solve reaches the FP64 target (its products with A are FP64).
@pytest.mark.parametrize("fmt", [2, 3], ids=["bf16", "fp8"])
@pytest.mark.parametrize("n,p,length,nugget", [(2048, 8, 0.1, 1e-3), (1500, 4, 0.2, 1e-2),
                                               (3000, 16, 0.1, 1e-3), (1031, 32, 0.2, 1e-2)])
def test_precond_reaches_fp64_on_ill_conditioned_kernel(env, fmt, n, p, length, nugget):
    A, b = wl.exp_kernel(n, seed=2, length=length, nugget=nugget)
    r, x = solve(env, A, b, p, fmt, method=2)
    assert r.status == 0, r
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert relres <= 1e-10 * 1.01, relres
    assert abs(relres - r.relres_true) <= 1e-3 * relres + 1e-16
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    ref = env["oracle"].ccg(A, b, X0, 1e-10, 20 * n, nthreads=8)
    err = np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= 1e-8, err
    # the preconditioner shortens the FP64 iteration
    assert r.iterations < ref["iterations"], (r.iterations, ref["iterations"])
    assert r.outer_steps >= 1


def test_precond_with_prequantised_matrix_and_degree_one(env):
    """A prequantised FP8 matrix reused by two solves; a polynomial of degree
    one (no product with the quantised A: Z = R / centre of the interval)
    reduces the method to FP64 cCG with scaled residues, so its count is held
    to the oracle's rounding envelope (tests/envelope.py)."""
    torch, ccg = env["torch"], env["ccg"]
    n, p = 1200, 8
    A, b = wl.exp_kernel(n, seed=5, length=0.1, nugget=1e-3)
    dA = torch.from_numpy(A).cuda()
    db = torch.from_numpy(b).cuda()
    with ccg.Solver(mixed_method=2) as s:
        m = s.lowp_matrix(dA, ccg.LOWP_FP8_E4M3)
        for _ in range(2):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            r = s.solve_mixed(m, dA, db, x, p=p, tol=1e-10, maxit=20 * n)
            assert r.status == 0, r
            xs = x.cpu().numpy()
            assert np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1.01e-10
        m.close()
    with ccg.Solver(precision=ccg.BF16_IR, mixed_method=2, cheb_degree=1) as s:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        r = s.solve(dA, db, x, p=p, tol=1e-10, maxit=20 * n)
    X0 = env["oracle"].initial_block(n, p, None, 1.0, 0)
    _, counts, _ = oracle_counts(env["oracle"], A, b, X0, 1e-10, 20 * n)
    assert r.status == 0, r
    assert within_envelope(r.iterations, counts), (r.iterations, counts)


@pytest.mark.parametrize("fmt", [2, 3], ids=["bf16", "fp8"])
def test_auto_method_probes_refinement_then_preconditions(env, fmt):
    """The default method: on a well-conditioned system refinement converges
    by itself; on an ill-conditioned kernel it hands over to the
    preconditioned FP64 solve, which reaches the FP64 bar against the
    oracle."""
    A, b = wl.gram_shift(1024, seed=4, shift=0.5 if fmt == 2 else 2.0)
    r, x = solve(env, A, b, 8, fmt)
    assert r.status == 0, r
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.01e-10
    n = 2048
    A, b = wl.exp_kernel(n, seed=2, length=0.1, nugget=1e-3)
    r, x = solve(env, A, b, 8, fmt)
    assert r.status == 0, r
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1.01e-10
    ref = env["oracle"].ccg(A, b, env["oracle"].initial_block(n, 8, None, 1.0, 0), 1e-10,
                            20 * n, nthreads=8)
    assert np.linalg.norm(x - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
