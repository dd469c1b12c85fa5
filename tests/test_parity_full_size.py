"""Full-size GPU parity on the benchmark system: the exponential kernel
exp(-|z_i - z_j| / 0.2) + 1e-2 I on 8192 points of [0,1]^3 (seed 1), b ~ N(0,1),
x0 = 0, tol 1e-10, for every agent count the workload names (p = 1, 4, 8, 16,
32), in the launch configuration the benchmark times (one CTA per SM).

Both FP64 solvers are held to the FP64 bar against the FP64 oracle
(Algorithm 2 with Algorithm 3's deflation and Algorithm 4's stopping rule):
status OK, true relative residual <= 1e-10 and ||x - x_oracle|| / ||x_oracle||
<= 1e-8.  The FP64-pipe solver forms A D_k in FP64; the sliced solver forms it
exactly on the FP8 tensor cores from 4-bit slices of A and D_k (p <= 16).

Iteration counts.  This system has kappa ~ 1e5, and its iteration count is
not a stable function of rounding: the oracle itself stops 4 to 6
iterations apart when only the summation order of its block product changes
(measured: 537 to 543 at p = 4, 251 to 256 at p = 16, 873 to 878 at p = 1),
because min_j ||R e_j|| crosses tol on a flat, oscillating stretch of the
residual curve.  Each GPU count is therefore held to the oracle's rounding
envelope on this input (tests/envelope.py): its counts over the four
summation orders, widened by 2 on either side.
"""
import numpy as np
import pytest
from envelope import oracle_counts, within_envelope

from paper_1204_0069_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10
N = 8192


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
    A, b = wl.exp_kernel(N, seed=1, length=0.2, nugget=1e-2)
    yield dict(torch=torch, ccg=ccg, oracle=oracle, A=A, b=b, dA=torch.from_numpy(A).cuda(),
               db=torch.from_numpy(b).cuda(), cache={})


def oracle_envelope(env, p):
    if p not in env["cache"]:
        X0 = env["oracle"].initial_block(N, p, None, 1.0, 0)
        ref, counts, status = oracle_counts(env["oracle"], env["A"], env["b"], X0, TOL, 5000)
        assert all(s == 0 for s in status), status
        env["cache"][p] = (ref, counts)
    return env["cache"][p]


def check(env, p, precision):
    torch, ccg = env["torch"], env["ccg"]
    x = torch.zeros(N, dtype=torch.float64, device="cuda:0")
    with ccg.Solver(device=0, precision=precision) as s:
        r = s.solve(env["dA"], env["db"], x, p=p, tol=TOL, maxit=5000)
    torch.cuda.synchronize()
    ref, counts = oracle_envelope(env, p)
    xg = x.cpu().numpy()
    A, b = env["A"], env["b"]
    assert r.status == 0, r
    assert r.relres_true <= TOL
    assert np.linalg.norm(A @ xg - b) / np.linalg.norm(b) <= TOL * 1.01
    err = np.linalg.norm(xg - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= 1e-8, err
    assert within_envelope(r.iterations, counts), (r.iterations, counts)
    assert r.p_final == ref["p_final"]


@pytest.mark.parametrize("p", [1, 4, 8, 16, 32])
def test_fp64_pipe_exp_kernel_n8192(env, p):
    check(env, p, env["ccg"].FP64)


@pytest.mark.parametrize("p", [1, 4, 8, 16])
def test_sliced_fp64_exp_kernel_n8192(env, p):
    check(env, p, env["ccg"].FP64_SLICED)
