"""ccg_solve_noalloc (the solve that allocates nothing) against ccg_solve.

Some callers cannot allocate device memory while they run -- their memory
belongs to a pool or a fixed budget, or the synchronisation an allocation can
cause is too costly -- so the library offers one solve whose scratch is a
fixed device array.  This file runs last (its name sorts last) so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.  Same tolerances as the parity tests:
||x - x_ref|| / ||x_ref|| <= 1e-8 and iterations within 2, on two calls in a
row (the second call reuses the scratch the first one left behind), and the
second call leaves the device's free memory where it found it.
"""
import numpy as np
import pytest

from paper_1204_0069_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_0069_gb300 import build as B
    B.build()
    from paper_1204_0069_gb300 import ccg
    return dict(torch=torch, ccg=ccg)


@pytest.mark.parametrize("case", ["gram_n1024_p8", "spd_n4096_p32"])
def test_noalloc_matches_solve_on_two_calls(env, case):
    torch, ccg = env["torch"], env["ccg"]
    if case == "gram_n1024_p8":
        A, b = wl.gram_shift(1024, seed=0, shift=0.5)
        p = 8
    else:
        A, b = wl.random_spd(4096, seed=7, cond=100.0)
        p = 32  # n * p = CCG_NOALLOC_MAX_NP, the largest accepted size
    n = b.shape[0]
    dA = torch.from_numpy(A).cuda()
    db = torch.from_numpy(b).cuda()
    x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    with ccg.Solver(device=0) as s:
        r_ref = s.solve(dA, db, x_ref, p=p, tol=1e-10, maxit=10 * n)
    assert r_ref.status == 0
    xr = x_ref.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        r = ccg.solve_noalloc(dA, db, x, p=p, tol=1e-10, maxit=10 * n, device=0, stream=stream)
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            # the first call loaded the module and looked up the scratch array;
            # the second one takes no device memory at all
            assert free1 >= free0, (free0, free1)
        assert r.status == 0, r
        assert r.relres_true <= 1e-10
        xg = x.cpu().numpy()
        assert np.linalg.norm(xg - xr) / np.linalg.norm(xr) <= 1e-8
        assert abs(r.iterations - r_ref.iterations) <= 2


def test_noalloc_rejects_oversize_and_host_buffers(env):
    torch, ccg = env["torch"], env["ccg"]
    n = 4097
    A, b = wl.random_spd(64, seed=1)
    dA = torch.eye(n, dtype=torch.float64, device="cuda")
    db = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert ccg.solve_noalloc(dA, db, x, p=32, tol=1e-8, maxit=10).status == -1  # n*p too big
    xh = np.zeros(64)
    assert ccg.solve_noalloc(A, b, xh, p=2, tol=1e-8, maxit=10).status == -1    # host pointers
