"""GPU tests of the batched solver: many independent SPD systems of uneven
size in one persistent launch (one CTA per system at a time, largest first).
Every system is checked against the FP64 oracle with the parity bar of the
single-system solver (relres <= 1e-10, ||x - x_oracle|| / ||x_oracle|| <=
1e-8, iterations within 2)."""
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
    import oracle
    oracle.build()
    from paper_1204_0069_gb300 import ccg
    return dict(torch=torch, ccg=ccg, oracle=oracle)


def make_batch(sizes, seed):
    rng = np.random.default_rng(seed)
    mats, rhs = [], []
    for k, n in enumerate(sizes):
        A, b = wl.gram_shift(int(n), seed=seed * 100003 + k, shift=float(rng.uniform(0.05, 1.0)))
        mats.append(A)
        rhs.append(b)
    return mats, rhs


def pack(ccg, torch, sizes, mats, rhs):
    a_off, v_off, at, vt = ccg.batch_offsets(sizes)
    Ap = np.zeros(at)
    bp = np.zeros(vt)
    for n, A, b, ao, vo in zip(sizes, mats, rhs, a_off, v_off):
        ld = n + (n & 1)
        Ap[ao:ao + n * ld].reshape(n, ld)[:, :n] = A
        bp[vo:vo + n] = b
    return torch.from_numpy(Ap).cuda(), torch.from_numpy(bp).cuda(), v_off


@pytest.mark.parametrize("p", [1, 4, 7])
def test_batched_matches_oracle_per_system(env, p):
    torch, ccg, oracle = env["torch"], env["ccg"], env["oracle"]
    rng = np.random.default_rng(p)
    sizes = [int(v) for v in np.round(np.exp(rng.uniform(np.log(8), np.log(300), 150)))]
    sizes = [max(s, p) for s in sizes] + [p, 301, 17]
    mats, rhs = make_batch(sizes, seed=p)
    dA, db, v_off = pack(ccg, torch, sizes, mats, rhs)
    x = torch.zeros_like(db)
    with ccg.Solver() as s:
        summ, st, it, rr = s.solve_batched(sizes, dA, db, x, p=p, tol=1e-10, maxit=10000)
    assert summ.status == 0, summ
    xs = x.cpu().numpy()
    for k, (n, A, b) in enumerate(zip(sizes, mats, rhs)):
        xi = xs[v_off[k]:v_off[k] + n]
        assert st[k] == 0
        relres = np.linalg.norm(b - A @ xi) / np.linalg.norm(b)
        assert relres <= 1.01e-10 and rr[k] <= 1e-10
        X0 = oracle.initial_block(n, p, None, 1.0, 0)
        ref = oracle.ccg(A, b, X0, 1e-10, 10000)
        err = np.linalg.norm(xi - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= 1e-8, (k, n, err)
        assert abs(int(it[k]) - ref["iterations"]) <= 2, (k, n, it[k], ref["iterations"])


def test_batched_empty_and_invalid(env):
    torch, ccg = env["torch"], env["ccg"]
    with ccg.Solver() as s:
        z = torch.zeros(4, dtype=torch.float64, device="cuda")
        summ, *_ = s.solve_batched([], z, z, z, p=2, tol=1e-8, maxit=10)
        assert summ.status == 0
        summ, *_ = s.solve_batched([1], z, z, z, p=2, tol=1e-8, maxit=10)  # p > n
        assert summ.status == -1


@pytest.mark.parametrize("p", [1, 4])
def test_batched_fp32_refinement_reaches_fp64_accuracy(env, p):
    """Batched FP32 + FP64 refinement: every system reaches the FP64 target
    (true relative residual <= 1e-10, checked here in NumPy) and every x
    agrees with the FP64 oracle's to the FP64 bar, 1e-8 relative."""
    torch, ccg, oracle = env["torch"], env["ccg"], env["oracle"]
    rng = np.random.default_rng(10 + p)
    sizes = [int(v) for v in np.round(np.exp(rng.uniform(np.log(8), np.log(400), 120)))]
    sizes = [max(s, p) for s in sizes] + [p, 401, 33]
    mats, rhs = make_batch(sizes, seed=20 + p)
    dA, db, v_off = pack(ccg, torch, sizes, mats, rhs)
    x = torch.zeros_like(db)
    with ccg.Solver(precision=ccg.FP32_IR) as s:
        summ, st, it, rr = s.solve_batched(sizes, dA, db, x, p=p, tol=1e-10, maxit=10000)
    assert summ.status == 0, summ
    assert 1 <= summ.outer_steps <= 30
    xs = x.cpu().numpy()
    for k, (n, A, b) in enumerate(zip(sizes, mats, rhs)):
        xi = xs[v_off[k]:v_off[k] + n]
        assert st[k] == 0, (k, n, st[k], rr[k])
        relres = np.linalg.norm(b - A @ xi) / np.linalg.norm(b)
        assert relres <= 1.01e-10 and abs(relres - rr[k]) <= 1e-12, (k, relres, rr[k])
        X0 = oracle.initial_block(n, p, None, 1.0, 0)
        ref = oracle.ccg(A, b, X0, 1e-10, 10000)
        err = np.linalg.norm(xi - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= 1e-8, (k, n, err)


def test_batched_rejects_tensor_core_precisions(env):
    torch, ccg = env["torch"], env["ccg"]
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    with ccg.Solver(precision=ccg.BF16_IR) as s:
        summ, *_ = s.solve_batched([2], z, z, z, p=1, tol=1e-8, maxit=10)
        assert summ.status == -1


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_batched_each_apass_variant_matches_oracle(env, variant):
    """Every A-pass shape the autotuner may pick gives the FP64 parity bar."""
    torch, ccg, oracle = env["torch"], env["ccg"], env["oracle"]
    p = 4
    sizes = [37, 64, 100, 129, 255, 300, 513, 700]
    mats, rhs = make_batch(sizes, seed=40 + variant)
    dA, db, v_off = pack(ccg, torch, sizes, mats, rhs)
    x = torch.zeros_like(db)
    with ccg.Solver(batch_autotune=False) as s:
        s.batch_tuning(p, ccg.FP64, [variant] * 8)
        summ, st, it, rr = s.solve_batched(sizes, dA, db, x, p=p, tol=1e-10, maxit=10000)
    assert summ.status == 0, summ
    xs = x.cpu().numpy()
    for k, (n, A, b) in enumerate(zip(sizes, mats, rhs)):
        xi = xs[v_off[k]:v_off[k] + n]
        X0 = oracle.initial_block(n, p, None, 1.0, 0)
        ref = oracle.ccg(A, b, X0, 1e-10, 10000)
        assert np.linalg.norm(b - A @ xi) / np.linalg.norm(b) <= 1.01e-10
        assert np.linalg.norm(xi - ref["x"]) / np.linalg.norm(ref["x"]) <= 1e-8
        assert abs(int(it[k]) - ref["iterations"]) <= 2, (k, n, it[k], ref["iterations"])


def test_batch_autotuner_fills_the_buckets_it_meets(env):
    torch, ccg = env["torch"], env["ccg"]
    p = 4
    sizes = [40, 50, 90, 200, 210, 600]          # buckets 0, 1, 2, 4
    mats, rhs = make_batch(sizes, seed=77)
    dA, db, v_off = pack(ccg, torch, sizes, mats, rhs)
    x = torch.zeros_like(db)
    with ccg.Solver() as s:
        assert s.batch_tuning(p) == [-1] * 8
        summ, st, it, rr = s.solve_batched(sizes, dA, db, x, p=p, tol=1e-10, maxit=10000)
        table = s.batch_tuning(p)
        assert summ.status == 0
        assert all(table[b] in (0, 1, 2) for b in (0, 1, 2, 4))
        assert all(table[b] == -1 for b in (3, 5, 6, 7))
        with pytest.raises(RuntimeError):
            s.batch_tuning(1, ccg.FP64, [1] * 8)  # no variant 1 for p <= 2
    xs = x.cpu().numpy()
    for k, (n, A, b) in enumerate(zip(sizes, mats, rhs)):
        xi = xs[v_off[k]:v_off[k] + n]
        assert np.linalg.norm(b - A @ xi) / np.linalg.norm(b) <= 1.01e-10
