"""GPU tests of the serving loop: continuous admission of solve requests.

* every result equals the same request solved alone (same worker share,
  hence the same grid): bitwise, which is within any stated tolerance;
* every served FP64 result matches the FP64 oracle run on the same request
  (Algorithm 2 with Algorithm 3's deflation and Algorithm 4's stop rule):
  iterations within 2 of the oracle's counts over its summation orders
  (tests/envelope.py; some requests have kappa ~ 5e4) and ||x - x_oracle|| / ||x_oracle|| <= 100 tol (1e-8 at
  tol 1e-10; two iterates that both stop at relres <= 1e-6 differ at that
  level); a served
  mixed-precision result meets its tolerance on the true residual and its
  distance to the oracle's answer is bounded by the conditioning;
* requests admitted while others run overlap (peak in-flight > 1);
* the device-memory budget is never exceeded and a request larger than the
  budget is refused at submission;
* the same holds for the slots mode, where one persistent kernel serves
  every request from a ring that the server appends to while it runs
  (continuous batching), including requests that arrive after the kernel
  has ended on idle.
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
    from paper_1204_0069_gb300 import ccg
    import oracle
    oracle.build()
    return dict(torch=torch, ccg=ccg, oracle=oracle)


def requests(torch, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(np.round(np.exp(rng.uniform(np.log(200), np.log(2500)))))
        A, b = wl.exp_kernel(n, seed=seed * 1000 + k, length=float(rng.uniform(0.05, 0.5)),
                             nugget=float(10 ** rng.uniform(-4, -1)))
        tol = [1e-6, 1e-10][k % 2]
        out.append((torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), tol, A, b))
    return out


def even_ld(torch, A):
    """A with an even leading dimension (the serving kernel's 16-byte loads)."""
    n = A.shape[0]
    if n % 2 == 0:
        return A
    Ap = torch.zeros((n, n + 1), dtype=torch.float64, device=A.device)
    Ap[:, :n] = A
    return Ap


def run_server(ccg, torch, reqs, workers, budget, precision=0, share=16, slots=0):
    srv = ccg.Server(workers=workers, budget_bytes=budget, precision=precision,
                     ctas_per_worker=share, slots=slots, max_n=4096)
    xs = [torch.zeros(b.shape[0], dtype=torch.float64, device="cuda") for _, b, *_ in reqs]
    # the matrices must stay allocated until their results are in
    mats = [even_ld(torch, A) if slots else A for A, *_ in reqs]
    for k, (A, b, tol, *_) in enumerate(reqs):
        assert srv.submit(k, mats[k], b, xs[k], p=8, tol=tol, maxit=50000) == 0
    got = {}
    while len(got) < len(reqs):
        for r in srv.poll(64, wait_ms=200):
            got[r["id"]] = r
    st = srv.stats()
    srv.close()
    return got, [x.cpu().numpy() for x in xs], st


@pytest.mark.parametrize("precision", [0, 1, 4], ids=["fp64", "fp32_ir", "fp64_sliced"])
def test_results_alone_equal_results_in_the_mix(env, precision):
    torch, ccg = env["torch"], env["ccg"]
    reqs = requests(torch, 10, seed=5)
    mix, xmix, st = run_server(ccg, torch, reqs, workers=6, budget=150e9, precision=precision)
    assert st["peak_in_flight"] > 1
    for k, (A, b, tol, An, bn) in enumerate(reqs):
        r = mix[k]
        assert r["status"] == 0, r
        relres = np.linalg.norm(bn - An @ xmix[k]) / np.linalg.norm(bn)
        assert relres <= tol * 1.01
        alone, xal, _ = run_server(ccg, torch, [reqs[k]], workers=1, budget=150e9,
                                   precision=precision)
        assert alone[0]["iterations"] == r["iterations"]
        assert np.array_equal(xal[0], xmix[k])
        # the served answer against the FP64 oracle on the same request
        n = bn.shape[0]
        ref, counts, status = oracle_counts(env["oracle"], An, bn,
                                            env["oracle"].initial_block(n, 8, None, 1.0, 0),
                                            tol, 50000)
        assert all(s == 0 for s in status), status
        err = np.linalg.norm(xmix[k] - ref["x"]) / np.linalg.norm(ref["x"])
        if precision in (0, 4):
            # FP64 bar scaled to the request's tolerance: 1e-8 at tol 1e-10
            assert within_envelope(r["iterations"], counts), (r["iterations"], counts)
            assert err <= 100.0 * tol, err
        else:
            # two answers that both meet relres <= tol differ by at most
            # 2 kappa tol relative (kappa bounded by ||A||_inf / lambda_min)
            kappa = np.abs(An).sum(axis=1).max() / (np.min(np.linalg.eigvalsh(An)))
            assert err <= 2.0 * kappa * tol, (err, kappa)


def test_budget_is_respected(env):
    torch, ccg = env["torch"], env["ccg"]
    reqs = requests(torch, 8, seed=9)
    biggest = max(int(b.shape[0]) for _, b, *_ in reqs)
    budget = 2.5 * biggest * biggest * 8 + 64e6  # room for about two of the largest
    got, xs, st = run_server(ccg, torch, reqs, workers=6, budget=budget)
    assert st["peak_reserved_bytes"] <= budget
    assert all(r["status"] == 0 for r in got.values())
    # admission waits for memory: some request was admitted after it was queued
    assert any(r["admit_ms"] - r["submit_ms"] > 0.0 for r in got.values())
    srv = ccg.Server(workers=1, budget_bytes=1e6)
    A, b, *_ = reqs[0]
    x = torch.zeros_like(b)
    assert srv.submit(0, A, b, x, p=4, tol=1e-8, maxit=100) == -4  # can never fit
    srv.close()


@pytest.mark.parametrize("slots", [6, 8])
def test_slots_mode_alone_equals_mix_and_matches_oracle(env, slots):
    torch, ccg = env["torch"], env["ccg"]
    reqs = requests(torch, 12, seed=7)
    mix, xmix, st = run_server(ccg, torch, reqs, workers=1, budget=150e9, slots=slots)
    assert st["peak_in_flight"] > 1
    assert len({r["worker"] for r in mix.values()}) > 1  # several slots served
    for k, (A, b, tol, An, bn) in enumerate(reqs):
        r = mix[k]
        assert r["status"] == 0, r
        relres = np.linalg.norm(bn - An @ xmix[k]) / np.linalg.norm(bn)
        assert relres <= tol * 1.01
        alone, xal, _ = run_server(ccg, torch, [reqs[k]], workers=1, budget=150e9, slots=slots)
        assert alone[0]["iterations"] == r["iterations"]
        assert np.array_equal(xal[0], xmix[k])
        n = bn.shape[0]
        ref, counts, status = oracle_counts(env["oracle"], An, bn,
                                            env["oracle"].initial_block(n, 8, None, 1.0, 0),
                                            tol, 50000)
        assert all(s_ == 0 for s_ in status), status
        assert within_envelope(r["iterations"], counts), (r["iterations"], counts)
        err = np.linalg.norm(xmix[k] - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= 100.0 * tol, err


def test_slots_mode_restarts_after_idle_and_respects_budget(env):
    import time
    torch, ccg = env["torch"], env["ccg"]
    reqs = requests(torch, 6, seed=11)
    biggest = max(int(b.shape[0]) for _, b, *_ in reqs)
    probe = ccg.Server(slots=4, max_n=4096)
    fixed = probe.stats()["reserved_bytes"]  # the slots' own blocks
    probe.close()
    budget = fixed + 2.2 * biggest * biggest * 8 + 16e6  # about two matrices at a time
    srv = ccg.Server(slots=4, budget_bytes=budget, max_n=4096)
    xs = [torch.zeros(b.shape[0], dtype=torch.float64, device="cuda") for _, b, *_ in reqs]
    mats = [even_ld(torch, A) for A, *_ in reqs]
    got = {}
    for k in range(3):
        A, b, tol, *_ = reqs[k]
        assert srv.submit(k, mats[k], b, xs[k], p=8, tol=tol, maxit=50000) == 0
    while len(got) < 3:
        for r in srv.poll(64, wait_ms=200):
            got[r["id"]] = r
    time.sleep(0.3)  # the kernel ends on idle; the next requests launch it again
    for k in range(3, 6):
        A, b, tol, *_ = reqs[k]
        assert srv.submit(k, mats[k], b, xs[k], p=8, tol=tol, maxit=50000) == 0
    while len(got) < 6:
        for r in srv.poll(64, wait_ms=200):
            got[r["id"]] = r
    st = srv.stats()
    srv.close()
    assert st["peak_reserved_bytes"] <= budget
    for k, (A, b, tol, An, bn) in enumerate(reqs):
        assert got[k]["status"] == 0, got[k]
        assert np.linalg.norm(bn - An @ xs[k].cpu().numpy()) / np.linalg.norm(bn) <= tol * 1.01


def test_slots_mode_rejects_what_it_cannot_serve(env):
    torch, ccg = env["torch"], env["ccg"]
    srv = ccg.Server(slots=2, max_n=256)
    n = 300
    A = torch.eye(n, dtype=torch.float64, device="cuda")
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    assert srv.submit(0, A, b, x, p=4, tol=1e-8, maxit=10) == -1          # n > max_n
    A2 = torch.eye(200, dtype=torch.float64, device="cuda")
    b2 = torch.ones(200, dtype=torch.float64, device="cuda")
    x2 = torch.zeros(200, dtype=torch.float64, device="cuda")
    assert srv.submit(1, A2, b2, x2, p=9, tol=1e-8, maxit=10) == -1       # p > max_p
    hA = np.eye(200)
    assert srv.submit(2, hA, b2, x2, p=4, tol=1e-8, maxit=10) == -1       # host matrix
    srv.close()
    with pytest.raises(RuntimeError):
        ccg.Server(slots=2, precision=ccg.FP32_IR)                       # FP64 only
