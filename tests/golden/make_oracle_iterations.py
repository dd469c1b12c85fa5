"""Write tests/golden/oracle_iterations.json: iteration counts of the FP64
oracle (and nothing else) on the benchmark workloads.

The CPU baseline of bench.py times a bounded sample of oracle iterations and
scales it to a full solve with these counts.  Run:  python tests/golden/make_oracle_iterations.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1204_0069_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")


def main():
    rows = []
    nthreads = os.cpu_count() or 1
    cases = [("gram_shift n=256 shift=0.5 seed=0", lambda: wl.gram_shift(256, 0, 0.5), [4]),
             ("exp_kernel n=8192 l=0.2 nugget=1e-2 seed=1",
              lambda: wl.exp_kernel(8192, 1, 0.2, 1e-2), [1, 4, 8, 16, 32])]
    for name, gen, ps in cases:
        A, b = gen()
        n = b.shape[0]
        for p in ps:
            X0 = oracle.initial_block(n, p, None, 1.0, 0)
            t = time.time()
            r = oracle.ccg(A, b, X0, 1e-10, 20000, nthreads=nthreads)
            rows.append(dict(workload=name, n=n, p=p, tol=1e-10, x0_spread=1.0, seed=0,
                             rank_tol=1e-12, status=r["status_name"], iterations=r["iterations"],
                             replacements=r["replacements"], drops=r["drops"],
                             relres_true=r["relres_true"], seconds=round(time.time() - t, 2),
                             threads=nthreads))
            print(rows[-1], flush=True)
    with open(OUT, "w") as f:
        json.dump({"generator": "tests/golden/make_oracle_iterations.py (oracle only)",
                   "rows": rows}, f, indent=1)


if __name__ == "__main__":
    main()
