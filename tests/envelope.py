"""The oracle's rounding envelope of an iteration count.

cCG fixes no summation order for the block product A D_k, and on an
ill-conditioned system the iteration count moves with the order: on the
benchmark system (exponential kernel, n = 8192, kappa ~ 1e5) the oracle alone
stops 4 to 6 iterations apart when its block product is summed ascending,
descending, in blocks of 64 or as 64 interleaved sums.  Solves whose
dynamics are set by rounding (agents started 1e6 away from the solution, so
that the recurrence residual drifts from the true one and a residual
replacement follows) move the same way: the more accurate the product, the
fewer iterations after the replacement.  A GPU solve sums in yet another
order (tiles and lanes), or, for the sliced product, more accurately than any
plain order.  Its count is held to the range of the oracle's counts over the
orders, widened by 2 on either side: the plain "within 2" rule wherever the
orders agree.  Up to n = 4096 the orders include the compensated product
(Dot2, nearly the exact sum rounded once); above, it is left out for time.
"""
import os

COMPENSATED_MAX_N = 4096


def oracle_counts(oracle, A, b, X0, tol, maxit, nthreads=None, **kw):
    """(oracle result in the default order, counts over the orders, statuses)."""
    nthreads = nthreads or (os.cpu_count() or 1)
    orders = [o for o in oracle.PRODUCT_ORDERS if o != 4 or b.shape[0] <= COMPENSATED_MAX_N]
    runs = [oracle.ccg(A, b, X0, tol, maxit, nthreads=nthreads, product_order=o, **kw)
            for o in orders]
    return runs[0], [r["iterations"] for r in runs], [r["status"] for r in runs]


def within_envelope(count, counts, slack=2):
    return min(counts) - slack <= count <= max(counts) + slack
