"""Pin of the oracle's Gram products against exact rational sums (CPU only).

Section 4 of the paper derives the matrix stepsizes in exact arithmetic; the
oracle therefore takes every p x p Gram (M = D'AD, G = R'D, H = R'AD) and the
residue norms as compensated dot products (Dot2 of Ogita, Rump and Oishi,
SIAM J. Sci. Comput. 26(6), 2005, built from Knuth's TwoSum and Dekker's
TwoProduct).  Their Proposition on Dot2 bounds the result by

    |dot2(x, y) - x'y| <= u |x'y| + gamma_n^2 sum |x_i y_i|,
    u = 2^-53, gamma_n = n u / (1 - n u),

the accuracy of a product evaluated in twice the working precision and then
rounded once.  The sum of products of doubles is a dyadic rational, computed
here exactly with Fractions.  The inputs are built with heavy cancellation
(condition numbers 1e10 to 1e30), where a plain FP64 sum misses the bound by
many orders of magnitude, so that a dropped error term of TwoProduct or of
TwoSum, or a plain accumulation, fails the test.
"""
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -53


def _gamma(n):
    return n * U / (1.0 - n * U)


def _exact(u, v):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, v)), Fraction(0))


def _cancelling_columns(rng, m, q, spread, rel):
    """n = 2m rows: the first m products are spread over 2^(+-spread), the
    second m nearly cancel them (relative perturbation 2^-rel), and the rows
    are shuffled, so that each column pair has a large condition number."""
    a = rng.standard_normal((m, q)) * np.exp2(rng.integers(-spread, spread + 1, (m, q)))
    b = rng.standard_normal((m, q))
    b2 = b * (1.0 + np.exp2(-rel) * rng.standard_normal((m, q)))
    Ucol = np.vstack([a, -a])
    Vcol = np.vstack([b, b2])
    perm = rng.permutation(2 * m)
    return Ucol[perm], Vcol[perm]


@pytest.mark.parametrize("m,q,spread,rel,seed", [
    (40, 3, 20, 30, 0),
    (100, 2, 40, 40, 1),
    (64, 4, 10, 50, 2),
])
def test_gram_meets_the_dot2_bound(oracle_mod, m, q, spread, rel, seed):
    rng = np.random.default_rng(seed)
    Ub, Vb = _cancelling_columns(rng, m, q, spread, rel)
    n = Ub.shape[0]
    G = oracle_mod.gram(Ub, Vb)
    worst_cond = 0.0
    plain_misses = 0
    for a in range(q):
        for c in range(q):
            x, y = Ub[:, a], Vb[:, c]
            S = _exact(x, y)
            absum = float(np.sum(np.abs(x * y)))
            bound = U * abs(float(S)) + _gamma(n) ** 2 * absum
            err = abs(Fraction(float(G[a, c])) - S)
            assert float(err) <= bound, (a, c, float(err), bound)
            if a == c:
                worst_cond = max(worst_cond, absum / max(abs(float(S)), 1e-300))
                plain = float(np.sum(x * y))  # the same sum without compensation
                if float(abs(Fraction(plain) - S)) > bound:
                    plain_misses += 1
    # the inputs are hard enough that an uncompensated sum fails the same bound
    assert worst_cond > 1e9
    assert plain_misses >= 1


def test_gram_orientation_and_exact_small_cases(oracle_mod):
    """G[a, c] = sum_i U[i, a] V[i, c] (not V'U); sums of a few exactly
    representable products are returned exactly."""
    Ub = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    Vb = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    G = oracle_mod.gram(Ub, Vb)
    np.testing.assert_array_equal(G, Ub.T @ Vb)
    # 1e16 + 1 - 1e16 cancels to 1 exactly only with compensation
    x = np.array([1e16, 1.0, -1e16])[:, None]
    y = np.ones((3, 1))
    assert oracle_mod.gram(x, y)[0, 0] == 1.0
    # a product whose exact value needs 106 bits: (1 + 2^-52)^2 - 1 - 2^-51
    e = 1.0 + 2.0 ** -52
    x = np.array([e, -1.0, -(2.0 ** -51)])[:, None]
    y = np.array([e, 1.0, 1.0])[:, None]
    assert oracle_mod.gram(x, y)[0, 0] == 2.0 ** -104


def test_gram_rejects_bad_shapes(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.gram(np.zeros((4, 33)), np.zeros((4, 33)))
    with pytest.raises(ValueError):
        oracle_mod.gram(np.zeros((4, 2)), np.zeros((4, 3)))
