"""CPU checks that the seeded input generators follow their stated recipes.

The generators hold none of the solver's arithmetic; these tests fix what the
recipes promise so that the parity and benchmark inputs are the systems they
are said to be: symmetry of the stored matrix, positive definiteness and the
spectrum, the diagonal of the kernel family, the value ranges of the paper's
own family (Sec. 5: spectrum uniform in [1, kappa], b and X_0 uniform in
[-10, 10]), the draw order within one seeded stream, and reproducibility.
"""
import math

import numpy as np
import pytest

from paper_1204_0069_gb300 import workloads as wl


def _contig_f64(*arrays):
    for a in arrays:
        assert a.dtype == np.float64 and a.flags.c_contiguous


def test_gram_shift_recipe():
    n, shift = 128, 0.5
    A, b = wl.gram_shift(n, seed=0, shift=shift)
    _contig_f64(A, b)
    assert A.shape == (n, n) and b.shape == (n,)
    np.testing.assert_array_equal(A, A.T)
    lam = np.linalg.eigvalsh(A)
    # G G^T / n is positive semidefinite; its largest eigenvalue sits near the
    # Marchenko-Pastur edge (1 + 1)^2 = 4 for a square G
    assert lam[0] >= shift - 1e-12
    assert lam[-1] <= shift + 5.0
    # b is the next draw of the same stream, after the n x n Gaussian G
    rng = np.random.default_rng(0)
    G = rng.standard_normal((n, n))
    np.testing.assert_array_equal(b, rng.standard_normal(n))
    np.testing.assert_allclose(A - shift * np.eye(n), G @ G.T / n, rtol=0, atol=1e-13)


def test_exp_kernel_recipe():
    n, length, nugget = 200, 0.2, 1e-2
    A, b = wl.exp_kernel(n, seed=1, length=length, nugget=nugget)
    _contig_f64(A, b)
    np.testing.assert_array_equal(A, A.T)
    np.testing.assert_array_equal(np.diag(A), np.full(n, 1.0 + nugget))
    off = A[~np.eye(n, dtype=bool)]
    assert np.all(off > 0.0) and np.all(off < 1.0)
    # points are the first draws of the stream, b the next
    rng = np.random.default_rng(1)
    z = rng.random((n, 3))
    np.testing.assert_array_equal(b, rng.standard_normal(n))
    for i, j in [(0, 1), (5, 199), (123, 17), (64, 65)]:
        ref = math.exp(-math.dist(z[i], z[j]) / length)
        assert abs(A[i, j] - ref) <= 4e-16 * ref
    # the exponential kernel is positive definite, so A - nugget I is PSD
    assert np.linalg.eigvalsh(A)[0] >= nugget * (1.0 - 1e-6)


def test_haar_spectrum_recipe():
    n, kappa, p = 60, 1e6, 3
    A, b, X0 = wl.haar_spectrum(n, seed=5, kappa=kappa, p=p)
    _contig_f64(A, b, X0)
    assert X0.shape == (n, p)
    np.testing.assert_array_equal(A, A.T)
    # spectrum: the uniform draws on [1, kappa] that follow the n x n Gaussian
    rng = np.random.default_rng(5)
    rng.standard_normal((n, n))
    lam_ref = np.sort(rng.uniform(1.0, kappa, size=n))
    lam = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(lam, lam_ref, rtol=0, atol=1e-7)
    assert lam[0] >= 1.0 - 1e-7 and lam[-1] <= kappa * (1 + 1e-12)
    assert np.all(np.abs(b) <= 10.0) and np.all(np.abs(X0) <= 10.0)
    # entries spread over the whole interval, not a narrower one
    assert b.min() < -8.0 and b.max() > 8.0


def test_random_spd_condition_number():
    for n, cond in [(8, 10.0), (30, 100.0), (40, 1e4)]:
        A, b = wl.random_spd(n, seed=n, cond=cond)
        _contig_f64(A, b)
        np.testing.assert_array_equal(A, A.T)
        lam = np.linalg.eigvalsh(A)
        np.testing.assert_allclose(lam, np.geomspace(1.0, cond, n), rtol=1e-9, atol=0)


@pytest.mark.parametrize("gen,args", [
    (wl.gram_shift, (48,)),
    (wl.exp_kernel, (48,)),
    (wl.haar_spectrum, (20,)),
    (wl.random_spd, (16, 3)),
])
def test_generators_are_reproducible_and_seed_dependent(gen, args):
    first = gen(*args) if gen is wl.random_spd else gen(*args, seed=11)
    again = gen(*args) if gen is wl.random_spd else gen(*args, seed=11)
    for x, y in zip(first, again):
        np.testing.assert_array_equal(x, y)
    if gen is not wl.random_spd:
        other = gen(*args, seed=12)
        assert not np.array_equal(first[0], other[0])
        assert not np.array_equal(first[1], other[1])


def test_random_block_shape_and_scale():
    V = wl.random_block(1000, 4, seed=2, scale=3.0)
    _contig_f64(V)
    assert V.shape == (1000, 4)
    assert 2.7 < V.std() < 3.3


@pytest.mark.parametrize("n,length,nugget", [(700, 0.1, 1e-3), (4500, 0.37, 1e-4)])
def test_device_kernel_builder_matches_the_host_recipe(n, length, nugget):
    """The on-device builder of the benchmark (run here on the CPU device) gives
    the exponential-kernel family of the host recipe: same points, diagonal
    exactly 1 + nugget, exactly symmetric, and every entry within a few ulps
    of the argument's size (exp multiplies a relative error of its argument
    t = |z_i - z_j| / length by t); the second case spans a ragged last row
    chunk."""
    torch = pytest.importorskip("torch")
    import bench
    A = bench.device_exp_kernel(n, 2, length, nugget, torch.device("cpu")).numpy()
    R, _ = wl.exp_kernel(n, seed=2, length=length, nugget=nugget)
    np.testing.assert_array_equal(np.diag(A), np.full(n, 1.0 + nugget))
    np.testing.assert_array_equal(A, A.T)
    t = -np.log(R - nugget * np.eye(n))
    assert np.max(np.abs(A - R) / (R * (1.0 + t))) <= 4 * 2.0 ** -52
