"""GPU parity of the tensor-core low-precision block product W = A_lp V.

The reference rounds the same operands the same way with torch's own BF16 /
FP8 E4M3 conversions (round to nearest even, saturating) and multiplies them
in FP64; the kernel accumulates in FP32 on the tensor cores: one FP32
addition per MMA (16 BF16 products, or 2 x 32 FP8 products), so each entry
may differ by at most about (n/16) FP32 roundings of (|A_lp| |V_lp|)_ij; the
test allows twice that, 2 (n/16 + 8) 2^-24 (|A_lp| |V_lp|)_ij.
Sizes span one ragged tile up to many tiles with ragged row and k tails, and
q = 1 .. 32 (both accumulator widths, N = 16 and 32).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [(100, 1), (128, 8), (300, 16), (1000, 17), (777, 32), (4100, 5), (2048, 32)]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1204_0069_gb300 import build as B
    B.build()
    from paper_1204_0069_gb300 import ccg
    s = ccg.Solver(device=0)
    yield dict(torch=torch, ccg=ccg, solver=s)
    s.close()


def round_to_format(x, sig_bits, min_exp=None, max_abs=None):
    """Round float64 x to nearest-even in a binary format with `sig_bits`
    significant bits, normal exponents down to min_exp (subnormal spacing
    below) and saturation at max_abs -- written out from the format
    definitions (bfloat16: 8 significant bits; FP8 E4M3: 4 significant bits,
    min normal 2^-6, max 448), so that no library conversion (which may round
    twice through float32) decides the expected value."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    expo = e - 1                             # floor(log2 |x|)
    if min_exp is not None:
        expo = np.maximum(expo, min_exp)
    step = np.ldexp(1.0, expo - (sig_bits - 1))
    q = np.rint(x / step) * step             # numpy rint: round half to even
    q[x == 0] = 0.0
    if max_abs is not None:
        q = np.clip(q, -max_abs, max_abs)
    return q


def bf16_round(torch, x):
    return round_to_format(x, 8)


def e4m3_round(torch, x):
    return round_to_format(x, 4, min_exp=-6, max_abs=448.0)


def tf32_trunc(x32):
    """TF32 part of FP32 values: the low 13 mantissa bits cleared."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


def reference(torch, A, V, fmt):
    if fmt == 2:
        # FP32 A; the four TF32 products (A_hi + A_lo)(D_hi + D_lo) with
        # hi = tf32(x), lo = tf32(x - hi) (x rounded to FP32 first)
        Af = A.astype(np.float32)
        Ah = tf32_trunc(Af)
        Al = tf32_trunc((Af.astype(np.float64) - Ah).astype(np.float32))
        Vf = V.astype(np.float32)
        Vh = tf32_trunc(Vf)
        Vl = tf32_trunc((Vf.astype(np.float64) - Vh).astype(np.float32))
        W = Ah @ Vh + Ah @ Vl + Al @ Vh + Al @ Vl
        mag = (np.abs(Ah) + np.abs(Al)) @ (np.abs(Vh) + np.abs(Vl))
        return W, mag
    if fmt == 0:
        Aq = bf16_round(torch, A)
        Vq = bf16_round(torch, V)
    else:
        s = (np.abs(A).max(axis=1) / 448.0).astype(np.float32).astype(np.float64)
        s[s == 0] = 1.0
        Aq = e4m3_round(torch, A * (1.0 / s)[:, None]) * s[:, None]
        sg = (np.abs(V).max(axis=0).astype(np.float32) / np.float32(448.0)).astype(np.float64)
        sg[sg == 0] = 1.0
        x = V / sg[None, :]
        hi = e4m3_round(torch, x)
        lo = e4m3_round(torch, x - hi)
        Vq = (hi + lo) * sg[None, :]
    return Aq @ Vq, np.abs(Aq) @ np.abs(Vq)


@pytest.mark.parametrize("fmt", [0, 1, 2], ids=["bf16", "fp8", "fp32_tf32x3"])
@pytest.mark.parametrize("n,q", CASES)
def test_lowp_block_product(env, fmt, n, q):
    torch = env["torch"]
    rng = np.random.default_rng(1000 * n + q + fmt)
    A = rng.standard_normal((n, n))
    A = 0.5 * (A + A.T)
    V = rng.standard_normal((n, q))
    dA = torch.from_numpy(A).cuda()
    m = env["solver"].lowp_matrix(dA, fmt)
    W = torch.zeros((n, q), dtype=torch.float64, device="cuda")
    rc, ms = m.block_product(torch.from_numpy(V).cuda(), W)
    assert rc == 0
    ref, mag = reference(torch, A, V, fmt)
    err = np.abs(W.cpu().numpy() - ref)
    if fmt == 2:
        # 2 MMAs per 8 k (K = 8 per TF32 MMA); plus the TF32 reading of the low
        # parts (truncation or rounding: one TF32 ulp of a low part)
        bound = 2.0 * (2 * n / 8 + 8) * 2.0 ** -24 * mag + 2.0 ** -19 * mag
        # and the product is FP32-accurate against the exact FP64 one
        exact = np.abs(W.cpu().numpy() - A @ V)
        assert np.all(exact <= 2.0 ** -16 * (np.abs(A) @ np.abs(V)))
    else:
        bound = 2.0 * (n / 16 + 8) * 2.0 ** -24 * mag
    assert np.all(err <= bound + 1e-300), (err / mag).max()
    # repeated call on the same operands is bitwise identical (fixed-order fixup)
    W2 = torch.zeros_like(W)
    assert m.block_product(torch.from_numpy(V).cuda(), W2)[0] == 0
    assert torch.equal(W, W2)
    m.close()


def test_lowp_bytes_and_host_operands(env):
    torch = env["torch"]
    n, q = 513, 4
    rng = np.random.default_rng(3)
    A = rng.standard_normal((n, n))
    m = env["solver"].lowp_matrix(A, 0)  # host A is staged inside the call
    assert m.nbytes() == n * 640 * 2      # rows padded to a multiple of 128
    V = rng.standard_normal((n, q))
    W = np.zeros((n, q))
    assert m.block_product(V, W)[0] == 0
    ref, mag = reference(torch, A, V, 0)
    assert np.all(np.abs(W - ref) <= 2.0 * (n / 16 + 8) * 2.0 ** -24 * mag)
    m.close()
