"""The error model behind the bf16x3 tolerances of the GPU tests, checked by
emulating the split product on the CPU.

a = hi + lo with hi = bf16(a) and lo = bf16(a - hi) (round to nearest even);
the tensor cores form hi_a hi_b + hi_a lo_b + lo_a hi_b with FP32
accumulation.  The dropped term lo_a lo_b and the split's own rounding leave
a relative error of at most 3 * 2^-16 per product (typically ~2^-18), so a
norm-wise relative error well below the tests' 2e-4 for random
contractions; the FP32 accumulation adds only ~K^(1/2) 2^-24.
"""
import numpy as np


def _bf16(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = ((u >> 16) & 1) + 0x7FFF
    r = ((u + bias) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _split(x):
    x32 = np.asarray(x, dtype=np.float32)
    hi = _bf16(x32)
    lo = _bf16(x32 - hi)  # exact in FP32 (Sterbenz): the remainder of a float32
    return hi, lo


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert _bf16(np.float32(1 + 2 ** -8)) == np.float32(1.0)
    assert _bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    assert _bf16(np.float32(1 + 2 ** -7)) == np.float32(1 + 2 ** -7)


def test_split_product_error_per_product():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(200000)
    b = rng.standard_normal(200000)
    ha, la = _split(a)
    hb, lb = _split(b)
    p3 = ha.astype(np.float64) * hb + ha.astype(np.float64) * lb + la.astype(np.float64) * hb
    rel = np.abs(p3 - a * b) / (np.abs(a) * np.abs(b))
    # bf16 keeps 8 significant bits: |a - hi| <= 2^-8 |a|, lo's own rounding <= 2^-16 |a|, and the
    # dropped lo_a lo_b <= 2^-16 |a b|: at most 3 * 2^-16 per product (plus FP32's 2^-24 terms)
    assert rel.max() <= 3 * 2.0 ** -16 + 2.0 ** -22
    assert np.median(rel) <= 2.0 ** -17


def test_split_gemm_normwise_error():
    rng = np.random.default_rng(2)
    for k in (64, 1024):
        A = rng.standard_normal((96, k))
        B = rng.standard_normal((k, 80))
        ha, la = _split(A)
        hb, lb = _split(B)
        f = lambda x, y: x.astype(np.float32) @ y.astype(np.float32)  # FP32 accumulation  # noqa: E731
        C3 = f(ha, hb).astype(np.float64) + f(ha, lb) + f(la, hb)
        ref = A @ B
        err = np.linalg.norm(C3 - ref) / np.linalg.norm(ref)
        assert err < 2e-5   # an order below the 2e-4 the GPU parity tests allow


def _split3(x):
    """a = hi + lo + lo2, each bf16, with the remainders taken in FP64 (the
    environment updates' operands are FP64): |a - hi - lo - lo2| <= 2^-24 |a|."""
    x = np.asarray(x, dtype=np.float64)
    hi = _bf16(x.astype(np.float32)).astype(np.float64)
    r1 = x - hi
    lo = _bf16(r1.astype(np.float32)).astype(np.float64)
    lo2 = _bf16((r1 - lo).astype(np.float32)).astype(np.float64)
    return hi, lo, lo2


def test_three_plane_split_product_error():
    """The environment updates' six products hi hi + hi lo + lo hi + hi lo2 +
    lo lo + lo2 hi: the dropped terms (lo lo2, lo2 lo, lo2 lo2) and the split's
    remainders leave about 2^-24 per product, two orders below bf16x3."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal(200000)
    b = rng.standard_normal(200000)
    ha, la, ma = _split3(a)
    hb, lb, mb = _split3(b)
    p6 = ha * hb + ha * lb + la * hb + ha * mb + la * lb + ma * hb
    rel = np.abs(p6 - a * b) / (np.abs(a) * np.abs(b))
    assert rel.max() <= 4 * 2.0 ** -24
    A = rng.standard_normal((96, 1024))
    B = rng.standard_normal((1024, 80))
    (ha, la, ma), (hb, lb, mb) = _split3(A), _split3(B)
    f = lambda x, y: (x.astype(np.float32) @ y.astype(np.float32)).astype(np.float64)  # noqa: E731
    C6 = f(ha, hb) + f(ha, lb) + f(la, hb) + f(ha, mb) + f(la, lb) + f(ma, hb)
    ref = A @ B
    err = np.linalg.norm(C6 - ref) / np.linalg.norm(ref)
    assert err < 1e-6  # below the 5e-6 the GPU environment-update tests allow
