"""The bottleneck GEMM kernels (tcgen05 split-BF16 and split-TF32, FP64 DFMA) against plain products."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (64, 64, 64), (128, 256, 64), (200, 300, 130), (257, 513, 1000), (96, 40, 72)]


@pytest.fixture(scope="module")
def pkg():
    import paper_2110_03607_gb300 as p

    p.load()
    return p


def _bf16_exact(rng, shape):
    # small integers times a power of two: exactly representable in BF16 (and TF32)
    return rng.integers(-8, 9, size=shape).astype(np.float64) * 0.25


def _split_modes(pkg):
    return (pkg.PREC_BF16X3, pkg.PREC_BF16X6, pkg.PREC_TF32, pkg.PREC_TF32X3)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_tc_gemm_bit_exact_on_bf16_representable_inputs(pkg, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = _bf16_exact(rng, (m, k))
    b = _bf16_exact(rng, (n, k))
    ref = a @ b.T          # integers/16 below 2^24: exact in FP32 and FP64
    for mode in _split_modes(pkg):
        c = pkg.hotrg_gemm_nt(mode, a, b)
        np.testing.assert_array_equal(c, ref, err_msg=f"mode {mode}")


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (257, 513, 1000)])
def test_tf32_pieces_keep_eleven_significant_bits(pkg, m, n, k):
    # A: 11-bit odd integers / 2048, exact in TF32 (10 stored bits) but not in BF16 (7);
    # B: integers in [-2, 2].  Every partial sum is an integer / 2048 below 2^24 / 2048,
    # exact in FP32 in any order, so one TF32 piece gives the product bit for bit.
    rng = np.random.default_rng(5 + m + k)
    a = (2 * rng.integers(512, 1024, size=(m, k)) + 1).astype(np.float64) / 2048.0
    b = rng.integers(-2, 3, size=(n, k)).astype(np.float64)
    bits = a.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0x1FFF == 0)      # TF32-exact
    assert np.all(bits & 0xFFFF != 0)      # none of them BF16-exact
    ref = a @ b.T
    np.testing.assert_array_equal(pkg.hotrg_gemm_nt(pkg.PREC_TF32, a, b), ref)


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_gemm_modes_against_fp64_product(pkg, m, n, k):
    rng = np.random.default_rng(1000 + m + n + k)
    a = rng.standard_normal((m, k))
    b = rng.standard_normal((n, k))
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T            # sum_k |a||b| bounds every rounding error
    c64 = pkg.hotrg_gemm_nt(pkg.PREC_FP64, a, b)
    assert np.max(np.abs(c64 - ref) / scale) <= 1e-14 * max(1, k)
    # 3 pieces: inputs to 2^-24 relative; FP32 accumulation error <= k 2^-24 sum|ab|
    c6 = pkg.hotrg_gemm_nt(pkg.PREC_BF16X6, a, b)
    assert np.max(np.abs(c6 - ref) / scale) <= 4 * 2.0 ** -24 * (1 + k ** 0.5) * 4
    # 2 pieces: inputs to 2^-16 relative
    c3 = pkg.hotrg_gemm_nt(pkg.PREC_BF16X3, a, b)
    assert np.max(np.abs(c3 - ref) / scale) <= 4 * 2.0 ** -16
    # 2 TF32 pieces: inputs to 2^-22 relative (round to nearest: 2^-23 each), the dropped
    # term x_1 y_1 below 2^-22 of |x||y|; plus the FP32 accumulation of the 3-piece form
    ct3 = pkg.hotrg_gemm_nt(pkg.PREC_TF32X3, a, b)
    assert np.max(np.abs(ct3 - ref) / scale) <= 4 * 2.0 ** -22 + 4 * 2.0 ** -24 * (1 + k ** 0.5) * 4
    # 1 TF32 piece: inputs to 2^-11 relative
    ct = pkg.hotrg_gemm_nt(pkg.PREC_TF32, a, b)
    err_t = np.max(np.abs(ct - ref) / scale)
    assert err_t <= 4 * 2.0 ** -11
    if k >= 64:   # and no better than one piece can be: the second piece is really dropped
        assert err_t >= 2.0 ** -20


def test_tc_gemm_long_accumulation_is_unbiased(pkg):
    # all products positive and exact in BF16: the only error is the FP32
    # accumulation; the tensor core truncates, so a single long accumulation
    # drifts low by ~1e-5 over K = 4096.  The chunked epilogue keeps it near RN.
    rng = np.random.default_rng(11)
    m, n, k = 256, 256, 4096
    a = rng.integers(1, 256, size=(m, k)).astype(np.float64) / 128.0
    b = rng.integers(1, 256, size=(n, k)).astype(np.float64) / 128.0
    ref = a @ b.T
    for mode in _split_modes(pkg):
        c = pkg.hotrg_gemm_nt(mode, a, b)
        rel = (c - ref) / ref
        assert abs(rel.mean()) <= 1.5e-7, rel.mean()
        assert np.abs(rel).max() <= 2e-6
