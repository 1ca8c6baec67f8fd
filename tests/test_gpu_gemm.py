"""The bottleneck GEMM kernels (tcgen05 split-BF16 and FP64 DFMA) against plain products."""

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
    # small integers times a power of two: exactly representable in BF16
    return rng.integers(-8, 9, size=shape).astype(np.float64) * 0.25


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_tc_gemm_bit_exact_on_bf16_representable_inputs(pkg, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    a = _bf16_exact(rng, (m, k))
    b = _bf16_exact(rng, (n, k))
    ref = a @ b.T          # integers/16 below 2^24: exact in FP32 and FP64
    for mode in (pkg.PREC_BF16X3, pkg.PREC_BF16X6):
        c = pkg.hotrg_gemm_nt(mode, a, b)
        np.testing.assert_array_equal(c, ref)


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


def test_tc_gemm_long_accumulation_is_unbiased(pkg):
    # all products positive and exact in BF16: the only error is the FP32
    # accumulation; the tensor core truncates, so a single long accumulation
    # drifts low by ~1e-5 over K = 4096.  The chunked epilogue keeps it near RN.
    rng = np.random.default_rng(11)
    m, n, k = 256, 256, 4096
    a = rng.integers(1, 256, size=(m, k)).astype(np.float64) / 128.0
    b = rng.integers(1, 256, size=(n, k)).astype(np.float64) / 128.0
    ref = a @ b.T
    for mode in (pkg.PREC_BF16X3, pkg.PREC_BF16X6):
        c = pkg.hotrg_gemm_nt(mode, a, b)
        rel = (c - ref) / ref
        assert abs(rel.mean()) <= 1.5e-7, rel.mean()
        assert np.abs(rel).max() <= 2e-6
