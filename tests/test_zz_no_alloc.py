"""hotrg_gemm_nt_noalloc: the bottleneck GEMM for callers that may not allocate
device memory (a framework that owns all device memory through its own pool, or
a loop where cudaMalloc/cudaFree would synchronise the device).  Its scratch is a
fixed device array inside the library.  The test calls it through the C ABI with
caller-owned device buffers, checks it against the plain FP64 product a @ b.T
(the error bounds of the allocating entry point's tests) and against the
allocating hotrg_gemm_nt bit for bit, twice in a row so that the second round
runs on scratch the first one left behind, and checks that the calls leave the
device's free memory unchanged.  Collected last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _fn():
    import paper_2110_03607_gb300 as pkg

    lib = pkg.load()
    fn = lib.hotrg_gemm_nt_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 4
    return pkg, fn


def _bound(pkg, mode, k):
    """Largest admitted |C - A B^T| / (|A| |B|^T), per element."""
    if mode == pkg.PREC_FP64:
        return 1e-14 * max(1, k)
    if mode == pkg.PREC_BF16X6:
        return 4 * 2.0 ** -24 * (1 + k ** 0.5) * 4     # 3 pieces: inputs to 2^-24, FP32 sums
    return 4 * 2.0 ** -16                               # 2 pieces: inputs to 2^-16


def test_noalloc_gemm_matches_plain_product_and_allocating_entry_point_twice():
    import torch

    pkg, fn = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    # ragged sizes: K not a multiple of 64 on the first call, so the pad must be cleared;
    # more than one 128 x 256 tile, and partial tiles
    cases = [(pkg.PREC_BF16X6, 300, 520, 200), (pkg.PREC_BF16X6, 257, 384, 130),
             (pkg.PREC_BF16X3, 129, 260, 64), (pkg.PREC_FP64, 200, 150, 333)]
    data = []
    for mode, m, n, k in cases:
        a = rng.standard_normal((m, k))
        b = rng.standard_normal((n, k))
        ref = pkg.hotrg_gemm_nt(mode, a, b)          # the allocating entry point, first
        da = torch.from_numpy(a).cuda()
        db = torch.from_numpy(b).cuda()
        dc = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        data.append((mode, m, n, k, a, b, ref, da, db, dc))
    # one call per mode loads every kernel module the calls use
    for mode, m, n, k, a, b, ref, da, db, dc in data:
        assert fn(mode, m, n, k, da.data_ptr(), db.data_ptr(), dc.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for mode, m, n, k, a, b, ref, da, db, dc in data:
            dc.fill_(float("nan"))
            st = fn(mode, m, n, k, da.data_ptr(), db.data_ptr(), dc.data_ptr(), stream)
            assert st == 0, pkg.hotrg_strerror(st)
            got = dc.cpu().numpy()
            exact = a @ b.T
            scale = np.abs(a) @ np.abs(b).T
            assert np.max(np.abs(got - exact) / scale) <= _bound(pkg, mode, k), (mode, m, n, k)
            # same kernels on the same inputs: the results agree bit for bit
            np.testing.assert_array_equal(got, ref)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the calls changed the device's free memory"


def test_noalloc_rejects_sizes_beyond_its_scratch_and_limits():
    import torch

    pkg, fn = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    m = n = 4096
    k = 4096      # 256 + 2*3*4096*4096*2 + 4*4096^2 bytes > 64 MiB
    da = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    dc = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    assert fn(pkg.PREC_BF16X6, m, n, k, da.data_ptr(), da.data_ptr(), dc.data_ptr(), stream) == -1
    # the size limits of hotrg_gemm_nt hold in every mode, FP64 included (no scratch)
    assert fn(pkg.PREC_FP64, 1 << 21, 1, 1, da.data_ptr(), da.data_ptr(), dc.data_ptr(), stream) == -1
    assert fn(pkg.PREC_BF16X6, 0, 1, 1, da.data_ptr(), da.data_ptr(), dc.data_ptr(), stream) == -1
