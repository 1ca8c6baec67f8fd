"""hotrg_gemm_nt_noalloc: the bottleneck GEMM for callers that may not allocate
device memory (a pool-owning framework, or a loop where cudaMalloc/cudaFree
would synchronise the device).  Its scratch is a fixed device array inside the
library; the test calls it through the C ABI with caller-owned device buffers
and compares with the allocating hotrg_gemm_nt, twice in a row so that the
second call runs on scratch the first one left behind.  Collected last.
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


def test_noalloc_gemm_matches_allocating_entry_point_twice():
    import torch

    pkg, fn = _fn()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(2024)
    # ragged sizes: K not a multiple of 64 on the first call, so the pad must be cleared
    cases = [(pkg.PREC_BF16X6, 300, 520, 200), (pkg.PREC_BF16X6, 257, 384, 130),
             (pkg.PREC_BF16X3, 129, 260, 64)]
    for mode, m, n, k in cases:
        a = rng.standard_normal((m, k))
        b = rng.standard_normal((n, k))
        ref = pkg.hotrg_gemm_nt(mode, a, b)
        scale = np.abs(a) @ np.abs(b).T
        da = torch.from_numpy(a).cuda()
        db = torch.from_numpy(b).cuda()
        dc = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(mode, m, n, k, da.data_ptr(), db.data_ptr(), dc.data_ptr(), stream)
        assert st == 0, pkg.hotrg_strerror(st)
        got = dc.cpu().numpy()
        tol = 4 * 2.0 ** -24 * (1 + k ** 0.5) * 4 if mode == pkg.PREC_BF16X6 else 4 * 2.0 ** -16
        assert np.max(np.abs(got - ref) / scale) <= tol
        # same kernels on the same inputs: the results agree bit for bit
        np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    pkg, fn = _fn()
    m = n = 4096
    k = 4096      # 2*3*8192*4096 + 4*4096^2 bytes > 64 MiB
    da = torch.zeros((m, k), dtype=torch.float64, device="cuda")
    dc = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    st = fn(pkg.PREC_BF16X6, m, n, k, da.data_ptr(), da.data_ptr(), dc.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == -1   # HOTRG_EINVAL
