"""ctypes binding of libhotrg.so: argument marshalling only.

Every function below has the name of the C entry point it wraps and raises
HotrgError on a non-zero status.  Tensors cross the boundary as numpy
float64 arrays in the interchange layout (axes x_1, x_1', ..., x_d, x_d'),
or as any object exposing a device/host pointer via ``data_ptr()`` (torch).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB = None

PREC_FP64 = 0
PREC_BF16X3 = 1
PREC_BF16X6 = 2
PREC_TF32 = 3
PREC_TF32X3 = 4

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class HotrgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().hotrg_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def library_path() -> str:
    return os.environ.get("HOTRG_LIBRARY", os.path.join(_PKG, "libhotrg.so"))


def load():
    """Load libhotrg.so (raises if it was not built: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libhotrg.so not found at {path}; build it with "
                          "`python -m paper_2110_03607_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    I64 = ctypes.c_int64
    sig = {
        "hotrg_init_ising": (I, [I, D, D, ctypes.POINTER(P)]),
        "hotrg_init_tensor": (I, [I, ctypes.POINTER(I), P, D, ctypes.POINTER(P)]),
        "hotrg_set_tensor": (I, [P, ctypes.POINTER(I), P]),
        "hotrg_set_stream": (I, [P, P]),
        "hotrg_set_allocator": (I, [P, _ALLOC_FN, _FREE_FN, P]),
        "hotrg_set_precision": (I, [P, I]),
        "hotrg_step": (I, [P, I, I]),
        "hotrg_isometry": (I, [P, I, P, I64, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "hotrg_spectrum": (I, [P, I, I, P, I64, ctypes.POINTER(I)]),
        "hotrg_truncation": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "hotrg_jacobi_sweeps": (I, [P, I, ctypes.POINTER(I)]),
        "hotrg_free_energy": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "hotrg_observables": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I)]),
        "hotrg_bond_dims": (I, [P, ctypes.POINTER(I)]),
        "hotrg_tensor": (I, [P, P, I64, ctypes.POINTER(I)]),
        "hotrg_gemm_nt": (I, [I, I, I, I, P, P, P]),
        "hotrg_gemm_nt_noalloc": (I, [I, I, I, I, P, P, P, P]),
        "hotrg_set_fp64_threshold": (I, [P, D]),
        "hotrg_set_slice_budget": (I, [P, D]),
        "hotrg_set_z2": (I, [P, I]),
        "hotrg_step_batch": (I, [ctypes.POINTER(P), I, ctypes.POINTER(I), ctypes.POINTER(I), I,
                                 ctypes.POINTER(I)]),
        "hotrg_set_parity": (I, [P, ctypes.POINTER(I)]),
        "hotrg_leg_parity": (I, [P, ctypes.POINTER(I), I, ctypes.POINTER(I)]),
        "hotrg_bottleneck_flops": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I)]),
        "hotrg_set_tangent": (I, [P, I]),
        "hotrg_energy": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I)]),
        "hotrg_specific_heat": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "hotrg_tangent_tensor": (I, [P, P, I64, ctypes.POINTER(I)]),
        "hotrg_profile": (I, [P, I]),
        "hotrg_step_times": (I, [P, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "hotrg_fp64_rate": (I, [ctypes.POINTER(D)]),
        "hotrg_gemm_rate": (I, [I, I, I, I, I, ctypes.POINTER(D)]),
        "hotrg_shard_env": (I, [P, I, I, I, I, P, I64, ctypes.POINTER(I64)]),
        "hotrg_shard_isometries": (I, [P, I, I, P, I64]),
        "hotrg_shard_contract": (I, [P, I, I, I, I, P, I64, ctypes.POINTER(I64)]),
        "hotrg_shard_finish": (I, [P, I, I, P, I64]),
        "hotrg_device_bytes": (I, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "hotrg_launch_count": (I, [P, ctypes.POINTER(I64)]),
        "hotrg_set_autotune": (I, [P, I]),
        "hotrg_autotune_entries": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), I]),
        "hotrg_graph_capture": (I, [P, I, ctypes.POINTER(I), I, ctypes.POINTER(P)]),
        "hotrg_graph_launch": (I, [P, P]),
        "hotrg_graph_free": (None, [P]),
        "hotrg_free": (None, [P]),
        "hotrg_strerror": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise HotrgError(status, where)


def _ptr(buf):
    if hasattr(buf, "data_ptr"):
        return ctypes.c_void_p(buf.data_ptr())
    return buf.ctypes.data_as(ctypes.c_void_p)


def hotrg_init_ising(d: int, beta: float, h: float):
    ctx = ctypes.c_void_p()
    _check(load().hotrg_init_ising(d, beta, h, ctypes.byref(ctx)), "hotrg_init_ising")
    return ctx


def hotrg_init_tensor(d: int, chis, t, beta: float):
    arr = np.ascontiguousarray(t, dtype=np.float64) if not hasattr(t, "data_ptr") else t
    c = (ctypes.c_int * 4)(*list(chis) + [0] * (4 - len(chis)))
    ctx = ctypes.c_void_p()
    _check(load().hotrg_init_tensor(d, c, _ptr(arr), beta, ctypes.byref(ctx)), "hotrg_init_tensor")
    return ctx


def hotrg_set_tensor(ctx, chis, t):
    arr = np.ascontiguousarray(t, dtype=np.float64) if not hasattr(t, "data_ptr") else t
    c = (ctypes.c_int * 4)(*list(chis) + [0] * (4 - len(chis)))
    _check(load().hotrg_set_tensor(ctx, c, _ptr(arr)), "hotrg_set_tensor")


def hotrg_set_stream(ctx, stream_handle: int):
    _check(load().hotrg_set_stream(ctx, ctypes.c_void_p(stream_handle)), "hotrg_set_stream")


def hotrg_set_precision(ctx, mode: int):
    _check(load().hotrg_set_precision(ctx, mode), "hotrg_set_precision")


def hotrg_step(ctx, axis: int, chi: int):
    _check(load().hotrg_step(ctx, axis, chi), "hotrg_step")


def hotrg_isometry(ctx, leg: int):
    rows, cols, prime = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib = load()
    st = lib.hotrg_isometry(ctx, leg, None, 0, ctypes.byref(rows), ctypes.byref(cols), ctypes.byref(prime))
    if st not in (0, -1) or rows.value == 0:
        _check(st, "hotrg_isometry")
    u = np.empty((rows.value, cols.value), dtype=np.float64)
    _check(lib.hotrg_isometry(ctx, leg, _ptr(u), u.size, ctypes.byref(rows), ctypes.byref(cols),
                              ctypes.byref(prime)), "hotrg_isometry")
    return u, bool(prime.value)


def hotrg_spectrum(ctx, leg: int, prime: int):
    n = ctypes.c_int()
    lib = load()
    st = lib.hotrg_spectrum(ctx, leg, prime, None, 0, ctypes.byref(n))
    if st not in (0, -1) or n.value == 0:
        _check(st, "hotrg_spectrum")
    lam = np.empty(n.value, dtype=np.float64)
    _check(lib.hotrg_spectrum(ctx, leg, prime, _ptr(lam), lam.size, ctypes.byref(n)), "hotrg_spectrum")
    return lam


def hotrg_truncation(ctx, leg: int):
    e, ep = ctypes.c_double(), ctypes.c_double()
    _check(load().hotrg_truncation(ctx, leg, ctypes.byref(e), ctypes.byref(ep)), "hotrg_truncation")
    return e.value, ep.value


def hotrg_jacobi_sweeps(ctx, leg: int) -> int:
    n = ctypes.c_int()
    _check(load().hotrg_jacobi_sweeps(ctx, leg, ctypes.byref(n)), "hotrg_jacobi_sweeps")
    return n.value


def hotrg_free_energy(ctx):
    lnz, f = ctypes.c_double(), ctypes.c_double()
    _check(load().hotrg_free_energy(ctx, ctypes.byref(lnz), ctypes.byref(f)), "hotrg_free_energy")
    return lnz.value, f.value


def hotrg_observables(ctx):
    tr, x, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().hotrg_observables(ctx, ctypes.byref(tr), ctypes.byref(x), ctypes.byref(n)),
           "hotrg_observables")
    return tr.value, x.value, n.value


def hotrg_bond_dims(ctx):
    dims = (ctypes.c_int * 4)()
    _check(load().hotrg_bond_dims(ctx, dims), "hotrg_bond_dims")
    return list(dims)


def hotrg_tensor(ctx, out=None):
    dims = (ctypes.c_int * 8)()
    lib = load()
    lib.hotrg_tensor(ctx, None, 0, dims)
    shape = [x for x in dims if x > 0]
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    n = int(np.prod(shape))
    _check(lib.hotrg_tensor(ctx, _ptr(out), n, dims), "hotrg_tensor")
    return out


def hotrg_gemm_nt(mode: int, a, b):
    """C = A . B^T with the bottleneck kernel of `mode` (numpy float64 in and out)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m, k = a.shape
    n, k2 = b.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    c = np.empty((m, n), dtype=np.float64)
    _check(load().hotrg_gemm_nt(mode, m, n, k, _ptr(a), _ptr(b), _ptr(c)), "hotrg_gemm_nt")
    return c


def hotrg_gemm_nt_noalloc(mode: int, a, b, c, stream=None):
    """C = A . B^T into the caller's `c` with no device allocation.

    a [M][K], b [N][K] and c [M][N] are CUDA float64 tensors, contiguous row-major,
    owned by the caller; `stream` is a cudaStream_t handle (an int, e.g. a torch
    stream's ``cuda_stream``; None = the legacy default stream).  The library
    cannot tell a host pointer or a wrong shape from a good one, so both are
    refused here before the call."""
    for name, x in (("a", a), ("b", b), ("c", c)):
        if not (hasattr(x, "is_cuda") and x.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if str(x.dtype) != "torch.float64" or x.dim() != 2 or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 2-d float64 tensor")
    m, k = a.shape
    n, k2 = b.shape
    if k != k2 or tuple(c.shape) != (m, n):
        raise ValueError("shapes must be a [M][K], b [N][K], c [M][N]")
    _check(load().hotrg_gemm_nt_noalloc(mode, m, n, k, _ptr(a), _ptr(b), _ptr(c),
                                        ctypes.c_void_p(stream or 0)), "hotrg_gemm_nt_noalloc")


def hotrg_set_fp64_threshold(ctx, flops: float):
    _check(load().hotrg_set_fp64_threshold(ctx, float(flops)), "hotrg_set_fp64_threshold")


def hotrg_set_slice_budget(ctx, nbytes: float):
    _check(load().hotrg_set_slice_budget(ctx, float(nbytes)), "hotrg_set_slice_budget")


def hotrg_step_batch(ctxs, axes, chis, nthreads: int = 0):
    """One step on each context, driven concurrently; returns the per-context statuses."""
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    ax = (ctypes.c_int * n)(*[int(a) for a in axes])
    ch = (ctypes.c_int * n)(*[int(x) for x in chis])
    st = (ctypes.c_int * n)()
    _check(load().hotrg_step_batch(arr, n, ax, ch, int(nthreads), st), "hotrg_step_batch")
    return [st[i] for i in range(n)]


def hotrg_set_z2(ctx, enable: bool):
    _check(load().hotrg_set_z2(ctx, 1 if enable else 0), "hotrg_set_z2")


def hotrg_set_parity(ctx, parity):
    """Declare the parities of every index (axis 0's indices first, then axis 1, ...);
    None forgets them (dense steps, no read-back)."""
    if parity is None:
        _check(load().hotrg_set_parity(ctx, None), "hotrg_set_parity")
        return
    arr = (ctypes.c_int * len(parity))(*[int(x) for x in parity])
    _check(load().hotrg_set_parity(ctx, arr), "hotrg_set_parity")


def hotrg_set_autotune(ctx, enable: bool = True):
    """Tune the chain stages' launch shapes on their first launch (results unchanged)."""
    _check(load().hotrg_set_autotune(ctx, 1 if enable else 0), "hotrg_set_autotune")


def hotrg_autotune_entries(ctx):
    """The tuned chain-stage shapes' choices (CTAs per SM)."""
    lib = load()
    n = ctypes.c_int()
    _check(lib.hotrg_autotune_entries(ctx, ctypes.byref(n), None, 0), "hotrg_autotune_entries")
    buf = (ctypes.c_int * max(1, n.value))()
    _check(lib.hotrg_autotune_entries(ctx, ctypes.byref(n), buf, max(1, n.value)), "hotrg_autotune_entries")
    return [buf[i] for i in range(n.value)]


def hotrg_graph_capture(ctx, axes, chi: int):
    """Record the steps (axes[i], chi) into a CUDA graph without running them; returns
    the graph handle (a closed sequence: see include/hotrg.h)."""
    n = len(axes)
    ax = (ctypes.c_int * n)(*[int(a) for a in axes])
    g = ctypes.c_void_p()
    _check(load().hotrg_graph_capture(ctx, n, ax, int(chi), ctypes.byref(g)), "hotrg_graph_capture")
    return g


def hotrg_graph_launch(ctx, graph):
    """Enqueue one replay of the captured steps on the context's stream."""
    _check(load().hotrg_graph_launch(ctx, graph), "hotrg_graph_launch")


def hotrg_graph_free(graph):
    load().hotrg_graph_free(graph)


def hotrg_leg_parity(ctx):
    """Known parities of every index, or None while they are unknown."""
    lib = load()
    n = ctypes.c_int()
    buf = (ctypes.c_int * 160)()
    st = lib.hotrg_leg_parity(ctx, buf, 160, ctypes.byref(n))
    if st == -7:
        return None
    _check(st, "hotrg_leg_parity")
    return [buf[i] for i in range(n.value)]


def hotrg_bottleneck_flops(ctx):
    """(dense flops, performed flops, Z2 block form used) of the last step's bottleneck."""
    dense, done, z2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().hotrg_bottleneck_flops(ctx, ctypes.byref(dense), ctypes.byref(done), ctypes.byref(z2)),
           "hotrg_bottleneck_flops")
    return dense.value, done.value, bool(z2.value)


def hotrg_set_tangent(ctx, enable=True):
    """Carry dT/d beta through the later steps (Ising context, before the first step);
    enable = 2 carries d^2 T / d beta^2 as well (FP64 form)."""
    order = int(enable) if not isinstance(enable, bool) else (1 if enable else 0)
    _check(load().hotrg_set_tangent(ctx, order), "hotrg_set_tangent")


def hotrg_specific_heat(ctx):
    """(d^2(ln Z/V)/d beta^2, specific heat per site beta^2 d^2(ln Z/V)/d beta^2) of the last step."""
    g2, c = ctypes.c_double(), ctypes.c_double()
    _check(load().hotrg_specific_heat(ctx, ctypes.byref(g2), ctypes.byref(c)), "hotrg_specific_heat")
    return g2.value, c.value


def hotrg_energy(ctx):
    """(d(ln Z/V)/d beta, internal energy per site, degenerate pairs left out) of the last step."""
    g, u, deg = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().hotrg_energy(ctx, ctypes.byref(g), ctypes.byref(u), ctypes.byref(deg)), "hotrg_energy")
    return g.value, u.value, deg.value


def hotrg_tangent_tensor(ctx, out=None):
    """d(T / Tr T)/d beta of the current tensor in the layout of hotrg_tensor."""
    dims = (ctypes.c_int * 8)()
    lib = load()
    lib.hotrg_tangent_tensor(ctx, None, 0, dims)
    shape = [x for x in dims if x > 0]
    if out is None:
        out = np.empty(shape, dtype=np.float64)
    n = int(np.prod(shape))
    _check(lib.hotrg_tangent_tensor(ctx, _ptr(out), n, dims), "hotrg_tangent_tensor")
    return out


def hotrg_profile(ctx, mode):
    """0: off; 1 (or True): every phase of each step; 2: bottleneck GEMMs, summed over steps."""
    _check(load().hotrg_profile(ctx, int(mode)), "hotrg_profile")


PHASES = ["permute", "environment", "jacobi", "select", "split", "prime_chain", "bottleneck",
          "nonprime_chain", "trace_norm", "jacobi_warm_start", "jacobi_fp32", "z2_gather_scatter"]


def hotrg_step_times(ctx):
    ms = (ctypes.c_double * 16)()
    nl = (ctypes.c_int * 16)()
    n, f64 = ctypes.c_int(), ctypes.c_int()
    _check(load().hotrg_step_times(ctx, ms, nl, ctypes.byref(n), ctypes.byref(f64)), "hotrg_step_times")
    return ({PHASES[k]: ms[k] for k in range(n.value)}, {PHASES[k]: nl[k] for k in range(n.value)},
            bool(f64.value))


def shard_sizes(ctx, axis: int, chi: int):
    """(Gram elements, c'-slices, elements of one slice) of a sharded step along `axis`."""
    dims = hotrg_bond_dims(ctx)
    d = sum(1 for x in dims if x > 0)
    chi_c = dims[axis]
    grams, pn = 0, 1
    for j in range(1, d):
        cj = dims[(axis + j) % d]
        grams += 4 * (cj * chi_c) ** 2
        pn *= min(cj * cj, chi)
    return grams, chi_c, chi_c * pn * pn


def _buf_len(buf):
    return int(buf.numel()) if hasattr(buf, "numel") and callable(buf.numel) else int(np.asarray(buf).size)


def hotrg_shard_env(ctx, axis: int, chi: int, part: int, nparts: int, out=None):
    """This rank's share of the step's environment Grams (numpy FP64, or `out`)."""
    n = shard_sizes(ctx, axis, chi)[0]
    if out is None:
        out = np.zeros(n, dtype=np.float64)
    got = ctypes.c_int64()
    _check(load().hotrg_shard_env(ctx, axis, chi, part, nparts, _ptr(out), _buf_len(out), ctypes.byref(got)),
           "hotrg_shard_env")
    return out


def hotrg_shard_isometries(ctx, axis: int, chi: int, grams):
    _check(load().hotrg_shard_isometries(ctx, axis, chi, _ptr(grams), _buf_len(grams)), "hotrg_shard_isometries")


def hotrg_shard_contract(ctx, axis: int, chi: int, c_lo: int, c_hi: int, out=None):
    """The new tensor's c'-slices [c_lo, c_hi) (numpy FP64 [c_hi - c_lo][Rn][Pn], or `out`)."""
    _, _, per = shard_sizes(ctx, axis, chi)
    if out is None:
        out = np.zeros((c_hi - c_lo) * per, dtype=np.float64)
    got = ctypes.c_int64()
    _check(load().hotrg_shard_contract(ctx, axis, chi, c_lo, c_hi, _ptr(out), _buf_len(out), ctypes.byref(got)),
           "hotrg_shard_contract")
    return out


def hotrg_shard_finish(ctx, axis: int, chi: int, slices):
    _check(load().hotrg_shard_finish(ctx, axis, chi, _ptr(slices), _buf_len(slices)), "hotrg_shard_finish")


def hotrg_gemm_rate(mode: int, m: int, n: int, k: int, iters: int) -> float:
    """Milliseconds per launch of the split GEMM kernel (BF16 or TF32 pieces of `mode`) on
    device-resident operands."""
    v = ctypes.c_double()
    _check(load().hotrg_gemm_rate(mode, m, n, k, iters, ctypes.byref(v)), "hotrg_gemm_rate")
    return v.value


def hotrg_fp64_rate() -> float:
    """Measured FP64 FMA rate of the current device, TFLOP/s."""
    v = ctypes.c_double()
    _check(load().hotrg_fp64_rate(ctypes.byref(v)), "hotrg_fp64_rate")
    return v.value


def hotrg_device_bytes(ctx) -> int:
    b = ctypes.c_size_t()
    _check(load().hotrg_device_bytes(ctx, ctypes.byref(b)), "hotrg_device_bytes")
    return b.value


def hotrg_launch_count(ctx) -> int:
    n = ctypes.c_int64()
    _check(load().hotrg_launch_count(ctx, ctypes.byref(n)), "hotrg_launch_count")
    return n.value


# ctx address -> the ctypes callbacks given to hotrg_set_allocator, referenced until
# hotrg_free (the library calls them until then)
_ALLOCATORS = {}


def hotrg_set_allocator(ctx, alloc=None, free=None):
    """Route the context's device allocations through alloc(nbytes) -> device pointer
    (an int; 0 or None on failure) and free(ptr); alloc = free = None returns to
    cudaMalloc.  Buffers already held are released through the previous hooks first."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        cb = (_ALLOC_FN(), _FREE_FN())
    else:
        cb = (_ALLOC_FN(lambda nbytes, _user: alloc(int(nbytes)) or None),
              _FREE_FN(lambda ptr, _user: free(ptr)))
    _check(load().hotrg_set_allocator(ctx, cb[0], cb[1], None), "hotrg_set_allocator")
    key = getattr(ctx, "value", ctx)
    if alloc is None:
        _ALLOCATORS.pop(key, None)
    else:
        _ALLOCATORS[key] = cb


def hotrg_free(ctx):
    load().hotrg_free(ctx)
    _ALLOCATORS.pop(getattr(ctx, "value", ctx), None)


def hotrg_strerror(status: int) -> str:
    return load().hotrg_strerror(status).decode()


class Hotrg:
    """Owning handle around one context, with torch streams and memory."""

    def __init__(self, d: int, beta: float, h: float = 0.0, precision: int = PREC_BF16X6,
                 use_torch: bool = True, tensor=None, chis=None, fp64_below: float | None = None,
                 z2: bool = True):
        self.d = d
        self.beta = beta
        if tensor is None:
            self.ctx = hotrg_init_ising(d, beta, h)
        else:
            self.ctx = hotrg_init_tensor(d, chis, tensor, beta)
        self._cb = None
        if use_torch:
            self.use_torch()
        hotrg_set_precision(self.ctx, precision)
        if fp64_below is not None:
            hotrg_set_fp64_threshold(self.ctx, fp64_below)
        hotrg_set_z2(self.ctx, z2)

    def use_torch(self):
        import torch

        def _alloc(nbytes, _user):
            return torch.cuda.caching_allocator_alloc(int(nbytes))

        def _free(ptr, _user):
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
        _check(load().hotrg_set_allocator(self.ctx, self._cb[0], self._cb[1], None), "hotrg_set_allocator")
        hotrg_set_stream(self.ctx, torch.cuda.current_stream().cuda_stream)

    def step(self, axis: int, chi: int):
        hotrg_step(self.ctx, axis, chi)

    def free_energy(self):
        return hotrg_free_energy(self.ctx)

    def energy(self):
        return hotrg_energy(self.ctx)

    def specific_heat(self):
        return hotrg_specific_heat(self.ctx)

    def close(self):
        if self.ctx:
            hotrg_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
