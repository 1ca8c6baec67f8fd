"""The C ABI library loads and exports every entry point include/hotrg.h declares (no GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hotrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hotrg_[a-z0-9_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2110_03607_gb300 import build

    return build.build()


def test_header_declares_the_core_calls():
    names = _declared()
    for n in ("hotrg_init_ising", "hotrg_step", "hotrg_isometry", "hotrg_free_energy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hotrg_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports_errors_without_a_gpu(lib_path):
    import paper_2110_03607_gb300 as pkg

    lib = pkg.load()
    assert lib.hotrg_strerror(-1).decode() == "invalid argument"
    # argument checks happen before any CUDA call
    ctx = ctypes.c_void_p()
    assert lib.hotrg_init_ising(1, 0.3, 0.0, ctypes.byref(ctx)) == -1
    assert lib.hotrg_init_ising(3, -0.1, 0.0, ctypes.byref(ctx)) == -1
    assert lib.hotrg_step(None, 0, 4) == -1
    assert lib.hotrg_gemm_nt(7, 1, 1, 1, None, None, None) == -1
    assert lib.hotrg_gemm_nt_noalloc(7, 1, 1, 1, None, None, None, None) == -1
    assert lib.hotrg_gemm_nt_noalloc(0, 0, 1, 1, None, None, None, None) == -1


def test_binding_wraps_every_declared_entry_point():
    from paper_2110_03607_gb300 import binding

    names = _declared()
    assert len(names) > 40
    assert [n for n in names if not callable(getattr(binding, n, None))] == []


def test_binding_refusals_before_the_library_call():
    import torch

    from paper_2110_03607_gb300 import binding

    # host tensors would reach the kernels as device pointers: refused in the binding
    a = torch.zeros((4, 8), dtype=torch.float64)
    with pytest.raises(ValueError):
        binding.hotrg_gemm_nt_noalloc(binding.PREC_FP64, a, a, torch.zeros((4, 4), dtype=torch.float64))
    with pytest.raises(ValueError):
        binding.hotrg_set_allocator(ctypes.c_void_p(), lambda n: 0, None)
    # a null context is refused by the library before any CUDA call
    with pytest.raises(binding.HotrgError) as e:
        binding.hotrg_set_allocator(ctypes.c_void_p(), lambda n: 0, lambda p: None)
    assert e.value.status == -1
    assert binding._ALLOCATORS == {}


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2110_03607_gb300.binding as b

    monkeypatch.setattr(b, "_LIB", None)
    monkeypatch.setenv("HOTRG_LIBRARY", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        b.load()


def test_binding_precision_constants_match_the_header():
    from paper_2110_03607_gb300 import binding

    src = open(os.path.join(ROOT, "include", "hotrg.h")).read()
    body = re.search(r"enum hotrg_precision \{(.*?)\};", src, flags=re.S).group(1)
    enum = {k: int(v) for k, v in re.findall(r"HOTRG_(PREC_[A-Z0-9]+)\s*=\s*(\d+)", body)}
    assert set(enum) == {"PREC_FP64", "PREC_BF16X3", "PREC_BF16X6", "PREC_TF32", "PREC_TF32X3"}
    for k, v in enum.items():
        assert getattr(binding, k) == v, k
