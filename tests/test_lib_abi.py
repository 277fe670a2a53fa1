"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/asm2.h declares
(no GPU compute here)."""
import ctypes as C
import os
import re

import pytest

from paper_1401_7227_gb300 import asm2
from paper_1401_7227_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return asm2.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "asm2.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(asm2.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_error_strings_and_defaults(lib):
    for st in range(0, 9):
        assert lib.asm_error_string(st)
    assert lib.asm_error_string(99) == b"unknown status"
    o = asm2.Options()
    lib.asm_default_options(C.byref(o))
    assert (o.precision, o.krylov, o.restart, o.local_solver, o.flexible, o.device) == (0, 0, 30, 0, -1, 0)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    h = C.c_void_p()
    o = asm2.Options()
    lib.asm_default_options(C.byref(o))
    o.restart = 0
    assert lib.asm_create(C.byref(h), C.byref(o), None) == 1
    assert lib.asm_create(None, None, None) == 1
    assert lib.asm_set_grid(None, 1, 1, 1) == 1
    assert lib.asm_factor(None) == 1
    assert lib.asm_destroy(None) == 0


def test_sources_compile_for_sm_103a_only():
    src = open(os.path.join(ROOT, "paper_1401_7227_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without libasm2.so the binding raises instead of computing anything."""
    monkeypatch.setattr(asm2, "_lib", None)
    monkeypatch.setattr(lib_build, "LIB", os.path.join(ROOT, "no-such-dir", "libasm2.so"))
    with pytest.raises(RuntimeError, match="missing"):
        asm2.load()


def test_no_device_is_a_cuda_error(lib):
    """Without a usable GPU both constructors return ASM_ERR_CUDA (6); a bad device index where
    devices exist would be ASM_ERR_INVALID_ARG.  Here, with no GPU, only the first case is reachable."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.asm_create(C.byref(h), None, None) == 6 and not h
    s = C.c_void_p()
    assert lib.asm_server_create(C.byref(s), None, None) == 6 and not s
    with pytest.raises(asm2.ASMError) as e:
        asm2.Solver(stream=0)
    assert e.value.status == 6
