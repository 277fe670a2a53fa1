"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/asm2.h declares; a
C program links against it; the host-side checks of the library and of the Python binding refuse
bad input before any device work, and nothing falls back to the CPU (no GPU compute here)."""
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
    assert (o.lump_precision, o.ortho) == (1, 0)


def test_invalid_arguments_are_rejected_on_the_host(lib):
    h = C.c_void_p()
    o = asm2.Options()
    lib.asm_default_options(C.byref(o))
    o.restart = 0
    assert lib.asm_create(C.byref(h), C.byref(o), None) == 1
    lib.asm_default_options(C.byref(o))
    o.ortho = 2
    assert lib.asm_create(C.byref(h), C.byref(o), None) == 1
    o.ortho = 1
    o.restart = 63  # classical Gram-Schmidt keeps at most 62 basis vectors
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


class _FakeLib:
    """Records the library calls the binding makes; every call returns ASM_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


def test_binding_refuses_wrong_lengths_before_calling_the_library(monkeypatch):
    """The library reads exactly 3N (vectors) or 9 nnzb (values) doubles from each pointer it gets,
    so the binding checks those counts first: a wrong length raises ValueError with no call made."""
    import numpy as np
    from paper_1401_7227_gb300 import synth
    fake = _FakeLib()
    monkeypatch.setattr(asm2, "_lib", fake)
    s = synth.grid_jacobian(2, 2, 1, 1)     # N = 4, nnzb = 12
    sol = object.__new__(asm2.Solver)
    sol._h, sol.n_cells, sol.nnzb, sol.device, sol.stream = C.c_void_p(1), s.n_cells, s.nnzb, 0, 0
    srv = object.__new__(asm2.Server)
    srv._h, srv._keep, srv._n, srv.stream = C.c_void_p(1), {}, {}, 0
    try:
        bad = [
            lambda: sol.solve(np.zeros(3 * s.n_cells - 1)),
            lambda: sol.apply(np.zeros(3 * s.n_cells + 1)),
            lambda: sol.spmv(np.zeros((3, 3))),
            lambda: sol.update_values(s.vals[:-1]),
            lambda: sol.set_matrix(s.row_ptr, s.col_idx, s.vals[:-1]),
            lambda: asm2.solve_batch([sol, sol], [s.b, s.b[:-1]]),
            lambda: asm2.solve_batch([sol, sol], [s.b]),
            lambda: srv.submit(s, s.b[:-3]),
            lambda: srv.submit(synth.GridSystem(s.nx, s.ny, s.nz, s.row_ptr[:-1], s.col_idx, s.vals, s.b, 1, 1.0),
                               s.b),
        ]
        for f in bad:
            with pytest.raises(ValueError):
                f()
        assert fake.calls == []
        # the right lengths reach the library
        sol.solve(s.b)
        sol.apply(s.b.reshape(-1, 3))
        sol.update_values(s.vals)
        asm2.solve_batch([sol, sol], [s.b, s.b])
        srv.submit(s, s.b)
        assert fake.calls == ["asm_solve", "asm_apply_precond", "asm_update_values", "asm_solve_batch",
                              "asm_server_submit"]
    finally:
        sol._h = None   # never hand the fake handle to the real library
        srv._h = None


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "asm2.h"
int main(void) {
    asm_options o;
    asm_server_options so;
    asm_handle h = 0;
    asm_default_options(&o);
    asm_server_default_options(&so);
    printf("%d %d %d %d %d %d\n", o.precision, o.krylov, o.restart, o.local_solver, o.flexible, o.device);
    printf("%d %d %d\n", so.precision, so.restart, so.max_cached);
    printf("%s|%s\n", asm_error_string(ASM_ERR_ZERO_PIVOT), asm_error_string(99));
    o.restart = 0;
    printf("%d %d\n", asm_create(&h, &o, NULL), h == 0);
    printf("%d %d\n", asm_set_grid(NULL, 1, 1, 1), asm_destroy(NULL));
    return 0;
}
"""


def test_c_program_links_against_the_library(lib, tmp_path):
    """The boundary is a C ABI: a C99 program includes include/asm2.h, links libasm2.so and calls
    the host-only entry points (no GPU needed)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no gcc")
    src, exe = tmp_path / "abi.c", tmp_path / "abi"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(lib_build.LIB)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe),
                    f"-L{libdir}", "-l:libasm2.so", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    assert out[0] == "0 0 30 0 -1 0"
    assert out[1].split()[1] == "30" and out[1].split()[2] == "16"
    zp, unknown = out[2].split("|")
    assert zp == lib.asm_error_string(3).decode() and unknown == "unknown status"
    assert out[3] == "1 1"          # restart 0 is refused on the host, the handle stays NULL
    assert out[4] == "1 0"
