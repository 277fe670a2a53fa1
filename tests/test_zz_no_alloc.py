"""The no-allocation residual entry point (asm_residual_noalloc), for callers that cannot allocate
device memory when they need a residual (a memory pool that forbids further allocations, or
allocations fixed after start-up).  It must give the same residual as the allocating path
(asm_spmv, then b - A x) on consecutive calls that reuse its fixed scratch, and the device's free
memory must not move across its calls: asm_create already loaded its kernel and scratch array.

This file is collected last so that, if it fails, a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

INVALID_ARG, STATE = 1, 8


def _call(sol, b, x, r, norm):
    return asm2.load().asm_residual_noalloc(sol.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                            C.c_void_p(r.data_ptr()), C.c_void_p(norm.data_ptr()))


@pytest.mark.parametrize("dims", [(10, 10, 5), (33, 17, 9)])
def test_noalloc_residual_matches_allocating_path_twice(dims):
    s = synth.grid_jacobian(*dims, seed=5)
    sol = asm2.Solver()
    sol.set_grid(*dims)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    rng = np.random.default_rng(11)
    xs = [rng.standard_normal(3 * s.n_cells) for _ in range(2)]
    refs = [s.b - sol.spmv(x) for x in xs]  # the existing entry point
    # every buffer of both calls exists before the first call, so that free memory can be compared
    b = torch.from_numpy(s.b).cuda()
    xd = [torch.from_numpy(x).cuda() for x in xs]
    rd = [torch.empty_like(b) for _ in xs]
    nd = [torch.empty(1, dtype=torch.float64, device="cuda") for _ in xs]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        st = _call(sol, b, xd[call], rd[call], nd[call])
        assert st == 0, asm2.STATUS.get(st, st)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, f"device free memory moved by {free0 - free1} bytes across the calls"
    for call in range(2):
        r = rd[call].cpu().numpy()
        ref = refs[call]
        assert np.linalg.norm(r - ref) <= 1e-14 * np.linalg.norm(ref), call
        assert abs(nd[call].item() - np.linalg.norm(ref)) <= 1e-12 * np.linalg.norm(ref), call
    sol.close()


def test_noalloc_rejects_missing_matrix_and_overlap():
    sol = asm2.Solver()
    sol.set_grid(2, 2, 2)
    b = torch.zeros(24, dtype=torch.float64, device="cuda")
    n = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(sol, b, b, b, n) == STATE
    s = synth.grid_jacobian(2, 2, 2, seed=5)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    x = torch.ones(48, dtype=torch.float64, device="cuda")
    assert _call(sol, b, x[:24], x[:24], n) == INVALID_ARG      # r is x
    assert _call(sol, b, x[:24], x[12:36], n) == INVALID_ARG    # r overlaps x
    r = torch.empty(24, dtype=torch.float64, device="cuda")
    assert _call(sol, b, x[:24], r, n) == 0
    sol.close()
