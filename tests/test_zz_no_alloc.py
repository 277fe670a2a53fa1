"""The no-allocation residual entry point (asm_residual_noalloc), for callers that cannot allocate
device memory when they need a residual (a pool that forbids further allocations, allocations
fixed after start-up, work about to be captured).  It must give the same residual as the
allocating path (asm_spmv, then b - A x), on consecutive calls that reuse its fixed scratch.

This file is collected last so that, if it fails, a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu


def _noalloc(sol, b, x):
    r = torch.empty_like(b)
    norm = torch.empty(1, dtype=torch.float64, device=b.device)
    st = asm2.load().asm_residual_noalloc(sol.handle, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                          C.c_void_p(r.data_ptr()), C.c_void_p(norm.data_ptr()))
    assert st == 0, asm2.STATUS.get(st, st)
    return r.cpu().numpy(), float(norm.item())


@pytest.mark.parametrize("dims", [(10, 10, 5), (33, 17, 9)])
def test_noalloc_residual_matches_allocating_path_twice(dims):
    s = synth.grid_jacobian(*dims, seed=5)
    sol = asm2.Solver()
    sol.set_grid(*dims)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    rng = np.random.default_rng(11)
    for call in range(2):
        x = rng.standard_normal(3 * s.n_cells)
        ref = s.b - sol.spmv(x)  # existing entry point
        r, norm = _noalloc(sol, torch.from_numpy(s.b).cuda(), torch.from_numpy(x).cuda())
        assert np.linalg.norm(r - ref) <= 1e-14 * np.linalg.norm(ref), call
        assert abs(norm - np.linalg.norm(ref)) <= 1e-12 * np.linalg.norm(ref), call
    sol.close()


def test_noalloc_rejects_missing_matrix():
    sol = asm2.Solver()
    sol.set_grid(2, 2, 2)
    b = torch.zeros(24, dtype=torch.float64, device="cuda")
    st = asm2.load().asm_residual_noalloc(sol.handle, C.c_void_p(b.data_ptr()), C.c_void_p(b.data_ptr()),
                                          C.c_void_p(b.data_ptr()), C.c_void_p(b.data_ptr()))
    assert st == 8
