"""Failure detection without a GPU fault: a bounded device wait that runs out.

The apply kernels stream the factor chunks (ILU sweeps) or line packets (nested factorisation) into
shared memory with bulk copies and wait on mbarriers with a poll limit.  ASM_TUNE_WAIT_LIMIT = 0
makes the first wait on every copy give up at once: each CTA records ASM_ERR_TIMEOUT in the
device status word, waits with the full bound for its own copies in flight, and returns.  The call
must then report ASM_ERR_TIMEOUT, and after the limit is restored the same handle must give the
bits it gave before and match the oracle again, so the context stayed usable.  Nothing here
faults, traps or hangs the GPU: the limit only shortens a loop that already ends on its own."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

TIMEOUT = 7
CASES = {
    # local solver, factor precision, geometry, oracle solver, apply tolerance against the oracle
    "ilu_fp64": ("colsum", "fp64", O.Geometry(16, 16, 8, 2, 2, 1, ov=1), O.BILU0_COLSUM, 1e-12),
    "ilu_fp32": ("colsum", "fp32", O.Geometry(16, 16, 8, 2, 2, 1, ov=1), O.BILU0_COLSUM, 1e-5),
    "nf_fp64": ("nf_colsum", "fp64", O.Geometry(12, 10, 8, 2, 2, 1, ov=1, near_width=0, far_mode=0), O.NF_COLSUM,
                1e-11),
}


@pytest.mark.parametrize("case", list(CASES))
def test_expired_wait_reports_timeout_and_handle_recovers(case):
    local, prec, g, osolver, tol = CASES[case]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 31)
    sol = asm2.Solver(precision=prec, local_solver=local)
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode)
    sol.factor()
    b = torch.from_numpy(s.b).cuda()
    z0 = sol.apply(b).clone()

    sol.set_tuning(wait_limit_log2=0)
    with pytest.raises(asm2.ASMError) as e:
        sol.apply(b)
    assert e.value.status == TIMEOUT

    sol.set_tuning(wait_limit_log2=22)
    z1 = sol.apply(b)
    assert torch.equal(z0, z1)
    zo = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=osolver).apply(s.b)
    z1 = z1.cpu().numpy()
    assert np.linalg.norm(z1 - zo) <= tol * np.linalg.norm(zo)
    # a solve on the same handle still converges to the FP64 tolerance
    x, info = sol.solve(b, rtol=1e-8, max_iter=500)
    assert info["converged"] and info["rel_residual"] <= 1e-8
    sol.close()


def test_wait_limit_argument_checked():
    sol = asm2.Solver()
    with pytest.raises(asm2.ASMError):
        sol.set_tuning(wait_limit_log2=31)
    sol.close()
