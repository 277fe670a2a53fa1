"""Classical Gram-Schmidt in the Arnoldi step (asm_options.ortho = ASM_ORTHO_CGS), a non-default
option next to the modified Gram-Schmidt of Section 2.

It rounds differently from MGS, so it is held to the solution tolerance: every solve reaches the
FP64 1e-8 true residual, its iteration count is within two of MGS's on the same system, and its
solution is within 1e-6 (relative) of the oracle's MGS solution (two iterates with residuals
below 1e-8 may differ by up to cond(A) times that; here they agree far more closely).  Batched solves ignore the
option (they run MGS), so a batch of CGS handles gives the bits of a batch of MGS handles."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

CASES = {
    # geometry, seed, factor precision
    "cfg1_fp64": (O.Geometry(10, 10, 5, 2, 2, 1, ov=1), 1, "fp64"),
    "k16_fp64": (O.Geometry(32, 32, 8, 4, 4, 1, ov=1), 5, "fp64"),
    "cfg2_fp32": (O.Geometry(64, 64, 16, 8, 8, 1, ov=1), 2, "fp32"),
}


def make(g, s, prec, ortho, restart=30):
    sol = asm2.Solver(precision=prec, restart=restart, ortho=ortho)
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov)
    sol.factor()
    return sol


@pytest.mark.parametrize("case", list(CASES))
def test_cgs_reaches_the_tolerance_near_mgs(case):
    g, seed, prec = CASES[case]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    b = torch.from_numpy(s.b).cuda()
    infos, xs = {}, {}
    for ortho in ("mgs", "cgs"):
        sol = make(g, s, prec, ortho)
        x, info = sol.solve(b, 1e-8, 1000)
        xs[ortho], infos[ortho] = x.cpu().numpy(), info
        sol.close()
    r = s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, xs["cgs"])
    assert infos["cgs"]["converged"] and np.linalg.norm(r) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(s.b)
    assert abs(infos["cgs"]["iterations"] - infos["mgs"]["iterations"]) <= 2, infos
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    xo, _ = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 1000)
    err = np.linalg.norm(xs["cgs"] - xo) / np.linalg.norm(xo)
    assert err <= 1e-6
    print(case, "iterations mgs", infos["mgs"]["iterations"], "cgs", infos["cgs"]["iterations"], "error", err)


def test_cgs_restart_62_and_a_short_restart():
    g, seed, prec = CASES["k16_fp64"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    b = torch.from_numpy(s.b).cuda()
    for m in (62, 3):
        sol = make(g, s, prec, "cgs", restart=m)
        x, info = sol.solve(b, 1e-8, 2000)
        assert info["converged"] and info["rel_residual"] <= 1e-8 * (1 + 1e-6), (m, info)
        sol.close()


def test_batches_run_mgs_whatever_the_option():
    g, seed, prec = CASES["cfg1_fp64"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    s2 = synth.grid_jacobian(g.nx, g.ny, g.nz, seed + 10)
    bs = [torch.from_numpy(s.b).cuda(), torch.from_numpy(s2.b).cuda()]
    out = {}
    for ortho in ("mgs", "cgs"):
        sols = [make(g, s, prec, ortho), make(g, s2, prec, ortho)]
        out[ortho] = asm2.solve_batch(sols, bs, 1e-8, 500)
        for x in sols:
            x.close()
    for a, c in zip(out["mgs"][0], out["cgs"][0]):
        assert torch.equal(a, c)
