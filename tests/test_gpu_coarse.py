"""Classical coarse-grid corrections on the GPU (Section 3, Eqs. 3.5-3.8) against the oracle: each
apply within 1e-12 relative (FP64), GMRES with the same iteration count and the solution within
1e-8; batching unchanged; bad arguments rejected."""
import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

CASES = [  # geometry, coarse box size (None: partition boxes)
    (O.Geometry(7, 5, 4, 2, 2, 1, ov=1), (3, 2, 2)),
    (O.Geometry(7, 5, 4, 2, 2, 1, ov=1), None),
    (O.Geometry(6, 6, 6, 2, 1, 2, ov=0, near_width=0, far_mode=0), (2, 2, 2)),
    (O.Geometry(8, 4, 5, 3, 2, 1, ov=1, near_width=1, cnear=(2, 2, 3)), (4, 4, 5)),
    (O.Geometry(16, 16, 8, 4, 4, 2, ov=0, near_width=0, far_mode=0), None),
    (O.Geometry(16, 16, 8, 4, 4, 1, ov=1), (4, 4, 4)),
]
MODES = {O.TWO_LEVEL: "two-level", O.TWO_STAGE: "two-stage"}


def solver(g, s, mode, cbox, precision="fp64", krylov="gmres", restart=30):
    sol = asm2.Solver(precision=precision, krylov=krylov, restart=restart)
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode,
                      g.cfar if g.far_mode == 2 else None)
    sol.set_coarse(MODES[mode] if mode else "none", cbox)
    sol.factor()
    return sol


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("mode", [O.TWO_LEVEL, O.TWO_STAGE])
def test_apply_matches_oracle(ci, mode):
    g, cbox = CASES[ci]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 40 + ci)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=mode, cbox=cbox)
    sol = solver(g, s, mode, cbox)
    for seed in (1, 2):
        r = synth.rhs(s.n_cells, seed)
        assert rel(sol.apply(r), pc.apply(r)) <= 1e-12


@pytest.mark.parametrize("ci", [1, 2, 4, 5])
@pytest.mark.parametrize("mode", [O.TWO_LEVEL, O.TWO_STAGE])
def test_gmres_matches_oracle(ci, mode):
    g, cbox = CASES[ci]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 50 + ci)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=mode, cbox=cbox)
    xo, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 2000)
    x, info = solver(g, s, mode, cbox).solve(s.b, rtol=1e-8, max_iter=2000)
    assert oi.converged and info["converged"]
    assert info["iterations"] == oi.iters and info["restarts"] == oi.restarts
    assert rel(x, xo) <= 1e-8


def test_two_stage_with_one_box_per_cell_converges_in_one_iteration():
    g = O.Geometry(5, 4, 3, 2, 2, 1, ov=0, near_width=0, far_mode=0)
    s = synth.grid_jacobian(5, 4, 3, 7)
    x, info = solver(g, s, O.TWO_STAGE, (1, 1, 1)).solve(s.b, rtol=1e-8, max_iter=10)
    assert info["iterations"] == 1 and info["converged"]
    assert rel(x, np.linalg.solve(s.dense(), s.b)) <= 1e-10


def test_mixed_precision_and_orthomin_with_coarse_correction():
    g, cbox = CASES[5]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 60)
    x, info = solver(g, s, O.TWO_STAGE, cbox, precision="fp32").solve(s.b, rtol=1e-8, max_iter=2000)
    r = s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, x)
    assert info["converged"] and np.linalg.norm(r) <= 1e-8 * np.linalg.norm(s.b)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=O.TWO_STAGE, cbox=cbox)
    xo, oi = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, pc, 10, 1e-8, 500)
    x, info = solver(g, s, O.TWO_STAGE, cbox, krylov="orthomin", restart=10).solve(s.b, rtol=1e-8, max_iter=500)
    assert info["iterations"] == oi.iters and info["converged"] == oi.converged
    assert rel(x, xo) <= 1e-8


def test_batch_with_mixed_corrections_equals_alone():
    picks = [(1, O.TWO_LEVEL), (2, O.TWO_STAGE), (4, None), (5, O.TWO_STAGE)]
    systems, alone = [], []
    for ci, mode in picks:
        g, cbox = CASES[ci]
        s = synth.grid_jacobian(g.nx, g.ny, g.nz, 70 + ci)
        systems.append((g, cbox, mode, s))
        sol = solver(g, s, mode, cbox)
        sol.set_tuning(coop_ortho=False)
        alone.append(sol.solve(s.b, 1e-8, 2000))
    solvers = [solver(g, s, mode, cbox) for g, cbox, mode, s in systems]
    xs, infos = asm2.solve_batch(solvers, [s.b for *_, s in systems], 1e-8, 2000)
    for (x, info), xb, ib in zip(alone, xs, infos):
        np.testing.assert_array_equal(x, xb)
        assert info == ib


def test_bad_coarse_arguments():
    g, _ = CASES[4]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 1)
    sol = asm2.Solver()
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    with pytest.raises(asm2.ASMError):
        sol.set_coarse("two-level", None)  # partition boxes before a partition
    sol.set_partition(g.px, g.py, g.pz, g.ov)
    for mode, cb in ((3, None), ("two-level", (0, 1, 1)), ("two-level", (1, 1, 1))):  # last: 2048 boxes
        with pytest.raises(asm2.ASMError):
            sol.set_coarse(mode, cb)
    sol.set_coarse("two-stage", (2, 2, 2))  # 512 boxes
    sol.factor()
    # removing the correction gives back the plain method: same 40 GMRES steps as the oracle's
    sol.set_coarse("none")
    sol.factor()
    x, info = sol.solve(s.b, 1e-8, 40)
    go = O.Geometry(g.nx, g.ny, g.nz, g.px, g.py, g.pz, ov=g.ov)
    xo, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, O.Precond(go, s.row_ptr, s.col_idx, s.vals), 30, 1e-8, 40)
    assert info["iterations"] == oi.iters == 40 and rel(x, xo) <= 1e-8
