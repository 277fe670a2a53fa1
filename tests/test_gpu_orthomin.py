"""ORTHOMIN(k) on the GPU (Section 2) against the oracle's ORTHOMIN: same step count, solution within
1e-8 relative, the same true residual; batching leaves each system's arithmetic unchanged.

ORTHOMIN(k) can stagnate where GMRES converges (the oracle's own ORTHOMIN stalls on the "ragged" and
"k32" geometries below for every k up to 40); convergence is tested where the oracle converges, and
the stalled cases are compared after a fixed number of steps."""
import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

GEOMS = {
    "cfg1": (O.Geometry(10, 10, 5, 2, 2, 1, ov=1), 1),
    "ragged": (O.Geometry(9, 7, 6, 3, 2, 2, ov=1, near_width=1, cnear=(2, 3, 2)), 2),
    "cfar": (O.Geometry(12, 6, 5, 3, 1, 1, ov=2, near_width=2, cnear=(3, 2, 2), far_mode=2, cfar=(4, 3, 5)), 3),
    "k32": (O.Geometry(16, 16, 8, 4, 4, 2, ov=1), 7),
    "nofar": (O.Geometry(8, 8, 4, 2, 2, 1, ov=1, near_width=2, far_mode=0), 4),
    "tall": (O.Geometry(5, 4, 40, 1, 2, 3, ov=2, near_width=2, cnear=(2, 2, 4)), 8),
}


def om_solver(g, s, k=10, precision="fp64"):
    sol = asm2.Solver(precision=precision, restart=k, krylov="orthomin")
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode,
                      g.cfar if g.far_mode == 2 else None)
    sol.factor()
    return sol


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def true_rel(s, x):
    return np.linalg.norm(s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, x)) / np.linalg.norm(s.b)


@pytest.mark.parametrize("name,k", [("cfg1", 10), ("cfg1", 1), ("cfar", 5), ("nofar", 20), ("tall", 40)])
def test_orthomin_matches_oracle(name, k):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    xo, oi = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, pc, k, 1e-8, 2000)
    x, info = om_solver(g, s, k).solve(s.b, rtol=1e-8, max_iter=2000)
    assert oi.converged and info["converged"] and info["status"] == 0
    assert info["iterations"] == oi.iters and info["restarts"] == 0
    assert true_rel(s, x) <= 1e-8
    assert abs(info["rel_residual"] - oi.relres) <= 1e-3 * oi.relres + 1e-15
    assert rel(x, xo) <= 1e-8


def test_orthomin_step_limit_matches_oracle():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    xo, oi = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, pc, 3, 1e-14, 7)
    x, info = om_solver(g, s, 3).solve(s.b, rtol=1e-14, max_iter=7)
    assert info["status"] == 4 and not info["converged"] and info["iterations"] == 7 == oi.iters
    assert rel(x, xo) <= 1e-10
    assert abs(info["rel_residual"] - oi.relres) <= 1e-8 * oi.relres


@pytest.mark.parametrize("name,k,steps", [("ragged", 10, 40), ("k32", 5, 25)])
def test_orthomin_stagnating_case_matches_oracle(name, k, steps):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    xo, oi = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, pc, k, 1e-8, steps)
    x, info = om_solver(g, s, k).solve(s.b, rtol=1e-8, max_iter=steps)
    assert not oi.converged and info["status"] == 4 and info["iterations"] == steps == oi.iters
    assert rel(x, xo) <= 1e-8
    assert abs(info["rel_residual"] - oi.relres) <= 1e-8 * oi.relres


def test_orthomin_zero_rhs_and_exact_preconditioner():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    x, info = om_solver(g, s).solve(np.zeros(3 * s.n_cells), rtol=1e-8, max_iter=10)
    assert info["converged"] and info["iterations"] == 0 and not np.any(x)
    # one vertical column, one subdomain: block ILU(0) of a block-tridiagonal matrix is exact
    g1 = O.Geometry(1, 1, 12, 1, 1, 1, ov=0, near_width=0)
    s1 = synth.grid_jacobian(1, 1, 12, 3)
    x, info = om_solver(g1, s1).solve(s1.b, rtol=1e-8, max_iter=10)
    assert info["iterations"] == 1 and info["converged"]
    assert rel(x, np.linalg.solve(s1.dense(), s1.b)) <= 1e-10


@pytest.mark.parametrize("prec", ["fp32", "fp16s"])
def test_orthomin_mixed_precision_reaches_fp64_tolerance(prec):
    g, seed = GEOMS["cfar"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    x, info = om_solver(g, s, 10, prec).solve(s.b, rtol=1e-8, max_iter=3000)
    assert info["converged"] and true_rel(s, x) <= 1e-8


def test_orthomin_batch_equals_alone_bitwise():
    cases = [GEOMS["cfg1"], GEOMS["cfar"], GEOMS["nofar"], GEOMS["tall"]]
    systems = [synth.grid_jacobian(g.nx, g.ny, g.nz, seed) for g, seed in cases]
    ks = [10, 4, 7, 40]
    alone = [om_solver(g, s, k).solve(s.b, 1e-8, 2000) for (g, _), s, k in zip(cases, systems, ks)]
    solvers = [om_solver(g, s, k) for (g, _), s, k in zip(cases, systems, ks)]
    xs, infos = asm2.solve_batch(solvers, [s.b for s in systems], 1e-8, 2000)
    for (x, info), xb, ib in zip(alone, xs, infos):
        np.testing.assert_array_equal(x, xb)
        assert info == ib


def test_batch_rejects_mixed_methods():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    a = om_solver(g, s)
    b = asm2.Solver()
    b.set_grid(g.nx, g.ny, g.nz)
    b.set_matrix(s.row_ptr, s.col_idx, s.vals)
    b.set_partition(g.px, g.py, g.pz, g.ov)
    b.factor()
    with pytest.raises(asm2.ASMError):
        asm2.solve_batch([a, b], [s.b, s.b], 1e-8, 100)
