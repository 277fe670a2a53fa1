"""Exact local solves on the GPU (the paper's own setting, Section 5: subdomain problems solved by
Gaussian elimination) against the oracle's dense-LU local solver.

Both sides solve A_i y = R_i r by a backward-stable dense elimination with partial pivoting (the
GPU inverts A_i by Gauss-Jordan, the oracle factors it by LU), so they agree to about
cond(A_i) * eps; each apply is checked against 100 * max_i cond(A_i) * eps (at least 1e-12)."""
import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

GEOMS = {
    "cfg1": (O.Geometry(10, 10, 5, 2, 2, 1, ov=1), 1),
    "ragged": (O.Geometry(9, 7, 6, 3, 2, 2, ov=1, near_width=1, cnear=(2, 3, 2)), 2),
    "cfar": (O.Geometry(12, 6, 5, 3, 1, 1, ov=2, near_width=2, cnear=(3, 2, 2), far_mode=2, cfar=(4, 3, 5)), 3),
    "nofar": (O.Geometry(8, 8, 4, 2, 2, 1, ov=1, near_width=2, far_mode=0), 4),
    "xsplit": (O.Geometry(20, 20, 6, 4, 1, 1, ov=0, near_width=2, cnear=(2, 2, 2)), 5),
}
EPS = np.finfo(float).eps


def exact_solver(g, s):
    sol = asm2.Solver(precision="fp64", local_solver="exact")
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode,
                      g.cfar if g.far_mode == 2 else None)
    sol.factor()
    return sol


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dense(rp, ci, v):
    n = rp.shape[0] - 1
    a = np.zeros((3 * n, 3 * n))
    for p in range(n):
        for t in range(rp[p], rp[p + 1]):
            a[3 * p:3 * p + 3, 3 * ci[t]:3 * ci[t] + 3] = v[t]
    return a


@pytest.mark.parametrize("name", list(GEOMS))
def test_apply_matches_oracle_dense_lu(name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
    cond = max(np.linalg.cond(dense(*pc.sub_matrix(k))) for k in range(g.n_sub))
    tol = max(1e-12, 100 * cond * EPS)
    sol = exact_solver(g, s)
    for seed_r in (1, 2):
        r = synth.rhs(s.n_cells, seed_r)
        assert rel(sol.apply(r), pc.apply(r)) <= tol, (cond, tol)


def test_single_subdomain_converges_in_one_iteration():
    g = O.Geometry(6, 5, 4, 1, 1, 1, ov=0, near_width=0)
    s = synth.grid_jacobian(6, 5, 4, 6)
    x, info = exact_solver(g, s).solve(s.b, rtol=1e-8, max_iter=10)
    assert info["iterations"] == 1 and info["converged"]
    assert rel(x, np.linalg.solve(s.dense(), s.b)) <= 1e-10


@pytest.mark.parametrize("name", ["cfg1", "ragged", "nofar", "xsplit"])
def test_gmres_with_exact_local_solves_matches_oracle(name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
    xo, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 500)
    x, info = exact_solver(g, s).solve(s.b, rtol=1e-8, max_iter=500)
    assert oi.converged and info["converged"]
    assert info["iterations"] == oi.iters
    assert rel(x, xo) <= 1e-8


def test_singular_local_matrix_is_reported():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    vals = s.vals.copy()
    cell = 3  # a cell owned by subdomain 0: zero its block row, so every A_i holding it as a fine row is singular
    vals[s.row_ptr[cell]:s.row_ptr[cell + 1]] = 0.0
    with pytest.raises(O.OracleError):
        O.Precond(g, s.row_ptr, s.col_idx, vals, solver=O.DENSE_LU)
    sol = asm2.Solver(precision="fp64", local_solver="exact")
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov)
    with pytest.raises(asm2.ASMError) as e:
        sol.factor()
    assert e.value.status == 3 and e.value.where[0] == 0


def test_batch_equals_alone_and_mixing_is_rejected():
    names = ["cfg1", "ragged", "nofar"]
    systems = []
    for n in names:
        g, seed = GEOMS[n]
        systems.append((g, synth.grid_jacobian(g.nx, g.ny, g.nz, seed)))
    alone = []
    for g, s in systems:
        sol = exact_solver(g, s)
        sol.set_tuning(coop_ortho=False)
        alone.append(sol.solve(s.b, 1e-8, 500))
    solvers = [exact_solver(g, s) for g, s in systems]
    xs, infos = asm2.solve_batch(solvers, [s.b for _, s in systems], 1e-8, 500)
    for (x, info), xb, ib in zip(alone, xs, infos):
        np.testing.assert_array_equal(x, xb)
        assert info == ib
    g, s = systems[0]
    ilu = asm2.Solver(precision="fp64")
    ilu.set_grid(g.nx, g.ny, g.nz)
    ilu.set_matrix(s.row_ptr, s.col_idx, s.vals)
    ilu.set_partition(g.px, g.py, g.pz, g.ov)
    ilu.factor()
    with pytest.raises(asm2.ASMError):
        asm2.solve_batch([solvers[0], ilu], [s.b, s.b], 1e-8, 10)


def test_exact_needs_fp64():
    with pytest.raises(asm2.ASMError):
        asm2.Solver(precision="fp32", local_solver="exact")
