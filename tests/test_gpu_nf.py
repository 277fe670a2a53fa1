"""Nested factorisation (Appendix A) as the GPU local solver, against the oracle's nested
factorisation on the same seeded systems.

Local problems without lumps (near width 0, no far field): each A_i is hepta-banded on the box of
its fine set.  Both sides compute the diagonal blocks G in the same order (Eq. A.6, or A.7 with the
column sums of L2 T^-1 U2 and L3 P^-1 U3 from row-vector line and plane solves) and apply
B_i^-1 by the same nested sweeps, so they differ by rounding only (the GPU contracts products into
fused multiply-adds): G to 1e-12 of max |G|, each apply to max(1e-12, 100 max_i cond(A_i) eps)."""
import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

GEOMS = {  # geometries whose local problems are boxes without lumps
    "one": (O.Geometry(5, 4, 3, 1, 1, 1, ov=0, near_width=0, far_mode=0), 20),
    "x2": (O.Geometry(6, 5, 4, 2, 1, 1, ov=1, near_width=0, far_mode=0), 21),
    "yz": (O.Geometry(5, 6, 4, 1, 2, 2, ov=1, near_width=0, far_mode=0), 22),
    "ragged": (O.Geometry(9, 7, 6, 3, 2, 2, ov=1, near_width=0, far_mode=0), 23),
    "tiles": (O.Geometry(24, 20, 16, 3, 2, 1, ov=2, near_width=0, far_mode=0), 24),
    "long": (O.Geometry(4, 3, 150, 2, 1, 1, ov=1, near_width=0, far_mode=0), 25),  # lines of 150 cells
    "flat": (O.Geometry(7, 6, 1, 2, 2, 1, ov=1, near_width=0, far_mode=0), 27),   # lines of one cell
    "thin": (O.Geometry(6, 5, 2, 2, 1, 1, ov=1, near_width=0, far_mode=0), 28),   # lines of two cells
}
SOLVERS = {"nf_colsum": O.NF_COLSUM, "nf": O.NF}
EPS = np.finfo(float).eps


def nf_solver(g, s, local="nf_colsum", krylov="gmres", restart=30, precision="fp64"):
    sol = asm2.Solver(precision=precision, local_solver=local, krylov=krylov, restart=restart)
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode)
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


@pytest.mark.parametrize("local", list(SOLVERS))
@pytest.mark.parametrize("name", ["one", "x2", "yz", "ragged"])
def test_diagonal_blocks_match_oracle(name, local):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=SOLVERS[local])
    sol = nf_solver(g, s, local)
    for sd in range(g.n_sub):
        np.testing.assert_array_equal(sol.local_map(sd), pc.sub_map(sd))  # same local rows
        _, G = pc.sub_nf(sd)
        Gg = sol.nf_diagonal(sd)
        assert np.abs(Gg - G).max() <= 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("local", list(SOLVERS))
@pytest.mark.parametrize("name", list(GEOMS))
def test_apply_matches_oracle(name, local):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=SOLVERS[local])
    cond = max(np.linalg.cond(dense(*pc.sub_matrix(k))) for k in range(g.n_sub)) if g.n_cells < 2000 else 1e3
    tol = max(1e-12, 100 * cond * EPS)
    sol = nf_solver(g, s, local)
    for seed_r in (1, 2):
        r = synth.rhs(s.n_cells, seed_r)
        z, zo = sol.apply(r), pc.apply(r)
        assert rel(z, zo) <= tol, (rel(z, zo), tol)
        assert np.abs(z - zo).max() <= tol * np.abs(zo).max()


def test_one_column_is_exact():
    """One vertical line: T is the exact block LU of the block tridiagonal A, so B = A."""
    g = O.Geometry(1, 1, 12, 1, 1, 1, ov=0, near_width=0, far_mode=0)
    s = synth.grid_jacobian(1, 1, 12, 3)
    for local in SOLVERS:
        z = nf_solver(g, s, local).apply(s.b)
        assert rel(z, np.linalg.solve(s.dense(), s.b)) <= 1e-12


@pytest.mark.parametrize("local", list(SOLVERS))
@pytest.mark.parametrize("name", ["x2", "ragged", "tiles"])
def test_gmres_matches_oracle(name, local):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=SOLVERS[local])
    xo, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 500)
    x, info = nf_solver(g, s, local).solve(s.b, rtol=1e-8, max_iter=500)
    assert oi.converged and info["converged"]
    assert info["iterations"] == oi.iters
    assert rel(x, xo) <= 1e-7
    assert rel(O.spmv(s.row_ptr, s.col_idx, s.vals, x), s.b) <= 1e-8


def test_orthomin_matches_oracle():
    g, seed = GEOMS["ragged"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM)
    xo, oi = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, pc, 10, 1e-14, 12)
    x, info = nf_solver(g, s, krylov="orthomin", restart=10).solve(s.b, rtol=1e-14, max_iter=12)
    assert info["iterations"] == oi.iters == 12
    assert rel(x, xo) <= 1e-9


def test_batch_equals_alone_bitwise():
    g, _ = GEOMS["ragged"]
    systems = [synth.grid_jacobian(g.nx, g.ny, g.nz, seed) for seed in (31, 32)]
    alone = []
    for s in systems:
        sol = nf_solver(g, s)
        sol.set_tuning(coop_ortho=False)  # the batch's per-kernel orthogonalisation path
        alone.append(sol.solve(s.b, rtol=1e-8, max_iter=500)[0])
    sols = [nf_solver(g, s) for s in systems]
    xs, infos = asm2.solve_batch(sols, [s.b for s in systems], rtol=1e-8, max_iter=500)
    for x, a, inf in zip(xs, alone, infos):
        assert inf["converged"]
        np.testing.assert_array_equal(x, a)


def test_with_two_level_coarse_correction_matches_oracle():
    g, seed = GEOMS["ragged"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM, coarse=O.TWO_LEVEL)
    sol = asm2.Solver(precision="fp64", local_solver="nf_colsum")
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode)
    sol.set_coarse("two-level")
    sol.factor()
    r = synth.rhs(s.n_cells, 4)
    assert rel(sol.apply(r), pc.apply(r)) <= 1e-11


def test_zero_pivot_location_matches_oracle():
    """A cell whose row and column blocks are all zero has G = 0 (every term of Eqs. A.6-A.7 that
    reaches it carries one of those blocks)."""
    g, seed = GEOMS["one"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    v = s.vals.copy()
    cell = 2 + g.nz * (1 + g.nx * 2)
    for p in range(s.n_cells):
        for t in range(s.row_ptr[p], s.row_ptr[p + 1]):
            if p == cell or s.col_idx[t] == cell:
                v[t] = 0.0
    with pytest.raises(O.OracleError) as eo:
        O.Precond(g, s.row_ptr, s.col_idx, v, solver=O.NF_COLSUM)
    sol = asm2.Solver(precision="fp64", local_solver="nf_colsum")
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, v)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode)
    with pytest.raises(asm2.ASMError) as eg:
        sol.factor()
    assert eg.value.status == 3
    assert eg.value.where == (0, cell) == tuple(eo.value.where)


def test_local_problems_with_lumps_are_rejected():
    g = O.Geometry(6, 5, 4, 2, 1, 1, ov=1, near_width=2)
    s = synth.grid_jacobian(6, 5, 4, 1)
    sol = asm2.Solver(precision="fp64", local_solver="nf_colsum")
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode)
    with pytest.raises(asm2.ASMError) as e:
        sol.factor()
    assert e.value.status == 1


def test_nf_refuses_fp16_storage():
    with pytest.raises(asm2.ASMError):
        asm2.Solver(precision="fp16s", local_solver="nf")


@pytest.mark.parametrize("local", list(SOLVERS))
@pytest.mark.parametrize("name", ["x2", "ragged", "tiles", "long", "flat", "thin"])
def test_fp32_apply_close_to_oracle(name, local):
    """FP32 apply (G from the FP64 factorisation, rounded): within 1e-5 of the FP64 oracle."""
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=SOLVERS[local])
    r = synth.rhs(s.n_cells, 3)
    assert rel(nf_solver(g, s, local, precision="fp32").apply(r), pc.apply(r)) <= 1e-5


@pytest.mark.parametrize("name", ["ragged", "tiles"])
def test_fp32_gmres_reaches_fp64_tolerance(name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM)
    _, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 500)
    x, info = nf_solver(g, s, precision="fp32").solve(s.b, rtol=1e-8, max_iter=500)
    assert info["converged"] and info["iterations"] <= oi.iters + 2
    assert rel(O.spmv(s.row_ptr, s.col_idx, s.vals, x), s.b) <= 1e-8


def test_line_too_long_for_fp64_apply_is_rejected():
    """An FP64 line packet of 250 cells does not fit the apply's two shared-memory slots; FP32 does."""
    g = O.Geometry(2, 2, 250, 1, 1, 1, ov=0, near_width=0, far_mode=0)
    s = synth.grid_jacobian(2, 2, 250, 26)
    with pytest.raises(asm2.ASMError) as e:
        nf_solver(g, s, precision="fp64")
    assert e.value.status == 1
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM)
    assert rel(nf_solver(g, s, precision="fp32").apply(s.b), pc.apply(s.b)) <= 1e-5


def test_update_values_then_factor_equals_fresh_solver():
    """New values on the same pattern (a Newton step): the band tables and packets are rebuilt from
    the re-assembled slots and the apply equals that of a solver built with the new values."""
    g, seed = GEOMS["ragged"]
    s1 = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    s2 = synth.grid_jacobian(g.nx, g.ny, g.nz, seed + 100)
    sol = nf_solver(g, s1)
    sol.update_values(s2.vals)
    sol.factor()
    r = synth.rhs(s2.n_cells, 6)
    np.testing.assert_array_equal(sol.apply(r), nf_solver(g, s2).apply(r))
