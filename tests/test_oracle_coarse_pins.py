"""Pins of the oracle's classical coarse-grid corrections (Section 3, Eqs. 3.5-3.8), the comparators
of the paper's Fig. 6, against dense linear algebra written out here (no GPU).

R_C sums each coarse box's cells, R_C^T copies a box value back to its cells, A_C = R_C A R_C^T.
  two-level  (Eq. 3.5): z = B_AS^{-1} r + R_C^T A_C^{-1} R_C r
  two-stage  (Eq. 3.7): z = B_AS^{-1} r + R_C^T A_C^{-1} R_C (r - A B_AS^{-1} r)
"""
import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import synth


def box_of_cells(g, cbox):
    """Coarse box of every cell, from the grid coordinates (independent of the oracle)."""
    box = np.empty(g.n_cells, dtype=np.int64)
    if cbox is None:
        # partition boxes: the owner's subdomain index tz + pz*(tx + px*ty)
        def part(n, p, x):
            return max(t for t in range(p) if (n * t) // p <= x)
        for j in range(g.ny):
            for i in range(g.nx):
                for k in range(g.nz):
                    box[k + g.nz * (i + g.nx * j)] = part(g.nz, g.pz, k) + g.pz * (part(g.nx, g.px, i)
                                                                                + g.px * part(g.ny, g.py, j))
        return box, g.px * g.py * g.pz
    nbx, nby, nbz = [-(-n // c) for n, c in zip((g.nx, g.ny, g.nz), cbox)]
    for j in range(g.ny):
        for i in range(g.nx):
            for k in range(g.nz):
                box[k + g.nz * (i + g.nx * j)] = k // cbox[2] + nbz * (i // cbox[0] + nbx * (j // cbox[1]))
    return box, nbx * nby * nbz


def dense_RC(box, nb):
    N = box.shape[0]
    R = np.zeros((3 * nb, 3 * N))
    for a in range(N):
        for c in range(3):
            R[3 * box[a] + c, 3 * a + c] = 1.0
    return R


CASES = [  # geometry, coarse box size (None: partition boxes)
    (O.Geometry(7, 5, 4, 2, 2, 1, ov=1), (3, 2, 2)),
    (O.Geometry(7, 5, 4, 2, 2, 1, ov=1), None),
    (O.Geometry(6, 6, 6, 2, 1, 2, ov=0, near_width=0, far_mode=0), (2, 2, 2)),
    (O.Geometry(8, 4, 5, 3, 2, 1, ov=1, near_width=1, cnear=(2, 2, 3)), (4, 4, 5)),
]


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_coarse_matrix_is_RC_A_RCt(ci):
    g, cbox = CASES[ci]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 11 + ci)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=O.TWO_LEVEL, cbox=cbox)
    ac, box = pc.coarse_matrix()
    want_box, nb = box_of_cells(g, cbox)
    np.testing.assert_array_equal(box, want_box)
    R = dense_RC(want_box, nb)
    np.testing.assert_allclose(ac, R @ s.dense() @ R.T, rtol=0, atol=1e-12 * np.abs(ac).max())


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("mode", [O.TWO_LEVEL, O.TWO_STAGE])
def test_corrections_equal_their_dense_formulas(ci, mode):
    g, cbox = CASES[ci]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 21 + ci)
    a = s.dense()
    r = s.b
    z_as = O.Precond(g, s.row_ptr, s.col_idx, s.vals).apply(r)
    z = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=mode, cbox=cbox).apply(r)
    box, nb = box_of_cells(g, cbox)
    R = dense_RC(box, nb)
    w = r if mode == O.TWO_LEVEL else r - a @ z_as
    want = z_as + R.T @ np.linalg.solve(R @ a @ R.T, R @ w)
    np.testing.assert_allclose(z, want, rtol=0, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_two_stage_leaves_no_coarse_residual(ci):
    """R_C (r - A z) = 0 after a two-stage apply: the coarse equations hold exactly."""
    g, cbox = CASES[ci]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 31 + ci)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=O.TWO_STAGE, cbox=cbox)
    z = pc.apply(s.b)
    box, nb = box_of_cells(g, cbox)
    res = s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, z)
    rc = np.zeros((nb, 3))
    np.add.at(rc, box, res.reshape(-1, 3))
    assert np.abs(rc).max() <= 1e-9 * np.abs(s.b).sum()


def test_two_stage_with_one_box_per_cell_is_exact():
    """With R_C = I, B_C = A^{-1} and the two-stage preconditioner is A^{-1} (Eq. 3.7)."""
    g = O.Geometry(5, 4, 3, 2, 2, 1, ov=0, near_width=0, far_mode=0)
    s = synth.grid_jacobian(5, 4, 3, 7)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=O.TWO_STAGE, cbox=(1, 1, 1))
    np.testing.assert_allclose(pc.apply(s.b), np.linalg.solve(s.dense(), s.b), rtol=1e-9, atol=0)
    x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 10)
    assert info.iters == 1 and info.converged


def test_two_level_single_box_closed_form():
    """One coarse box over the whole grid: the correction is the same 3-vector in every cell,
    (sum of all blocks of A)^{-1} (sum of r over the cells)."""
    g = O.Geometry(6, 5, 4, 2, 1, 2, ov=1)
    s = synth.grid_jacobian(6, 5, 4, 9)
    z_as = O.Precond(g, s.row_ptr, s.col_idx, s.vals).apply(s.b)
    z = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=O.TWO_LEVEL, cbox=(6, 5, 4)).apply(s.b)
    corr = np.linalg.solve(s.vals.sum(axis=0), s.b.reshape(-1, 3).sum(axis=0))
    np.testing.assert_allclose((z - z_as).reshape(-1, 3), np.broadcast_to(corr, (s.n_cells, 3)),
                               rtol=1e-10, atol=0)


def test_no_coarse_mode_is_the_plain_apply():
    g = O.Geometry(7, 5, 4, 2, 2, 1, ov=1)
    s = synth.grid_jacobian(7, 5, 4, 3)
    a = O.Precond(g, s.row_ptr, s.col_idx, s.vals).apply(s.b)
    b = O.Precond(g, s.row_ptr, s.col_idx, s.vals, coarse=O.NO_COARSE, cbox=(2, 2, 2)).apply(s.b)
    np.testing.assert_array_equal(a, b)
