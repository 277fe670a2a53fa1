"""The synthetic inputs have the properties their recipe states (they stand in for the paper's
matrices, which are not available):

- A conservative finite-volume Jacobian (Section 2: material balance).  Every 3x3 block column sum
  is the cell's diagonal accumulation, plus the well term on the two well columns.
- Upwinding.  Across every face, exactly one of the two cells is upstream, and only the upstream
  neighbour's block carries saturation derivatives.
- Vertical transmissibility about 250 times the horizontal one (the strongest band is vertical,
  Section 2 and Appendix A).
- A pattern that is structurally symmetric, sorted, with a diagonal block in every row.
- A condition number inside the range of the paper's Table 1 on the 10 x 10 x 5 grid.
- Counter-based random draws: any entry regenerates on its own.
"""
import numpy as np
import pytest

from paper_1401_7227_gb300 import synth


@pytest.fixture(scope="module")
def s():
    return synth.grid_jacobian(10, 10, 5, 1)


def coo(s):
    rows = np.repeat(np.arange(s.n_cells), np.diff(s.row_ptr))
    return rows, s.col_idx.astype(np.int64)


def test_pattern_is_a_sorted_symmetric_7_point_stencil(s):
    rows, cols = coo(s)
    for r in range(s.n_cells):
        c = s.col_idx[s.row_ptr[r]:s.row_ptr[r + 1]]
        assert np.all(np.diff(c) > 0) and r in c
    pairs = set(zip(rows.tolist(), cols.tolist()))
    assert all((c, r) in pairs for r, c in pairs)
    # interior cells have all six neighbours
    nx, ny, nz = s.nx, s.ny, s.nz
    inner = 1 + nz * (1 + nx * 1)
    assert s.row_ptr[inner + 1] - s.row_ptr[inner] == 7
    assert s.nnzb == s.n_cells + 2 * ((nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1))


def test_block_column_sums_are_the_accumulation(s):
    """Sum over p of A[p, q] = diag(eps_p, eps_s, eps_s) * U[0.5, 1.5] * (transmissibility sum of q),
    plus WELL * T_NOMINAL * I on the well columns: diagonal and positive, the off-diagonal part zero
    to rounding."""
    rows, cols = coo(s)
    csum = np.zeros((s.n_cells, 3, 3))
    np.add.at(csum, cols, s.vals)
    scale = np.abs(s.vals).max()
    off = csum.copy()
    off[:, [0, 1, 2], [0, 1, 2]] = 0.0
    assert np.abs(off).max() <= 1e-12 * scale
    d = csum[:, [0, 1, 2], [0, 1, 2]]
    assert np.all(d > 0)
    c, i, j, k = synth.cell_coords(s.nx, s.ny, s.nz)
    well = ((i == 0) & (j == 0)) | ((i == s.nx - 1) & (j == s.ny - 1))
    # without the well term what is left is eps * U[0.5, 1.5] * tsum per component, so the ratio of
    # a saturation to the pressure accumulation lies in eps_s / eps_p * [1/3, 3]
    acc = d - np.where(well[:, None], synth.WELL * synth.T_NOMINAL, 0.0)
    assert np.all(acc > 0)
    ratio = acc[:, 1] / acc[:, 0]
    lo, hi = synth.EPS_S / synth.EPS_P / 3.0, synth.EPS_S / synth.EPS_P * 3.0
    assert np.all((ratio >= lo) & (ratio <= hi))


def test_exactly_one_upstream_cell_across_every_face(s):
    """The saturation columns of an off-diagonal block are non-zero only when the neighbour is
    upstream, and across each face exactly one of the two blocks has them."""
    rows, cols = coo(s)
    offd = rows != cols
    sat = np.abs(s.vals[:, 1:, 1:]).sum(axis=(1, 2)) > 0
    up = {(r, c): u for r, c, u in zip(rows[offd].tolist(), cols[offd].tolist(), sat[offd].tolist())}
    for (r, c), u in up.items():
        assert u != up[(c, r)], (r, c)


def test_vertical_transmissibility_dominates(s):
    """T_z / T_x ~ 250: the pressure entry of vertical blocks against horizontal ones."""
    rows, cols = coo(s)
    d = np.abs(cols - rows)
    pz = np.abs(s.vals[d == 1, 0, 0])
    px = np.abs(s.vals[d == s.nz, 0, 0])
    ratio = np.median(pz) / np.median(px)
    assert 100 <= ratio <= 600, ratio


def test_condition_number_in_the_papers_range(s):
    """Table 1 lists condition numbers from 6.7e3 to 2.3e8 for the paper's matrices."""
    cond = np.linalg.cond(s.dense())
    assert 6.7e3 <= cond <= 2.3e8, cond


def test_draws_are_counter_based():
    idx = np.arange(1000)
    u = synth.uniform(7, synth.F_M, idx)
    for t in (0, 17, 999):
        assert synth.uniform(7, synth.F_M, np.array([t]))[0] == u[t]
    assert np.all((u >= 0) & (u < 1))
    assert abs(u.mean() - 0.5) < 0.05
    g = synth.normal(7, synth.F_GCELL, np.arange(20000))
    assert abs(g.mean()) < 0.05 and abs(g.std() - 1.0) < 0.05
    # different seeds and fields give different streams
    assert not np.array_equal(u, synth.uniform(8, synth.F_M, idx))
    assert not np.array_equal(u, synth.uniform(7, synth.F_M + 1, idx))


def test_same_seed_same_system():
    a, b = synth.grid_jacobian(6, 5, 4, 3), synth.grid_jacobian(6, 5, 4, 3)
    assert np.array_equal(a.vals, b.vals) and np.array_equal(a.b, b.b)
    c = synth.grid_jacobian(6, 5, 4, 4)
    assert not np.array_equal(a.vals, c.vals)
