"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed form, an invariant, a
special case that reduces to a library routine, a brute-force dense computation, or a value the
paper prints (tests/golden).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sysm(nx, ny, nz, seed=1, sigma=1.0):
    return synth.grid_jacobian(nx, ny, nz, seed, sigma)


def dense_local(rp, ci, v):
    n = rp.shape[0] - 1
    a = np.zeros((3 * n, 3 * n))
    for p in range(n):
        for t in range(rp[p], rp[p + 1]):
            q = ci[t]
            a[3 * p:3 * p + 3, 3 * q:3 * q + 3] = v[t]
    return a


def restriction(m, n):
    """Dense R_s (3n x 3N) from a cell -> local map (Eq. 4.1: identity on fine cells, a row of
    ones over each lump)."""
    N = m.shape[0]
    R = np.zeros((3 * n, 3 * N))
    for a in range(N):
        if m[a] >= 0:
            for c in range(3):
                R[3 * m[a] + c, 3 * a + c] = 1.0
    return R


# ---------------------------------------------------------------------------------------------
# 3x3 inverse ("dense sub-matrices inverted directly", Section 2)
# ---------------------------------------------------------------------------------------------
def test_inv3_matches_library_inverse():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a = rng.standard_normal((3, 3))
        np.testing.assert_allclose(O.inv3(a), np.linalg.inv(a), rtol=1e-10, atol=1e-12)
    # a block that needs a row interchange
    a = np.array([[0.0, 1.0, 2.0], [3.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    np.testing.assert_allclose(O.inv3(a) @ a, np.eye(3), atol=1e-14)
    with pytest.raises(ZeroDivisionError):
        O.inv3(np.ones((3, 3)))


# ---------------------------------------------------------------------------------------------
# Geometry of Section 4 (Eq. 4.1, Figs. 2-3)
# ---------------------------------------------------------------------------------------------
def test_counts_match_hand_count():
    rows = np.loadtxt(os.path.join(GOLDEN, "cfg_10x10x5_counts.txt"), dtype=int, comments="#")
    g = O.Geometry(10, 10, 5, 2, 2, 1, ov=1, near_width=2, cnear=(2, 2, 2), far_mode=1)
    for s, nf, nn, nfar in rows:
        _, cnt = O.local_map(g, int(s))
        assert cnt == (nf, nn, nfar)


def test_appendix_b_lumping_matrix():
    """Eq. B.1: on a 1 x 1 x 12 column split in four, subdomain 0 without overlap or near field
    sees the other three parts as lumps of three consecutive cells: exactly the printed E."""
    E = np.loadtxt(os.path.join(GOLDEN, "appendix_b_lumping.txt"), comments="#")
    g = O.Geometry(1, 1, 12, 1, 1, 4, ov=0, near_width=0, far_mode=1)
    m, cnt = O.local_map(g, 0)
    assert cnt == (3, 0, 3)
    lump_of = m[3:] - 3
    Eo = np.zeros((3, 9))
    Eo[lump_of, np.arange(9)] = 1.0
    np.testing.assert_array_equal(Eo, E)


def test_appendix_b_identity_lumped_residuals_sum_to_zero():
    """Appendix B: with A = E a E^T and dX = A^{-1} E r, the lumped new residual E(r - a E^T dX)
    is zero.  Checked for the E of Eq. B.1 on the oracle's lumping of a real local problem."""
    s = sysm(1, 1, 12)
    g = O.Geometry(1, 1, 12, 1, 1, 4, ov=0, near_width=0, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
    m = pc.sub_map(0)
    R = restriction(m, pc.sub_n(0))
    a = s.dense()
    r = s.b
    dX = pc.local_solve(0, R @ r)
    r_new = r - a @ (R.T @ dX)
    assert np.abs(R @ r_new).max() <= 1e-10 * np.abs(r).max()


GEOMS = [
    O.Geometry(10, 10, 5, 2, 2, 1, ov=1, near_width=2, cnear=(2, 2, 2), far_mode=1),
    O.Geometry(9, 7, 6, 3, 2, 2, ov=1, near_width=1, cnear=(2, 3, 2), far_mode=1),
    O.Geometry(12, 6, 5, 3, 1, 1, ov=2, near_width=2, cnear=(3, 2, 2), far_mode=2, cfar=(4, 3, 5)),
    O.Geometry(8, 8, 4, 2, 2, 1, ov=1, near_width=2, cnear=(2, 2, 2), far_mode=0),
    O.Geometry(8, 8, 4, 2, 2, 1, ov=0, near_width=0, far_mode=1),
]


def _coords(g):
    c = np.arange(g.n_cells)
    return c % g.nz, (c // g.nz) % g.nx, c // (g.nz * g.nx)  # k, i, j


def _split(n, p, t):
    return n * t // p


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_geometry_invariants(gi):
    g = GEOMS[gi]
    k, i, j = _coords(g)
    own = O.owner(g)
    assert own.min() == 0 and own.max() == g.n_sub - 1
    for s in range(g.n_sub):
        m, (nf, nn, nfar) = O.local_map(g, s)
        n = nf + nn + nfar
        # local indices are exactly 0..n-1
        used = np.unique(m[m >= 0])
        np.testing.assert_array_equal(used, np.arange(n))
        # every cell is in the local problem unless there is no far field
        if g.far_mode != 0:
            assert (m >= 0).all()
        # fine set = owned box grown by ov and clipped, in ascending global order
        tz, tx, ty = s % g.pz, (s // g.pz) % g.px, s // (g.pz * g.px)
        lo = [max(0, _split(g.nx, g.px, tx) - g.ov), max(0, _split(g.ny, g.py, ty) - g.ov),
              max(0, _split(g.nz, g.pz, tz) - g.ov)]
        hi = [min(g.nx, _split(g.nx, g.px, tx + 1) + g.ov), min(g.ny, _split(g.ny, g.py, ty + 1) + g.ov),
              min(g.nz, _split(g.nz, g.pz, tz + 1) + g.ov)]
        infine = (i >= lo[0]) & (i < hi[0]) & (j >= lo[1]) & (j < hi[1]) & (k >= lo[2]) & (k < hi[2])
        fine_cells = np.nonzero(infine)[0]
        assert nf == fine_cells.size
        np.testing.assert_array_equal(m[fine_cells], np.arange(nf))
        # owned cells are fine cells
        assert (m[own == s] < nf).all() and (m[own == s] >= 0).all()
        # ring = fine set grown by near_width minus fine set
        w = g.near_width
        inouter = ((i >= lo[0] - w) & (i < hi[0] + w) & (j >= lo[1] - w) & (j < hi[1] + w) &
                   (k >= lo[2] - w) & (k < hi[2] + w))
        ring = inouter & ~infine
        if w > 0:
            cx, cy, cz = g.cnear
            nbx, nbz = -(-g.nx // cx), -(-g.nz // cz)
            box = (k // cz) + nbz * ((i // cx) + nbx * (j // cy))
            near_boxes = np.unique(box[ring])
            assert nn == near_boxes.size
            # near lump t is box near_boxes[t] minus the fine set, in box-index order
            for t, b in enumerate(near_boxes):
                cells = np.nonzero((box == b) & ~infine)[0]
                assert (m[cells] == nf + t).all()
                assert (m == nf + t).sum() == cells.size
        else:
            assert nn == 0
        # far lumps: one per far box with cells left, in box order, inside that box
        far = m >= nf + nn
        if g.far_mode == 1:
            fbox = own
        elif g.far_mode == 2:
            fx, fy, fz = g.cfar
            fbox = (k // fz) + (-(-g.nz // fz)) * ((i // fx) + (-(-g.nx // fx)) * (j // fy))
        else:
            assert nfar == 0 and not far.any()
            continue
        boxes = np.unique(fbox[far])
        assert boxes.size == nfar
        for t, b in enumerate(boxes):
            assert (m[far & (fbox == b)] == nf + nn + t).all()
            assert ((m == nf + nn + t) == (far & (fbox == b))).all()


# ---------------------------------------------------------------------------------------------
# Local matrices A_s = R_s A R_s^T (Eq. 3.4 with the R_s of Eq. 4.1; Eq. B.3)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("gi", [0, 1, 2, 3])
def test_local_matrix_is_RART(gi):
    g = GEOMS[gi]
    s = sysm(g.nx, g.ny, g.nz, seed=7)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.BILU0)
    a = s.dense()
    for sd in range(g.n_sub):
        n = pc.sub_n(sd)
        R = restriction(pc.sub_map(sd), n)
        ref = R @ a @ R.T
        got = dense_local(*pc.sub_matrix(sd))
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(a).max())
        # the pattern holds exactly the blocks that receive a coupling
        rp, ci, v = pc.sub_matrix(sd)
        assert rp[-1] == ci.size


# ---------------------------------------------------------------------------------------------
# Block ILU(0) with column-sum compensation (Section 2, Eq. A.7 analogue)
# ---------------------------------------------------------------------------------------------
def factors_dense(pc, sd):
    rp, ci, _ = pc.sub_matrix(sd)
    lu, dp = pc.sub_factors(sd)
    n = rp.shape[0] - 1
    L = np.eye(3 * n)
    U = np.zeros((3 * n, 3 * n))
    for p in range(n):
        for t in range(rp[p], rp[p + 1]):
            q = ci[t]
            if q < p:
                L[3 * p:3 * p + 3, 3 * q:3 * q + 3] = lu[t]
            elif q > p:
                U[3 * p:3 * p + 3, 3 * q:3 * q + 3] = lu[t]
            else:
                U[3 * p:3 * p + 3, 3 * p:3 * p + 3] = dp[p]
                np.testing.assert_allclose(lu[t] @ dp[p], np.eye(3), atol=1e-9)
    return L, U


def pattern_mask(rp, ci):
    n = rp.shape[0] - 1
    P = np.zeros((n, n), dtype=bool)
    for p in range(n):
        P[p, ci[rp[p]:rp[p + 1]]] = True
    return P


@pytest.mark.parametrize("gi", [0, 1, 2])
def test_P2_colsum_error_matrix(gi):
    """E = LU - A_s is zero on the off-diagonal pattern and has zero 3x3 block column sums; with
    plain ILU(0) E is zero on the whole pattern instead.  Together these fix the factors."""
    g = GEOMS[gi]
    s = sysm(g.nx, g.ny, g.nz, seed=3)
    for solver in (O.BILU0_COLSUM, O.BILU0):
        pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=solver)
        for sd in range(g.n_sub):
            rp, ci, v = pc.sub_matrix(sd)
            A = dense_local(rp, ci, v)
            L, U = factors_dense(pc, sd)
            E = L @ U - A
            n = rp.shape[0] - 1
            Eb = E.reshape(n, 3, n, 3).transpose(0, 2, 1, 3)
            P = pattern_mask(rp, ci)
            scale = np.abs(A).max()
            off = P & ~np.eye(n, dtype=bool)
            assert np.abs(Eb[off]).max() <= 1e-11 * scale
            if solver == O.BILU0_COLSUM:
                colsum = Eb.sum(axis=0)  # [q, 3, 3]
                assert np.abs(colsum).max() <= 1e-11 * scale
            else:
                assert np.abs(Eb[np.eye(n, dtype=bool)]).max() <= 1e-11 * scale
    # the compensation actually did something on a lumped problem (triangles create fill)
    pc0 = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.BILU0_COLSUM)
    pc1 = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.BILU0)
    assert np.abs(pc0.sub_factors(0)[1] - pc1.sub_factors(0)[1]).max() > 0


def test_P1_closed_form_on_triangle_free_graph():
    """K = 1 without lumps: the local graph is the 7-point grid (no triangles), so no in-pattern
    update exists and D_q = A_qq - sum_{k<q adj} (sum_{p>k adj k} A_pk) D_k^{-1} A_kq."""
    s = sysm(4, 3, 5, seed=11)
    g = O.Geometry(4, 3, 5, 1, 1, 1, ov=0, near_width=0, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    _, dp = pc.sub_factors(0)
    A = {}
    for r in range(s.n_cells):
        for e in range(s.row_ptr[r], s.row_ptr[r + 1]):
            A[(r, int(s.col_idx[e]))] = s.vals[e]
    adj = {r: [int(c) for c in s.col_idx[s.row_ptr[r]:s.row_ptr[r + 1]] if c != r] for r in range(s.n_cells)}
    D = {}
    for q in range(s.n_cells):
        d = A[(q, q)].copy()
        for k in adj[q]:
            if k < q:
                colsum_k = sum(A[(p, k)] for p in adj[k] if p > k)
                d -= colsum_k @ np.linalg.inv(D[k]) @ A[(k, q)]
        D[q] = d
        np.testing.assert_allclose(dp[q], d, rtol=1e-10, atol=1e-10 * np.abs(d).max())


def test_P3_tridiagonal_is_exact_lu():
    s = sysm(1, 1, 9, seed=5)
    g = O.Geometry(1, 1, 9, 1, 1, 1, ov=0, near_width=0, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    L, U = factors_dense(pc, 0)
    np.testing.assert_allclose(L @ U, s.dense(), atol=1e-10 * np.abs(s.vals).max())
    x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 50)
    assert info.iters == 1 and info.converged


def test_P4_single_subdomain_is_global_bilu0():
    s = sysm(5, 4, 3, seed=9)
    g = O.Geometry(5, 4, 3, 1, 1, 1, ov=1, near_width=2, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    m, cnt = O.local_map(g, 0)
    assert cnt == (s.n_cells, 0, 0)
    np.testing.assert_array_equal(m, np.arange(s.n_cells))
    rp, ci, v = pc.sub_matrix(0)
    np.testing.assert_array_equal(rp, s.row_ptr)
    np.testing.assert_array_equal(ci, s.col_idx)
    np.testing.assert_array_equal(v, s.vals)
    # apply == one global ILU solve: L U z = r
    L, U = factors_dense(pc, 0)
    z = pc.apply(s.b)
    np.testing.assert_allclose(L @ (U @ z), s.b, rtol=0, atol=1e-9 * np.abs(s.b).max())


def test_P5_exact_local_solve_single_subdomain_one_iteration():
    s = sysm(4, 4, 3, seed=2)
    g = O.Geometry(4, 4, 3, 1, 1, 1, ov=0, near_width=0, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
    np.testing.assert_allclose(s.dense() @ pc.apply(s.b), s.b, atol=1e-9)
    x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 10)
    assert info.iters == 1 and info.converged


@pytest.mark.parametrize("gi", [0, 1, 2, 3])
def test_P6_lumped_residuals_vanish_with_exact_local_solves(gi):
    """Appendix B applied to every local problem: R_s (r - A R_s^T A_s^{-1} R_s r) = 0."""
    g = GEOMS[gi]
    s = sysm(g.nx, g.ny, g.nz, seed=4)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
    a = s.dense()
    r = s.b
    for sd in range(g.n_sub):
        R = restriction(pc.sub_map(sd), pc.sub_n(sd))
        rr = r - a @ (R.T @ pc.local_solve(sd, R @ r))
        assert np.abs(R @ rr).max() <= 1e-9 * np.abs(R @ r).max()


@pytest.mark.parametrize("gi", [0, 1, 3])
def test_apply_is_restricted_additive_schwarz(gi):
    """Eqs. 4.2-4.3 with exact local solves, written with dense matrices:
    B^{-1} = sum_s P_s R_s^T A_s^{-1} R_s, P_s = diag(owned by s)."""
    g = GEOMS[gi]
    s = sysm(g.nx, g.ny, g.nz, seed=6)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
    a = s.dense()
    own = np.repeat(O.owner(g), 3)
    z = np.zeros(3 * s.n_cells)
    for sd in range(g.n_sub):
        R = restriction(pc.sub_map(sd), pc.sub_n(sd))
        As = R @ a @ R.T
        z += np.where(own == sd, R.T @ np.linalg.solve(As, R @ s.b), 0.0)
    np.testing.assert_allclose(pc.apply(s.b), z, rtol=1e-9, atol=1e-9 * np.abs(z).max())


def test_colsum_zero_residual_sum_per_component():
    """Section 2: with the column-sum choice the residual after a preconditioning step sums to
    zero, per component (zero material-balance error).  Plain ILU(0) does not have it."""
    s = sysm(6, 5, 4, seed=8)
    g = O.Geometry(6, 5, 4, 1, 1, 1, ov=0, near_width=0, far_mode=1)
    a = s.dense()
    for solver, zero in ((O.BILU0_COLSUM, True), (O.BILU0, False)):
        pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=solver)
        r = s.b
        rn = r - a @ pc.apply(r)
        sums = rn.reshape(-1, 3).sum(axis=0)
        if zero:
            assert np.abs(sums).max() <= 1e-9 * np.abs(r).sum()
        else:
            assert np.abs(sums).max() > 1e-6 * np.abs(r).sum()


def test_singular_pivot_reported():
    s = sysm(3, 3, 2, seed=1)
    v = s.vals.copy()
    diag_pos = [e for r in range(s.n_cells) for e in range(s.row_ptr[r], s.row_ptr[r + 1])
                if s.col_idx[e] == r]
    v[diag_pos[4]] = 0.0
    # cut row 4's couplings so that its pivot stays exactly zero
    for e in range(s.row_ptr[4], s.row_ptr[5]):
        v[e] = 0.0
    for r in range(s.n_cells):
        for e in range(s.row_ptr[r], s.row_ptr[r + 1]):
            if s.col_idx[e] == 4:
                v[e] = 0.0
    g = O.Geometry(3, 3, 2, 1, 1, 1, ov=0, near_width=0, far_mode=1)
    with pytest.raises(O.OracleError) as ei:
        O.Precond(g, s.row_ptr, s.col_idx, v)
    assert ei.value.status == O.ERR_PIVOT and ei.value.where == (0, 4)


# ---------------------------------------------------------------------------------------------
# Krylov accelerators (Section 2)
# ---------------------------------------------------------------------------------------------
def krylov_min_residual(a, b, j):
    K = np.zeros((b.size, j))
    v = b.copy()
    for t in range(j):
        K[:, t] = v
        v = a @ v
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(a @ Q, b, rcond=None)
    return np.linalg.norm(b - a @ Q @ y)


def test_gmres_minimises_residual_over_krylov_space():
    s = sysm(3, 2, 2, seed=12)
    a = s.dense()
    for j in (1, 2, 4, 7):
        x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, None, 30, 1e-30, j)
        assert info.iters == j
        ref = krylov_min_residual(a, s.b, j)
        np.testing.assert_allclose(np.linalg.norm(s.b - a @ x), ref, rtol=1e-6)
        np.testing.assert_allclose(info.history[-1] * np.linalg.norm(s.b), ref, rtol=1e-6)


def test_right_preconditioned_gmres_minimises_over_preconditioned_space():
    s = sysm(3, 3, 2, seed=13)
    a = s.dense()
    g = O.Geometry(3, 3, 2, 1, 1, 1, ov=0, near_width=0, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    Binv = np.stack([pc.apply(e) for e in np.eye(a.shape[0])], axis=1)
    for j in (1, 3, 5):
        x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-30, j)
        ref = krylov_min_residual(a @ Binv, s.b, j)
        np.testing.assert_allclose(np.linalg.norm(s.b - a @ x), ref, rtol=1e-6)


def test_gmres_restart_and_solution():
    """P7: solution against a dense solve, with restarts (m = 5)."""
    s = sysm(4, 4, 3, seed=14)
    a = s.dense()
    xs = np.linalg.solve(a, s.b)
    g = O.Geometry(4, 4, 3, 2, 2, 1, ov=1, near_width=1, far_mode=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 5, 1e-10, 500)
    assert info.converged and info.restarts > 1
    assert np.linalg.norm(s.b - a @ x) <= 1e-10 * np.linalg.norm(s.b) * 1.0001
    cond = np.linalg.cond(a)
    assert np.linalg.norm(x - xs) <= cond * 1e-10 * np.linalg.norm(xs)
    assert np.all(np.diff(info.history) <= 1e-12)  # |g| never grows within a cycle


def test_orthomin_matches_gmres_residual_while_directions_are_kept():
    """ORTHOMIN(k) with all directions kept is GCR, which minimises the residual over the same
    Krylov space as GMRES (exact arithmetic)."""
    s = sysm(3, 2, 2, seed=15)
    a = s.dense()
    for j in (1, 3, 6):
        x, info = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, None, 10, 1e-30, j)
        assert info.iters == j
        np.testing.assert_allclose(np.linalg.norm(s.b - a @ x), krylov_min_residual(a, s.b, j), rtol=1e-6)


def test_orthomin_converges_with_the_preconditioner():
    s = sysm(6, 6, 4, seed=16)
    g = O.Geometry(6, 6, 4, 2, 2, 1, ov=1)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    x, info = O.orthomin(s.row_ptr, s.col_idx, s.vals, s.b, pc, 20, 1e-8, 400)
    assert info.converged and info.relres <= 1e-8


def test_spmv_matches_dense():
    s = sysm(4, 3, 3, seed=17)
    np.testing.assert_allclose(O.spmv(s.row_ptr, s.col_idx, s.vals, s.b), s.dense() @ s.b, rtol=1e-12,
                               atol=1e-12 * np.abs(s.vals).max())


def test_configuration_10x10x5_converges():
    w = synth.WORKLOADS["grid10x10x5_k4"]
    s = synth.make(w)
    g = O.Geometry(w.nx, w.ny, w.nz, w.px, w.py, w.pz, ov=w.overlap)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    x, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, w.restart, 1e-8, 1000)
    assert info.converged and info.relres <= 1e-8
    xs = np.linalg.solve(s.dense(), s.b)
    assert np.linalg.norm(x - xs) <= 1e-4 * np.linalg.norm(xs)


@pytest.mark.parametrize("nx,ny,nz,K,C", [(10, 10, 5, 2, 2), (10, 10, 5, 5, 2), (10, 10, 5, 5, 4), (12, 12, 4, 4, 3),
                                          (16, 16, 4, 4, 4), (16, 16, 4, 8, 4)])
def test_P8_near_and_far_together_need_no_more_iterations(nx, ny, nz, K, C):
    """Section 5 (Figs. 5-8): with exact local solves and no overlap, the near field and the far
    field together take no more GMRES iterations than either one alone.  K subdomains split in x;
    near ring of 2x2x2 lumps, width 2; far lumps of C x C x min(C, nz) cells.  A qualitative check
    of the lump construction, not an exact value."""
    s = synth.grid_jacobian(nx, ny, nz, 1)
    cb = (C, C, min(C, nz))

    def iters(near_width, far_mode):
        g = O.Geometry(nx, ny, nz, K, 1, 1, ov=0, near_width=near_width, cnear=(2, 2, 2), far_mode=far_mode,
                       cfar=cb if far_mode == 2 else (0, 0, 0))
        pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU)
        _, info = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 300)
        assert info.converged
        return info.iters

    near, far, both = iters(2, 0), iters(0, 2), iters(2, 2)
    assert both <= min(near, far), (near, far, both)


@pytest.mark.parametrize("g", [
    O.Geometry(4, 4, 2, 5, 1, 1),                                   # more boxes than cells in x
    O.Geometry(4, 4, 2, 1, 1, 1, ov=-1),
    O.Geometry(4, 4, 2, 1, 1, 1, near_width=2, cnear=(0, 2, 2)),
    O.Geometry(4, 4, 2, 1, 1, 1, far_mode=2, cfar=(0, 1, 1)),
    O.Geometry(4, 4, 2, 1, 1, 1, far_mode=3),
    O.Geometry(0, 4, 2),
])
def test_invalid_geometry_is_refused(g):
    """Section 4's geometry needs 1 <= p <= n per axis, ov >= 0, near and far boxes of >= 1 cell:
    the oracle refuses anything else instead of building from it."""
    s = synth.grid_jacobian(4, 4, 2, 1)
    with pytest.raises(ValueError):
        O.local_map(g, 0)
    with pytest.raises(O.OracleError):
        O.Precond(g, s.row_ptr, s.col_idx, s.vals)
