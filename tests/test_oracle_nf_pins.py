"""Pins of the oracle's nested factorisation (Appendix A, Eqs. A.1-A.7) against dense matrices built
here from the definitions (no GPU).

For a box of bx * by * bz cells (local cell p = z + bz (x + bx y)) the local matrix is
A = D + L1 + U1 + L2 + U2 + L3 + U3 and
  B = (P + L3)(I + P^-1 U3),  P = (T + L2)(I + T^-1 U2),  T = (G + L1)(I + G^-1 U1),
with G block diagonal: G = D - L1 G^-1 U1 (A.6), or with colsum also minus the block column sums of
L2 T^-1 U2 and L3 P^-1 U3 (A.7).  The tests rebuild T, P, B densely from the oracle's G and check
what the appendix states about E = B - A.
"""
import numpy as np
import pytest

import oracle as O
from paper_1401_7227_gb300 import synth

CASES = [  # geometries whose local problems are boxes without lumps
    O.Geometry(5, 4, 3, 1, 1, 1, ov=0, near_width=0, far_mode=0),
    O.Geometry(6, 5, 4, 2, 1, 1, ov=1, near_width=0, far_mode=0),
    O.Geometry(5, 6, 4, 1, 2, 2, ov=1, near_width=0, far_mode=0),
    O.Geometry(5, 4, 1, 2, 1, 1, ov=1, near_width=0, far_mode=0),  # lines of one cell
    O.Geometry(1, 5, 4, 1, 2, 1, ov=1, near_width=0, far_mode=0),  # planes of one line
]


def dense(rp, ci, v):
    n = rp.shape[0] - 1
    a = np.zeros((3 * n, 3 * n))
    for p in range(n):
        for t in range(rp[p], rp[p + 1]):
            a[3 * p:3 * p + 3, 3 * ci[t]:3 * ci[t] + 3] = v[t]
    return a


def bands(a, dims):
    """The seven band matrices of A (dense), by the cell offsets of the box."""
    bx, by, bz = dims
    n = bx * by * bz
    S = bx * bz
    out = {k: np.zeros_like(a) for k in ("D", "L1", "U1", "L2", "U2", "L3", "U3")}
    for p in range(n):
        z, x, y = p % bz, (p // bz) % bx, p // S
        def put(name, q):
            out[name][3 * p:3 * p + 3, 3 * q:3 * q + 3] = a[3 * p:3 * p + 3, 3 * q:3 * q + 3]
        put("D", p)
        if z > 0: put("L1", p - 1)
        if z < bz - 1: put("U1", p + 1)
        if x > 0: put("L2", p - bz)
        if x < bx - 1: put("U2", p + bz)
        if y > 0: put("L3", p - S)
        if y < by - 1: put("U3", p + S)
    assert np.allclose(sum(out.values()), a, rtol=0, atol=0), "A is not hepta-banded on the box"
    return out


def nested(G, bd):
    n3 = G.shape[0] * 3
    Gm = np.zeros((n3, n3))
    for p in range(G.shape[0]):
        Gm[3 * p:3 * p + 3, 3 * p:3 * p + 3] = G[p]
    I = np.eye(n3)
    T = (Gm + bd["L1"]) @ (I + np.linalg.solve(Gm, bd["U1"]))
    P = (T + bd["L2"]) @ (I + np.linalg.solve(T, bd["U2"]))
    B = (P + bd["L3"]) @ (I + np.linalg.solve(P, bd["U3"]))
    return T, P, B


def colsum(M):
    """Block diagonal matrix of the 3x3 block column sums of M."""
    n = M.shape[0] // 3
    out = np.zeros_like(M)
    for j in range(n):
        out[3 * j:3 * j + 3, 3 * j:3 * j + 3] = M[:, 3 * j:3 * j + 3].reshape(n, 3, 3).sum(axis=0)
    return out


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("solver", [O.NF, O.NF_COLSUM])
def test_nf_error_matrix_and_solve(ci, solver):
    g = CASES[ci]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 20 + ci)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=solver)
    for sd in range(g.n_sub):
        dims, G = pc.sub_nf(sd)
        a = dense(*pc.sub_matrix(sd))
        bd = bands(a, dims)
        T, P, B = nested(G, bd)
        M2 = bd["L2"] @ np.linalg.solve(T, bd["U2"])
        M3 = bd["L3"] @ np.linalg.solve(P, bd["U3"])
        E = B - a
        scale = np.abs(a).max()
        if solver == O.NF:      # Eq. A.6: E = L2 T^-1 U2 + L3 P^-1 U3
            want = M2 + M3
        else:                   # Eq. A.7: the same terms with their block column sums removed
            want = M2 - colsum(M2) + M3 - colsum(M3)
            assert np.abs(colsum(E)).max() <= 1e-10 * scale
        np.testing.assert_allclose(E, want, rtol=0, atol=1e-10 * scale)
        r = synth.rhs(pc.sub_n(sd), 5 + sd)
        np.testing.assert_allclose(pc.local_solve(sd, r), np.linalg.solve(B, r), rtol=1e-9,
                                   atol=1e-12 * np.abs(np.linalg.solve(B, r)).max())


def test_nf_on_one_column_is_exact():
    """One vertical line: T is the exact block LU of the tridiagonal A, so B = A."""
    g = O.Geometry(1, 1, 12, 1, 1, 1, ov=0, near_width=0, far_mode=0)
    s = synth.grid_jacobian(1, 1, 12, 3)
    for solver in (O.NF, O.NF_COLSUM):
        pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=solver)
        np.testing.assert_allclose(pc.apply(s.b), np.linalg.solve(s.dense(), s.b), rtol=1e-10, atol=0)


def test_nf_colsum_preserves_residual_sums():
    """1^T (B - A) = 0 per component, so the preconditioned residual r - A B^-1 r sums to zero."""
    g = CASES[1]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 8)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM)
    for sd in range(g.n_sub):
        a = dense(*pc.sub_matrix(sd))
        r = synth.rhs(pc.sub_n(sd), 9)
        res = r - a @ pc.local_solve(sd, r)
        assert np.abs(res.reshape(-1, 3).sum(axis=0)).max() <= 1e-10 * np.abs(r).sum()


def test_nf_needs_local_problems_without_lumps():
    g = O.Geometry(6, 5, 4, 2, 1, 1, ov=1, near_width=2)
    s = synth.grid_jacobian(6, 5, 4, 1)
    with pytest.raises(O.OracleError):
        O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM)
