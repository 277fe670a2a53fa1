"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerances (relative): local matrices and factors 1e-12 per block row; each preconditioner apply
1e-12 (||dz|| / ||z||); GMRES solution 1e-8.  Integer structure (maps, patterns, level counts,
iteration counts) must be identical.  Mixed precision (factors computed in FP64, then stored):
FP32 applies 1e-5 (unit roundoff 6e-8 times the local triangular solves' amplification); FP16S
applies 5e-3 (unit roundoff 2^-11 = 4.9e-4 of the stored values, same amplification); lump rows
in FP64 or FP32 alike.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

GEOMS = {
    "cfg1": (O.Geometry(10, 10, 5, 2, 2, 1, ov=1), 1),
    "ragged": (O.Geometry(9, 7, 6, 3, 2, 2, ov=1, near_width=1, cnear=(2, 3, 2)), 2),
    "cfar": (O.Geometry(12, 6, 5, 3, 1, 1, ov=2, near_width=2, cnear=(3, 2, 2), far_mode=2, cfar=(4, 3, 5)), 3),
    "nofar": (O.Geometry(8, 8, 4, 2, 2, 1, ov=1, near_width=2, far_mode=0), 4),
    "nonear": (O.Geometry(8, 8, 4, 2, 2, 1, ov=0, near_width=0, far_mode=1), 5),
    "k1": (O.Geometry(6, 5, 4, 1, 1, 1, ov=0, near_width=0), 6),
    "k32": (O.Geometry(16, 16, 8, 4, 4, 2, ov=1), 7),
    "tall": (O.Geometry(5, 4, 40, 1, 2, 3, ov=2, near_width=2, cnear=(2, 2, 4)), 8),
}


MIXED_TOL = {"fp32": 1e-5, "fp16s": 5e-3}


def gpu_solver(g, s, precision="fp64", local_solver="colsum", restart=30, lumps="fp64"):
    sol = asm2.Solver(precision=precision, restart=restart, local_solver=local_solver, lumps=lumps)
    sol.set_grid(g.nx, g.ny, g.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(g.px, g.py, g.pz, g.ov, g.near_width, g.cnear, g.far_mode,
                      g.cfar if g.far_mode == 2 else None)
    sol.factor()
    return sol


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def rowwise_rel(a, b, rp):
    worst = 0.0
    for p in range(rp.shape[0] - 1):
        d = np.linalg.norm(a[rp[p]:rp[p + 1]] - b[rp[p]:rp[p + 1]])
        worst = max(worst, d / max(np.linalg.norm(b[rp[p]:rp[p + 1]]), 1e-300))
    return worst


@pytest.mark.parametrize("name", list(GEOMS))
def test_spmv(name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s)
    y = sol.spmv(s.b)
    assert rel(y, O.spmv(s.row_ptr, s.col_idx, s.vals, s.b)) <= 1e-14
    yd = sol.spmv(torch.from_numpy(s.b).cuda()).cpu().numpy()
    np.testing.assert_array_equal(y, yd)


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("local_solver", ["colsum", "plain"])
def test_local_structure_matrix_factors(name, local_solver):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s, local_solver=local_solver)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.BILU0_COLSUM if local_solver == "colsum" else O.BILU0)
    for sd in range(g.n_sub):
        info = sol.local_info(sd)
        assert info["counts"] == pc.sub_counts(sd)
        np.testing.assert_array_equal(sol.local_map(sd), pc.sub_map(sd))
        rp, ci, v = sol.local_matrix(sd)
        orp, oci, ov = pc.sub_matrix(sd)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        assert rowwise_rel(v.reshape(-1, 9), ov.reshape(-1, 9), rp) <= 1e-12
        lu, dp = sol.local_factors(sd)
        olu, odp = pc.sub_factors(sd)
        assert rowwise_rel(lu.reshape(-1, 9), olu.reshape(-1, 9), rp) <= 1e-12
        assert rowwise_rel(dp.reshape(-1, 9), odp.reshape(-1, 9), np.arange(rp.shape[0])) <= 1e-12


@pytest.mark.parametrize("name", list(GEOMS))
@pytest.mark.parametrize("local_solver", ["colsum", "plain"])
def test_apply(name, local_solver):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s, local_solver=local_solver)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.BILU0_COLSUM if local_solver == "colsum" else O.BILU0)
    rng = np.random.default_rng(seed)
    for r in (s.b, rng.standard_normal(3 * s.n_cells), np.zeros(3 * s.n_cells)):
        z = sol.apply(r)
        zo = pc.apply(r)
        if np.linalg.norm(zo) == 0:
            assert np.linalg.norm(z) == 0
        else:
            assert rel(z, zo) <= 1e-12
    # device buffers give the same bits as host buffers
    zd = sol.apply(torch.from_numpy(s.b).cuda()).cpu().numpy()
    np.testing.assert_array_equal(zd, sol.apply(s.b))


@pytest.mark.parametrize("lumps", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["cfg1", "ragged", "cfar", "k32", "tall"])
def test_apply_mixed_precision_close_to_fp64(name, lumps):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    zo = pc.apply(s.b)
    for prec, tol in MIXED_TOL.items():
        z = gpu_solver(g, s, precision=prec, lumps=lumps).apply(s.b)
        assert rel(z, zo) <= tol, prec


@pytest.mark.parametrize("name", ["cfg1", "ragged", "cfar", "nofar", "k32", "tall"])
def test_gmres_solution(name):
    g, seed = GEOMS[name]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    xo, oinfo = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 2000)
    x, info = sol.solve(s.b, rtol=1e-8, max_iter=2000)
    assert oinfo.converged and info["converged"]
    assert info["iterations"] == oinfo.iters
    assert info["restarts"] == oinfo.restarts
    r = s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, x)
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-8
    assert abs(info["rel_residual"] - oinfo.relres) <= 1e-3 * oinfo.relres + 1e-15
    assert rel(x, xo) <= 1e-8


def test_gmres_restart_short_cycles():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s, restart=5)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    xo, oinfo = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 5, 1e-8, 3000)
    x, info = sol.solve(s.b, rtol=1e-8, max_iter=3000)
    assert info["iterations"] == oinfo.iters and info["restarts"] == oinfo.restarts
    assert rel(x, xo) <= 1e-8


@pytest.mark.parametrize("lumps", ["fp64", "fp32"])
@pytest.mark.parametrize("prec", ["fp32", "fp16s"])
def test_mixed_precision_reaches_fp64_tolerance(prec, lumps):
    g, seed = GEOMS["k32"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s, precision=prec, lumps=lumps)
    x, info = sol.solve(s.b, rtol=1e-8, max_iter=3000)
    r = s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, x)
    assert info["converged"]
    assert np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-8
    xs = np.linalg.solve(s.dense(), s.b) if s.n_cells <= 600 else None
    if xs is not None:
        assert rel(x, xs) <= 1e-4


def test_tridiagonal_one_iteration():
    g = O.Geometry(1, 1, 12, 1, 1, 1, ov=0, near_width=0)
    s = synth.grid_jacobian(1, 1, 12, 3)
    sol = gpu_solver(g, s)
    x, info = sol.solve(s.b, rtol=1e-8, max_iter=10)
    assert info["iterations"] == 1 and info["converged"]
    assert rel(x, np.linalg.solve(s.dense(), s.b)) <= 1e-10


def test_zero_rhs():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s)
    x, info = sol.solve(np.zeros(3 * s.n_cells), rtol=1e-8, max_iter=10)
    assert info["converged"] and info["iterations"] == 0
    assert not np.any(x)


def test_not_converged_status():
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s)
    x, info = sol.solve(s.b, rtol=1e-14, max_iter=3)
    assert info["status"] == 4 and not info["converged"] and info["iterations"] == 3
    xo, oinfo = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, O.Precond(g, s.row_ptr, s.col_idx, s.vals), 30, 1e-14, 3)
    assert rel(x, xo) <= 1e-10


def test_zero_pivot_location_matches_oracle():
    s = synth.grid_jacobian(3, 3, 2, 1)
    v = s.vals.copy()
    for r in range(s.n_cells):
        for e in range(s.row_ptr[r], s.row_ptr[r + 1]):
            if r == 4 or s.col_idx[e] == 4:
                v[e] = 0.0
    g = O.Geometry(3, 3, 2, 1, 1, 1, ov=0, near_width=0)
    with pytest.raises(O.OracleError) as eo:
        O.Precond(g, s.row_ptr, s.col_idx, v)
    sol = asm2.Solver()
    sol.set_grid(3, 3, 2)
    sol.set_matrix(s.row_ptr, s.col_idx, v)
    sol.set_partition(1, 1, 1, 0, 0)
    with pytest.raises(asm2.ASMError) as eg:
        sol.factor()
    assert eg.value.status == 3 and eg.value.where == eo.value.where


def test_pattern_errors_are_rejected():
    s = synth.grid_jacobian(3, 3, 2, 1)
    sol = asm2.Solver()
    sol.set_grid(3, 3, 2)
    rp, ci = s.row_ptr.copy(), s.col_idx.copy()
    # drop the (0, 1) block only: the pattern is no longer structurally symmetric
    keep = np.ones(ci.size, dtype=bool)
    keep[np.nonzero(ci[rp[0]:rp[1]] == 1)[0][0] + rp[0]] = False
    rp2 = rp.copy()
    rp2[1:] -= 1
    with pytest.raises(asm2.ASMError) as e:
        sol.set_matrix(rp2, ci[keep], s.vals[keep])
    assert e.value.status == 2
    bad = ci.copy()
    bad[3] = 10 ** 6
    with pytest.raises(asm2.ASMError) as e:
        sol.set_matrix(rp, bad, s.vals)
    assert e.value.status == 1
    with pytest.raises(asm2.ASMError) as e:
        sol.factor()
    assert e.value.status == 8


def test_update_values_matches_fresh_factorisation():
    g, seed = GEOMS["ragged"]
    s1 = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    s2 = synth.grid_jacobian(g.nx, g.ny, g.nz, seed + 100)
    sol = gpu_solver(g, s1)
    sol.update_values(s2.vals)
    sol.factor()
    fresh = gpu_solver(g, s2)
    np.testing.assert_array_equal(sol.apply(s2.b), fresh.apply(s2.b))
    zo = O.Precond(g, s2.row_ptr, s2.col_idx, s2.vals).apply(s2.b)
    assert rel(sol.apply(s2.b), zo) <= 1e-12


def test_batch_equals_alone_bitwise():
    """A system's arithmetic does not depend on the other systems of a batch (same per-kernel
    orthogonalisation path for the lone solve)."""
    cases = [GEOMS["cfg1"], GEOMS["ragged"], GEOMS["k32"]]
    systems = [synth.grid_jacobian(g.nx, g.ny, g.nz, seed) for g, seed in cases]
    alone = []
    for (g, _), s in zip(cases, systems):
        sol = gpu_solver(g, s)
        sol.set_tuning(coop_ortho=False)
        x, info = sol.solve(s.b, 1e-8, 2000)
        alone.append((x, info))
    solvers = [gpu_solver(g, s) for (g, _), s in zip(cases, systems)]
    xs, infos = asm2.solve_batch(solvers, [s.b for s in systems], 1e-8, 2000)
    for (x, info), xb, ib in zip(alone, xs, infos):
        np.testing.assert_array_equal(x, xb)
        assert info == ib


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_mixing_chunk_capacities_equals_alone(precision):
    """Subdomains whose largest wavefront level needs larger stream chunks (a 40x40x24 grid in 2x2
    boxes) share a batch with subdomains that keep the smallest chunks (10x10x5): every CTA uses its
    own ring-slot size inside the launch's shared memory, and the bits do not change."""
    cases = [GEOMS["cfg1"], (O.Geometry(40, 40, 24, 2, 2, 1, ov=1), 11)]
    systems = [synth.grid_jacobian(g.nx, g.ny, g.nz, seed) for g, seed in cases]
    alone = []
    for (g, _), s in zip(cases, systems):
        sol = gpu_solver(g, s, precision=precision)
        sol.set_tuning(coop_ortho=False)
        alone.append(sol.solve(s.b, 1e-8, 2000))
    solvers = [gpu_solver(g, s, precision=precision) for (g, _), s in zip(cases, systems)]
    xs, infos = asm2.solve_batch(solvers, [s.b for s in systems], 1e-8, 2000)
    for (x, info), xb, ib in zip(alone, xs, infos):
        assert ib["converged"]
        np.testing.assert_array_equal(x, xb)
        assert info == ib


@pytest.mark.parametrize("precision, tol, lumps", [("fp64", 1e-12, "fp64"), ("fp32", 1e-5, "fp64"),
                                                   ("fp32", 1e-5, "fp32"), ("fp16s", 5e-3, "fp32")])
def test_lump_rows_longer_than_the_smallest_chunk(precision, tol, lumps):
    """Far lumps that touch many near lumps (32x32x64 in 4x4 boxes): lump rows of ~130 blocks (~10 KB
    in FP64) need stream chunks above the 8 KB minimum capacity; the apply matches the oracle."""
    g = O.Geometry(32, 32, 64, 4, 4, 1, ov=1)
    s = synth.grid_jacobian(32, 32, 64, 9)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    r = synth.rhs(s.n_cells, 1)
    assert rel(gpu_solver(g, s, precision=precision, lumps=lumps).apply(r), pc.apply(r)) <= tol


def test_configuration_64x64x16_k64():
    w = synth.WORKLOADS["grid64x64x16_k64"]
    s = synth.make(w)
    g = O.Geometry(w.nx, w.ny, w.nz, w.px, w.py, w.pz, ov=w.overlap)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    sol = gpu_solver(g, s)
    assert rel(sol.apply(s.b), pc.apply(s.b)) <= 1e-12
    xo, oinfo = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, w.restart, 1e-8, 2000)
    x, info = sol.solve(s.b, 1e-8, 2000)
    assert info["iterations"] == oinfo.iters
    assert rel(x, xo) <= 1e-8
    s32 = gpu_solver(g, s, precision="fp32")
    x32, i32 = s32.solve(s.b, 1e-8, 2000)
    r = s.b - O.spmv(s.row_ptr, s.col_idx, s.vals, x32)
    assert i32["converged"] and np.linalg.norm(r) / np.linalg.norm(s.b) <= 1e-8


@pytest.mark.parametrize("prec, lumps", [("fp64", "fp64"), ("fp32", "fp64"), ("fp16s", "fp64"), ("fp32", "fp32"),
                                         ("fp16s", "fp32")])
def test_kernel_variants(prec, lumps):
    """Shared-memory vs device-memory local vectors give the same bits; the cooperative and the
    per-projection Gram-Schmidt paths differ only in the order of the reduction sums."""
    g, seed = GEOMS["k32"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    sol = gpu_solver(g, s, precision=prec, lumps=lumps)
    z1 = sol.apply(s.b)
    x1, i1 = sol.solve(s.b, 1e-8, 2000)
    sol.set_tuning(apply_smem=False)
    np.testing.assert_array_equal(z1, sol.apply(s.b))
    x2, i2 = sol.solve(s.b, 1e-8, 2000)
    np.testing.assert_array_equal(x1, x2)
    sol.set_tuning(coop_ortho=False)
    x3, i3 = sol.solve(s.b, 1e-8, 2000)
    assert i1 == i2 and i3["iterations"] == i1["iterations"]
    assert rel(x3, x1) <= 1e-10


@pytest.mark.parametrize("lumps", ["fp64", "fp32"])
@pytest.mark.parametrize("prec", ["fp32", "fp16s"])
def test_device_memory_local_vectors_with_more_lumps_than_fine_rows(prec, lumps):
    """Subdomains of 4 cells with ~60 far lumps each: the device-memory local vectors (lumps in
    FP64 with an FP32 mirror, or in FP32; fine rows at the factor precision) must not spill into
    the next subdomain's; the result equals the shared-memory variant bit for bit."""
    g = O.Geometry(8, 8, 4, 8, 8, 1, ov=0, near_width=2)
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 9)
    pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals)
    assert max(pc.sub_n(k) - pc.sub_counts(k)[0] for k in range(g.n_sub)) > 4 * pc.sub_counts(0)[0]
    sol = gpu_solver(g, s, precision=prec, lumps=lumps)
    z1 = sol.apply(s.b)
    sol.set_tuning(apply_smem=False)
    np.testing.assert_array_equal(z1, sol.apply(s.b))
    assert rel(z1, pc.apply(s.b)) <= MIXED_TOL[prec]


@pytest.mark.parametrize("prec, lumps", [("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "fp32"), ("fp16s", "fp32")])
def test_local_vector_placements_agree(prec, lumps):
    """512 subdomains (more than one wave of the shared-memory variant, so the automatic choice is
    lumps in shared memory): every placement of the apply's local vectors gives the same bits, and
    the FP64 apply matches the oracle."""
    g = O.Geometry(32, 32, 4, 16, 16, 2, ov=1)
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, 12)
    sol = gpu_solver(g, s, precision=prec, lumps=lumps)
    z = sol.apply(s.b)
    for place in ("device", "lumps", "shared", "auto"):
        sol.set_tuning(apply_smem=place)
        np.testing.assert_array_equal(z, sol.apply(s.b))
    assert rel(z, O.Precond(g, s.row_ptr, s.col_idx, s.vals).apply(s.b)) <= MIXED_TOL.get(prec, 1e-12)
    x1, i1 = sol.solve(s.b, 1e-8, 2000)
    sol.set_tuning(apply_smem="device")
    x2, i2 = sol.solve(s.b, 1e-8, 2000)
    assert i1 == i2
    np.testing.assert_array_equal(x1, x2)


def test_graphs_and_online_tuner_leave_results_unchanged():
    """Batched steps replayed as CUDA graphs and the online placement tuner change no bit of any
    result; a handle's second solve (with the tuner's remembered choice) repeats its first."""
    cases = [GEOMS["cfg1"], GEOMS["ragged"], GEOMS["k32"], (O.Geometry(32, 32, 4, 16, 16, 2, ov=1), 12)]
    systems = [synth.grid_jacobian(g.nx, g.ny, g.nz, seed) for g, seed in cases]

    def batch(**tuning):
        solvers = []
        for (g, _), s in zip(cases, systems):
            sol = gpu_solver(g, s, precision="fp32")
            sol.set_tuning(**tuning)
            solvers.append(sol)
        return asm2.solve_batch(solvers, [s.b for s in systems], 1e-8, 2000)

    ref_x, ref_i = batch(graphs=False, autotune=False)
    for tuning in ({"graphs": True, "autotune": False}, {"graphs": False, "autotune": True}, {}):
        xs, infos = batch(**tuning)
        for a, b_ in zip(xs, ref_x):
            np.testing.assert_array_equal(a, b_)
        assert infos == ref_i
    g, seed = cases[3]
    s = systems[3]
    sol = gpu_solver(g, s, precision="fp32")
    x1, i1 = sol.solve(s.b, 1e-8, 2000)
    x2, i2 = sol.solve(s.b, 1e-8, 2000)
    np.testing.assert_array_equal(x1, x2)
    assert i1 == i2


def test_batch_refuses_mixed_lump_precisions():
    """Every system of a batch runs in the same apply launch, so all must store lump rows alike."""
    g, seed = GEOMS["cfg1"]
    s = synth.grid_jacobian(g.nx, g.ny, g.nz, seed)
    a = gpu_solver(g, s, precision="fp32", lumps="fp64")
    b = gpu_solver(g, s, precision="fp32", lumps="fp32")
    with pytest.raises(asm2.ASMError) as e:
        asm2.solve_batch([a, b], [s.b, s.b], 1e-8, 100)
    assert e.value.status == 1
    xs, infos = asm2.solve_batch([b], [s.b], 1e-8, 2000)
    assert infos[0]["converged"]
