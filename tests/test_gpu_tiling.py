"""The tiling switches and the tiling tuner (asm_set_tuning ASM_TUNE_CHUNK_KB / ASM_TUNE_APPLY_SLOTS,
asm_tune_tiling), on 40 x 40 x 24 with 2 x 2 x 1 subdomains and overlap 2: local problems of
~11,000 block rows whose widest levels need more than the smallest chunk capacity, so the
capacities 8-24 KB give different chunkings.

- A capacity only regroups rows into chunks: with FP32 fine and lump rows every row computes the
  same bits under every capacity and every ring-slot count, and the tuner's result leaves the
  apply's bits and the solve's iteration count unchanged.
- With FP64 lump rows the entry slots of a lump row are chosen per chunk, so their rounding may
  change: the FP64 apply is checked against the oracle (1e-12) instead.
- The tuner reports every measured configuration, leaves the fastest in place (the handle's stats
  show it), and refuses what it cannot tune."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1401_7227_gb300 import asm2, synth

pytestmark = pytest.mark.gpu

G = O.Geometry(40, 40, 24, 2, 2, 1, ov=2)


@pytest.fixture(scope="module")
def system():
    return synth.grid_jacobian(G.nx, G.ny, G.nz, 5)


def solver(system, prec="fp32", lumps="fp32", local="colsum"):
    sol = asm2.Solver(precision=prec, restart=30, lumps=lumps, local_solver=local)
    sol.set_grid(G.nx, G.ny, G.nz)
    sol.set_matrix(system.row_ptr, system.col_idx, system.vals)
    if local == "colsum":
        sol.set_partition(G.px, G.py, G.pz, G.ov)
    else:
        sol.set_partition(G.px, G.py, G.pz, 1, 0, (2, 2, 2), "none")
    sol.factor()
    return sol


@pytest.fixture(scope="module")
def oracle_z(system):
    return O.Precond(G, system.row_ptr, system.col_idx, system.vals).apply(system.b)


def test_rule_chunks_exceed_the_smallest_capacity(system):
    sol = solver(system)
    st = sol.stats()
    assert st["chunk_max_kb"] > 8 and st["stream_chunks"] > 0
    sol.close()


@pytest.mark.parametrize("kb", [8, 12, 16, 20, 24])
def test_chunk_capacity_keeps_the_bits_of_fp32_rows(system, kb):
    sol = solver(system)
    b = torch.from_numpy(system.b).cuda()
    z0 = sol.apply(b).clone()
    n0 = sol.stats()["stream_chunks"]
    sol.set_tuning(chunk_kb=kb)
    sol.factor()
    st = sol.stats()
    assert st["chunk_max_kb"] == kb
    if kb == 8:
        assert st["stream_chunks"] > n0
    for place in ("auto", "device", "lumps", "shared"):
        sol.set_tuning(apply_smem=place)
        assert torch.equal(sol.apply(b), z0), (kb, place)
    sol.close()


@pytest.mark.parametrize("place", ["shared", "device", "lumps"])
@pytest.mark.parametrize("slots", [2, 3, 4])
def test_ring_slots_keep_the_bits(system, slots, place):
    """With 8 KB chunks all local vectors (186 KB per subdomain here) and 2-4 ring slots fit one
    CTA's shared memory, which 24 KB slots do not allow; the other placements take 2-4 slots too."""
    sol = solver(system)
    b = torch.from_numpy(system.b).cuda()
    z0 = sol.apply(b).clone()
    sol.set_tuning(chunk_kb=8)
    sol.factor()
    sol.set_tuning(apply_smem=place, apply_slots=slots)
    st = sol.stats()
    assert st["apply_placement"] == place and st["apply_slots"] == slots
    assert torch.equal(sol.apply(b), z0)
    sol.close()


@pytest.mark.parametrize("kb", [8, 24])
def test_chunk_capacity_fp64_matches_the_oracle(system, oracle_z, kb):
    sol = solver(system, prec="fp64", lumps="fp64")
    sol.set_tuning(chunk_kb=kb)
    sol.factor()
    z = sol.apply(torch.from_numpy(system.b).cuda()).cpu().numpy()
    assert np.linalg.norm(z - oracle_z) <= 1e-12 * np.linalg.norm(oracle_z)
    sol.close()


def test_tuner_leaves_the_fastest_and_the_same_results(system):
    sol = solver(system)
    b = torch.from_numpy(system.b).cuda()
    z0 = sol.apply(b).clone()
    _, info0 = sol.solve(b, 1e-8, 500)
    rep = sol.tune_tiling(reps=3)
    rows = rep["measured"]
    assert len(rows) >= 4 and rep["rule_ms"] > 0
    assert {r["chunk_kb"] for r in rows} >= {0, 8}
    assert all(r["apply_ms"] > 0 and r["ctas_per_sm"] >= 1 for r in rows)
    best = rep["best"]
    assert best["apply_ms"] == min(r["apply_ms"] for r in rows)
    st = sol.stats()
    assert st["chunk_max_kb"] == best["chunk_max_kb"] and st["stream_chunks"] == best["chunks"]
    assert st["apply_placement"] == best["placement"] and st["apply_slots"] == best["slots"]
    assert torch.equal(sol.apply(b), z0)
    _, info1 = sol.solve(b, 1e-8, 500)
    assert info1["converged"] and info1["iterations"] == info0["iterations"]
    print("tiling:", rep["rule_ms"], best)
    sol.close()


def test_tuner_fp64_stays_within_the_oracle_tolerance(system, oracle_z):
    sol = solver(system, prec="fp64", lumps="fp64")
    sol.tune_tiling(reps=2)
    z = sol.apply(torch.from_numpy(system.b).cuda()).cpu().numpy()
    assert np.linalg.norm(z - oracle_z) <= 1e-12 * np.linalg.norm(oracle_z)
    sol.close()


def test_tuner_and_switch_errors(system):
    sol = asm2.Solver()
    with pytest.raises(asm2.ASMError):
        sol.tune_tiling()  # not factored
    for bad in (4, 10, 28, 32):
        with pytest.raises(asm2.ASMError):
            sol.set_tuning(chunk_kb=bad)
    for bad in (1, 5):
        with pytest.raises(asm2.ASMError):
            sol.set_tuning(apply_slots=bad)
    sol.close()
    sol = solver(system)
    with pytest.raises(asm2.ASMError):
        sol.tune_tiling(reps=0)
    sol.close()
    nf = solver(system, local="nf_colsum")
    with pytest.raises(asm2.ASMError):
        nf.tune_tiling()
    nf.close()


def test_batch_tuner_keeps_every_solution(system):
    """Six systems of different sizes (8 KB to 24 KB rule capacities) solved as one batch: the
    batch tuner's choice gives the bits of the solve before tuning."""
    grids = [(8, 8, 4, 2, 2, 1), (16, 16, 8, 2, 2, 1), (24, 24, 8, 4, 4, 1), (40, 40, 24, 2, 2, 1),
             (12, 20, 6, 2, 3, 1), (32, 32, 16, 4, 4, 1)]
    sols, bs = [], []
    for k, (nx, ny, nz, px, py, pz) in enumerate(grids):
        s = synth.grid_jacobian(nx, ny, nz, 200 + k)
        sol = asm2.Solver(precision="fp32", restart=20, lumps="fp32")
        sol.set_grid(nx, ny, nz)
        sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
        sol.set_partition(px, py, pz, 2 if nx == 40 else 1)
        sol.factor()
        sols.append(sol)
        bs.append(torch.from_numpy(s.b).cuda())
    caps = {s_.stats()["chunk_max_kb"] for s_ in sols}
    assert len(caps) > 1
    x0, i0 = asm2.solve_batch(sols, bs, 1e-8, 500)
    rep = asm2.tune_tiling_batch(sols, bs, 1e-8, 500)
    assert len(rep["measured"]) >= 2 and rep["rule_ms"] > 0
    best = rep["best"]
    assert best["apply_ms"] == min(r["apply_ms"] for r in rep["measured"])
    if best["chunk_kb"] > 0:
        assert all(s_.stats()["chunk_max_kb"] >= best["chunk_kb"] for s_ in sols)
    x1, i1 = asm2.solve_batch(sols, bs, 1e-8, 500)
    for a, b_, u, v in zip(x0, x1, i0, i1):
        assert torch.equal(a, b_) and u["iterations"] == v["iterations"] and v["converged"]
    st = sols[0].stats()
    assert st["last_solve_placement"] in ("device", "lumps", "shared") and st["last_solve_slots"] >= 2
    print("batch tiling:", rep["rule_ms"], best)
    for s_ in sols:
        s_.close()
