"""The variant sweep (analogue of the paper's Figs. 5-9) runs, and its configurations are the ones the
oracle builds for the same method names: one entry per method checked against the oracle."""
import io
from contextlib import redirect_stdout

import pytest

import oracle as O
from paper_1401_7227_gb300 import sweep, synth

pytestmark = pytest.mark.gpu


def test_sweep_entries_match_oracle_iterations():
    buf = io.StringIO()
    with redirect_stdout(buf):
        sweep.main(["--grid", "8", "8", "4", "--K", "2", "--C", "2", "--max-iter", "300"])
    rows = {line.split("|")[1].strip(): line.split("|")[2].strip() for line in buf.getvalue().splitlines()
            if line.startswith("| ") and not line.startswith("| method")}
    assert set(rows) == set(sweep.METHODS)
    s = synth.grid_jacobian(8, 8, 4, 1)
    geo = {
        "near": (O.Geometry(8, 8, 4, 2, 1, 1, ov=0, near_width=2, far_mode=0), O.NO_COARSE),
        "far": (O.Geometry(8, 8, 4, 2, 1, 1, ov=0, near_width=0, far_mode=2, cfar=(2, 2, 2)), O.NO_COARSE),
        "near+far": (O.Geometry(8, 8, 4, 2, 1, 1, ov=0, near_width=2, far_mode=2, cfar=(2, 2, 2)), O.NO_COARSE),
        "two-level": (O.Geometry(8, 8, 4, 2, 1, 1, ov=0, near_width=0, far_mode=0), O.TWO_LEVEL),
        "two-stage": (O.Geometry(8, 8, 4, 2, 1, 1, ov=0, near_width=0, far_mode=0), O.TWO_STAGE),
    }
    for m, (g, coarse) in geo.items():
        pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.DENSE_LU, coarse=coarse,
                       cbox=(2, 2, 2) if coarse else None)
        _, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 300)
        assert oi.converged
        assert rows[m].split()[0] == str(oi.iters), (m, rows[m], oi.iters)


def test_sweep_with_nested_factorisation_matches_oracle():
    """--local nf: the two classical corrections with NF + colsum local solves equal the oracle's
    iteration counts; the methods with lumps are reported as not applicable."""
    buf = io.StringIO()
    with redirect_stdout(buf):
        sweep.main(["--grid", "8", "8", "4", "--K", "2", "--C", "2", "--max-iter", "300", "--local", "nf"])
    rows = {line.split("|")[1].strip(): line.split("|")[2].strip() for line in buf.getvalue().splitlines()
            if line.startswith("| ") and not line.startswith("| method")}
    assert rows["near"] == rows["far"] == rows["near+far"] == "n/a"
    s = synth.grid_jacobian(8, 8, 4, 1)
    g = O.Geometry(8, 8, 4, 2, 1, 1, ov=0, near_width=0, far_mode=0)
    for m, coarse in (("two-level", O.TWO_LEVEL), ("two-stage", O.TWO_STAGE)):
        pc = O.Precond(g, s.row_ptr, s.col_idx, s.vals, solver=O.NF_COLSUM, coarse=coarse, cbox=(2, 2, 2))
        _, oi = O.gmres(s.row_ptr, s.col_idx, s.vals, s.b, pc, 30, 1e-8, 300)
        assert oi.converged
        assert rows[m].split()[0] == str(oi.iters), (m, rows[m], oi.iters)
