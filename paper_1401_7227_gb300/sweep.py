"""Iteration-count sweep of the preconditioner variants the paper compares (Section 5, Figs. 5-9),
on synthetic black-oil Jacobians, through the GPU library.

For each subdomain count K (a 1-D split in x, or a 2-D split in x and y) and coarsening C:
  near       near field only: the fine set plus a ring of lumps (2x2x2 boxes, width 2), nothing
             beyond -- additive Schwarz with coarsened boundary cells
  far        far field only: the fine set plus the far lumps (C x C x C boxes)
  near+far   the paper's method: fine set, near ring and far lumps
  two-level  classical additive Schwarz plus the coarse-grid correction of Eq. 3.5 (C x C x C boxes)
  two-stage  classical additive Schwarz plus the two-stage correction of Eqs. 3.7-3.8
No overlap (as in the paper's comparisons), GMRES(30) to a 1e-8 relative residual, local problems
solved exactly (the paper's setting; --local colsum for block ILU(0) + column sum, --local nf for
nested factorisation with column sums (Appendix A), which needs local problems without lumps and so
serves the two classical corrections only).  "blocks" is the mean local size n_i, the paper's measure
of preconditioner work.

    python -m paper_1401_7227_gb300.sweep --grid 20 20 6 --K 2 4 5 10 --C 2 4 5 [--split x|xy]
"""
from __future__ import annotations

import argparse
import sys

import numpy as np

from . import asm2, synth

METHODS = ("near", "far", "near+far", "two-level", "two-stage")


def split(K: int, mode: str, nx: int, ny: int):
    if mode == "x":
        return K, 1, 1
    px = int(np.floor(np.sqrt(K)))
    while K % px:
        px -= 1
    return K // px, px, 1  # the longer side in x


def run_one(system, g, method: str, K: int, C: int, mode: str, local: str, tol: float, max_iter: int):
    nx, ny, nz = g
    px, py, pz = split(K, mode, nx, ny)
    if local == "nf_colsum" and method in ("near", "far", "near+far"):
        return "n/a", None  # lumps: nested factorisation needs boxes without them
    sol = asm2.Solver(precision="fp64", restart=30, local_solver=local)
    try:
        sol.set_grid(nx, ny, nz)
        sol.set_matrix(system.row_ptr, system.col_idx, system.vals)
        cbox = (C, C, min(C, nz))
        if method == "near":
            sol.set_partition(px, py, pz, 0, 2, (2, 2, 2), "none")
        elif method == "far":
            sol.set_partition(px, py, pz, 0, 0, (2, 2, 2), "boxes", cbox)
        elif method == "near+far":
            sol.set_partition(px, py, pz, 0, 2, (2, 2, 2), "boxes", cbox)
        else:
            sol.set_partition(px, py, pz, 0, 0, (2, 2, 2), "none")
            sol.set_coarse(method, cbox)
        sol.factor()
        st = sol.stats()
        x, info = sol.solve(system.b, rtol=tol, max_iter=max_iter)
        blocks = st["local_rows"] / st["n_sub"]
        return info["iterations"] if info["converged"] else None, blocks
    finally:
        sol.close()


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--grid", type=int, nargs=3, default=[20, 20, 6])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--sigma", type=float, default=1.0)
    ap.add_argument("--K", type=int, nargs="+", default=[2, 4, 5, 10])
    ap.add_argument("--C", type=int, nargs="+", default=[2, 4, 5])
    ap.add_argument("--split", choices=["x", "xy"], default="x")
    ap.add_argument("--local", choices=["exact", "colsum", "nf"], default="exact")
    ap.add_argument("--methods", nargs="+", default=list(METHODS))
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=1000)
    args = ap.parse_args(argv)
    nx, ny, nz = args.grid
    local = "nf_colsum" if args.local == "nf" else args.local
    system = synth.grid_jacobian(nx, ny, nz, args.seed, args.sigma)
    print(f"grid {nx}x{ny}x{nz} ({system.n_cells} cells, seed {args.seed}, sigma {args.sigma}), "
          f"{args.split} split, overlap 0, local solves: {args.local}, GMRES(30) to {args.tol:g}")
    print()
    cols = [(K, C) for K in args.K for C in args.C]
    print("| method | " + " | ".join(f"K={K} C={C}" for K, C in cols) + " |")
    print("|---|" + "---|" * len(cols))
    for m in args.methods:
        cells = []
        for K, C in cols:
            it, blocks = run_one(system, (nx, ny, nz), m, K, C, args.split, local, args.tol, args.max_iter)
            cells.append("n/a" if it == "n/a" else f"{it if it is not None else '—'} ({blocks:.0f})")
        print(f"| {m} | " + " | ".join(cells) + " |")
        sys.stdout.flush()
    print()
    print("entries: GMRES iterations (mean local size n_i in blocks); — = not converged in --max-iter;"
          " n/a = the local solver does not apply to local problems with lumps")
    return 0


if __name__ == "__main__":
    sys.exit(main())
