"""The benchmark's algorithmic byte count of the nested-factorisation apply, checked against an
enumeration of the apply's line solves (no GPU): forward planes j = 0 .. by-1, then backward planes
j = by-2 .. 0; in each plane the forward lines l = 0 .. bx-1, then the backward lines l = bx-2 .. 0.
A forward line reads G^-1, M, N, P, Q and two of L2, L3, U3; a backward line G^-1, M, N, P, Q and U2."""
import bench
from paper_1401_7227_gb300 import synth


def enumerated_bytes(w, elem):
    def spans(n, p, ov):
        out = []
        for t in range(p):
            lo, hi = n * t // p, n * (t + 1) // p
            out.append(min(n, hi + ov) - max(0, lo - ov))
        return out

    total = 24 * w.nx * w.ny * w.nz  # the owned cells of z, once
    for bx in spans(w.nx, w.px, w.overlap):
        for by in spans(w.ny, w.py, w.overlap):
            for bz in spans(w.nz, w.pz, w.overlap):
                field = 9 * elem * bz
                planes = list(range(by)) + list(range(by - 2, -1, -1))
                for _ in planes:
                    for _ in range(bx):
                        total += 7 * field       # forward lines
                    for _ in range(bx - 1):
                        total += 6 * field       # backward lines
                total += 24 * bx * by * bz       # the box's part of r
                total += 2 * 3 * elem * bx * bz * (by - 1)  # y_j out and back, every plane but the last
    return total


def test_nf_apply_bytes_match_the_line_solve_schedule():
    for name in ("grid10x10x5_k4", "grid64x64x16_k64", "grid128x128x64_k512"):
        w = synth.WORKLOADS[name]
        for elem in (4, 8):
            assert bench.nf_apply_bytes(w, elem) == enumerated_bytes(w, elem), (name, elem)
