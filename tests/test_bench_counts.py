"""Host logic of the benchmark line (no GPU).

The algorithmic byte count of the nested-factorisation apply is checked against an
enumeration of the apply's line solves (no GPU): forward planes j = 0 .. by-1, then backward planes
j = by-2 .. 0; in each plane the forward lines l = 0 .. bx-1, then the backward lines l = bx-2 .. 0.
A forward line reads G^-1, M, N, P, Q and two of L2, L3, U3; a backward line G^-1, M, N, P, Q and U2.

The clocks summary (median SM clock, maximum, throttle reasons) is checked against sample rows."""
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


def test_clock_summary_reads_throttle_reasons():
    """The clocks object of the bench line: median SM clock under load, the maximum, and every
    throttle reason seen Active in any sample (nvidia-smi csv rows, noheader, nounits)."""
    cs = bench.ClockSampler(0)
    cs.rows = [
        ["0", "2070", "2070", "900.5", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1980", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2032", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["garbage"],
        ["0", "[N/A]", "2070"],
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.rows.append(["0", "1500", "2070", "800", "0x8", "Active", "Not Active", "Active", "Not Active"])
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_ortho_roofline_counts_the_mgs_passes():
    """The Gram-Schmidt roofline's flops: every Arnoldi step j of a GMRES(m) cycle makes j + 2
    passes of 2 FMAs per element (the first pass: (w, v_0) and (w, w); then w -= h v and the next
    dot; the last: w -= h v_j and (w, w)) and one scaling pass, enumerated here pass by pass."""
    class Sys:
        n_cells = 1000

    for iters, m in ((87, 30), (30, 30), (5, 30), (61, 20)):
        n3 = 3.0 * Sys.n_cells
        flops = 0.0
        done = 0
        while done < iters:
            for j in range(min(m, iters - done)):
                passes = [2] + [2] * j + [2]  # FMAs per element of each pass
                flops += sum(2 * f for f in passes) * n3 + n3  # 2 flops per FMA; the scaling: 1 per element
                done += 1
        res = {"info": {"iterations": iters, "restarts": 0}, "prof": {"ortho_ms": 1000.0}}
        line = bench.ortho_roofline(res, Sys, 1, m)
        assert abs(line["achieved"] * 1e12 * 1.0 - flops) <= 1e-9 * flops, (iters, m)
