"""Benchmark: time to solve the 1M-cell (128 x 128 x 64, 3 unknowns per cell) system to a 1e-8
FP64 true relative residual with two-level additive Schwarz + block ILU(0)/colsum GMRES(30), on
one GB300, FP32-stored factors (the mixed-precision path) with the FP64 path measured beside it.

A step = one whole pass of the hot path on the resident system: new matrix values in (device),
local matrices re-assembled and re-factored, GMRES to 1e-8.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--precision fp32]
  python bench.py --impl reference ...     # the CPU oracle, timed on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1401_7227_gb300 import synth  # noqa: E402

METRIC = "1M-cell solve time to 1e-8 rel. residual, FP32-prec vs FP64; served p50/p99 latency"
UNIT = "ms/solve"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        gid = vis.split(",")[self.index] if vis else str(self.index)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gid}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """The largest value of x over the ranks (the job's time is its slowest replica's)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# CPU oracle: measured in full on the small workloads, estimated from a bounded sample on the
# 1M-cell one
# ---------------------------------------------------------------------------------------------
# GMRES(30) iterations to 1e-8 of each workload (FP64 path; the oracle takes the same count at the
# two smaller sizes): the reference arm extrapolates its sample to this many iterations
ITERS_MEASURED = {"grid10x10x5_k4": 26, "grid64x64x16_k64": 38, "grid128x128x64_k512": 87}

# readings of the generator that differ from the workload text, stated in every line's config
GENERATOR = {"diagonal": "accumulation minus the COLUMN sum of the off-diagonal blocks (conservative form)",
             "eps_p": synth.EPS_P, "eps_s": synth.EPS_S,
             "wells": f"{synth.WELL} x T_nominal x I3 on every layer of columns (0,0) and (nx-1,ny-1)",
             "sigma": f"scales the layer term of ln k; the cell term is fixed at {synth.CELL_NOISE}"}


def cpu_info():
    """(CPU model, logical cores) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return model or "unknown", os.cpu_count()


def cycles(iters: int, m: int):
    """Lengths of the GMRES(m) cycles of a solve of `iters` iterations."""
    out = [m] * (iters // m)
    if iters % m:
        out.append(iters % m)
    return out or [0]


def krylov_model(w, system, points=(1, 2, 6)):
    """Oracle GMRES(m) time without a preconditioner, T(n) = c + a n + b n (n + 1) / 2 for n
    iterations of one cycle (c: setup and true residual, a: SpMV and the rest of an iteration,
    b: one Gram-Schmidt projection), fitted to runs of `points` iterations.  Returns (c, a, b)
    and the seconds spent."""
    import oracle as O
    t0 = time.perf_counter()
    T = []
    for n in points:
        t1 = time.perf_counter()
        O.gmres(system.row_ptr, system.col_idx, system.vals, system.b, None, w.restart, 1e-30, n)
        T.append(time.perf_counter() - t1)
    M = np.array([[1.0, n, n * (n + 1) / 2] for n in points])
    c, a, b = np.linalg.lstsq(M, np.array(T), rcond=None)[0]
    return (float(c), float(a), max(0.0, float(b))), time.perf_counter() - t0


def subdomain_sample(w, system, subs):
    """Oracle setup (local problem + factorisation) and one apply of each subdomain in `subs`."""
    import oracle as O
    g = O.Geometry(w.nx, w.ny, w.nz, w.px, w.py, w.pz, ov=w.overlap)
    t_setup, t_apply = [], []
    for s in subs:
        t0 = time.perf_counter()
        pc = O.Precond(g, system.row_ptr, system.col_idx, system.vals, only=int(s))
        t_setup.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        pc.apply(system.b)
        t_apply.append(time.perf_counter() - t0)
        del pc
    return float(np.mean(t_setup)), float(np.mean(t_apply))


def estimate_ms(w, iters: int, t_setup: float, t_apply: float, kry):
    """Oracle ms per solve: every subdomain set up once; one apply per iteration and one per cycle
    (x += B^{-1} V y); the Krylov part of each cycle from the fitted model."""
    K = w.px * w.py * w.pz
    c, a, b = kry
    cyc = cycles(iters, w.restart)
    krylov = sum(c + a * L + b * L * (L + 1) / 2 for L in cyc)
    return 1e3 * (K * t_setup + (iters + len(cyc)) * K * t_apply + krylov), {
        "setup_s": K * t_setup, "apply_s": (iters + len(cyc)) * K * t_apply, "krylov_s": krylov}


def sample_subs(K: int, n: int, seed: int = 0):
    return sorted(int(x) for x in np.random.default_rng(1000 + K + seed).choice(K, size=min(n, K), replace=False))


def oracle_estimate(w, system, iters: int, n_subs: int = 6):
    """Estimated oracle ms per solve of workload w from a bounded sample (n_subs random
    subdomains, three short unpreconditioned GMRES runs)."""
    K = w.px * w.py * w.pz
    subs = sample_subs(K, n_subs)
    t0 = time.perf_counter()
    t_setup, t_apply = subdomain_sample(w, system, subs)
    kry, _ = krylov_model(w, system)
    ms, parts = estimate_ms(w, iters, t_setup, t_apply, kry)
    sample = (f"oracle setup+factor and one apply of subdomains {subs} (of {K}), scaled to all {K}; "
              f"unpreconditioned oracle GMRES({w.restart}) runs of 1, 2 and 6 iterations on the full grid, "
              f"fitted per cycle; combined for {iters} iterations")
    return ms, sample, {"per_subdomain_setup_s": t_setup, "per_subdomain_apply_s": t_apply,
                        "parts_s": parts, "sample_wall_s": time.perf_counter() - t0}


def oracle_measured(name: str):
    """One full oracle solve of a named workload (setup + factorisation, then GMRES to 1e-8),
    timed, with its solution; beside it the estimator's prediction from a bounded sample."""
    import oracle as O
    w = synth.WORKLOADS[name]
    system = synth.make(w)
    g = O.Geometry(w.nx, w.ny, w.nz, w.px, w.py, w.pz, ov=w.overlap)
    t0 = time.perf_counter()
    pc = O.Precond(g, system.row_ptr, system.col_idx, system.vals)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, info = O.gmres(system.row_ptr, system.col_idx, system.vals, system.b, pc, w.restart, 1e-8, 3000)
    t_solve = time.perf_counter() - t0
    del pc
    est, _, _ = oracle_estimate(w, system, info.iters)
    total = 1e3 * (t_setup + t_solve)
    rec = {"setup_factor_ms": 1e3 * t_setup, "solve_ms": 1e3 * t_solve, "total_ms": total,
           "iterations": info.iters, "true_rel_residual": info.relres, "estimator_ms": est,
           "estimator_error": (est - total) / total}
    return rec, system, x


def serving_pool(n_pool: int, seed0: int = 5_000_000):
    """Synthetic matrices for the serving stream: cells log-uniform on [2000, 1048576],
    nx = ny = round((2n)^(1/3)), nz = max(2, round(n / nx^2)), px = py = clamp(round(nx / 8), 1, 16),
    pz = 2 if nz > 32 else 1, overlap 1."""
    import math
    pool = []
    for k in range(n_pool):
        u = float(synth.uniform(seed0 + k, 98, np.arange(1))[0])
        n = math.exp(math.log(2000) + u * (math.log(1048576) - math.log(2000)))
        nx = max(2, int(round((2 * n) ** (1 / 3))))
        nz = max(2, int(round(n / nx ** 2)))
        p = min(16, max(1, int(round(nx / 8))))
        pz = 2 if nz > 32 else 1
        s = synth.grid_jacobian(nx, nx, nz, seed0 + k, 1.0)
        rhs = [synth.rhs(s.n_cells, seed0 + 100000 + 10 * k + j) for j in range(4)]
        pool.append((s, (p, p, pz), rhs))
    return pool


def serve_stream(srv, pool, n_req: int, rate: float, seed: int = 5):
    """One Poisson stream through the serving loop.  30% of requests repeat an earlier matrix
    (factors reused), the rest carry a new matrix (full set-up: values uploaded, local matrices
    assembled and factored).  Latency = completion - arrival (host wall clock); generation is off
    the clock."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_req)
    arrivals = np.cumsum(gaps)
    reqs = []
    key0 = seed * 10_000_000  # matrix keys of this stream: a key always names the same matrix
    for i in range(n_req):
        if i > 0 and rng.random() < 0.3:
            j = int(rng.integers(0, i))
            key, pidx = reqs[j][0], reqs[j][1]
        else:
            key, pidx = key0 + i, int(rng.integers(0, len(pool)))
        reqs.append((key, pidx, int(rng.integers(0, 4))))
    st0 = srv.stats()
    t0 = time.perf_counter()
    nxt = 0
    inflight = {}
    lat = []
    done_t = []
    while nxt < n_req or inflight:
        now = time.perf_counter() - t0
        while nxt < n_req and arrivals[nxt] <= now:
            key, pidx, bj = reqs[nxt]
            s, part, rhs = pool[pidx]
            t = srv.submit(s, rhs[bj], partition=part, overlap=1, matrix_key=key, max_iter=2000)
            inflight[t] = arrivals[nxt]
            nxt += 1
        a, pend = srv.progress(2)
        now = time.perf_counter() - t0
        for t in list(inflight):
            r = srv.result(t)
            if r is not None:
                lat.append(now - inflight.pop(t))
                done_t.append(now)
        if a == 0 and pend == 0 and not inflight and nxt < n_req:
            time.sleep(max(0.0, min(0.002, arrivals[nxt] - now)))
    st1 = srv.stats()
    stats = {k: st1[k] - st0[k] for k in st1 if k not in ("resident_bytes", "budget_bytes", "active", "pending")}
    lat_ms = np.array(lat) * 1e3
    span = max(done_t) - arrivals[0]
    wall_ms = 1e3 * (time.perf_counter() - t0)
    return {"requests": n_req, "offered_per_s": rate, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "mean_ms": float(lat_ms.mean()),
            "solves_per_s": n_req / span, "reuse_hits": stats["reuse_hits"],
            "structure_builds": stats["structure_builds"], "structure_reuses": stats["structure_reuses"],
            "new_device_systems": n_req - stats["reuse_hits"] - stats["structure_reuses"],
            "steps": stats["steps"], "progress_calls": stats["progress_calls"],
            # host wall time by phase (the analysis runs on a worker thread, beside the rest)
            "phases_ms": {"loop_wall": wall_ms, "analysis_worker": stats["analysis_ms"], "admit": stats["admit_ms"],
                          "of_which_build": stats["build_ms"], "of_which_rekey": stats["rekey_ms"],
                          "build_factorisation": stats["build_factor_ms"],
                          "steps": stats["step_ms"], "retire": stats["retire_ms"]}}


def run_serving(args, stream):
    """The serving stream with the FP32 and the FP64 preconditioner, on one long-lived server per
    precision (the contract stream is 20,000 requests, so the first requests' structure analysis
    and device allocations are a warm-up, not the steady state): an untimed warm-up stream, then the
    stream at the offered rate (200/s).  One GB300 cannot keep up with that rate on this stream, so
    that run measures capacity (solves/s under overload) and its latencies mostly measure
    queueing; a second stream at 70% of the measured capacity gives p50/p99 at a sustainable load."""
    from paper_1401_7227_gb300 import asm2
    pool = serving_pool(args.serve_pool)
    out = {"sample": f"Poisson arrivals, 30% repeated matrices (factors reused), {len(pool)} distinct "
                     f"synthetic matrices of 2e3-1e6 cells, overlap 1, GMRES(30) to 1e-8; one server per "
                     f"precision, warmed by {args.serve_warm} untimed requests",
           "contract_rate_per_s": args.serve_rate}
    for prec in ("fp32", "fp64"):
        srv = asm2.Server(precision=prec, restart=30, max_active=args.serve_max_active, max_cached=128,
                          stream=stream.cuda_stream)
        warm = serve_stream(srv, pool, args.serve_warm, args.serve_rate, seed=4)
        over = serve_stream(srv, pool, args.serve_requests, args.serve_rate)
        cap = over["solves_per_s"]
        sus = serve_stream(srv, pool, args.serve_requests, 0.7 * cap, seed=6)
        srv.close()
        out[prec] = {"warm_up": {k: warm[k] for k in ("requests", "solves_per_s", "new_device_systems")},
                     "offered_rate": over, "capacity_solves_per_s": cap, "at_70pct_capacity": sus}
    return out


def run_batch(args, stream):
    """The batched workload: 256 independent systems from the same generator, grids (8, 8, 4) * s
    with s log-uniform on [1, 6] (256 - 55,296 cells), p_x = p_y = clamp(round(n_x / 6), 2, 8),
    overlap 1, FP32 factors, GMRES(20) to 1e-8; one step = all 256 solved together (every kernel
    launch serves all unfinished systems; steps replayed as CUDA graphs)."""
    import torch
    from paper_1401_7227_gb300 import asm2
    n_sys = args.batch_systems
    systems, solvers, bs = [], [], []
    for i in range(n_sys):
        nx, ny, nz, px, py, pz = synth.batch_grid(i)
        s = synth.grid_jacobian(nx, ny, nz, 1000 + i)
        sol = asm2.Solver(precision="fp32", restart=20, stream=stream.cuda_stream)
        sol.set_grid(nx, ny, nz)
        sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
        sol.set_partition(px, py, pz, 1)
        sol.factor()
        systems.append(s)
        solvers.append(sol)
        bs.append(torch.from_numpy(s.b).cuda())
    infos = None
    tiling = None
    if not args.no_tune:
        rep = asm2.tune_tiling_batch(solvers, bs, 1e-8, 3000)
        tiling = {"rule_ms_per_batch": rep["rule_ms"], "chosen": rep["best"],
                  "chosen_vs_rule": rep["best"]["apply_ms"] / rep["rule_ms"],
                  "measured": [[r["chunk_kb"], r["chunk_max_kb"], r["placement"], r["slots"], r["ctas_per_sm"],
                                round(r["apply_ms"], 3)] for r in rep["measured"]]}
    for _ in range(max(1, args.warmup)):
        xs, infos = asm2.solve_batch(solvers, bs, 1e-8, 3000)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        xs, infos = asm2.solve_batch(solvers, bs, 1e-8, 3000)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    its = [i["iterations"] for i in infos]
    worst = max(i["rel_residual"] for i in infos)
    cells = sum(s.n_cells for s in systems)
    st0 = solvers[0].stats()
    caps = {}
    for sol in solvers:
        c = sol.stats()["chunk_max_kb"]
        caps[c] = caps.get(c, 0) + 1
    apply_tiling = {"systems_per_chunk_kb": {str(k): v for k, v in sorted(caps.items())},
                    "ring_slot_kb": st0["last_solve_chunk_kb"], "placement": st0["last_solve_placement"],
                    "slots": st0["last_solve_slots"]}
    for sol in solvers:
        sol.close()
    return {"workload": f"{n_sys} systems, 256-55,296 cells each (total {cells}), K 4-64, ov 1, FP32 factors, GMRES(20)",
            "ms_per_batch": ms, "solves_per_s": 1e3 * n_sys / ms, "cells": cells,
            "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
            "all_converged": all(i["converged"] for i in infos), "worst_true_rel_residual": worst,
            "tiling": tiling, "apply_tiling": apply_tiling}


def nf_apply_bytes(w, elem: int) -> int:
    """Algorithmic bytes of one nested-factorisation apply on workload w: every line solve reads the
    fields of its line's packet it needs (G^-1, M, N, the two-step products P and Q, then L2 + L3,
    L2 + U3 or U2: 9 values per cell each), r comes in once (FP64), y_j goes out and back once per
    plane but the last, and the owned cells go out once (FP64)."""
    def spans(n, p, ov):
        return [min(n, n * (t + 1) // p + ov) - max(0, n * t // p - ov) for t in range(p)]
    tot = 24 * w.nx * w.ny * w.nz
    for bx in spans(w.nx, w.px, w.overlap):
        for by in spans(w.ny, w.py, w.overlap):
            for bz in spans(w.nz, w.pz, w.overlap):
                field = 9 * elem * bz
                fwd = by * bx + (by - 1) * bx            # forward lines of the forward and backward planes
                bwd = by * (bx - 1) + (by - 1) * (bx - 1)  # backward lines
                tot += (7 * fwd + 6 * bwd) * field + 24 * bx * by * bz + 2 * 3 * elem * bx * bz * (by - 1)
    return tot


def run_nf(args, stream, w, w_system, vals_d, b_d):
    """Nested factorisation with column-sum compensation (Appendix A) as the local solver, on the
    same system, partition and overlap without lumps (near width 0, no far field); FP32 apply,
    GMRES(restart) to 1e-8.  A step is the main line's: update values + re-factor + solve."""
    import torch
    from paper_1401_7227_gb300 import asm2
    sol = asm2.Solver(precision="fp32", restart=w.restart, local_solver="nf_colsum", stream=stream.cuda_stream)
    sol.set_grid(w.nx, w.ny, w.nz)
    sol.set_matrix(w_system[0], w_system[1], vals_d)
    sol.set_partition(w.px, w.py, w.pz, w.overlap, 0, (2, 2, 2), "none")
    sol.factor()

    def step():
        sol.update_values(vals_d)
        sol.factor()
        return sol.solve(b_d, rtol=1e-8, max_iter=args.max_iter)

    for _ in range(max(1, args.warmup)):
        step()
    sol.reset_profile()
    sol.set_profiling(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x, info = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    prof = sol.profile()
    st = sol.stats()
    sol.close()
    apply_ms = prof["apply_ms"] / max(1, prof["apply_launches"])
    alg = nf_apply_bytes(w, 4)
    peak, peak_kind = peaks()
    ach = alg / (apply_ms * 1e-3) / 1e9
    return {"workload": f"{w.name} without lumps (near width 0, no far field), NF + colsum, FP32 apply",
            "ms_per_step": ms, "iterations": info["iterations"], "converged": info["converged"],
            "true_rel_residual": info["rel_residual"], "local_rows": st["local_rows"],
            "breakdown_ms_per_step": {k: prof[k] / args.steps for k in ("apply_ms", "spmv_ms", "ortho_ms", "factor_ms")},
            "apply": {"kernel": "k_nf_apply", "launch_ms": apply_ms, "alg_bytes_per_launch": alg, "achieved": ach,
                      "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": peak_kind,
                      "bound": "latency (sequential line recurrences)"}}


def run_profile_case(args):
    """Small case for ncu captures: 128 x 128 x 32 (16 x 16 x 1 subdomains, overlap 2), three
    preconditioner applies then one GMRES solve.  The apply runs with the local-vector placement the
    1M-cell workload runs with (the placement rule and the tiling tuner both give all local vectors
    in device memory, 256-thread CTAs, four per SM, two ring slots)."""
    import torch
    from paper_1401_7227_gb300 import asm2
    from paper_1401_7227_gb300 import build as lib_build
    lib_build.build()
    s = synth.grid_jacobian(128, 128, 32, 3, 2.0)
    sol = asm2.Solver(precision=args.precision, restart=30, lumps=args.lumps)
    sol.set_grid(128, 128, 32)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(16, 16, 1, 2)
    sol.factor()
    sol.set_tuning(apply_smem="device", autotune=False)
    b = torch.from_numpy(s.b).cuda()
    for _ in range(3):
        sol.apply(b)
    torch.cuda.synchronize()
    x, info = sol.solve(b, 1e-8, 400)
    print(json.dumps({"profile_case": "grid128x128x32_k256", "info": info, "stats": sol.stats()}))
    sol.close()
    return 0


def run_profile_nf(args):
    """Case for ncu captures of the nested-factorisation apply: the 1M-cell workload's system
    (128 x 128 x 64, 16 x 16 x 2 subdomains, overlap 2, no lumps), FP32 apply, three applies."""
    import torch
    from paper_1401_7227_gb300 import asm2
    from paper_1401_7227_gb300 import build as lib_build
    lib_build.build()
    w = synth.WORKLOADS["grid128x128x64_k512"]
    s = synth.make(w)
    sol = asm2.Solver(precision="fp32", restart=w.restart, local_solver="nf_colsum")
    sol.set_grid(w.nx, w.ny, w.nz)
    sol.set_matrix(s.row_ptr, s.col_idx, s.vals)
    sol.set_partition(w.px, w.py, w.pz, w.overlap, 0, (2, 2, 2), "none")
    sol.factor()
    b = torch.from_numpy(s.b).cuda()
    for _ in range(3):
        z = sol.apply(b)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "nf_grid128x128x64_k512", "z_norm": float(torch.linalg.norm(z)),
                      "alg_bytes_per_apply": nf_apply_bytes(w, 4), "stats": sol.stats()}))
    sol.close()
    return 0


def run_profile_kernels(args):
    """Case for one ncu capture of every kernel family (time and DRAM bytes per launch): on
    128 x 128 x 32 (524,288 cells, 16 x 16 x 1 subdomains, overlap 2; inputs larger than L2):
    the ILU path with FP32 factors (set-up, applies, a few GMRES steps), ORTHOMIN, the two-level
    coarse correction, nested factorisation; exact local solves on 16 x 16 x 8 (4 subdomains of
    ~2,200 unknowns: their dense inverses stay within a few hundred MB); and two systems of
    32 x 32 x 16 through the batched per-projection Gram-Schmidt path."""
    import torch
    from paper_1401_7227_gb300 import asm2
    from paper_1401_7227_gb300 import build as lib_build
    lib_build.build()
    s = synth.grid_jacobian(128, 128, 32, 3, 2.0)
    b = torch.from_numpy(s.b).cuda()

    def make(local="colsum", prec="fp32", krylov="gmres", near_width=2, far="partition", sys=s, part=(16, 16, 1),
             ov=2, coarse=None):
        sol = asm2.Solver(precision=prec, restart=30, local_solver=local, krylov=krylov)
        sol.set_grid(sys.nx, sys.ny, sys.nz)
        sol.set_matrix(sys.row_ptr, sys.col_idx, sys.vals)
        sol.set_partition(*part, ov, near_width, (2, 2, 2), far)
        if coarse:
            sol.set_coarse(coarse)
        sol.factor()
        return sol

    out = {}
    sol = make()
    for _ in range(2):
        sol.apply(b)
    x, info = sol.solve(b, 1e-8, 6)
    out["ilu_fp32"] = info
    sol.close()
    sol = make(krylov="orthomin")
    out["orthomin"] = sol.solve(b, 1e-8, 4)[1]
    sol.close()
    sol = make(prec="fp64", near_width=0, far="none", coarse="two-level")
    sol.apply(b)
    out["two_level"] = sol.solve(b, 1e-8, 3)[1]
    sol.close()
    sol = make(local="nf_colsum", near_width=0, far="none")
    sol.apply(b)
    out["nf"] = sol.solve(b, 1e-8, 3)[1]
    sol.close()
    small = synth.grid_jacobian(32, 32, 16, 4)
    tiny = synth.grid_jacobian(16, 16, 8, 4)
    sol = make(local="exact", prec="fp64", sys=tiny, part=(2, 2, 1), ov=1)
    sol.apply(torch.from_numpy(tiny.b).cuda())
    out["exact"] = sol.solve(torch.from_numpy(tiny.b).cuda(), 1e-8, 3)[1]
    sol.close()
    bs = [make(sys=small, part=(4, 4, 1), ov=1) for _ in range(2)]
    out["batch"] = asm2.solve_batch(bs, [torch.from_numpy(small.b).cuda()] * 2, 1e-8, 3)[1]
    for x_ in bs:
        x_.close()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "kernels_grid128x128x32_k256", "infos": out}, default=str))
    return 0


FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64 (no measured figure for it is given)


def spmv_roofline(res, system, steps: int):
    """The SpMV is bound by the FP64 pipe on this GPU (18 flops per 3x3 block against ~76 bytes):
    achieved TFLOP/s of one launch against the nominal FP64 rate.  Launches per solve: one per
    Arnoldi step and one per restart (true residual)."""
    info = res["info"]
    launches = info["iterations"] + info["restarts"] + 1
    ms = res["prof"]["spmv_ms"] / steps / launches
    flops = 18.0 * system.col_idx.size
    ach = flops / (ms * 1e-3) / 1e12
    return {"kernel": "k_spmv", "bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_NOMINAL_TFLOPS, "peak_kind": "nominal FP64", "launch_ms": ms,
            "hbm_frac": (76.0 * system.col_idx.size + 48.0 * system.n_cells) / (ms * 1e-3) / 1e9 / peaks()[0]}


def ortho_roofline(res, system, steps: int, m: int):
    """Modified Gram-Schmidt (k_ortho_coop, one cooperative launch per Arnoldi step; the timer also
    holds the small per-step control kernels).  Step j of a cycle makes j + 2 fused passes over
    the 3N-vector w, each 2 FP64 FMAs per element (w -= h v_prev; dot with the next v, or the
    norm), and one scaling pass: 4 * 3N * (j + 2) + 3N flops.  It reads v_0..v_j, w once and writes
    v_{j+1}: 8 * 3N * (j + 3) algorithmic bytes (w stays in L2 between passes).  Bound: the FP64
    pipe, against the nominal 1.25 TFLOP/s."""
    info = res["info"]
    n3 = 3.0 * system.n_cells
    flops = byt = 0.0
    for L in cycles(info["iterations"], m):
        for j in range(L):
            flops += 4.0 * n3 * (j + 2) + n3
            byt += 8.0 * n3 * (j + 3)
    sec = res["prof"]["ortho_ms"] / steps * 1e-3
    ach = flops / sec / 1e12
    return {"kernel": "k_ortho_coop", "bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS,
            "unit": "TFLOP/s", "frac": ach / FP64_NOMINAL_TFLOPS, "peak_kind": "nominal FP64",
            "ms_per_solve": sec * 1e3, "launch_ms": sec * 1e3 / max(1, info["iterations"]),
            "hbm_frac": byt / sec / 1e9 / peaks()[0]}


def apply_traffic(alg_bytes: int):
    """DRAM bytes per apply from the committed ncu record, scaled by algorithmic bytes; None when
    the kernel source changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "apply_traffic.json")))
        src = open(os.path.join(ROOT, "paper_1401_7227_gb300", "csrc", "kernels_solve.cu"), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != rec["kernel_source_sha256_16"]:
            return None
        return int(rec["dram_bytes_per_launch"] * alg_bytes / rec["alg_bytes_per_launch"])
    except Exception:
        return None


def workload_config(w, system, precision: str, lumps: str = "fp32"):
    """The `config` object of both arms' lines (the same dict, so that the two lines compare)."""
    return {"workload": w.name, "grid": [w.nx, w.ny, w.nz], "cells": system.n_cells,
            "partition": [w.px, w.py, w.pz], "overlap": w.overlap, "near_width": 2, "c_near": [2, 2, 2],
            "far": "partition boxes", "krylov": f"GMRES({w.restart})", "precision": precision,
            "lump_rows": "fp64" if precision == "fp64" else lumps,
            "tol": 1e-8, "l2": "inputs larger than L2 (A 0.56 GB, factors > 0.5 GB)",
            "step": "update values + re-assemble + re-factor + GMRES to 1e-8", "generator": GENERATOR}


def run_reference(args):
    """The oracle as it stands, on the host cores, for the GPU arm's workload and metric.  A full
    1M-cell oracle solve takes many minutes, so each step is a bounded sample of it: the setup and
    one apply of one subdomain (a different random one each step) and three short
    unpreconditioned GMRES runs on the full grid, extrapolated to the whole solve (ms per solve,
    `value`).  `ms_per_step` is the time the sample itself took."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = synth.WORKLOADS[args.workload]
    system = synth.make(w)
    iters = args.ref_iters if args.ref_iters is not None else ITERS_MEASURED[w.name]
    K = w.px * w.py * w.pz
    order = sample_subs(K, K, seed=1)
    est, wall = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t_setup, t_apply = subdomain_sample(w, system, [order[k % K]])
        kry, _ = krylov_model(w, system)
        ms, _ = estimate_ms(w, iters, t_setup, t_apply, kry)
        if k >= args.warmup:
            est.append(ms)
            wall.append(1e3 * (time.perf_counter() - t0))
    v = float(np.mean(est))
    model, nproc = cpu_info()
    sample = (f"per step: oracle setup+factor and one apply of one random subdomain (of {K}), scaled to all {K}, "
              f"plus unpreconditioned oracle GMRES({w.restart}) runs of 1, 2 and 6 iterations on the full grid; "
              f"extrapolated to {iters} iterations; value = mean of the steps' estimates")
    # n_gpus: the launch's world size, as in the GPU arm; the work itself ran on one host core
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(wall)), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference", "estimated": True,
            "config": workload_config(w, system, args.precision, args.lumps), "iterations_assumed": iters,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": model, "nproc": nproc, "estimated": True},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def run_small(args, stream):
    """The two smaller workloads end to end on both sides: one full oracle solve each (setup +
    factorisation and GMRES timed separately, single-threaded) beside the GPU's solve in each factor
    precision (a step as in the main line: update values, re-factor, solve), with each GPU
    solution's error against the oracle's."""
    import torch
    from paper_1401_7227_gb300 import asm2
    model, nproc = cpu_info()
    out = {"kind": "oracle", "cores": 1, "cpu_model": model, "nproc": nproc, "workloads": {}}
    for name in ("grid10x10x5_k4", "grid64x64x16_k64"):
        w = synth.WORKLOADS[name]
        rec, system, xo = oracle_measured(name)
        vals_d = torch.from_numpy(system.vals.reshape(-1)).cuda()
        b_d = torch.from_numpy(system.b).cuda()
        gpu = {}
        for prec in ("fp64", "fp32", "fp16s"):
            sol = asm2.Solver(precision=prec, restart=w.restart, stream=stream.cuda_stream)
            sol.set_grid(w.nx, w.ny, w.nz)
            sol.set_matrix(system.row_ptr, system.col_idx, vals_d)
            sol.set_partition(w.px, w.py, w.pz, w.overlap)
            sol.factor()

            def step():
                sol.update_values(vals_d)
                sol.factor()
                return sol.solve(b_d, rtol=1e-8, max_iter=3000)

            for _ in range(max(3, args.warmup)):
                step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                x, info = step()
            e1.record(stream)
            torch.cuda.synchronize()
            xh = x.cpu().numpy()
            gpu[prec] = {"ms_per_solve": e0.elapsed_time(e1) / args.steps, "iterations": info["iterations"],
                         "true_rel_residual": info["rel_residual"],
                         "err_vs_oracle": float(np.linalg.norm(xh - xo) / np.linalg.norm(xo))}
            sol.close()
        rec["gpu"] = gpu
        rec["oracle_over_gpu_fp64"] = rec["total_ms"] / gpu["fp64"]["ms_per_solve"]
        out["workloads"][name] = rec
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1401_7227_gb300 import asm2
    from paper_1401_7227_gb300 import build as lib_build

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    lib_build.build()
    w = synth.WORKLOADS[args.workload]
    system = synth.make(w)
    n3 = 3 * system.n_cells
    vals_d = torch.from_numpy(system.vals.reshape(-1)).cuda()
    b_d = torch.from_numpy(system.b).cuda()
    stream = torch.cuda.current_stream()

    def make_solver(prec, lumps, ortho="mgs"):
        s = asm2.Solver(precision=prec, restart=w.restart, device=local, stream=stream.cuda_stream, lumps=lumps,
                        ortho=ortho)
        s.set_grid(w.nx, w.ny, w.nz)
        s.set_matrix(system.row_ptr, system.col_idx, vals_d)
        s.set_partition(w.px, w.py, w.pz, w.overlap)
        if args.chunk_kb is not None:
            s.set_tuning(chunk_kb=args.chunk_kb)
        s.factor()
        if args.placement is not None:  # a fixed placement: no online tuning
            s.set_tuning(apply_smem=args.placement, autotune=False)
        return s

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step(sol):
        sol.update_values(vals_d)
        sol.factor()
        x, info = sol.solve(b_d, rtol=1e-8, max_iter=args.max_iter)
        return x, info

    results = {}
    def vkey(prec, lumps, ortho="mgs"):  # "fp64", "fp32", "fp16s" (FP32 lumps), "fp32_lumps_fp64", "fp32_cgs"
        k = prec if prec == "fp64" or lumps == "fp32" else f"{prec}_lumps_fp64"
        return k if ortho == "mgs" else f"{k}_cgs"

    main_key = vkey(args.precision, args.lumps)
    variants = [(args.precision, args.lumps, "mgs")]
    if not args.no_precisions:
        for pv in (("fp64", "fp64", "mgs"), ("fp32", "fp32", "mgs"), ("fp16s", "fp32", "mgs"), ("fp32", "fp64", "mgs"),
                   ("fp32", "fp32", "cgs")):
            if vkey(*pv) != main_key:
                variants.append(pv)
    def tiling_summary(rep):
        """the tuner's choice against the default tiling, and every measured configuration as
        [chunk KB asked (0: rule), largest chunk KB, placement, ring slots, CTAs per SM, ms]"""
        if rep is None:
            return None
        b = rep["best"]
        return {"rule_ms": rep["rule_ms"], "chosen": b, "chosen_vs_rule": b["apply_ms"] / rep["rule_ms"],
                "measured": [[r["chunk_kb"], r["chunk_max_kb"], r["placement"], r["slots"], r["ctas_per_sm"],
                              round(r["apply_ms"], 4)] for r in rep["measured"]]}

    for prec, lumps, ortho in variants:
        sol = make_solver(prec, lumps, ortho)
        tiling = None if args.no_tune else tiling_summary(sol.tune_tiling(reps=7))
        for _ in range(args.warmup):
            step(sol)
        sol.reset_profile()
        sol.set_profiling(True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            infos = []
            for _ in range(args.steps):
                x, info = step(sol)
                infos.append(info)
            e1.record(stream)
            barrier()
        ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
        prof = sol.profile()
        sol.set_profiling(False)
        st = sol.stats()
        xh = x.cpu().numpy()
        import oracle as O
        r = system.b - O.spmv(system.row_ptr, system.col_idx, system.vals, xh)
        results[vkey(prec, lumps, ortho)] = {"ms": ms, "info": infos[-1], "prof": prof, "stats": st, "clocks": clk.summary(),
                         "host_check_relres": float(np.linalg.norm(r) / np.linalg.norm(system.b)), "solver": sol,
                         "x": xh, "tiling": tiling}

    main = results[main_key]
    sol = main["solver"]
    # end to end through the public API with pinned host buffers (matrix values + b in, x out)
    vals_h = torch.from_numpy(system.vals.reshape(-1)).pin_memory()
    b_h = torch.from_numpy(system.b).pin_memory()
    x_h = torch.empty(n3, dtype=torch.float64).pin_memory()
    import ctypes as C
    L = asm2.load()

    def e2e_step():
        asm2._check(L.asm_update_values(sol.handle, C.c_void_p(vals_h.data_ptr()), 0), "update")
        sol.factor()
        info = asm2.SolveInfo()
        st_ = L.asm_solve(sol.handle, C.c_void_p(b_h.data_ptr()), C.c_void_p(x_h.data_ptr()), 1e-8, args.max_iter, 0,
                          C.byref(info))
        if st_ not in (0, 4):
            raise asm2.ASMError(st_, "solve")

    for _ in range(max(1, args.warmup // 2)):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, ws)

    def err_vs_fp64(x):
        """relative distance to the FP64 GPU solution (itself checked against the oracle at the
        smaller sizes and against the oracle's apply on sampled subdomains at this size)"""
        if "fp64" not in results:
            return None
        x64 = results["fp64"]["x"]
        return float(np.linalg.norm(x - x64) / np.linalg.norm(x64))

    prof = main["prof"]
    st = main["stats"]
    n_apply = max(1, prof["apply_launches"])
    apply_ms = prof["apply_ms"] / n_apply
    alg_bytes = st["alg_apply_bytes"]
    peak, peak_kind = peaks()
    achieved = alg_bytes / (apply_ms * 1e-3) / 1e9
    launches = prof["kernel_launches"]
    line = {
        "metric": METRIC, "value": main["ms"], "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main["ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 Krylov / f32 factors" if args.precision == "fp32" else args.precision, "data": "synthetic",
        "config": workload_config(w, system, args.precision, args.lumps),
        "solves_per_s": 1e3 * ws / main["ms"],
        "iterations": main["info"]["iterations"], "restarts": main["info"]["restarts"],
        "true_rel_residual": main["info"]["rel_residual"], "host_check_rel_residual": main["host_check_relres"],
        "mean_local_rows": st["local_rows"] / st["n_sub"],
        "precisions": {p_: {"ms_per_solve": r_["ms"], "iterations": r_["info"]["iterations"],
                            "converged": bool(r_["info"]["converged"]), "true_rel_residual": r_["info"]["rel_residual"],
                            "host_check_rel_residual": r_["host_check_relres"],
                            "err_vs_fp64": err_vs_fp64(r_["x"]),
                            "ortho_ms_per_solve": r_["prof"]["ortho_ms"] / args.steps,
                            "tiling": None if r_["tiling"] is None else
                            {k: r_["tiling"][k] for k in ("rule_ms", "chosen", "chosen_vs_rule")}}
                       for p_, r_ in results.items() if p_ != main_key},
        "err_vs_fp64": err_vs_fp64(main["x"]),
        "tiling": main["tiling"],
        "apply_tiling": {k: st[k] for k in ("chunk_max_kb", "stream_chunks", "apply_placement", "apply_slots")},
        "breakdown_ms_per_solve": {k: prof[k] / args.steps for k in ("apply_ms", "spmv_ms", "ortho_ms", "factor_ms")},
        "roofline": {"bound": "hbm", "kernel": "precond apply (boxsum + fused local solves)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": apply_traffic(alg_bytes),
                     "alg_bytes_per_launch": alg_bytes, "launch_ms": apply_ms, "peak_kind": peak_kind},
        "rooflines_other": [spmv_roofline(main, system, args.steps), ortho_roofline(main, system, args.steps, w.restart)],
        "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(system.vals.nbytes + system.b.nbytes),
                "d2h_bytes_per_step": int(system.b.nbytes)},
        "gpu_launches": int(launches),
        "clocks": main["clocks"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        cpu_ms, sample, detail = oracle_estimate(w, system, main["info"]["iterations"])
        model, nproc = cpu_info()
        line["cpu_baseline"] = {"value": cpu_ms, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                "estimated": True, "cpu_model": model, "nproc": nproc, "detail": detail}
        line["cpu_baseline_measured"] = run_small(args, stream)
    for r_ in results.values():
        r_["solver"].close()
    if not args.no_nf and rank == 0:
        line["nf_local_solver"] = run_nf(args, stream, w, (system.row_ptr, system.col_idx), vals_d, b_d)
    if not args.no_batch and rank == 0:
        line["batch"] = run_batch(args, stream)
    if not args.no_serve and rank == 0:
        line["serving"] = run_serving(args, stream)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="grid128x128x64_k512", choices=list(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16s"])
    ap.add_argument("--lumps", default="fp32", choices=["fp64", "fp32"],
                    help="lump rows' precision under FP32/FP16S fine rows (asm_options.lump_precision)")
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--ref-iters", type=int, default=None,
                    help="iterations the reference arm extrapolates to (default: the workload's measured count)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-nf", action="store_true", help="skip the nested-factorisation leg")
    ap.add_argument("--no-precisions", action="store_true", help="time the --precision path only")
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--profile-case", action="store_true", help="small case for ncu captures")
    ap.add_argument("--profile-nf", action="store_true", help="nested-factorisation apply case for ncu captures")
    ap.add_argument("--profile-kernels", action="store_true", help="every kernel family, for one ncu capture")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tiling (no asm_tune_tiling)")
    ap.add_argument("--placement", choices=["auto", "device", "lumps", "shared"], default=None,
                    help="with --no-tune: fix the apply's placement (for profiling runs)")
    ap.add_argument("--chunk-kb", type=int, default=None, help="with --no-tune: fix the stream-chunk capacity")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-warm", type=int, default=300)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-pool", type=int, default=12)
    ap.add_argument("--serve-max-active", type=int, default=64)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.profile_nf:
        return run_profile_nf(args)
    if args.profile_kernels:
        return run_profile_kernels(args)
    if args.placement is not None or args.chunk_kb is not None:
        args.no_tune = True
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
