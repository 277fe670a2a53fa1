"""Thin ctypes binding of ``libasm2.so`` (include/asm2.h): the boundary-conditioned additive
Schwarz preconditioner (Section 4) with GMRES / ORTHOMIN (Section 2).  Argument marshalling only:
every step of the solver runs in the library's CUDA kernels.  Device buffers are torch CUDA
tensors, host buffers numpy arrays; the stream is torch's current CUDA stream unless one is given.

There is no fallback: if the library is missing or no CUDA device is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

ASM_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "pattern", 3: "zero pivot", 4: "not converged", 5: "out of memory",
          6: "cuda error", 7: "timeout", 8: "state"}
PREC = {"fp64": 0, "fp32": 1, "fp16s": 2}
LUMPS = {"fp64": 0, "fp32": 1}
FAR = {"none": 0, "partition": 1, "boxes": 2}
COARSE = {"none": 0, "two-level": 1, "two-stage": 2}
#: placements of the apply's local vectors (ASM_TUNE_APPLY_SMEM values)
PLACEMENT_NAMES = {0: "device", 2: "lumps", 3: "shared", -1: None}

#: every symbol include/asm2.h declares
EXPORTS = [
    "asm_default_options", "asm_error_string", "asm_create", "asm_destroy", "asm_set_grid", "asm_set_matrix_bsr",
    "asm_update_values", "asm_set_partition_boxes", "asm_set_coarse_correction", "asm_factor", "asm_apply_precond", "asm_spmv", "asm_solve",
    "asm_solve_batch", "asm_get_stats", "asm_get_error_location", "asm_get_local_info", "asm_get_local_map",
    "asm_get_local_matrix", "asm_get_local_factors", "asm_set_profiling", "asm_get_profile", "asm_reset_profile", "asm_set_tuning", "asm_tune_tiling", "asm_tune_tiling_batch",
    "asm_residual_noalloc",
    "asm_server_default_options", "asm_server_create", "asm_server_submit", "asm_server_progress",
    "asm_server_result", "asm_server_get_stats", "asm_server_destroy",
]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("krylov", C.c_int), ("restart", C.c_int), ("local_solver", C.c_int),
                ("flexible", C.c_int), ("device", C.c_int), ("lump_precision", C.c_int), ("ortho", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("rel_residual", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("n_cells", C.c_int), ("n_sub", C.c_int), ("local_rows", C.c_longlong), ("max_local_rows", C.c_int),
                ("max_levels", C.c_int), ("local_blocks", C.c_longlong), ("factor_bytes", C.c_longlong),
                ("apply_index_bytes", C.c_longlong), ("matrix_bytes", C.c_longlong), ("alg_apply_bytes", C.c_longlong),
                ("setup_ms", C.c_double),
                ("factor_ms", C.c_double), ("chunk_max_kb", C.c_int), ("stream_chunks", C.c_longlong),
                ("apply_placement", C.c_int), ("apply_slots", C.c_int), ("last_solve_placement", C.c_int),
                ("last_solve_slots", C.c_int), ("last_solve_chunk_kb", C.c_int)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for k in ("apply_placement", "last_solve_placement"):
            d[k] = PLACEMENT_NAMES.get(d[k], d[k])
        return d


class Profile(C.Structure):
    _fields_ = [("apply_ms", C.c_double), ("spmv_ms", C.c_double), ("ortho_ms", C.c_double), ("factor_ms", C.c_double),
                ("apply_launches", C.c_longlong), ("kernel_launches", C.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TilingEntry(C.Structure):
    _fields_ = [("chunk_kb", C.c_int), ("chunk_max_kb", C.c_int), ("chunks", C.c_longlong), ("placement", C.c_int),
                ("slots", C.c_int), ("ctas_per_sm", C.c_int), ("apply_ms", C.c_double)]


TILING_MAX = 64


class TilingReport(C.Structure):
    _fields_ = [("n", C.c_int), ("best", C.c_int), ("rule_ms", C.c_double), ("e", TilingEntry * TILING_MAX)]

    def as_dict(self):
        rows = [{"chunk_kb": e.chunk_kb, "chunk_max_kb": e.chunk_max_kb, "chunks": e.chunks,
                 "placement": PLACEMENT_NAMES.get(e.placement, e.placement), "slots": e.slots,
                 "ctas_per_sm": e.ctas_per_sm, "apply_ms": e.apply_ms} for e in self.e[:self.n]]
        return {"rule_ms": self.rule_ms, "best": rows[self.best] if rows else None, "measured": rows}


class ServerOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("restart", C.c_int), ("device", C.c_int), ("max_active", C.c_int),
                ("max_cached", C.c_int), ("hbm_budget", C.c_longlong), ("lump_precision", C.c_int)]


class Request(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("n_cells", C.c_int), ("nnzb", C.c_int),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("vals", C.c_void_p),
                ("px", C.c_int), ("py", C.c_int), ("pz", C.c_int), ("overlap", C.c_int), ("near_width", C.c_int),
                ("c_near", C.c_int * 3), ("far_mode", C.c_int), ("c_far", C.c_int * 3),
                ("b", C.c_void_p), ("rtol", C.c_double), ("max_iter", C.c_int), ("matrix_key", C.c_longlong)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("admitted", C.c_longlong), ("completed", C.c_longlong),
                ("steps", C.c_longlong), ("reuse_hits", C.c_longlong), ("structure_builds", C.c_longlong),
                ("evictions", C.c_longlong), ("resident_bytes", C.c_longlong), ("budget_bytes", C.c_longlong),
                ("active", C.c_int), ("pending", C.c_int), ("analysis_ms", C.c_double), ("admit_ms", C.c_double),
                ("build_ms", C.c_double), ("rekey_ms", C.c_double), ("step_ms", C.c_double),
                ("retire_ms", C.c_double), ("progress_calls", C.c_longlong), ("structure_reuses", C.c_longlong),
                ("build_factor_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ASMError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"asm2: {what}: {STATUS.get(status, status)} ({status})")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libasm2.so (built by paper_1401_7227_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_1401_7227_gb300.build.build() first")
        _build.build()
    L = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    L.asm_default_options.argtypes = [C.POINTER(Options)]
    L.asm_default_options.restype = None
    L.asm_error_string.argtypes = [I]
    L.asm_error_string.restype = C.c_char_p
    L.asm_create.argtypes = [C.POINTER(P), C.POINTER(Options), P]
    L.asm_destroy.argtypes = [P]
    L.asm_set_grid.argtypes = [P, I, I, I]
    L.asm_set_matrix_bsr.argtypes = [P, I, I, P, P, P, I]
    L.asm_update_values.argtypes = [P, P, I]
    L.asm_set_partition_boxes.argtypes = [P, I, I, I, I, I, P, I, P]
    L.asm_factor.argtypes = [P]
    L.asm_apply_precond.argtypes = [P, P, P, I]
    L.asm_spmv.argtypes = [P, P, P, I]
    L.asm_solve.argtypes = [P, P, P, D, I, I, C.POINTER(SolveInfo)]
    L.asm_solve_batch.argtypes = [P, I, P, P, D, I, I, P]
    L.asm_get_stats.argtypes = [P, C.POINTER(Stats)]
    L.asm_get_error_location.argtypes = [P, C.POINTER(I), C.POINTER(I)]
    L.asm_get_local_info.argtypes = [P, I, P, P, P, P]
    L.asm_get_local_map.argtypes = [P, I, P]
    L.asm_get_local_matrix.argtypes = [P, I, P, P, P]
    L.asm_get_local_factors.argtypes = [P, I, P, P]
    L.asm_set_profiling.argtypes = [P, I]
    L.asm_get_profile.argtypes = [P, C.POINTER(Profile)]
    L.asm_reset_profile.argtypes = [P]
    L.asm_set_tuning.argtypes = [P, I, I]
    L.asm_tune_tiling.argtypes = [P, I, C.POINTER(TilingReport)]
    L.asm_tune_tiling_batch.argtypes = [P, I, P, P, D, I, I, C.POINTER(TilingReport)]
    L.asm_residual_noalloc.argtypes = [P, P, P, P, P]
    L.asm_server_default_options.argtypes = [C.POINTER(ServerOptions)]
    L.asm_server_default_options.restype = None
    L.asm_server_create.argtypes = [C.POINTER(P), C.POINTER(ServerOptions), P]
    L.asm_server_submit.argtypes = [P, C.POINTER(Request), C.POINTER(C.c_longlong)]
    L.asm_server_progress.argtypes = [P, I, C.POINTER(I), C.POINTER(I)]
    L.asm_server_result.argtypes = [P, C.c_longlong, P, C.POINTER(SolveInfo)]
    L.asm_server_get_stats.argtypes = [P, C.POINTER(ServerStats)]
    L.asm_server_destroy.argtypes = [P]
    for name in EXPORTS:
        if name not in ("asm_default_options", "asm_error_string", "asm_server_default_options"):
            getattr(L, name).restype = I
    _lib = L
    return L


def _check(st: int, what: str):
    if st != ASM_OK:
        raise ASMError(st, what)


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _values(x, n: int, what: str):
    """(x as contiguous float64 with exactly n values, on_device).  CUDA tensors stay on the device;
    anything else becomes a host array.  The library reads exactly n values from the pointer, so a
    shorter or narrower buffer is refused here instead of being read past its end."""
    if _is_torch(x) and x.is_cuda:
        import torch
        xi = x.contiguous().to(torch.float64)
        got = xi.numel()
        dev = True
    else:
        xi = np.ascontiguousarray(x, dtype=np.float64)
        got = xi.size
        dev = False
    if got != n:
        raise ValueError(f"{what}: expected {n} values, got {got}")
    return xi, dev


def _ptr(a, on_device: bool):
    return C.c_void_p(a.data_ptr()) if on_device else _host_ptr(a)


def _current_stream(device: int):
    import torch
    return torch.cuda.current_stream(device).cuda_stream


# local solvers: block ILU(0) with / without column-sum compensation, exact (Gauss-Jordan), and
# nested factorisation (Appendix A) with / without column-sum compensation (boxes without lumps)
LOCAL = {"colsum": 0, "plain": 1, "exact": 2, "nf_colsum": 3, "nf": 4}


class Solver:
    """One system: grid, BSR 3x3 matrix, partition, factorisation and solves."""

    def __init__(self, precision: str = "fp64", restart: int = 30, local_solver: str = "colsum",
                 flexible: int = -1, device: int = 0, stream: int | None = None, krylov: str = "gmres",
                 lumps: str = "fp32", ortho: str = "mgs"):
        """lumps: "fp32" (default) or "fp64", the lump rows' precision under FP32/FP16S fine rows
        (asm_options.lump_precision).  ortho: "mgs" (default) or "cgs", the Arnoldi step's
        Gram-Schmidt (asm_options.ortho)."""
        L = load()
        o = Options()
        L.asm_default_options(C.byref(o))
        o.lump_precision = LUMPS[lumps]
        o.precision = PREC[precision]
        o.restart = restart
        o.local_solver = LOCAL[local_solver]
        o.flexible = flexible
        o.device = device
        o.krylov = {"gmres": 0, "orthomin": 1}[krylov]
        o.ortho = {"mgs": 0, "cgs": 1}[ortho]
        self.device = device
        self.stream = stream if stream is not None else _current_stream(device)
        h = C.c_void_p()
        _check(L.asm_create(C.byref(h), C.byref(o), C.c_void_p(self.stream)), "create")
        self._h = h
        self.n_cells = 0
        self.nnzb = None

    def close(self):
        if getattr(self, "_h", None):
            load().asm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_grid(self, nx: int, ny: int, nz: int):
        _check(load().asm_set_grid(self._h, nx, ny, nz), "set_grid")
        self.n_cells = nx * ny * nz

    def set_matrix(self, row_ptr, col_idx, vals):
        """row_ptr int32 [N+1], col_idx int32 [nnzb], vals [nnzb, 3, 3] float64 (host or CUDA)."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32).ravel()
        ci = np.ascontiguousarray(col_idx, dtype=np.int32).ravel()
        v, dev = _values(vals, 9 * ci.shape[0], "set_matrix")
        _check(load().asm_set_matrix_bsr(self._h, rp.shape[0] - 1, ci.shape[0], _host_ptr(rp), _host_ptr(ci),
                                         _ptr(v, dev), int(dev)), "set_matrix")
        self.nnzb = ci.shape[0]

    def update_values(self, vals):
        """New values on the pattern of set_matrix (vals [nnzb, 3, 3], host or CUDA)."""
        if self.nnzb is None:  # no matrix yet: the library reports STATE without reading vals
            _check(load().asm_update_values(self._h, _host_ptr(np.zeros(9)), 0), "update_values")
        v, dev = _values(vals, 9 * self.nnzb, "update_values")
        _check(load().asm_update_values(self._h, _ptr(v, dev), int(dev)), "update_values")

    def set_partition(self, px: int, py: int, pz: int, overlap: int = 1, near_width: int = 2,
                      c_near=(2, 2, 2), far_mode: str | int = "partition", c_far=None):
        fm = FAR[far_mode] if isinstance(far_mode, str) else int(far_mode)
        cn = (C.c_int * 3)(*c_near)
        cf = (C.c_int * 3)(*(c_far if c_far is not None else (1, 1, 1)))
        _check(load().asm_set_partition_boxes(self._h, px, py, pz, overlap, near_width, cn, fm, cf), "set_partition")

    def set_coarse(self, mode: str | int = "two-level", c_box=None):
        """Classical coarse-grid correction (Section 3): "none", "two-level" (Eq. 3.5) or
        "two-stage" (Eqs. 3.7-3.8), on the partition boxes (c_box None) or aligned boxes of c_box
        cells.  Takes effect at the next factor()."""
        m = COARSE[mode] if isinstance(mode, str) else int(mode)
        cb = None if c_box is None else (C.c_int * 3)(*c_box)
        _check(load().asm_set_coarse_correction(self._h, m, cb), "set_coarse")

    def factor(self):
        st = load().asm_factor(self._h)
        if st == 3:
            s, r = C.c_int(), C.c_int()
            load().asm_get_error_location(self._h, C.byref(s), C.byref(r))
            err = ASMError(st, f"factor (subdomain {s.value}, local row {r.value})")
            err.where = (s.value, r.value)
            raise err
        _check(st, "factor")

    def _vec_call(self, fn, x, what):
        xi, dev = _values(x, 3 * self.n_cells, what)
        if dev:
            import torch
            out = torch.empty_like(xi)
        else:
            out = np.empty_like(xi)
        _check(fn(self._h, _ptr(xi, dev), _ptr(out, dev), int(dev)), what)
        return out

    def apply(self, r):
        """z = B^{-1} r (Eqs. 4.2-4.5)."""
        return self._vec_call(load().asm_apply_precond, r, "apply_precond")

    def spmv(self, x):
        return self._vec_call(load().asm_spmv, x, "spmv")

    def solve(self, b, rtol: float = 1e-8, max_iter: int = 1000, check: bool = False):
        """x with ||b - A x|| <= rtol ||b||; returns (x, info dict)."""
        info = SolveInfo()
        bi, dev = _values(b, 3 * self.n_cells, "solve")
        if dev:
            import torch
            x = torch.empty_like(bi)
        else:
            x = np.empty_like(bi)
        st = load().asm_solve(self._h, _ptr(bi, dev), _ptr(x, dev), rtol, max_iter, int(dev), C.byref(info))
        if st not in (ASM_OK, 4) or (check and st != ASM_OK):
            raise ASMError(st, "solve")
        return x, info.as_dict()

    def stats(self) -> dict:
        s = Stats()
        _check(load().asm_get_stats(self._h, C.byref(s)), "stats")
        return s.as_dict()

    def set_tuning(self, apply_smem: bool | str | None = None, coop_ortho: bool | None = None,
                   autotune: bool | None = None, graphs: bool | None = None, wait_limit_log2: int | None = None,
                   chunk_kb: int | None = None, apply_slots: int | None = None):
        """apply_smem: True / "auto" (default placement), False / "device", "lumps" (lump vector in
        shared memory), "shared" (all local vectors in shared memory); see ASM_TUNE_APPLY_SMEM.
        autotune: the online placement tuner (ASM_TUNE_AUTOTUNE); graphs: CUDA graphs for batched
        solves (ASM_TUNE_GRAPHS); wait_limit_log2: the apply kernels' chunk waits give up after
        2^value polls (0: at once; default 22), a failure-detection hook (ASM_TUNE_WAIT_LIMIT).
        chunk_kb: stream-chunk capacity (0 rule, 8..24 KB; ASM_TUNE_CHUNK_KB, applied by the next
        factor()); apply_slots: the apply's ring slots (0 rule, 2..4; ASM_TUNE_APPLY_SLOTS)."""
        if chunk_kb is not None:
            _check(load().asm_set_tuning(self._h, 5, int(chunk_kb)), "set_tuning")
        if apply_slots is not None:
            _check(load().asm_set_tuning(self._h, 6, int(apply_slots)), "set_tuning")
        if wait_limit_log2 is not None:
            _check(load().asm_set_tuning(self._h, 4, int(wait_limit_log2)), "set_tuning")
        if autotune is not None:
            _check(load().asm_set_tuning(self._h, 2, int(autotune)), "set_tuning")
        if graphs is not None:
            _check(load().asm_set_tuning(self._h, 3, int(graphs)), "set_tuning")
        if apply_smem is not None:
            v = {"device": 0, "auto": 1, "lumps": 2, "shared": 3}[apply_smem] if isinstance(apply_smem, str) \
                else int(apply_smem)
            _check(load().asm_set_tuning(self._h, 0, v), "set_tuning")
        if coop_ortho is not None:
            _check(load().asm_set_tuning(self._h, 1, int(coop_ortho)), "set_tuning")

    def tune_tiling(self, reps: int = 9) -> dict:
        """asm_tune_tiling: measure the apply under every stream-chunk capacity and placement, leave
        the fastest in place (the handle stays factored) and return the measurements."""
        rep = TilingReport()
        _check(load().asm_tune_tiling(self._h, int(reps), C.byref(rep)), "tune_tiling")
        return rep.as_dict()

    def set_profiling(self, on: bool = True):
        _check(load().asm_set_profiling(self._h, 1 if on else 0), "set_profiling")

    def profile(self) -> dict:
        p = Profile()
        _check(load().asm_get_profile(self._h, C.byref(p)), "profile")
        return p.as_dict()

    def reset_profile(self):
        _check(load().asm_reset_profile(self._h), "reset_profile")

    # parity hooks -----------------------------------------------------------------------------
    def local_info(self, s: int):
        n, nnz, lv = C.c_int(), C.c_int(), C.c_int()
        cnt = (C.c_int * 3)()
        _check(load().asm_get_local_info(self._h, s, C.byref(n), C.byref(nnz), cnt, C.byref(lv)), "local_info")
        return {"n": n.value, "nnzb": nnz.value, "counts": tuple(cnt), "levels": lv.value}

    def local_map(self, s: int) -> np.ndarray:
        m = np.empty(self.n_cells, dtype=np.int32)
        _check(load().asm_get_local_map(self._h, s, _host_ptr(m)), "local_map")
        return m

    def local_matrix(self, s: int):
        inf = self.local_info(s)
        rp = np.empty(inf["n"] + 1, dtype=np.int32)
        ci = np.empty(inf["nnzb"], dtype=np.int32)
        v = np.empty((inf["nnzb"], 3, 3))
        _check(load().asm_get_local_matrix(self._h, s, _host_ptr(rp), _host_ptr(ci), _host_ptr(v)), "local_matrix")
        return rp, ci, v

    def nf_diagonal(self, s: int):
        """Nested factorisation: the diagonal blocks G (Eqs. A.6-A.7) of subdomain s, by local row."""
        inf = self.local_info(s)
        g = np.empty((inf["n"], 3, 3))
        _check(load().asm_get_local_factors(self._h, s, None, _host_ptr(g)), "nf_diagonal")
        return g

    def local_factors(self, s: int):
        inf = self.local_info(s)
        lu = np.empty((inf["nnzb"], 3, 3))
        dp = np.empty((inf["n"], 3, 3))
        _check(load().asm_get_local_factors(self._h, s, _host_ptr(lu), _host_ptr(dp)), "local_factors")
        return lu, dp


def _batch_args(solvers, bs, what):
    """handle array, b and x pointer arrays, the x arrays (allocated here), on-device flag, and the
    arrays the pointers refer to (kept alive by the caller)"""
    n = len(solvers)
    if len(bs) != n:
        raise ValueError(f"{what}: one right-hand side per solver")
    hs = (C.c_void_p * n)(*[s.handle for s in solvers])
    on_dev = all(_is_torch(b) and b.is_cuda for b in bs)
    if on_dev:
        import torch
        bi = [_values(b, 3 * s.n_cells, what)[0] for s, b in zip(solvers, bs)]
        xs = [torch.empty_like(b) for b in bi]
        bp = (C.c_void_p * n)(*[b.data_ptr() for b in bi])
        xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    else:  # all on the host (CUDA tensors in a mixed list are copied to the host)
        bi = [np.ascontiguousarray(b.cpu() if _is_torch(b) else b, dtype=np.float64) for b in bs]
        bi = [_values(b, 3 * s.n_cells, what)[0] for s, b in zip(solvers, bi)]
        xs = [np.empty_like(b) for b in bi]
        bp = (C.c_void_p * n)(*[b.ctypes.data for b in bi])
        xp = (C.c_void_p * n)(*[x.ctypes.data for x in xs])
    return hs, bp, xp, xs, on_dev, bi


def solve_batch(solvers, bs, rtol: float = 1e-8, max_iter: int = 1000):
    """Solve several factored systems in the same launches; returns ([x], [info])."""
    n = len(solvers)
    hs, bp, xp, xs, on_dev, _keep = _batch_args(solvers, bs, "solve_batch")
    infos = (SolveInfo * n)()
    st = load().asm_solve_batch(hs, n, bp, xp, rtol, max_iter, 1 if on_dev else 0, infos)
    if st not in (ASM_OK, 4):
        raise ASMError(st, "solve_batch")
    return xs, [i.as_dict() for i in infos]


def tune_tiling_batch(solvers, bs, rtol: float = 1e-8, max_iter: int = 1000) -> dict:
    """asm_tune_tiling_batch: time a batched solve under every stream-chunk capacity, leave the
    fastest in place and return the measurements (apply_ms: the batched solve's time)."""
    n = len(solvers)
    hs, bp, xp, _xs, on_dev, _keep = _batch_args(solvers, bs, "tune_tiling_batch")
    rep = TilingReport()
    _check(load().asm_tune_tiling_batch(hs, n, bp, xp, rtol, max_iter, 1 if on_dev else 0, C.byref(rep)),
           "tune_tiling_batch")
    return rep.as_dict()


@dataclass
class Problem:
    """Convenience: a Solver set up for a grid system and partition."""
    solver: Solver
    n_cells: int


def setup(system, px, py, pz, overlap=1, near_width=2, c_near=(2, 2, 2), far_mode="partition", c_far=None,
          precision="fp64", restart=30, local_solver="colsum", flexible=-1, device=0, factor=True) -> Solver:
    """Solver for a paper_1401_7227_gb300.synth.GridSystem."""
    s = Solver(precision=precision, restart=restart, local_solver=local_solver, flexible=flexible, device=device)
    s.set_grid(system.nx, system.ny, system.nz)
    s.set_matrix(system.row_ptr, system.col_idx, system.vals)
    s.set_partition(px, py, pz, overlap, near_width, c_near, far_mode, c_far)
    if factor:
        s.factor()
    return s


class Server:
    """Continuous-batching serving loop (asm_server_*): submit solves of any grid size as they
    arrive, call progress() to admit and advance them, collect results by ticket."""

    def __init__(self, precision: str = "fp32", restart: int = 30, device: int = 0, max_active: int = 64,
                 max_cached: int = 16, hbm_budget: int = 0, stream: int | None = None, lumps: str = "fp32"):
        L = load()
        o = ServerOptions()
        L.asm_server_default_options(C.byref(o))
        o.precision, o.restart, o.device = PREC[precision], restart, device
        o.max_active, o.max_cached, o.hbm_budget = max_active, max_cached, hbm_budget
        o.lump_precision = LUMPS[lumps]
        self.stream = stream if stream is not None else _current_stream(device)
        h = C.c_void_p()
        _check(L.asm_server_create(C.byref(h), C.byref(o), C.c_void_p(self.stream)), "server_create")
        self._h = h
        self._keep = {}  # ticket -> host arrays borrowed by the request
        self._n = {}

    def close(self):
        if getattr(self, "_h", None):
            load().asm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, system, b, partition=(1, 1, 1), overlap=1, near_width=2, c_near=(2, 2, 2), far_mode="partition",
               c_far=None, rtol=1e-8, max_iter=1000, matrix_key=-1) -> int:
        # host copies: the request borrows these pointers until its result is collected
        host = lambda a: a.detach().cpu() if _is_torch(a) else a  # noqa: E731
        n_cells = system.nx * system.ny * system.nz
        rp = np.ascontiguousarray(host(system.row_ptr), dtype=np.int32).ravel()
        ci = np.ascontiguousarray(host(system.col_idx), dtype=np.int32).ravel()
        if rp.shape[0] != n_cells + 1:
            raise ValueError(f"submit: row_ptr needs {n_cells + 1} entries, got {rp.shape[0]}")
        v, _ = _values(host(system.vals), 9 * ci.shape[0], "submit")
        bb, _ = _values(host(b), 3 * n_cells, "submit")
        q = Request()
        q.nx, q.ny, q.nz = system.nx, system.ny, system.nz
        q.n_cells, q.nnzb = n_cells, ci.shape[0]
        q.row_ptr, q.col_idx, q.vals = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
        q.px, q.py, q.pz = partition
        q.overlap, q.near_width = overlap, near_width
        q.c_near = (C.c_int * 3)(*c_near)
        q.far_mode = FAR[far_mode] if isinstance(far_mode, str) else int(far_mode)
        q.c_far = (C.c_int * 3)(*(c_far if c_far is not None else (1, 1, 1)))
        q.b, q.rtol, q.max_iter, q.matrix_key = bb.ctypes.data, rtol, max_iter, matrix_key
        t = C.c_longlong()
        _check(load().asm_server_submit(self._h, C.byref(q), C.byref(t)), "server_submit")
        self._keep[t.value] = (rp, ci, v)
        self._n[t.value] = q.n_cells
        return t.value

    def progress(self, max_steps: int = 1):
        a, p = C.c_int(), C.c_int()
        _check(load().asm_server_progress(self._h, max_steps, C.byref(a), C.byref(p)), "server_progress")
        return a.value, p.value

    def result(self, ticket: int):
        """(x, info) once the request is finished, else None."""
        x = np.empty(3 * self._n[ticket])
        info = SolveInfo()
        st = load().asm_server_result(self._h, ticket, _host_ptr(x), C.byref(info))
        if st == 8:
            return None
        self._keep.pop(ticket, None)
        self._n.pop(ticket, None)
        _check(st, "server_result")
        return x, info.as_dict()

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().asm_server_get_stats(self._h, C.byref(s)), "server_stats")
        return s.as_dict()
