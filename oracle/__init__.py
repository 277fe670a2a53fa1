"""ctypes wrapper of the plain FP64 CPU oracle (``asm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg are the only callers.  The CUDA library never imports this package, and this package never
imports the library.

Every routine follows the paper step by step (see the header of ``asm_oracle.c`` for the readings
of points the paper leaves open):

* :func:`local_map`, :func:`owner` -- Section 4, Eq. 4.1 and Figs. 2-3: the fine set, the near and
  far lumps and the local ordering of each subdomain.
* :class:`Precond` -- Eqs. 3.4, 4.1-4.5 and B.3: the local matrices R_s A R_s^T, their block
  ILU(0) with column-sum compensation (Section 2) or exact dense LU (Section 5), and the apply
  B^{-1} r = sum_s P_s R_s^T A_s^{-1} R_s r.
* :func:`gmres`, :func:`orthomin` -- Section 2: the Krylov accelerators, right-preconditioned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")

BILU0_COLSUM = 0
BILU0 = 1
DENSE_LU = 2
NF_COLSUM = 3  # nested factorisation with column-sum compensation (Appendix A, Eq. A.7)
NF = 4         # nested factorisation, G = D - L1 G^{-1} U1 only (Eq. A.6)

OK, ERR_ARG, ERR_PIVOT, ERR_PATTERN, ERR_NOMEM = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle with plain -O2 and no floating-point contraction."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("px", C.c_int), ("py", C.c_int), ("pz", C.c_int),
                ("ov", C.c_int), ("near_width", C.c_int), ("cnear", C.c_int * 3),
                ("far_mode", C.c_int), ("cfar", C.c_int * 3)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("relres", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.orc_pc_create.restype = P
        L.orc_pc_create.argtypes = [C.POINTER(_Geom), P, P, P, C.c_int, C.c_int, C.POINTER(C.c_int), P]
        L.orc_pc_destroy.argtypes = [P]
        L.orc_pc_sub_n.argtypes = [P, C.c_int]
        L.orc_pc_sub_nnz.argtypes = [P, C.c_int]
        L.orc_pc_sub_counts.argtypes = [P, C.c_int, P]
        L.orc_pc_sub_map.argtypes = [P, C.c_int, P]
        L.orc_pc_sub_matrix.argtypes = [P, C.c_int, P, P, P]
        L.orc_pc_sub_factors.argtypes = [P, C.c_int, P, P]
        L.orc_pc_local_solve.argtypes = [P, C.c_int, P, P]
        L.orc_pc_restrict.argtypes = [P, C.c_int, P, P]
        L.orc_pc_apply.argtypes = [P, P, P]
        L.orc_local_map.argtypes = [C.POINTER(_Geom), C.c_int, P, P]
        L.orc_owner.argtypes = [C.POINTER(_Geom), P]
        L.orc_n_sub.argtypes = [C.POINTER(_Geom)]
        L.orc_spmv.argtypes = [C.c_int, P, P, P, P, P]
        L.orc_inv3.argtypes = [P, P]
        L.orc_gmres.argtypes = [C.c_int, P, P, P, P, P, P, C.c_int, C.c_double, C.c_int,
                                C.POINTER(_Info), P]
        L.orc_orthomin.argtypes = L.orc_gmres.argtypes
        L.orc_pc_set_coarse.argtypes = [P, P, P, P, C.c_int, P, C.POINTER(C.c_int)]
        L.orc_pc_coarse_nb.argtypes = [P]
        L.orc_pc_coarse_matrix.argtypes = [P, P, P]
        L.orc_pc_sub_nf.argtypes = [P, C.c_int, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Geometry:
    """Grid, box partition and coarsening parameters of the boundary-conditioned AS (Section 4).

    far_mode: 0 no far field (classical AS, outer cells discarded), 1 far lumps = partition boxes,
    2 far lumps = aligned boxes of size ``cfar``.
    """

    nx: int
    ny: int
    nz: int
    px: int = 1
    py: int = 1
    pz: int = 1
    ov: int = 1
    near_width: int = 2
    cnear: tuple = (2, 2, 2)
    far_mode: int = 1
    cfar: tuple = (0, 0, 0)

    def c(self) -> _Geom:
        return _Geom(self.nx, self.ny, self.nz, self.px, self.py, self.pz, self.ov, self.near_width,
                     (C.c_int * 3)(*self.cnear), self.far_mode, (C.c_int * 3)(*self.cfar))

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_sub(self) -> int:
        return self.px * self.py * self.pz


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def local_map(g: Geometry, s: int):
    """(map[N], (n_fine, n_near, n_far)) of subdomain s."""
    m = np.empty(g.n_cells, dtype=np.int32)
    cnt = np.zeros(3, dtype=np.int32)
    gc = g.c()
    n = lib().orc_local_map(C.byref(gc), s, _p(m), _p(cnt))
    if n < 0:
        raise ValueError(f"oracle: bad geometry ({n})")
    return m, tuple(int(x) for x in cnt)


def owner(g: Geometry) -> np.ndarray:
    o = np.empty(g.n_cells, dtype=np.int32)
    gc = g.c()
    if lib().orc_owner(C.byref(gc), _p(o)) != 0:
        raise ValueError("oracle: bad geometry")
    return o


def spmv(row_ptr, col_idx, vals, x) -> np.ndarray:
    rp, ci, v, x = _i32(row_ptr), _i32(col_idx), _f64(vals), _f64(x)
    n = rp.shape[0] - 1
    y = np.empty(3 * n)
    lib().orc_spmv(n, _p(rp), _p(ci), _p(v), _p(x), _p(y))
    return y


def inv3(a) -> np.ndarray:
    a = _f64(a)
    out = np.empty((3, 3))
    if lib().orc_inv3(_p(a), _p(out)) != 0:
        raise ZeroDivisionError("singular 3x3 block")
    return out


class OracleError(RuntimeError):
    def __init__(self, status, where=None):
        super().__init__(f"oracle status {status} at {where}")
        self.status = status
        self.where = where


NO_COARSE, TWO_LEVEL, TWO_STAGE = 0, 1, 2


class Precond:
    """B^{-1} = sum_s P_s R_s^T A_s^{-1} R_s with A_s = R_s A R_s^T (Eqs. 3.4, 4.1-4.5).

    ``only`` builds a single subdomain (sampled checks on large grids).  ``coarse`` adds the
    classical coarse-grid correction the paper compares with (Section 3): TWO_LEVEL (Eq. 3.5) or
    TWO_STAGE (Eqs. 3.7-3.8), on the partition boxes (``cbox`` None) or aligned boxes of ``cbox``
    cells."""

    def __init__(self, g: Geometry, row_ptr, col_idx, vals, solver: int = BILU0_COLSUM, only: int = -1,
                 coarse: int = NO_COARSE, cbox=None):
        self.g = g
        self.solver = solver
        self.only = only
        self._rp, self._ci, self._v = _i32(row_ptr), _i32(col_idx), _f64(vals)
        st = C.c_int(0)
        loc = np.full(2, -1, dtype=np.int32)
        gc = g.c()
        self._h = lib().orc_pc_create(C.byref(gc), _p(self._rp), _p(self._ci), _p(self._v), solver,
                                      only, C.byref(st), _p(loc))
        if not self._h:
            raise OracleError(st.value, tuple(int(x) for x in loc))
        self.coarse = coarse
        if coarse != NO_COARSE:
            cb = None if cbox is None else np.asarray(cbox, dtype=np.int32)
            bad = C.c_int(-1)
            st = lib().orc_pc_set_coarse(self._h, _p(self._rp), _p(self._ci), _p(self._v), coarse,
                                         None if cb is None else _p(cb), C.byref(bad))
            if st != 0:
                raise OracleError(st, ("coarse", bad.value))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_pc_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def sub_n(self, s: int) -> int:
        return lib().orc_pc_sub_n(self._h, s)

    def sub_counts(self, s: int):
        c = np.zeros(3, dtype=np.int32)
        lib().orc_pc_sub_counts(self._h, s, _p(c))
        return tuple(int(x) for x in c)

    def sub_map(self, s: int) -> np.ndarray:
        m = np.empty(self.g.n_cells, dtype=np.int32)
        lib().orc_pc_sub_map(self._h, s, _p(m))
        return m

    def sub_matrix(self, s: int):
        n, nnz = self.sub_n(s), lib().orc_pc_sub_nnz(self._h, s)
        rp = np.empty(n + 1, dtype=np.int32)
        ci = np.empty(nnz, dtype=np.int32)
        v = np.empty((nnz, 3, 3))
        lib().orc_pc_sub_matrix(self._h, s, _p(rp), _p(ci), _p(v))
        return rp, ci, v

    def sub_factors(self, s: int):
        """(lu, dpiv): L below, U above, D^{-1} on the diagonal of A_s's pattern; pivot blocks."""
        n, nnz = self.sub_n(s), lib().orc_pc_sub_nnz(self._h, s)
        lu = np.empty((nnz, 3, 3))
        dp = np.empty((n, 3, 3))
        if lib().orc_pc_sub_factors(self._h, s, _p(lu), _p(dp)) != 0:
            raise ValueError("no ILU factors for this local solver")
        return lu, dp

    def restrict(self, s: int, r) -> np.ndarray:
        r = _f64(r)
        out = np.empty(3 * self.sub_n(s))
        lib().orc_pc_restrict(self._h, s, _p(r), _p(out))
        return out

    def local_solve(self, s: int, rhs) -> np.ndarray:
        rhs = _f64(rhs)
        out = np.empty_like(rhs)
        lib().orc_pc_local_solve(self._h, s, _p(rhs), _p(out))
        return out

    def sub_nf(self, s: int):
        """Nested factorisation of subdomain s: ((bx, by, bz), G blocks (n, 3, 3)); local cell
        p = z + bz (x + bx y)."""
        dims = np.zeros(3, dtype=np.int32)
        G = np.empty((self.sub_n(s), 3, 3))
        if lib().orc_pc_sub_nf(self._h, s, _p(dims), _p(G)) != 0:
            raise ValueError("no nested factorisation for this local solver")
        return tuple(int(x) for x in dims), G

    def coarse_matrix(self):
        """(A_C as a dense (3 nb, 3 nb) array, coarse box of every cell)."""
        nb = lib().orc_pc_coarse_nb(self._h)
        ac = np.empty((3 * nb, 3 * nb))
        box = np.empty(self.g.n_cells, dtype=np.int32)
        lib().orc_pc_coarse_matrix(self._h, _p(ac), _p(box))
        return ac, box

    def apply(self, r, z=None) -> np.ndarray:
        r = _f64(r)
        if z is None:
            z = np.zeros_like(r)
        lib().orc_pc_apply(self._h, _p(r), _p(z))
        return z


@dataclass
class SolveInfo:
    iters: int
    restarts: int
    converged: bool
    relres: float
    history: np.ndarray


def _krylov(fn, row_ptr, col_idx, vals, b, pc, m, tol, max_iter):
    rp, ci, v, b = _i32(row_ptr), _i32(col_idx), _f64(vals), _f64(b)
    n = rp.shape[0] - 1
    x = np.empty(3 * n)
    info = _Info()
    hist = np.zeros(max_iter + 1)
    st = fn(n, _p(rp), _p(ci), _p(v), pc.handle if pc is not None else None, _p(b), _p(x), m, tol,
            max_iter, C.byref(info), _p(hist))
    if st != 0:
        raise OracleError(st)
    return x, SolveInfo(info.iters, info.restarts, bool(info.converged), info.relres,
                        hist[:info.iters + 1].copy())


def gmres(row_ptr, col_idx, vals, b, pc: Precond | None, m: int = 30, tol: float = 1e-8,
          max_iter: int = 1000):
    """Right-preconditioned GMRES(m) with MGS and Givens rotations, x0 = 0 (Section 2)."""
    return _krylov(lib().orc_gmres, row_ptr, col_idx, vals, b, pc, m, tol, max_iter)


def orthomin(row_ptr, col_idx, vals, b, pc: Precond | None, k: int = 10, tol: float = 1e-8,
             max_iter: int = 1000):
    """Right-preconditioned ORTHOMIN(k), x0 = 0 (Section 2)."""
    return _krylov(lib().orc_orthomin, row_ptr, col_idx, vals, b, pc, k, tol, max_iter)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
