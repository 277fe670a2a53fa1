"""Seeded synthetic inputs: fully implicit black-oil-like Jacobians on a Cartesian grid.

This module only makes test and benchmark inputs.  It holds none of the preconditioner's or the
solver's arithmetic, so the CPU oracle and the CUDA library can both be fed from it.

The paper's test matrices (ORSREG1 and the SPE1 variants of Section 5, Table 1) are not available,
so these stand in for them with the same character: 3 unknowns per cell (pressure and two
saturations, Section 1), a 7-point stencil of 3x3 blocks, a layered lognormal permeability whose
vertical transmissibility is ~250x the horizontal one (Section 2: vertical flow is the strongest
band), marginal diagonal dominance, a full pressure row and upwinded saturation rows in every
off-diagonal block, and one injector and one producer well.

Cell numbering is z fastest: ``cell = k + nz * (i + nx * j)`` for grid position (i, j, k) =
(x, y, z).  Block columns within a row are sorted ascending, so a row lists its neighbours in the
order -y, -x, -z, diagonal, +z, +x, +y.

Random numbers come from a counter-based splitmix64: draw(seed, field, i) hashes a per-(seed,
field) key with the counter i, so any entry can be regenerated on its own and the stream does not
depend on the order of generation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_KEYMUL = np.uint64(0x100000001B3)
_CTRMUL = np.uint64(0xD1B54A32D192ED03)

# stream ("field") identifiers; each names one independent random stream per seed
F_GLAYER = 1      # per-layer normal of ln k (two fields: Box-Muller pair)
F_GCELL = 3       # per-cell normal of ln k (two fields)
F_PHI = 5         # potential noise (upwind direction)
F_ACC = 6         # accumulation scale, one per component (3 fields)
F_M = 16          # off-diagonal mobility/derivative entries, one field per block entry (9 fields)
F_B = 40          # right-hand side

#: nominal x transmissibility, k = 100 on a 100 x 100 x 2 cell: k * (dy * dz) / dx
T_NOMINAL = 200.0
#: pressure accumulation relative to the cell's transmissibility sum (sets the conditioning:
#: cond(A) ~ 1e4 on the 10 x 10 x 5 grid, inside the 6.7e3 - 2.3e8 range of the paper's Table 1)
EPS_P = 1.0e-3
#: saturation accumulation relative to the cell's transmissibility sum
EPS_S = 0.5
#: well index added to the diagonal of every perforated cell, relative to T_NOMINAL
WELL = 1.0
#: standard deviation of the within-layer (cell) part of ln k; sigma scales the layer part
CELL_NOISE = 0.6


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def draw_u64(seed: int, field: int, idx: np.ndarray) -> np.ndarray:
    """splitmix64 of (stream key XOR scrambled counter); stream key = splitmix64(seed*P + field)."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed], dtype=np.uint64) * _KEYMUL + np.uint64(field) + _GAMMA)[0]
        ctr = np.asarray(idx, dtype=np.uint64) * _CTRMUL
        return _mix((key ^ ctr) + _GAMMA)


def uniform(seed: int, field: int, idx, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Uniform on [lo, hi) from the top 53 bits of the draw."""
    u = (draw_u64(seed, field, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, field: int, idx) -> np.ndarray:
    """Standard normal by Box-Muller from the streams ``field`` and ``field + 1``."""
    u1 = ((draw_u64(seed, field, idx) >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = uniform(seed, field + 1, idx)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class GridSystem:
    """A BSR 3x3 system on an nx x ny x nz grid plus its right-hand side."""

    nx: int
    ny: int
    nz: int
    row_ptr: np.ndarray   # int32 [N+1]
    col_idx: np.ndarray   # int32 [nnzb], ascending within a row
    vals: np.ndarray      # float64 [nnzb, 3, 3], row-major blocks
    b: np.ndarray         # float64 [3N]
    seed: int
    sigma: float

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    def dense(self) -> np.ndarray:
        """Dense (3N x 3N) copy; for tiny grids only."""
        n = self.n_cells
        a = np.zeros((3 * n, 3 * n))
        for r in range(n):
            for e in range(self.row_ptr[r], self.row_ptr[r + 1]):
                c = self.col_idx[e]
                a[3 * r:3 * r + 3, 3 * c:3 * c + 3] = self.vals[e]
        return a


def cell_coords(nx: int, ny: int, nz: int):
    c = np.arange(nx * ny * nz, dtype=np.int64)
    k = c % nz
    i = (c // nz) % nx
    j = c // (nz * nx)
    return c, i, j, k


def rhs(n_cells: int, seed: int) -> np.ndarray:
    """b ~ U[-1, 1] per unknown (3 per cell)."""
    return uniform(seed, F_B, np.arange(3 * n_cells), -1.0, 1.0)


def grid_jacobian(nx: int, ny: int, nz: int, seed: int, sigma: float = 1.0, b_seed: int | None = None,
                  eps_p: float = EPS_P, eps_s: float = EPS_S, cell_noise: float | None = None) -> GridSystem:
    """Anisotropic black-oil-like Jacobian with a 7-point stencil of 3x3 blocks.

    ln k_x = ln 100 + 0.8 sigma g_layer + CELL_NOISE g_cell (sigma sets the layer-to-layer
    contrast of the layered field), k_y = k_x, k_z = 0.1 k_x, cells
    100 x 100 x 2, so T = harmonic-mean(k) * area / distance gives T_z / T_x ~ 250.
    Off-diagonal block (row cell c, neighbour n) = -T_cn * M, with
    M = [[lt, c01, c02], [w1, u*d11, u*d12], [w2, u*d21, u*d22]] and u = 1 when n is upstream of c
    under a seeded potential (injector at column (0,0), producer at (nx-1, ny-1); ties make the
    lower cell index upstream).  The matrix is conservative like a finite-volume Jacobian (the
    material balance of Section 2): every diagonal block is the accumulation minus the sum of the
    off-diagonal blocks in its *column*, so the saturation derivative of an outflow lands on the
    upstream cell's diagonal.  Accumulation = diag(eps_p, eps_s, eps_s) * U[0.5, 1.5] * (the
    cell's transmissibility sum); both well columns add WELL * T_NOMINAL * I on every layer.
    """
    n = nx * ny * nz
    c, i, j, k = cell_coords(nx, ny, nz)
    g_layer = normal(seed, F_GLAYER, np.arange(nz))
    g_cell = normal(seed, F_GCELL, c)
    cn = CELL_NOISE if cell_noise is None else cell_noise
    kx = 100.0 * np.exp(sigma * 0.8 * g_layer[k] + cn * g_cell)
    kz = 0.1 * kx

    fx = i / (nx - 1) if nx > 1 else np.zeros(n)
    fy = j / (ny - 1) if ny > 1 else np.zeros(n)
    phi = 1.0 - 0.5 * (fx + fy) + 0.1 * uniform(seed, F_PHI, c, -1.0, 1.0)

    # neighbour slots in ascending column order: -y, -x, -z, (diag), +z, +x, +y
    offs = [(-nz * nx, j > 0), (-nz, i > 0), (-1, k > 0), (1, k < nz - 1), (nz, i < nx - 1),
            (nz * nx, j < ny - 1)]
    geo = [2.0, 2.0, 5000.0, 5000.0, 2.0, 2.0]      # area / distance per direction
    perm = [kx, kx, kz, kz, kx, kx]

    ts = [np.where(valid, geo[d] * 2.0 * perm[d] * perm[d][np.where(valid, c + off, c)]
                   / (perm[d] + perm[d][np.where(valid, c + off, c)]), 0.0)
          for d, (off, valid) in enumerate(offs)]
    tsum = np.sum(ts, axis=0)
    diag = np.zeros((n, 3, 3))
    acc = np.stack([uniform(seed, F_ACC + m, c, 0.5, 1.5) for m in range(3)], axis=1)
    diag[:, 0, 0] = eps_p * tsum * acc[:, 0]
    diag[:, 1, 1] = eps_s * tsum * acc[:, 1]
    diag[:, 2, 2] = eps_s * tsum * acc[:, 2]
    well = ((i == 0) & (j == 0)) | ((i == nx - 1) & (j == ny - 1))
    for m in range(3):
        diag[well, m, m] += WELL * T_NOMINAL

    blocks = []
    for d, (off, valid) in enumerate(offs):
        nb = np.where(valid, c + off, c)
        t = ts[d]
        up = (phi[nb] > phi) | ((phi[nb] == phi) & (nb < c))
        u = up.astype(np.float64)
        idx = c * 6 + d
        m = np.empty((n, 3, 3))
        m[:, 0, 0] = uniform(seed, F_M + 0, idx, 0.8, 1.2)
        m[:, 0, 1] = uniform(seed, F_M + 1, idx, -0.2, 0.2)
        m[:, 0, 2] = uniform(seed, F_M + 2, idx, -0.2, 0.2)
        m[:, 1, 0] = uniform(seed, F_M + 3, idx, 0.2, 0.6)
        m[:, 2, 0] = uniform(seed, F_M + 4, idx, 0.2, 0.6)
        m[:, 1, 1] = u * uniform(seed, F_M + 5, idx, 0.5, 1.0)
        m[:, 1, 2] = u * uniform(seed, F_M + 6, idx, -0.1, 0.1)
        m[:, 2, 1] = u * uniform(seed, F_M + 7, idx, -0.1, 0.1)
        m[:, 2, 2] = u * uniform(seed, F_M + 8, idx, 0.5, 1.0)
        blk = -t[:, None, None] * m
        # conservative: the diagonal block of column nb collects minus this block
        np.subtract.at(diag, nb[valid], blk[valid])
        blocks.append((valid, nb, blk))

    slots = blocks[:3] + [(np.ones(n, dtype=bool), c, diag)] + blocks[3:]
    valid = np.stack([s[0] for s in slots], axis=1)            # [n, 7]
    cols = np.stack([s[1] for s in slots], axis=1)
    vals = np.stack([s[2] for s in slots], axis=1)             # [n, 7, 3, 3]
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(counts)
    col_idx = cols[valid].astype(np.int32)
    bvals = np.ascontiguousarray(vals[valid])
    b = rhs(n, seed if b_seed is None else b_seed)
    return GridSystem(nx, ny, nz, row_ptr, col_idx, bvals, b, seed, sigma)


# ---------------------------------------------------------------------------------------------
# Named workloads.  Each is (grid, partition, overlap, restart, sigma, seed).
# ---------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    px: int
    py: int
    pz: int
    overlap: int
    restart: int
    sigma: float
    seed: int


WORKLOADS = {
    "grid10x10x5_k4": Workload("grid10x10x5_k4", 10, 10, 5, 2, 2, 1, 1, 30, 1.0, 1),
    "grid64x64x16_k64": Workload("grid64x64x16_k64", 64, 64, 16, 8, 8, 1, 1, 30, 1.0, 2),
    "grid128x128x64_k512": Workload("grid128x128x64_k512", 128, 128, 64, 16, 16, 2, 2, 30, 2.0, 3),
}


def make(w: Workload, b_seed: int | None = None) -> GridSystem:
    return grid_jacobian(w.nx, w.ny, w.nz, w.seed, w.sigma, b_seed=b_seed)


def batch_grid(s_index: int, seed_base: int = 1000):
    """Grid of system s of the batched workload: (8, 8, 4) * scale, scale log-uniform on [1, 6]."""
    sc = math.exp(float(uniform(seed_base + s_index, 99, np.arange(1))[0]) * math.log(6.0))
    nx = max(2, int(round(8 * sc)))
    nz = max(2, int(round(4 * sc)))
    p = min(8, max(2, int(round(nx / 6))))
    return nx, nx, nz, p, p, 1
