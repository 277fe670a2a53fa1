/*
 * Plain, slow, single-threaded FP64 CPU oracle of the two-level ("boundary conditioning")
 * additive Schwarz preconditioner of Jackson, Taroni & Ponting (arXiv:1401.7227), with block
 * ILU(0) + column-sum compensation as the local solver (or exact dense LU, or the nested
 * factorisation of Appendix A on local problems without lumps), of the classical two-level and
 * two-stage coarse-grid corrections it is compared with (Section 3), and of the GMRES and
 * ORTHOMIN accelerators it is used in.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load this file.  It shares no code with the CUDA library and must stay readable against the
 * paper: no blocking, fusion or reordering beyond what each cited definition states.
 *
 * Conventions (readings of points the paper leaves open):
 *  - cell = k + nz*(i + nx*j) for grid position (i,j,k) = (x,y,z): z fastest (the vertical,
 *    strongest band innermost, Section 2 and Appendix A).
 *  - 3 unknowns per cell, 3x3 blocks stored row-major (Section 1).
 *  - Box partition px*py*pz, part t of n cells in a dimension is [n*t/p, n*(t+1)/p) (floor).
 *    Subdomain s = tz + pz*(tx + px*ty).
 *  - Fine set F_s = owned box grown by `ov` in every dimension, clipped to the grid.
 *  - Near field: the grid is tiled by boxes of cnear[0] x cnear[1] x cnear[2] cells aligned at 0;
 *    every such box that meets the ring (F_s grown by near_width, clipped, minus F_s) gives one
 *    lump: its cells outside F_s.
 *  - Far field: boxes (partition boxes, or cfar-sized aligned boxes); each gives one lump: its
 *    cells in neither F_s nor a near lump.  Empty lumps are dropped.  With far_mode 0 there is no
 *    far field: the remaining cells are left out of the local problem (classical additive
 *    Schwarz with a zero outer boundary, Eqs. 3.3-3.4).
 *  - Local order: F_s cells by ascending global index, then near lumps by box index, then far
 *    lumps by box index; box index = bz + nbz*(bx + nbx*by), like cells.
 *  - A lump sums whole 3x3 blocks (Section 4: coarsening by plain element summation; Appendix B).
 *  - Column-sum compensation: a fill block dropped at (p,q) is subtracted from the diagonal block
 *    (q,q) of its column before pivot q is taken, so E = LU - A has zero block column sums
 *    (Section 2; the colsum form of Eq. A.7).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_PIVOT -2
#define ORC_ERR_PATTERN -3
#define ORC_ERR_NOMEM -4

typedef struct {
    int nx, ny, nz;
    int px, py, pz;
    int ov;
    int near_width;
    int cnear[3];
    int far_mode; /* 0: none, 1: partition boxes, 2: cfar boxes */
    int cfar[3];
} orc_geom;

/* ------------------------------------------------------------------------------------------ */
/* 3x3 block helpers                                                                           */
/* ------------------------------------------------------------------------------------------ */

/* c = a * b */
static void mul3(const double* a, const double* b, double* c) {
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double t = 0.0;
            for (int k = 0; k < 3; k++) t += a[3 * r + k] * b[3 * k + s];
            c[3 * r + s] = t;
        }
}

/* y = a * x for a 3-vector */
static void mulv3(const double* a, const double* x, double* y) {
    for (int r = 0; r < 3; r++) y[r] = a[3 * r] * x[0] + a[3 * r + 1] * x[1] + a[3 * r + 2] * x[2];
}

/* inverse of a 3x3 block by Gauss-Jordan elimination with partial pivoting ("dense sub-matrices
 * inverted directly", Section 2).  Returns 0, or -1 for a zero pivot. */
static int inv3(const double* a, double* inv) {
    double m[3][6];
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            m[r][s] = a[3 * r + s];
            m[r][3 + s] = (r == s) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 3; c++) {
        int piv = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (m[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int s = 0; s < 6; s++) {
                double t = m[c][s];
                m[c][s] = m[piv][s];
                m[piv][s] = t;
            }
        double d = m[c][c];
        for (int s = 0; s < 6; s++) m[c][s] /= d;
        for (int r = 0; r < 3; r++) {
            if (r == c) continue;
            double f = m[r][c];
            if (f == 0.0) continue;
            for (int s = 0; s < 6; s++) m[r][s] -= f * m[c][s];
        }
    }
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) inv[3 * r + s] = m[r][3 + s];
    return 0;
}

int orc_inv3(const double* a, double* inv) { return inv3(a, inv); }

/* ------------------------------------------------------------------------------------------ */
/* Geometry: partition, fine set, near and far lumps (Section 4, Eq. 4.1; Figs. 2-3)           */
/* ------------------------------------------------------------------------------------------ */

static int split_lo(int n, int p, int t) { return (int)(((long long)n * t) / p); }

static int imax(int a, int b) { return a > b ? a : b; }
static int imin(int a, int b) { return a < b ? a : b; }

typedef struct {
    int lo[3], hi[3]; /* half-open, dimension order x, y, z */
} box3;

static int in_box(const box3* b, int x, int y, int z) {
    return x >= b->lo[0] && x < b->hi[0] && y >= b->lo[1] && y < b->hi[1] && z >= b->lo[2] &&
           z < b->hi[2];
}

static int geom_ok(const orc_geom* g) {
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return 0;
    if (g->px < 1 || g->py < 1 || g->pz < 1) return 0;
    if (g->px > g->nx || g->py > g->ny || g->pz > g->nz) return 0;
    if (g->ov < 0 || g->near_width < 0) return 0;
    if (g->near_width > 0 && (g->cnear[0] < 1 || g->cnear[1] < 1 || g->cnear[2] < 1)) return 0;
    if (g->far_mode < 0 || g->far_mode > 2) return 0;
    if (g->far_mode == 2 && (g->cfar[0] < 1 || g->cfar[1] < 1 || g->cfar[2] < 1)) return 0;
    return 1;
}

static box3 owned_box(const orc_geom* g, int s) {
    int tz = s % g->pz, tx = (s / g->pz) % g->px, ty = s / (g->pz * g->px);
    box3 b;
    b.lo[0] = split_lo(g->nx, g->px, tx);
    b.hi[0] = split_lo(g->nx, g->px, tx + 1);
    b.lo[1] = split_lo(g->ny, g->py, ty);
    b.hi[1] = split_lo(g->ny, g->py, ty + 1);
    b.lo[2] = split_lo(g->nz, g->pz, tz);
    b.hi[2] = split_lo(g->nz, g->pz, tz + 1);
    return b;
}

static box3 grow_clip(const orc_geom* g, box3 b, int w) {
    int n[3] = {g->nx, g->ny, g->nz};
    for (int d = 0; d < 3; d++) {
        b.lo[d] = imax(0, b.lo[d] - w);
        b.hi[d] = imin(n[d], b.hi[d] + w);
    }
    return b;
}

int orc_n_sub(const orc_geom* g) { return g->px * g->py * g->pz; }

/* owner[c] = subdomain whose owned box holds cell c */
int orc_owner(const orc_geom* g, int* owner) {
    if (!geom_ok(g)) return ORC_ERR_ARG;
    int K = orc_n_sub(g);
    for (int s = 0; s < K; s++) {
        box3 b = owned_box(g, s);
        for (int j = b.lo[1]; j < b.hi[1]; j++)
            for (int i = b.lo[0]; i < b.hi[0]; i++)
                for (int k = b.lo[2]; k < b.hi[2]; k++) owner[k + g->nz * (i + g->nx * j)] = s;
    }
    return ORC_OK;
}

/* map[c] = local unknown (block) index of cell c in subdomain s, or -1 when c is outside the
 * local problem.  counts[0..2] = number of fine cells, near lumps, far lumps.  Returns n_s. */
int orc_local_map(const orc_geom* g, int s, int* map, int* counts) {
    if (!geom_ok(g)) return ORC_ERR_ARG;
    if (s < 0 || s >= orc_n_sub(g)) return ORC_ERR_ARG;
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const int N = nx * ny * nz;
    for (int c = 0; c < N; c++) map[c] = -1;

    box3 own = owned_box(g, s);
    box3 fine = grow_clip(g, own, g->ov);
    box3 outer = grow_clip(g, fine, g->near_width);
    int idx = 0;

    /* fine cells, ascending global index */
    for (int c = 0; c < N; c++) {
        int k = c % nz, i = (c / nz) % nx, j = c / (nz * nx);
        if (in_box(&fine, i, j, k)) map[c] = idx++;
    }
    int n_fine = idx;

    /* near lumps: aligned cnear boxes meeting the ring outer \ fine */
    int n_near = 0;
    if (g->near_width > 0) {
        const int cx = g->cnear[0], cy = g->cnear[1], cz = g->cnear[2];
        const int nbx = (nx + cx - 1) / cx, nby = (ny + cy - 1) / cy, nbz = (nz + cz - 1) / cz;
        for (int bj = 0; bj < nby; bj++)
            for (int bi = 0; bi < nbx; bi++)
                for (int bk = 0; bk < nbz; bk++) {
                    box3 b = {{bi * cx, bj * cy, bk * cz},
                              {imin(nx, (bi + 1) * cx), imin(ny, (bj + 1) * cy), imin(nz, (bk + 1) * cz)}};
                    int meets = 0;
                    for (int j = b.lo[1]; j < b.hi[1]; j++)
                        for (int i = b.lo[0]; i < b.hi[0]; i++)
                            for (int k = b.lo[2]; k < b.hi[2]; k++)
                                if (in_box(&outer, i, j, k) && !in_box(&fine, i, j, k)) meets = 1;
                    if (!meets) continue;
                    for (int j = b.lo[1]; j < b.hi[1]; j++)
                        for (int i = b.lo[0]; i < b.hi[0]; i++)
                            for (int k = b.lo[2]; k < b.hi[2]; k++)
                                if (!in_box(&fine, i, j, k)) map[k + nz * (i + nx * j)] = idx;
                    idx++;
                    n_near++;
                }
    }

    /* far lumps: the remaining cells of each far box */
    int n_far = 0;
    if (g->far_mode != 0) {
        int nb;
        if (g->far_mode == 1)
            nb = orc_n_sub(g);
        else
            nb = ((nx + g->cfar[0] - 1) / g->cfar[0]) * ((ny + g->cfar[1] - 1) / g->cfar[1]) *
                 ((nz + g->cfar[2] - 1) / g->cfar[2]);
        for (int t = 0; t < nb; t++) {
            box3 b;
            if (g->far_mode == 1) {
                b = owned_box(g, t);
            } else {
                const int cx = g->cfar[0], cy = g->cfar[1], cz = g->cfar[2];
                const int nbx = (nx + cx - 1) / cx, nbz = (nz + cz - 1) / cz;
                int bk = t % nbz, bi = (t / nbz) % nbx, bj = t / (nbz * nbx);
                b.lo[0] = bi * cx;
                b.hi[0] = imin(nx, (bi + 1) * cx);
                b.lo[1] = bj * cy;
                b.hi[1] = imin(ny, (bj + 1) * cy);
                b.lo[2] = bk * cz;
                b.hi[2] = imin(nz, (bk + 1) * cz);
            }
            int any = 0;
            for (int j = b.lo[1]; j < b.hi[1]; j++)
                for (int i = b.lo[0]; i < b.hi[0]; i++)
                    for (int k = b.lo[2]; k < b.hi[2]; k++) {
                        int c = k + nz * (i + nx * j);
                        if (map[c] == -1) {
                            map[c] = idx;
                            any = 1;
                        }
                    }
            if (any) {
                idx++;
                n_far++;
            }
        }
    }
    if (counts) {
        counts[0] = n_fine;
        counts[1] = n_near;
        counts[2] = n_far;
    }
    return idx;
}

/* ------------------------------------------------------------------------------------------ */
/* Local matrices A_s = R_s A R_s^T (Eq. 3.4 with R_s of Eq. 4.1; Eq. B.3)                     */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int n;        /* block rows */
    int nnz;      /* blocks */
    int* rp;      /* [n+1] */
    int* ci;      /* [nnz], ascending in a row */
    int* diag;    /* [n] position of (p,p) */
    double* v;    /* [nnz*9] */
} bsr_t;

static void bsr_free(bsr_t* m) {
    free(m->rp);
    free(m->ci);
    free(m->diag);
    free(m->v);
    memset(m, 0, sizeof(*m));
}

/* position of (p,q) in m, or -1 */
static int bsr_find(const bsr_t* m, int p, int q) {
    int lo = m->rp[p], hi = m->rp[p + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (m->ci[mid] == q) return mid;
        if (m->ci[mid] < q)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

static int cmp_pair(const void* a, const void* b) {
    const long long x = *(const long long*)a, y = *(const long long*)b;
    return (x > y) - (x < y);
}

/* A_s[p,q] = sum over cells a in p, b in q of A[a,b], by direct summation over A's blocks in
 * row order; pattern = every (p,q) that receives a block of A. */
static int assemble_local(int N, const int* rp, const int* ci, const double* v, const int* map, int n,
                          bsr_t* out) {
    memset(out, 0, sizeof(*out));
    long long npair = 0;
    for (int a = 0; a < N; a++)
        if (map[a] >= 0)
            for (int e = rp[a]; e < rp[a + 1]; e++)
                if (map[ci[e]] >= 0) npair++;
    long long* pairs = (long long*)malloc(sizeof(long long) * (size_t)(npair > 0 ? npair : 1));
    if (!pairs) return ORC_ERR_NOMEM;
    long long w = 0;
    for (int a = 0; a < N; a++)
        if (map[a] >= 0)
            for (int e = rp[a]; e < rp[a + 1]; e++)
                if (map[ci[e]] >= 0) pairs[w++] = (long long)map[a] * n + map[ci[e]];
    qsort(pairs, (size_t)npair, sizeof(long long), cmp_pair);
    int nnz = 0;
    for (long long t = 0; t < npair; t++)
        if (t == 0 || pairs[t] != pairs[t - 1]) pairs[nnz++] = pairs[t];
    out->n = n;
    out->nnz = nnz;
    out->rp = (int*)calloc((size_t)n + 1, sizeof(int));
    out->ci = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    out->diag = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    out->v = (double*)calloc((size_t)nnz * 9 + 1, sizeof(double));
    if (!out->rp || !out->ci || !out->diag || !out->v) {
        free(pairs);
        bsr_free(out);
        return ORC_ERR_NOMEM;
    }
    for (int t = 0; t < nnz; t++) {
        int p = (int)(pairs[t] / n);
        out->ci[t] = (int)(pairs[t] % n);
        out->rp[p + 1]++;
    }
    free(pairs);
    for (int p = 0; p < n; p++) out->rp[p + 1] += out->rp[p];
    for (int p = 0; p < n; p++) {
        out->diag[p] = bsr_find(out, p, p);
        if (out->diag[p] < 0) {
            bsr_free(out);
            return ORC_ERR_PATTERN;
        }
    }
    /* values: direct summation over A's blocks */
    for (int a = 0; a < N; a++) {
        if (map[a] < 0) continue;
        for (int e = rp[a]; e < rp[a + 1]; e++) {
            int q = map[ci[e]];
            if (q < 0) continue;
            int pos = bsr_find(out, map[a], q);
            for (int t = 0; t < 9; t++) out->v[9 * (size_t)pos + t] += v[9 * (size_t)e + t];
        }
    }
    /* the factorisation below reads column k through row k's pattern: require symmetry */
    for (int p = 0; p < n; p++)
        for (int t = out->rp[p]; t < out->rp[p + 1]; t++)
            if (bsr_find(out, out->ci[t], p) < 0) {
                bsr_free(out);
                return ORC_ERR_PATTERN;
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Local solvers                                                                               */
/* ------------------------------------------------------------------------------------------ */

enum { ORC_BILU0_COLSUM = 0, ORC_BILU0 = 1, ORC_DENSE_LU = 2, ORC_NF_COLSUM = 3, ORC_NF = 4 };

/* Right-looking block ILU(0) (Section 2: ILU with zero fill on the 3x3 block structure, the
 * diagonal blocks inverted directly), in place on m.  With colsum != 0, every fill block that
 * falls outside the pattern is moved to the diagonal block of its column, so that E = LU - A has
 * zero block column sums (Section 2; the colsum choice of Eq. A.7).
 * On return, for q < p: L_pq; for q > p: U_pq; at (p,p): D_p^{-1}.  dpiv (n*9) receives the
 * final pivot blocks D_p.  Returns 0, or ORC_ERR_PIVOT with *bad_row = the singular pivot. */
static int bilu0_factor(bsr_t* m, int colsum, double* dpiv, int* bad_row) {
    const int n = m->n;
    double Dinv[9], F[9];
    for (int k = 0; k < n; k++) {
        double* Akk = m->v + 9 * (size_t)m->diag[k];
        if (dpiv) memcpy(dpiv + 9 * (size_t)k, Akk, sizeof(double) * 9);
        if (inv3(Akk, Dinv)) {
            *bad_row = k;
            return ORC_ERR_PIVOT;
        }
        memcpy(Akk, Dinv, sizeof(Dinv));
        /* column k below the diagonal: L_pk = A_pk D_k^{-1} (column pattern = row pattern) */
        for (int t = m->diag[k] + 1; t < m->rp[k + 1]; t++) {
            int p = m->ci[t];
            double* Apk = m->v + 9 * (size_t)bsr_find(m, p, k);
            double tmp[9];
            mul3(Apk, Dinv, tmp);
            memcpy(Apk, tmp, sizeof(tmp));
        }
        /* Schur update of the trailing pattern */
        for (int tq = m->diag[k] + 1; tq < m->rp[k + 1]; tq++) {
            int q = m->ci[tq];
            const double* Akq = m->v + 9 * (size_t)tq;
            for (int tp = m->diag[k] + 1; tp < m->rp[k + 1]; tp++) {
                int p = m->ci[tp];
                const double* Lpk = m->v + 9 * (size_t)bsr_find(m, p, k);
                mul3(Lpk, Akq, F);
                int pos = bsr_find(m, p, q);
                double* tgt;
                if (pos >= 0)
                    tgt = m->v + 9 * (size_t)pos; /* in the pattern */
                else if (colsum)
                    tgt = m->v + 9 * (size_t)m->diag[q]; /* dropped: into column q's diagonal */
                else
                    continue; /* dropped */
                for (int e = 0; e < 9; e++) tgt[e] -= F[e];
            }
        }
    }
    return 0;
}

/* forward L y = rhs (unit lower), then backward z_p = D_p^{-1} (y_p - sum_{q>p} U_pq z_q) */
static void bilu0_solve(const bsr_t* m, const double* rhs, double* z) {
    const int n = m->n;
    double* y = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int p = 0; p < n; p++) {
        double acc[3] = {rhs[3 * p], rhs[3 * p + 1], rhs[3 * p + 2]};
        for (int t = m->rp[p]; t < m->diag[p]; t++) {
            double tmp[3];
            mulv3(m->v + 9 * (size_t)t, y + 3 * (size_t)m->ci[t], tmp);
            for (int r = 0; r < 3; r++) acc[r] -= tmp[r];
        }
        for (int r = 0; r < 3; r++) y[3 * p + r] = acc[r];
    }
    for (int p = n - 1; p >= 0; p--) {
        double acc[3] = {y[3 * p], y[3 * p + 1], y[3 * p + 2]};
        for (int t = m->diag[p] + 1; t < m->rp[p + 1]; t++) {
            double tmp[3];
            mulv3(m->v + 9 * (size_t)t, z + 3 * (size_t)m->ci[t], tmp);
            for (int r = 0; r < 3; r++) acc[r] -= tmp[r];
        }
        mulv3(m->v + 9 * (size_t)m->diag[p], acc, z + 3 * (size_t)p);
    }
    free(y);
}

/* Dense LU with partial pivoting of the scalar 3n x 3n local matrix: the exact Gaussian
 * elimination of the local problems used for the paper's experiments (Section 5). */
typedef struct {
    int n3;
    double* a;  /* n3*n3 row-major LU */
    int* piv;
} dense_lu_t;

static int dense_alloc(dense_lu_t* d, int n3) {
    d->n3 = n3;
    d->a = (double*)calloc((size_t)n3 * n3 + 1, sizeof(double));
    d->piv = (int*)malloc(sizeof(int) * (size_t)(n3 > 0 ? n3 : 1));
    return (!d->a || !d->piv) ? ORC_ERR_NOMEM : ORC_OK;
}

/* Gaussian elimination with partial pivoting (whole rows swapped) of the filled d->a, in place:
 * unit-lower multipliers below the diagonal, U on and above it.  *bad_row = block row of a zero
 * pivot. */
static int dense_factor(dense_lu_t* d, int* bad_row) {
    const int n3 = d->n3;
    double* a = d->a;
    for (int c = 0; c < n3; c++) {
        int pr = c;
        for (int r = c + 1; r < n3; r++)
            if (fabs(a[(size_t)r * n3 + c]) > fabs(a[(size_t)pr * n3 + c])) pr = r;
        d->piv[c] = pr;
        if (a[(size_t)pr * n3 + c] == 0.0) {
            *bad_row = c / 3;
            return ORC_ERR_PIVOT;
        }
        if (pr != c)
            for (int s = 0; s < n3; s++) {
                double t = a[(size_t)c * n3 + s];
                a[(size_t)c * n3 + s] = a[(size_t)pr * n3 + s];
                a[(size_t)pr * n3 + s] = t;
            }
        for (int r = c + 1; r < n3; r++) {
            double f = a[(size_t)r * n3 + c] / a[(size_t)c * n3 + c];
            a[(size_t)r * n3 + c] = f;
            if (f != 0.0)
                for (int s = c + 1; s < n3; s++) a[(size_t)r * n3 + s] -= f * a[(size_t)c * n3 + s];
        }
    }
    return 0;
}

static int dense_lu_factor(const bsr_t* m, dense_lu_t* d, int* bad_row) {
    const int n3 = 3 * m->n;
    if (dense_alloc(d, n3)) return ORC_ERR_NOMEM;
    double* a = d->a;
    for (int p = 0; p < m->n; p++)
        for (int t = m->rp[p]; t < m->rp[p + 1]; t++)
            for (int r = 0; r < 3; r++)
                for (int s = 0; s < 3; s++)
                    a[(size_t)(3 * p + r) * n3 + 3 * m->ci[t] + s] = m->v[9 * (size_t)t + 3 * r + s];
    return dense_factor(d, bad_row);
}

static void dense_lu_solve(const dense_lu_t* d, const double* rhs, double* x) {
    const int n3 = d->n3;
    const double* a = d->a;
    for (int r = 0; r < n3; r++) x[r] = rhs[r];
    /* the factorisation swapped whole rows, so all interchanges come first */
    for (int c = 0; c < n3; c++) {
        int pr = d->piv[c];
        if (pr != c) {
            double t = x[c];
            x[c] = x[pr];
            x[pr] = t;
        }
    }
    for (int c = 0; c < n3; c++)
        for (int r = c + 1; r < n3; r++) x[r] -= a[(size_t)r * n3 + c] * x[c];
    for (int r = n3 - 1; r >= 0; r--) {
        double acc = x[r];
        for (int s = r + 1; s < n3; s++) acc -= a[(size_t)r * n3 + s] * x[s];
        x[r] = acc / a[(size_t)r * n3 + r];
    }
}


/* ------------------------------------------------------------------------------------------ */
/* Nested factorisation (Appendix A) of a local matrix on a box of bx * by * bz cells           */
/* ------------------------------------------------------------------------------------------ */
/* Local cell p = z + bz*(x + bx*y) (the local order of a box without lumps).  The hepta-banded
 * A = D + L1 + U1 + L2 + U2 + L3 + U3 (Eq. A.1) is held per cell: D[p] = A(p,p), L1[p] = A(p,p-1),
 * U1[p] = A(p,p+1), L2[p] = A(p,p-bz), U2[p] = A(p,p+bz), L3[p] = A(p,p-S), U3[p] = A(p,p+S),
 * S = bz*bx (zero blocks where a neighbour is missing).  The preconditioner (Eqs. A.2-A.4) is
 *   B = (P + L3)(I + P^{-1} U3),  P = (T + L2)(I + T^{-1} U2),  T = (G + L1)(I + G^{-1} U1)
 * with G block diagonal: G = D - L1 G^{-1} U1 (Eq. A.6), and with colsum (Eq. A.7) also minus the
 * block column sums of L2 T^{-1} U2 and of L3 P^{-1} U3.  T is block diagonal over the lines of a
 * plane (each line a block tridiagonal factor), P block diagonal over the planes. */
typedef struct {
    int bx, by, bz, n;
    double *D, *L1, *U1, *L2, *U2, *L3, *U3, *G, *Gi; /* [n*9] each */
} nf_t;

static void nf_free(nf_t* f) {
    free(f->D);
    free(f->L1);
    free(f->U1);
    free(f->L2);
    free(f->U2);
    free(f->L3);
    free(f->U3);
    free(f->G);
    free(f->Gi);
    memset(f, 0, sizeof(*f));
}

static void sub3(double* a, const double* b) { /* a -= b */
    for (int e = 0; e < 9; e++) a[e] -= b[e];
}
static void mulv3_sub(double* y, const double* a, const double* x) { /* y -= a x (3-vectors) */
    double t[3];
    mulv3(a, x, t);
    for (int r = 0; r < 3; r++) y[r] -= t[r];
}

/* T^{-1} b on the line starting at cell q0 (b, out: 3-vectors of the line's bz cells) */
static void nf_line_solve(const nf_t* f, int q0, const double* b, double* out) {
    const int bz = f->bz;
    double* s = (double*)malloc(sizeof(double) * 3 * (size_t)bz);
    for (int q = 0; q < bz; q++) { /* (G + L1) s = b */
        double t[3] = {b[3 * q], b[3 * q + 1], b[3 * q + 2]};
        if (q > 0) mulv3_sub(t, f->L1 + 9 * (size_t)(q0 + q), s + 3 * (q - 1));
        mulv3(f->Gi + 9 * (size_t)(q0 + q), t, s + 3 * q);
    }
    for (int q = bz - 1; q >= 0; q--) { /* (I + G^{-1} U1) out = s */
        double t[3] = {s[3 * q], s[3 * q + 1], s[3 * q + 2]};
        if (q < bz - 1) {
            double u[3], w[3];
            mulv3(f->U1 + 9 * (size_t)(q0 + q), out + 3 * (q + 1), u);
            mulv3(f->Gi + 9 * (size_t)(q0 + q), u, w);
            for (int r = 0; r < 3; r++) t[r] -= w[r];
        }
        for (int r = 0; r < 3; r++) out[3 * q + r] = t[r];
    }
    free(s);
}

/* W = u T^{-1} for a row of 3x3 blocks u over the line starting at q0 (W T = u) */
static void nf_line_solve_row(const nf_t* f, int q0, const double* u, double* W) {
    const int bz = f->bz;
    double* v = (double*)malloc(sizeof(double) * 9 * (size_t)bz);
    double t[9], t2[9];
    for (int q = 0; q < bz; q++) { /* v (I + G^{-1} U1) = u */
        memcpy(v + 9 * q, u + 9 * q, sizeof(double) * 9);
        if (q > 0) {
            mul3(v + 9 * (q - 1), f->Gi + 9 * (size_t)(q0 + q - 1), t);
            mul3(t, f->U1 + 9 * (size_t)(q0 + q - 1), t2);
            sub3(v + 9 * q, t2);
        }
    }
    for (int q = bz - 1; q >= 0; q--) { /* W (G + L1) = v */
        memcpy(t, v + 9 * q, sizeof(double) * 9);
        if (q < bz - 1) {
            mul3(W + 9 * (q + 1), f->L1 + 9 * (size_t)(q0 + q + 1), t2);
            sub3(t, t2);
        }
        mul3(t, f->Gi + 9 * (size_t)(q0 + q), W + 9 * q);
    }
    free(v);
}

/* P^{-1} b on the plane starting at cell c0 (3-vectors of its S cells) */
static void nf_plane_solve(const nf_t* f, int c0, const double* b, double* out) {
    const int bz = f->bz, bx = f->bx, S = bz * bx;
    double* z = (double*)malloc(sizeof(double) * 3 * (size_t)S);
    double* t = (double*)malloc(sizeof(double) * 3 * (size_t)bz);
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)bz);
    for (int l = 0; l < bx; l++) { /* (T + L2) z = b */
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            for (int r = 0; r < 3; r++) t[3 * q + r] = b[3 * c + r];
            if (l > 0) mulv3_sub(t + 3 * q, f->L2 + 9 * (size_t)(c0 + c), z + 3 * (c - bz));
        }
        nf_line_solve(f, c0 + l * bz, t, z + 3 * l * bz);
    }
    for (int l = bx - 1; l >= 0; l--) { /* (I + T^{-1} U2) out = z */
        if (l == bx - 1) {
            memcpy(out + 3 * l * bz, z + 3 * l * bz, sizeof(double) * 3 * (size_t)bz);
            continue;
        }
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            mulv3(f->U2 + 9 * (size_t)(c0 + c), out + 3 * (c + bz), t + 3 * q);
        }
        nf_line_solve(f, c0 + l * bz, t, w);
        for (int i = 0; i < 3 * bz; i++) out[3 * l * bz + i] = z[3 * l * bz + i] - w[i];
    }
    free(z);
    free(t);
    free(w);
}

/* W = u P^{-1} for a row of 3x3 blocks u over the plane starting at c0 (W P = u) */
static void nf_plane_solve_row(const nf_t* f, int c0, const double* u, double* W) {
    const int bz = f->bz, bx = f->bx, S = bz * bx;
    double* v = (double*)malloc(sizeof(double) * 9 * (size_t)S);
    double* x = (double*)malloc(sizeof(double) * 9 * (size_t)bz);
    double* y = (double*)malloc(sizeof(double) * 9 * (size_t)bz);
    double t[9];
    for (int l = 0; l < bx; l++) { /* v (I + T^{-1} U2) = u: v_l = u_l - (v_{l-1} T^{-1}) U2 */
        memcpy(v + 9 * (size_t)l * bz, u + 9 * (size_t)l * bz, sizeof(double) * 9 * (size_t)bz);
        if (l > 0) {
            nf_line_solve_row(f, c0 + (l - 1) * bz, v + 9 * (size_t)(l - 1) * bz, x);
            for (int q = 0; q < bz; q++) {
                mul3(x + 9 * q, f->U2 + 9 * (size_t)(c0 + (l - 1) * bz + q), t);
                sub3(v + 9 * ((size_t)l * bz + q), t);
            }
        }
    }
    for (int l = bx - 1; l >= 0; l--) { /* W (T + L2) = v: W_l = (v_l - W_{l+1} L2) T^{-1} */
        memcpy(y, v + 9 * (size_t)l * bz, sizeof(double) * 9 * (size_t)bz);
        if (l < bx - 1)
            for (int q = 0; q < bz; q++) {
                mul3(W + 9 * ((size_t)(l + 1) * bz + q), f->L2 + 9 * (size_t)(c0 + (l + 1) * bz + q), t);
                sub3(y + 9 * q, t);
            }
        nf_line_solve_row(f, c0 + l * bz, y, W + 9 * (size_t)l * bz);
    }
    free(v);
    free(x);
    free(y);
}

/* Factor: the G blocks, plane by plane, line by line, cell by cell (Eqs. A.6 / A.7). */
static int nf_factor(nf_t* f, int colsum, int* bad_row) {
    const int bz = f->bz, bx = f->bx, by = f->by, S = bz * bx;
    double* cs = (double*)calloc(9 * (size_t)S, sizeof(double)); /* colsum terms of one line/plane */
    double* u = (double*)malloc(sizeof(double) * 9 * (size_t)S);
    double* W = (double*)malloc(sizeof(double) * 9 * (size_t)S);
    double t[9], t2[9];
    for (int j = 0; j < by; j++) {
        const int c0 = j * S;
        /* colsum(L3 P^{-1} U3) on plane j: W3 = u3 P_{j-1}^{-1}, u3[c'] = L3[c'+S]; term[c] = W3[c-S] U3[c-S] */
        double* cs3 = (double*)calloc(9 * (size_t)S, sizeof(double));
        if (colsum && j > 0) {
            for (int c = 0; c < S; c++) memcpy(u + 9 * c, f->L3 + 9 * (size_t)(c0 + c), sizeof(double) * 9);
            nf_plane_solve_row(f, c0 - S, u, W);
            for (int c = 0; c < S; c++) mul3(W + 9 * c, f->U3 + 9 * (size_t)(c0 - S + c), cs3 + 9 * c);
        }
        for (int l = 0; l < bx; l++) {
            const int q0 = c0 + l * bz;
            /* colsum(L2 T^{-1} U2) on line l: W2 = u2 T_{l-1}^{-1}, u2[q'] = L2[q'+bz]; term[q] = W2[q-bz] U2[q-bz] */
            memset(cs, 0, sizeof(double) * 9 * (size_t)bz);
            if (colsum && l > 0) {
                for (int q = 0; q < bz; q++) memcpy(u + 9 * q, f->L2 + 9 * (size_t)(q0 + q), sizeof(double) * 9);
                nf_line_solve_row(f, q0 - bz, u, W);
                for (int q = 0; q < bz; q++) mul3(W + 9 * q, f->U2 + 9 * (size_t)(q0 - bz + q), cs + 9 * q);
            }
            for (int q = 0; q < bz; q++) {
                const int p = q0 + q;
                double* G = f->G + 9 * (size_t)p;
                memcpy(G, f->D + 9 * (size_t)p, sizeof(double) * 9);
                if (q > 0) { /* - L1 G^{-1} U1 */
                    mul3(f->L1 + 9 * (size_t)p, f->Gi + 9 * (size_t)(p - 1), t);
                    mul3(t, f->U1 + 9 * (size_t)(p - 1), t2);
                    sub3(G, t2);
                }
                sub3(G, cs + 9 * q);
                sub3(G, cs3 + 9 * (size_t)(l * bz + q));
                if (inv3(G, f->Gi + 9 * (size_t)p)) {
                    *bad_row = p;
                    free(cs3);
                    free(cs);
                    free(u);
                    free(W);
                    return ORC_ERR_PIVOT;
                }
            }
        }
        free(cs3);
    }
    free(cs);
    free(u);
    free(W);
    return ORC_OK;
}

/* B^{-1} r: (P + L3) y = r plane by plane, then (I + P^{-1} U3) x = y */
static void nf_solve(const nf_t* f, const double* r, double* x) {
    const int S = f->bz * f->bx, by = f->by;
    double* y = (double*)malloc(sizeof(double) * 3 * (size_t)f->n);
    double* t = (double*)malloc(sizeof(double) * 3 * (size_t)S);
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)S);
    for (int j = 0; j < by; j++) {
        for (int c = 0; c < S; c++) {
            for (int k = 0; k < 3; k++) t[3 * c + k] = r[3 * ((size_t)j * S + c) + k];
            if (j > 0) mulv3_sub(t + 3 * c, f->L3 + 9 * ((size_t)j * S + c), y + 3 * ((size_t)(j - 1) * S + c));
        }
        nf_plane_solve(f, j * S, t, y + 3 * (size_t)j * S);
    }
    for (int j = by - 1; j >= 0; j--) {
        if (j == by - 1) {
            memcpy(x + 3 * (size_t)j * S, y + 3 * (size_t)j * S, sizeof(double) * 3 * (size_t)S);
            continue;
        }
        for (int c = 0; c < S; c++) mulv3(f->U3 + 9 * ((size_t)j * S + c), x + 3 * ((size_t)(j + 1) * S + c), t + 3 * c);
        nf_plane_solve(f, j * S, t, w);
        for (int i = 0; i < 3 * S; i++) x[3 * (size_t)j * S + i] = y[3 * (size_t)j * S + i] - w[i];
    }
    free(y);
    free(t);
    free(w);
}

/* Bands of a box's local matrix; ORC_ERR_PATTERN if A_s has a block outside the seven bands. */
static int nf_setup(const bsr_t* A, int bx, int by, int bz, nf_t* f) {
    f->bx = bx;
    f->by = by;
    f->bz = bz;
    f->n = bx * by * bz;
    if (f->n != A->n) return ORC_ERR_ARG;
    double** band[7] = {&f->D, &f->L1, &f->U1, &f->L2, &f->U2, &f->L3, &f->U3};
    for (int k = 0; k < 7; k++) {
        *band[k] = (double*)calloc(9 * (size_t)f->n + 1, sizeof(double));
        if (!*band[k]) return ORC_ERR_NOMEM;
    }
    f->G = (double*)calloc(9 * (size_t)f->n + 1, sizeof(double));
    f->Gi = (double*)calloc(9 * (size_t)f->n + 1, sizeof(double));
    if (!f->G || !f->Gi) return ORC_ERR_NOMEM;
    const int S = bz * bx;
    /* the band of an entry follows from the two cells' box coordinates (z, x, y): neighbours in z
     * are L1/U1, in x L2/U2, in y L3/U3 (an index offset alone is ambiguous when bz or bx is 1) */
    for (int p = 0; p < f->n; p++) {
        const int pz = p % bz, px = (p / bz) % bx, py = p / S;
        for (int e = A->rp[p]; e < A->rp[p + 1]; e++) {
            const int q = A->ci[e];
            const int dz = q % bz - pz, dx = (q / bz) % bx - px, dy = q / S - py;
            double* dst = NULL;
            if (dx == 0 && dy == 0 && (dz == 0 || dz == -1 || dz == 1))
                dst = dz == 0 ? f->D : dz < 0 ? f->L1 : f->U1;
            else if (dz == 0 && dy == 0 && (dx == -1 || dx == 1))
                dst = dx < 0 ? f->L2 : f->U2;
            else if (dz == 0 && dx == 0 && (dy == -1 || dy == 1))
                dst = dy < 0 ? f->L3 : f->U3;
            if (!dst) return ORC_ERR_PATTERN;
            memcpy(dst + 9 * (size_t)p, A->v + 9 * (size_t)e, sizeof(double) * 9);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* The preconditioner B^{-1} = sum_s P_s R_s^T A_s^{-1} R_s (Eqs. 4.2-4.3, 4.5)               */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int* map;       /* [N] local index or -1 */
    int counts[3];
    bsr_t A;        /* assembled local matrix */
    bsr_t LU;       /* ILU factors (solver 0/1) */
    double* dpiv;   /* final pivot blocks (solver 0/1) */
    dense_lu_t dlu; /* solver 2 */
    nf_t nf;        /* solvers 3/4 */
} orc_sub;

/* Classical coarse-grid correction (Section 3, Eqs. 3.5-3.8): R_C sums the 3-vectors of each coarse
 * box's cells, R_C^T copies a box's value to each of its cells, A_C = R_C A R_C^T (Eq. 3.6) is
 * solved exactly (dense LU with partial pivoting). */
typedef struct {
    int mode;       /* 0 none, 1 two-level (Eq. 3.5), 2 two-stage (Eqs. 3.7-3.8) */
    int nb;         /* coarse boxes */
    int* box;       /* [N] coarse box of each cell */
    dense_lu_t lu;  /* of A_C, 3 nb unknowns */
    double* ac;     /* A_C before factorisation (3 nb x 3 nb, row-major), for inspection */
    const int *rp, *ci; /* A (caller-owned, kept alive by the caller) for the two-stage residual */
    const double* v;
} orc_coarse;

typedef struct {
    orc_geom g;
    int N, K, solver;
    int* owner;
    orc_sub* sub;
    int only; /* -1: all subdomains built; else the one subdomain that was built */
    orc_coarse cc;
} orc_pc;

static void sub_free(orc_sub* s) {
    free(s->map);
    bsr_free(&s->A);
    bsr_free(&s->LU);
    free(s->dpiv);
    free(s->dlu.a);
    free(s->dlu.piv);
    nf_free(&s->nf);
    memset(s, 0, sizeof(*s));
}

void orc_pc_destroy(orc_pc* pc) {
    if (!pc) return;
    free(pc->cc.box);
    free(pc->cc.lu.a);
    free(pc->cc.lu.piv);
    free(pc->cc.ac);
    if (pc->sub)
        for (int s = 0; s < pc->K; s++) sub_free(&pc->sub[s]);
    free(pc->sub);
    free(pc->owner);
    free(pc);
}

static int bsr_copy(const bsr_t* a, bsr_t* b) {
    b->n = a->n;
    b->nnz = a->nnz;
    b->rp = (int*)malloc(sizeof(int) * ((size_t)a->n + 1));
    b->ci = (int*)malloc(sizeof(int) * (size_t)(a->nnz > 0 ? a->nnz : 1));
    b->diag = (int*)malloc(sizeof(int) * (size_t)(a->n > 0 ? a->n : 1));
    b->v = (double*)malloc(sizeof(double) * ((size_t)a->nnz * 9 + 1));
    if (!b->rp || !b->ci || !b->diag || !b->v) return ORC_ERR_NOMEM;
    memcpy(b->rp, a->rp, sizeof(int) * ((size_t)a->n + 1));
    memcpy(b->ci, a->ci, sizeof(int) * (size_t)a->nnz);
    memcpy(b->diag, a->diag, sizeof(int) * (size_t)a->n);
    memcpy(b->v, a->v, sizeof(double) * (size_t)a->nnz * 9);
    return ORC_OK;
}

/* Build (and factor) the local problems.  only = -1 builds every subdomain; only = s builds just
 * subdomain s (for sampled checks on large grids).  Returns NULL on failure, with *status set
 * and, for a singular pivot, err_loc = {subdomain, local block row}. */
orc_pc* orc_pc_create(const orc_geom* g, const int* rp, const int* ci, const double* v, int solver,
                      int only, int* status, int* err_loc) {
    *status = ORC_ERR_ARG;
    if (!geom_ok(g) || solver < 0 || solver > 4) return NULL;
    orc_pc* pc = (orc_pc*)calloc(1, sizeof(orc_pc));
    pc->g = *g;
    pc->N = g->nx * g->ny * g->nz;
    pc->K = orc_n_sub(g);
    pc->solver = solver;
    pc->only = only;
    if (only < -1 || only >= pc->K) {
        free(pc);
        return NULL;
    }
    pc->owner = (int*)malloc(sizeof(int) * (size_t)pc->N);
    pc->sub = (orc_sub*)calloc((size_t)pc->K, sizeof(orc_sub));
    orc_owner(g, pc->owner);
    for (int s = 0; s < pc->K; s++) {
        if (only >= 0 && s != only) continue;
        orc_sub* S = &pc->sub[s];
        S->map = (int*)malloc(sizeof(int) * (size_t)pc->N);
        int n = orc_local_map(g, s, S->map, S->counts);
        int st = assemble_local(pc->N, rp, ci, v, S->map, n, &S->A);
        if (st) {
            *status = st;
            orc_pc_destroy(pc);
            return NULL;
        }
        int bad = -1;
        if (solver == ORC_DENSE_LU) {
            st = dense_lu_factor(&S->A, &S->dlu, &bad);
        } else if (solver == ORC_NF_COLSUM || solver == ORC_NF) {
            /* nested factorisation needs a box without lumps (Appendix A: hepta-banded matrix) */
            if (S->counts[1] != 0 || S->counts[2] != 0) {
                st = ORC_ERR_ARG;
            } else {
                const box3 F = grow_clip(g, owned_box(g, s), g->ov);
                st = nf_setup(&S->A, F.hi[0] - F.lo[0], F.hi[1] - F.lo[1], F.hi[2] - F.lo[2], &S->nf);
                if (!st) st = nf_factor(&S->nf, solver == ORC_NF_COLSUM, &bad);
            }
        } else {
            st = bsr_copy(&S->A, &S->LU);
            S->dpiv = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
            if (!st) st = bilu0_factor(&S->LU, solver == ORC_BILU0_COLSUM, S->dpiv, &bad);
        }
        if (st) {
            *status = st;
            if (err_loc) {
                err_loc[0] = s;
                err_loc[1] = bad;
            }
            orc_pc_destroy(pc);
            return NULL;
        }
    }
    *status = ORC_OK;
    return pc;
}

int orc_pc_sub_n(const orc_pc* pc, int s) { return pc->sub[s].A.n; }
int orc_pc_sub_nnz(const orc_pc* pc, int s) { return pc->sub[s].A.nnz; }
void orc_pc_sub_counts(const orc_pc* pc, int s, int* counts) {
    memcpy(counts, pc->sub[s].counts, sizeof(int) * 3);
}
void orc_pc_sub_map(const orc_pc* pc, int s, int* map) {
    memcpy(map, pc->sub[s].map, sizeof(int) * (size_t)pc->N);
}
/* local matrix A_s (pattern + values) */
void orc_pc_sub_matrix(const orc_pc* pc, int s, int* rp, int* ci, double* v) {
    const bsr_t* A = &pc->sub[s].A;
    memcpy(rp, A->rp, sizeof(int) * ((size_t)A->n + 1));
    memcpy(ci, A->ci, sizeof(int) * (size_t)A->nnz);
    memcpy(v, A->v, sizeof(double) * 9 * (size_t)A->nnz);
}
/* ILU factors in A_s's pattern: L below, U above, D^{-1} on the diagonal; and the pivots D */
int orc_pc_sub_factors(const orc_pc* pc, int s, double* lu, double* dpiv) {
    const orc_sub* S = &pc->sub[s];
    if (pc->solver >= ORC_DENSE_LU) return ORC_ERR_ARG;
    memcpy(lu, S->LU.v, sizeof(double) * 9 * (size_t)S->LU.nnz);
    if (dpiv) memcpy(dpiv, S->dpiv, sizeof(double) * 9 * (size_t)S->LU.n);
    return ORC_OK;
}

/* Nested factorisation of subdomain s: box dims {bx, by, bz} and the G blocks [n*9] */
int orc_pc_sub_nf(const orc_pc* pc, int s, int* dims, double* G) {
    const orc_sub* S = &pc->sub[s];
    if (pc->solver != ORC_NF_COLSUM && pc->solver != ORC_NF) return ORC_ERR_ARG;
    dims[0] = S->nf.bx;
    dims[1] = S->nf.by;
    dims[2] = S->nf.bz;
    if (G) memcpy(G, S->nf.G, sizeof(double) * 9 * (size_t)S->nf.n);
    return ORC_OK;
}

/* local solve A_s^{-1} (or B_s^{-1}) of a local right-hand side */
void orc_pc_local_solve(const orc_pc* pc, int s, const double* rhs, double* sol) {
    const orc_sub* S = &pc->sub[s];
    if (pc->solver == ORC_DENSE_LU)
        dense_lu_solve(&S->dlu, rhs, sol);
    else if (pc->solver == ORC_NF_COLSUM || pc->solver == ORC_NF)
        nf_solve(&S->nf, rhs, sol);
    else
        bilu0_solve(&S->LU, rhs, sol);
}

/* R_s r: fine entries copied, lump entries summed over the lump's cells (Eqs. 4.1, B.2) */
void orc_pc_restrict(const orc_pc* pc, int s, const double* r, double* rl) {
    const orc_sub* S = &pc->sub[s];
    const int n = S->A.n;
    for (int p = 0; p < 3 * n; p++) rl[p] = 0.0;
    for (int a = 0; a < pc->N; a++) {
        int p = S->map[a];
        if (p < 0) continue;
        for (int c = 0; c < 3; c++) rl[3 * p + c] += r[3 * a + c];
    }
}

/* Coarse boxes and A_C = R_C A R_C^T of the classical correction.  mode 1: two-level (Eq. 3.5),
 * 2: two-stage (Eqs. 3.7-3.8), 0: none.  cbox = NULL or {0,0,0}: the coarse boxes are the
 * partition boxes (box = owning subdomain); else aligned boxes of cbox cells, numbered
 * bz + nbz*(bx + nbx*by) like cells.  A (rp, ci, v) must outlive the preconditioner.  Returns
 * ORC_OK, ORC_ERR_ARG, ORC_ERR_NOMEM, or ORC_ERR_PIVOT with *bad_box = the coarse block row. */
int orc_pc_set_coarse(orc_pc* pc, const int* rp, const int* ci, const double* v, int mode, const int* cbox,
                      int* bad_box) {
    if (mode < 0 || mode > 2) return ORC_ERR_ARG;
    free(pc->cc.box);
    free(pc->cc.lu.a);
    free(pc->cc.lu.piv);
    free(pc->cc.ac);
    memset(&pc->cc, 0, sizeof(pc->cc));
    if (mode == 0) return ORC_OK;
    const orc_geom* g = &pc->g;
    const int N = pc->N;
    orc_coarse* cc = &pc->cc;
    cc->box = (int*)malloc(sizeof(int) * (size_t)N);
    if (!cc->box) return ORC_ERR_NOMEM;
    const int partition = cbox == NULL || (cbox[0] == 0 && cbox[1] == 0 && cbox[2] == 0);
    if (partition) {
        cc->nb = pc->K;
        memcpy(cc->box, pc->owner, sizeof(int) * (size_t)N);
    } else {
        if (cbox[0] < 1 || cbox[1] < 1 || cbox[2] < 1) return ORC_ERR_ARG;
        const int nbx = (g->nx + cbox[0] - 1) / cbox[0], nby = (g->ny + cbox[1] - 1) / cbox[1],
                  nbz = (g->nz + cbox[2] - 1) / cbox[2];
        cc->nb = nbx * nby * nbz;
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++)
                for (int k = 0; k < g->nz; k++)
                    cc->box[k + g->nz * (i + g->nx * j)] = k / cbox[2] + nbz * (i / cbox[0] + nbx * (j / cbox[1]));
    }
    for (int a = 0; a < N; a++) /* every cell in one of the nb boxes, before A_C is indexed by them */
        if (cc->box[a] < 0 || cc->box[a] >= cc->nb) return ORC_ERR_ARG;
    const int n3 = 3 * cc->nb;
    if (dense_alloc(&cc->lu, n3)) return ORC_ERR_NOMEM;
    /* A_C(I, J) = sum of the blocks A(a, b) over cells a in box I and b in box J */
    for (int a = 0; a < N; a++)
        for (int e = rp[a]; e < rp[a + 1]; e++) {
            const int I = cc->box[a], J = cc->box[ci[e]];
            for (int r = 0; r < 3; r++)
                for (int s = 0; s < 3; s++)
                    cc->lu.a[(size_t)(3 * I + r) * n3 + 3 * J + s] += v[9 * (size_t)e + 3 * r + s];
        }
    cc->ac = (double*)malloc(sizeof(double) * ((size_t)n3 * n3 + 1));
    if (!cc->ac) return ORC_ERR_NOMEM;
    memcpy(cc->ac, cc->lu.a, sizeof(double) * (size_t)n3 * n3);
    int bad = -1;
    const int st = dense_factor(&cc->lu, &bad);
    if (st) {
        if (bad_box) *bad_box = bad;
        return st;
    }
    cc->mode = mode;
    cc->rp = rp;
    cc->ci = ci;
    cc->v = v;
    return ORC_OK;
}

int orc_pc_coarse_nb(const orc_pc* pc) { return pc->cc.nb; }

/* A_C (3 nb x 3 nb, row-major) and the coarse box of every cell */
void orc_pc_coarse_matrix(const orc_pc* pc, double* ac, int* box) {
    const int n3 = 3 * pc->cc.nb;
    if (ac) memcpy(ac, pc->cc.ac, sizeof(double) * (size_t)n3 * n3);
    if (box) memcpy(box, pc->cc.box, sizeof(int) * (size_t)pc->N);
}

void orc_spmv(int N, const int* rp, const int* ci, const double* v, const double* x, double* y);

/* z += R_C^T A_C^{-1} R_C r (two-level, Eq. 3.5) or z += R_C^T A_C^{-1} R_C (r - A z) (two-stage,
 * Eq. 3.7 with z = B_AS^{-1} r on entry) */
static void coarse_correct(const orc_pc* pc, const double* r, double* z) {
    const orc_coarse* cc = &pc->cc;
    const int N = pc->N, n3 = 3 * cc->nb;
    double* w = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* rc = (double*)calloc((size_t)n3 + 1, sizeof(double));
    double* yc = (double*)malloc(sizeof(double) * ((size_t)n3 + 1));
    if (cc->mode == 2) {
        orc_spmv(N, cc->rp, cc->ci, cc->v, z, w);
        for (int i = 0; i < 3 * N; i++) w[i] = r[i] - w[i];
    } else {
        memcpy(w, r, sizeof(double) * 3 * (size_t)N);
    }
    for (int a = 0; a < N; a++)
        for (int c = 0; c < 3; c++) rc[3 * cc->box[a] + c] += w[3 * a + c];
    dense_lu_solve(&cc->lu, rc, yc);
    for (int a = 0; a < N; a++)
        for (int c = 0; c < 3; c++) z[3 * a + c] += yc[3 * cc->box[a] + c];
    free(w);
    free(rc);
    free(yc);
}

/* z = sum_s P_s R_s^T A_s^{-1} R_s r: each cell takes its owner's local solution (Eq. 4.2; the
 * off-processor coarse solution is discarded, Section 4).  With a single-subdomain build
 * (only >= 0), only that subdomain's owned rows of z are written. */
void orc_pc_apply(const orc_pc* pc, const double* r, double* z) {
    for (int s = 0; s < pc->K; s++) {
        if (pc->only >= 0 && s != pc->only) continue;
        const orc_sub* S = &pc->sub[s];
        const int n = S->A.n;
        double* rl = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
        double* zl = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
        orc_pc_restrict(pc, s, r, rl);
        orc_pc_local_solve(pc, s, rl, zl);
        for (int a = 0; a < pc->N; a++)
            if (pc->owner[a] == s)
                for (int c = 0; c < 3; c++) z[3 * a + c] = zl[3 * (size_t)S->map[a] + c];
        free(rl);
        free(zl);
    }
    if (pc->cc.mode != 0) coarse_correct(pc, r, z);
}

/* ------------------------------------------------------------------------------------------ */
/* Global block ILU(0) (+colsum) on A itself, the K = 1 special case                          */
/* ------------------------------------------------------------------------------------------ */

/* y = A x for the global BSR matrix */
void orc_spmv(int N, const int* rp, const int* ci, const double* v, const double* x, double* y) {
    for (int a = 0; a < N; a++) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int e = rp[a]; e < rp[a + 1]; e++) {
            double t[3];
            mulv3(v + 9 * (size_t)e, x + 3 * (size_t)ci[e], t);
            for (int r = 0; r < 3; r++) acc[r] += t[r];
        }
        for (int r = 0; r < 3; r++) y[3 * a + r] = acc[r];
    }
}

static double dot(int n, const double* a, const double* b) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------------------------ */
/* Krylov accelerators on r = b - A x (Section 2)                                              */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int iters;     /* preconditioned matrix-vector products */
    int restarts;  /* completed cycles */
    int converged;
    double relres; /* final true ||b - A x|| / ||b|| */
} orc_info;

static void precond(const orc_pc* pc, int n3, const double* r, double* z) {
    if (pc)
        orc_pc_apply(pc, r, z);
    else
        memcpy(z, r, sizeof(double) * (size_t)n3);
}

/* Right-preconditioned restarted GMRES(m): modified Gram-Schmidt Arnoldi on A B^{-1}, Givens
 * rotations on the Hessenberg matrix, x0 = 0.  A cycle ends when |g_{j+1}| <= tol ||b||, at
 * j = m, or on breakdown (h_{j+1,j} <= 1e-14 ||w before orthogonalisation||); then
 * x += B^{-1} V y and the true residual b - A x decides convergence.  resid_hist (optional,
 * max_iter+1 entries) receives |g| after each step, relative to ||b||. */
int orc_gmres(int N, const int* rp, const int* ci, const double* v, const orc_pc* pc, const double* b,
              double* x, int m, double tol, int max_iter, orc_info* info, double* resid_hist) {
    const int n3 = 3 * N;
    double* V = (double*)malloc(sizeof(double) * (size_t)n3 * (m + 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)n3);
    double* z = (double*)malloc(sizeof(double) * (size_t)n3);
    double* r = (double*)malloc(sizeof(double) * (size_t)n3);
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * m);
    double* sn = (double*)malloc(sizeof(double) * m);
    double* g = (double*)malloc(sizeof(double) * (m + 1));
    double* y = (double*)malloc(sizeof(double) * m);
    if (!V || !w || !z || !r || !H || !cs || !sn || !g || !y) return ORC_ERR_NOMEM;

    for (int i = 0; i < n3; i++) x[i] = 0.0;
    const double bnorm = sqrt(dot(n3, b, b));
    info->iters = 0;
    info->restarts = 0;
    info->converged = 0;
    info->relres = 0.0;
    if (bnorm == 0.0) {
        info->converged = 1;
        goto done;
    }
    memcpy(r, b, sizeof(double) * n3);
    double beta = bnorm;
    if (resid_hist) resid_hist[0] = 1.0;
    while (1) {
        for (int i = 0; i < n3; i++) V[i] = r[i] / beta;
        for (int i = 0; i <= m; i++) g[i] = 0.0;
        g[0] = beta;
        int jend = 0;
        for (int j = 0; j < m; j++) {
            double* vj = V + (size_t)j * n3;
            precond(pc, n3, vj, z);
            orc_spmv(N, rp, ci, v, z, w);
            const double w0 = sqrt(dot(n3, w, w));
            for (int k = 0; k <= j; k++) {
                const double* vk = V + (size_t)k * n3;
                double h = dot(n3, w, vk);
                H[k * m + j] = h;
                for (int i = 0; i < n3; i++) w[i] -= h * vk[i];
            }
            const double hn = sqrt(dot(n3, w, w));
            H[(j + 1) * m + j] = hn;
            for (int k = 0; k < j; k++) {
                double a = H[k * m + j], bb = H[(k + 1) * m + j];
                H[k * m + j] = cs[k] * a + sn[k] * bb;
                H[(k + 1) * m + j] = -sn[k] * a + cs[k] * bb;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double rr = hypot(a, bb);
            if (rr == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = a / rr;
                sn[j] = bb / rr;
            }
            H[j * m + j] = cs[j] * a + sn[j] * bb;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            info->iters++;
            if (resid_hist) resid_hist[info->iters] = fabs(g[j + 1]) / bnorm;
            jend = j + 1;
            int breakdown = hn <= 1e-14 * w0;
            if (fabs(g[j + 1]) <= tol * bnorm || breakdown || info->iters >= max_iter) break;
            double* vn = V + (size_t)(j + 1) * n3;
            for (int i = 0; i < n3; i++) vn[i] = w[i] / hn;
        }
        /* y = H^{-1} g (upper triangular), x += B^{-1} V y */
        for (int k = jend - 1; k >= 0; k--) {
            double acc = g[k];
            for (int l = k + 1; l < jend; l++) acc -= H[k * m + l] * y[l];
            y[k] = acc / H[k * m + k];
        }
        for (int i = 0; i < n3; i++) w[i] = 0.0;
        for (int k = 0; k < jend; k++) {
            const double* vk = V + (size_t)k * n3;
            for (int i = 0; i < n3; i++) w[i] += y[k] * vk[i];
        }
        precond(pc, n3, w, z);
        for (int i = 0; i < n3; i++) x[i] += z[i];
        orc_spmv(N, rp, ci, v, x, r);
        for (int i = 0; i < n3; i++) r[i] = b[i] - r[i];
        beta = sqrt(dot(n3, r, r));
        info->restarts++;
        info->relres = beta / bnorm;
        if (info->relres <= tol) {
            info->converged = 1;
            break;
        }
        if (info->iters >= max_iter || beta == 0.0) break;
    }
done:
    free(V);
    free(w);
    free(z);
    free(r);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    return ORC_OK;
}

/* ORTHOMIN(k) (Section 2, Vinsome's method), right-preconditioned, x0 = 0: the new direction
 * p = B^{-1} r is A-orthogonalised against the last k directions in the sense
 * (A p_j, A p_i) = 0, then x += alpha p, r -= alpha A p with alpha = (r, Ap)/(Ap, Ap).
 * Convergence on the recurrence residual, confirmed by a true residual at exit. */
int orc_orthomin(int N, const int* rp, const int* ci, const double* v, const orc_pc* pc, const double* b,
                 double* x, int kdir, double tol, int max_iter, orc_info* info, double* resid_hist) {
    const int n3 = 3 * N;
    double* P = (double*)malloc(sizeof(double) * (size_t)n3 * (kdir + 1));
    double* Q = (double*)malloc(sizeof(double) * (size_t)n3 * (kdir + 1));
    double* qq = (double*)malloc(sizeof(double) * (kdir + 1));
    double* r = (double*)malloc(sizeof(double) * (size_t)n3);
    double* t = (double*)malloc(sizeof(double) * (size_t)n3);
    if (!P || !Q || !qq || !r || !t) return ORC_ERR_NOMEM;
    for (int i = 0; i < n3; i++) x[i] = 0.0;
    memcpy(r, b, sizeof(double) * n3);
    const double bnorm = sqrt(dot(n3, b, b));
    info->iters = 0;
    info->restarts = 0;
    info->converged = 0;
    info->relres = 0.0;
    if (resid_hist) resid_hist[0] = 1.0;
    if (bnorm == 0.0) {
        info->converged = 1;
        goto done;
    }
    int stored = 0; /* directions held, at most kdir (ring of kdir+1 slots) */
    for (int it = 0; it < max_iter; it++) {
        int slot = it % (kdir + 1);
        double* p = P + (size_t)slot * n3;
        double* q = Q + (size_t)slot * n3;
        precond(pc, n3, r, p);
        orc_spmv(N, rp, ci, v, p, q);
        for (int l = 1; l <= stored; l++) {
            int os = ((it - l) % (kdir + 1) + (kdir + 1)) % (kdir + 1);
            const double* po = P + (size_t)os * n3;
            const double* qo = Q + (size_t)os * n3;
            double beta = dot(n3, q, qo) / qq[os];
            for (int i = 0; i < n3; i++) {
                p[i] -= beta * po[i];
                q[i] -= beta * qo[i];
            }
        }
        qq[slot] = dot(n3, q, q);
        if (qq[slot] == 0.0) break;
        double alpha = dot(n3, r, q) / qq[slot];
        for (int i = 0; i < n3; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        if (stored < kdir) stored++;
        info->iters++;
        double rn = sqrt(dot(n3, r, r));
        if (resid_hist) resid_hist[info->iters] = rn / bnorm;
        if (rn <= tol * bnorm) break;
    }
    orc_spmv(N, rp, ci, v, x, t);
    for (int i = 0; i < n3; i++) t[i] = b[i] - t[i];
    info->relres = sqrt(dot(n3, t, t)) / bnorm;
    info->converged = info->relres <= tol;
done:
    free(P);
    free(Q);
    free(qq);
    free(r);
    free(t);
    return ORC_OK;
}
