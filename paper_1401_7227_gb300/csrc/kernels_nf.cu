// Nested factorisation (Appendix A) as the local solver of local problems without lumps: each
// subdomain's A_i is hepta-banded on its box of bx * by * bz cells (local cell p = z + bz (x + bx y)),
// A = D + L1 + U1 + L2 + U2 + L3 + U3, and
//   B = (P + L3)(I + P^{-1} U3),  P = (T + L2)(I + T^{-1} U2),  T = (G + L1)(I + G^{-1} U1)
// with G block diagonal, G = D - L1 G^{-1} U1 (Eq. A.6), with colsum also minus the block column sums
// of L2 T^{-1} U2 and L3 P^{-1} U3 (Eq. A.7).  The factorisation and the solve are sequential along
// the cells of a subdomain (each line depends on the previous one, each plane on the previous
// plane), so one warp takes one subdomain and its lanes share the 3x3 block algebra: nine lanes for
// a block product (lane 3 r + c holds element (r, c)), three for a block times a 3-vector.
#include <cuda_runtime.h>

#include <algorithm>

#include "asm2_internal.h"

namespace asm2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- 3x3 blocks held one element per lane (lanes 0..8; other lanes carry zeros) --------------

// element (r, c) of a block stored row-major at p (nullptr: a zero block)
__device__ __forceinline__ double bload(const double* p, int lane) { return (p && lane < 9) ? p[lane] : 0.0; }

// a * b for blocks held per lane
__device__ __forceinline__ double bmul(double a, double b, int lane) {
    const int r = lane < 9 ? lane / 3 : 0, c = lane < 9 ? lane - 3 * (lane / 3) : 0;
    const double a0 = __shfl_sync(kFull, a, 3 * r), a1 = __shfl_sync(kFull, a, 3 * r + 1),
                 a2 = __shfl_sync(kFull, a, 3 * r + 2);
    const double b0 = __shfl_sync(kFull, b, c), b1 = __shfl_sync(kFull, b, 3 + c), b2 = __shfl_sync(kFull, b, 6 + c);
    return lane < 9 ? a0 * b0 + a1 * b1 + a2 * b2 : 0.0;
}

// inverse of a block held per lane: lane 0 runs Gauss-Jordan with partial pivoting, the result is
// spread back.  false (on every lane) for a zero pivot.
__device__ bool binv(double a, double& inv, int lane) {
    double m[3][6];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m[r][c] = __shfl_sync(kFull, a, 3 * r + c);
            m[r][3 + c] = r == c ? 1.0 : 0.0;
        }
    int ok = 1;
    if (lane == 0) {
        for (int c = 0; c < 3 && ok; c++) {
            int p = c;
            for (int r = c + 1; r < 3; r++)
                if (fabs(m[r][c]) > fabs(m[p][c])) p = r;
            if (m[p][c] == 0.0) {
                ok = 0;
                break;
            }
            if (p != c)
                for (int k = 0; k < 6; k++) {
                    const double t = m[c][k];
                    m[c][k] = m[p][k];
                    m[p][k] = t;
                }
            const double id = 1.0 / m[c][c];
            for (int k = 0; k < 6; k++) m[c][k] *= id;
            for (int r = 0; r < 3; r++) {
                if (r == c) continue;
                const double f = m[r][c];
                for (int k = 0; k < 6; k++) m[r][k] -= f * m[c][k];
            }
        }
    }
    ok = __shfl_sync(kFull, ok, 0);
    double out = 0.0;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double v = __shfl_sync(kFull, m[r][3 + c], 0);
            if (lane == 3 * r + c) out = v;
        }
    inv = out;
    return ok != 0;
}

// ---- 3-vectors held one component per lane (lanes 0..2) --------------------------------------

__device__ __forceinline__ double vload(const double* p, int lane) { return lane < 3 ? p[lane] : 0.0; }
__device__ __forceinline__ void vstore(double* p, double v, int lane) {
    if (lane < 3) p[lane] = v;
}

// (block at p) * x for x held per lane (nullptr: zero)
__device__ __forceinline__ double bvmul(const double* p, double x, int lane) {
    const double x0 = __shfl_sync(kFull, x, 0), x1 = __shfl_sync(kFull, x, 1), x2 = __shfl_sync(kFull, x, 2);
    if (!p || lane >= 3) return 0.0;
    return p[3 * lane] * x0 + p[3 * lane + 1] * x1 + p[3 * lane + 2] * x2;
}

struct NFView {
    const NFDesc& d;
    __device__ const double* band(int k, int p) const {  // k: 0 D, 1 L1, 2 U1, 3 L2, 4 U2, 5 L3, 6 U3
        const int s = d.bands[7 * p + k];
        return s >= 0 ? d.slot + 9LL * s : nullptr;
    }
    __device__ const double* gi(int p) const { return d.gi + 9LL * p; }
};

// W = u T^{-1} on the line starting at cell q0: W (G + L1)(I + G^{-1} U1) = u (rows of blocks)
__device__ void line_row_solve(const NFView& v, int q0, const double* u, double* vtmp, double* W, int lane) {
    const int bz = v.d.bz;
    double prev = 0.0;
    for (int q = 0; q < bz; q++) {  // vtmp (I + G^{-1} U1) = u
        double x = bload(u + 9 * q, lane);
        if (q > 0) x -= bmul(bmul(prev, bload(v.gi(q0 + q - 1), lane), lane), bload(v.band(2, q0 + q - 1), lane), lane);
        if (lane < 9) vtmp[9 * q + lane] = x;
        prev = x;
    }
    double next = 0.0;
    for (int q = bz - 1; q >= 0; q--) {  // W (G + L1) = vtmp
        double x = bload(vtmp + 9 * q, lane);
        if (q < bz - 1) x -= bmul(next, bload(v.band(1, q0 + q + 1), lane), lane);
        const double w = bmul(x, bload(v.gi(q0 + q), lane), lane);
        if (lane < 9) W[9 * q + lane] = w;
        next = w;
    }
    __syncwarp();
}

// out = T^{-1} b on the line starting at q0 (3-vectors); b and out may not alias
__device__ void line_solve(const NFView& v, int q0, const double* b, double* out, int lane) {
    const int bz = v.d.bz;
    double s = 0.0;
    for (int q = 0; q < bz; q++) {  // (G + L1) s = b
        double t = vload(b + 3 * q, lane);
        if (q > 0) t -= bvmul(v.band(1, q0 + q), s, lane);
        s = bvmul(v.gi(q0 + q), t, lane);
        vstore(out + 3 * q, s, lane);
    }
    __syncwarp();
    double o = 0.0;
    for (int q = bz - 1; q >= 0; q--) {  // (I + G^{-1} U1) out = s
        double t = vload(out + 3 * q, lane);
        if (q < bz - 1) t -= bvmul(v.gi(q0 + q), bvmul(v.band(2, q0 + q), o, lane), lane);
        vstore(out + 3 * q, t, lane);
        o = t;
    }
    __syncwarp();
}

// out = P^{-1} b on the plane starting at c0; scratch: 3 bz + 3 bz doubles
__device__ void plane_solve(const NFView& v, int c0, const double* b, double* out, double* t1, double* t2, int lane) {
    const int bz = v.d.bz, bx = v.d.bx;
    for (int l = 0; l < bx; l++) {  // (T + L2) z = b, z kept in out
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            double t = vload(b + 3 * c, lane);
            if (l > 0) t -= bvmul(v.band(3, c0 + c), vload(out + 3 * (c - bz), lane), lane);
            vstore(t1 + 3 * q, t, lane);
        }
        __syncwarp();
        line_solve(v, c0 + l * bz, t1, out + 3 * l * bz, lane);
    }
    for (int l = bx - 2; l >= 0; l--) {  // (I + T^{-1} U2) out = z
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            vstore(t1 + 3 * q, bvmul(v.band(4, c0 + c), vload(out + 3 * (c + bz), lane), lane), lane);
        }
        __syncwarp();
        line_solve(v, c0 + l * bz, t1, t2, lane);
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            vstore(out + 3 * c, vload(out + 3 * c, lane) - vload(t2 + 3 * q, lane), lane);
        }
        __syncwarp();
    }
}

// W = u P^{-1} on the plane starting at c0 (rows of blocks); scratch: vb (9 S), x, y, vt (9 bz each)
__device__ void plane_row_solve(const NFView& v, int c0, const double* u, double* vb, double* x, double* y, double* vt,
                                double* W, int lane) {
    const int bz = v.d.bz, bx = v.d.bx;
    for (int l = 0; l < bx; l++) {  // vb (I + T^{-1} U2) = u
        if (l > 0) line_row_solve(v, c0 + (l - 1) * bz, vb + 9 * (l - 1) * bz, vt, x, lane);
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            double e = bload(u + 9 * c, lane);
            if (l > 0) e -= bmul(bload(x + 9 * q, lane), bload(v.band(4, c0 + c - bz), lane), lane);
            if (lane < 9) vb[9 * c + lane] = e;
        }
        __syncwarp();
    }
    for (int l = bx - 1; l >= 0; l--) {  // W (T + L2) = vb
        for (int q = 0; q < bz; q++) {
            const int c = l * bz + q;
            double e = bload(vb + 9 * c, lane);
            if (l < bx - 1) e -= bmul(bload(W + 9 * (c + bz), lane), bload(v.band(3, c0 + c + bz), lane), lane);
            if (lane < 9) y[9 * q + lane] = e;
        }
        __syncwarp();
        line_row_solve(v, c0 + l * bz, y, vt, W + 9 * l * bz, lane);
    }
}

// Factorisation: G^{-1} of every cell, plane by plane, line by line, cell by cell
__global__ void __launch_bounds__(128) k_nf_factor(const NFDesc* __restrict__ descs, int ndesc, FactErr* err) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= ndesc) return;
    const NFDesc& d = descs[w];
    const NFView v{d};
    const int bz = d.bz, bx = d.bx, by = d.by, S = bz * bx;
    // scratch: cs3 (9 S), u (9 S), W (9 S), vb (9 S), x, y, vt, cs2 (9 bz each)
    double* cs3 = d.work;
    double* u = cs3 + 9 * S;
    double* W = u + 9 * S;
    double* vb = W + 9 * S;
    double* x = vb + 9 * S;
    double* y = x + 9 * bz;
    double* vt = y + 9 * bz;
    double* cs2 = vt + 9 * bz;
    for (int j = 0; j < by; j++) {
        const int c0 = j * S;
        const bool plane_term = d.colsum && j > 0;
        if (plane_term) {  // block column sums of L3 P_{j-1}^{-1} U3 on plane j
            for (int c = 0; c < S; c++)
                if (lane < 9) u[9 * c + lane] = bload(v.band(5, c0 + c), lane);
            __syncwarp();
            plane_row_solve(v, c0 - S, u, vb, x, y, vt, W, lane);
            for (int c = 0; c < S; c++) {
                const double e = bmul(bload(W + 9 * c, lane), bload(v.band(6, c0 - S + c), lane), lane);
                if (lane < 9) cs3[9 * c + lane] = e;
            }
            __syncwarp();
        }
        for (int l = 0; l < bx; l++) {
            const int q0 = c0 + l * bz;
            const bool line_term = d.colsum && l > 0;
            if (line_term) {  // block column sums of L2 T_{l-1}^{-1} U2 on line l
                for (int q = 0; q < bz; q++)
                    if (lane < 9) u[9 * q + lane] = bload(v.band(3, q0 + q), lane);
                __syncwarp();
                line_row_solve(v, q0 - bz, u, vt, W, lane);
                for (int q = 0; q < bz; q++) {
                    const double e = bmul(bload(W + 9 * q, lane), bload(v.band(4, q0 - bz + q), lane), lane);
                    if (lane < 9) cs2[9 * q + lane] = e;
                }
                __syncwarp();
            }
            for (int q = 0; q < bz; q++) {
                const int p = q0 + q;
                double g = bload(v.band(0, p), lane);
                if (q > 0) g -= bmul(bmul(bload(v.band(1, p), lane), bload(v.gi(p - 1), lane), lane),
                                     bload(v.band(2, p - 1), lane), lane);
                if (line_term) g -= bload(cs2 + 9 * q, lane);
                if (plane_term) g -= bload(cs3 + 9 * (l * bz + q), lane);
                if (lane < 9) d.g[9LL * p + lane] = g;
                double gi;
                if (!binv(g, gi, lane)) {
                    if (lane == 0 && atomicCAS(&err->flag, 0, 1) == 0) {
                        err->sub = d.sub;
                        err->row = p;
                    }
                    return;  // the whole warp leaves together (binv's result is warp-uniform)
                }
                if (lane < 9) d.gi[9LL * p + lane] = gi;
                __syncwarp();
            }
        }
    }
}

// Apply: y = R_i r (the box's cells), x = B^{-1} y, z[owned cells] = x[owned]
__global__ void __launch_bounds__(128) k_nf_apply(const SysTab* __restrict__ tab, const NFDesc* __restrict__ descs,
                                                 int ndesc) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= ndesc) return;
    const NFDesc& d = descs[w];
    const SysTab& st = tab[d.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const double* r = st.ws + (long long)in * st.n3p;
    double* z = st.ws + (long long)st.ctl[C_APPLY_OUT] * st.n3p;
    const NFView v{d};
    const int bz = d.bz, bx = d.bx, by = d.by, S = bz * bx, n = d.n;
    // scratch: yv (3 n), xv (3 n), t (3 S), wv (3 S), t1, t2 (3 bz each)
    double* yv = d.work;
    double* xv = yv + 3 * n;
    double* t = xv + 3 * n;
    double* wv = t + 3 * S;
    double* t1 = wv + 3 * S;
    double* t2 = t1 + 3 * bz;
    for (int j = 0; j < by; j++) {  // (P + L3) yv = R r
        for (int c = 0; c < S; c++) {
            const int p = j * S + c;
            double e = vload(r + 3LL * d.cell[p], lane);
            if (j > 0) e -= bvmul(v.band(5, p), vload(yv + 3 * (p - S), lane), lane);
            vstore(t + 3 * c, e, lane);
        }
        __syncwarp();
        plane_solve(v, j * S, t, yv + 3 * j * S, t1, t2, lane);
    }
    for (int c = (by - 1) * S; c < by * S; c++) vstore(xv + 3 * c, vload(yv + 3 * c, lane), lane);
    for (int j = by - 2; j >= 0; j--) {  // (I + P^{-1} U3) xv = yv
        for (int c = 0; c < S; c++) {
            const int p = j * S + c;
            vstore(t + 3 * c, bvmul(v.band(6, p), vload(xv + 3 * (p + S), lane), lane), lane);
        }
        __syncwarp();
        plane_solve(v, j * S, t, wv, t1, t2, lane);
        for (int c = 0; c < S; c++) {
            const int p = j * S + c;
            vstore(xv + 3 * p, vload(yv + 3 * p, lane) - vload(wv + 3 * c, lane), lane);
        }
        __syncwarp();
    }
    // owned cells take this subdomain's solution (P_i R_i^T)
    for (int i = lane; i < 3 * d.n_own; i += 32) {
        const int p = d.own[i / 3], c = i - 3 * (i / 3);
        z[3LL * d.cell[p] + c] = xv[3 * p + c];
    }
}

}  // namespace

size_t nf_work_doubles(int bx, int by, int bz) {
    const size_t S = (size_t)bx * bz, n = S * by;
    return std::max<size_t>(36 * (S + (size_t)bz), 6 * (n + S + (size_t)bz));
}

void launch_nf_factor(const NFDesc* descs, int ndesc, FactErr* err, cudaStream_t st) {
    if (ndesc > 0) k_nf_factor<<<(ndesc + 3) / 4, 128, 0, st>>>(descs, ndesc, err);
}

void launch_nf_apply(const SysTab* tab, const NFDesc* descs, int ndesc, cudaStream_t st) {
    if (ndesc > 0) k_nf_apply<<<(ndesc + 3) / 4, 128, 0, st>>>(tab, descs, ndesc);
}

}  // namespace asm2
