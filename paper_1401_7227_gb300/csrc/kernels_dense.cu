// Dense inverses by Gauss-Jordan elimination with partial pivoting, for several matrices in one
// cooperative launch (the exact local solves A_i^{-1} of Section 5 and the coarse matrix A_C^{-1}
// of Eq. 3.5), and the exact-local-solve apply.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "asm2_internal.h"

namespace asm2 {
namespace {

// Every matrix is an augmented [A | I] (n x 2n, row-major) inverted in place; G / nmat CTAs work on
// each.  Per pivot column k (all groups step together, a matrix with n <= k idles):
//  (A) each CTA finds the largest |a(i,k)|, i >= k, among its rows of its matrix;
//  (B) every CTA of the group reduces its group's partials in the same order (ties: lowest row),
//      then the group saves the pivot row scaled by 1/pivot and the column multipliers;
//  (C) every row is updated, rows k and p exchanged on the way.
// A zero pivot column marks the matrix (err[m] = 1 + k) and its group stops working on it, but every
// CTA still meets every grid barrier.
__global__ void __launch_bounds__(256) k_gj_batched(const GJMat* __restrict__ mats, int nmat, int nmax,
                                                    double* __restrict__ part, int* __restrict__ err) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int per = gridDim.x / nmat;  // CTAs per matrix (the launch makes this >= 1)
    const int m = blockIdx.x / per, rank = blockIdx.x - m * per;
    const bool mine = m < nmat;
    GJMat M{};
    if (mine) M = mats[m];
    const int n = mine ? M.n : 0;
    const long long W = 2LL * n;
    const long long gtid = (long long)rank * blockDim.x + threadIdx.x;
    const long long gstride = (long long)per * blockDim.x;
    __shared__ double sval[256];
    __shared__ int sidx[256];
    __shared__ int piv_row;
    __shared__ double piv_val;
    __shared__ bool dead;
    if (threadIdx.x == 0) dead = !mine;
    __syncthreads();
    for (int k = 0; k < nmax; k++) {
        const bool active = !dead && k < n;
        // (A)
        double best = -1.0;
        int bi = n;
        if (active)
            for (long long i = k + gtid; i < n; i += gstride) {
                const double a = fabs(M.aug[i * W + k]);
                if (a > best) {
                    best = a;
                    bi = (int)i;
                }
            }
        sval[threadIdx.x] = best;
        sidx[threadIdx.x] = bi;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                const double o = sval[threadIdx.x + s];
                const int oi = sidx[threadIdx.x + s];
                if (o > sval[threadIdx.x] || (o == sval[threadIdx.x] && oi < sidx[threadIdx.x])) {
                    sval[threadIdx.x] = o;
                    sidx[threadIdx.x] = oi;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = sval[0];
            part[2 * blockIdx.x + 1] = (double)sidx[0];
        }
        grid.sync();
        // (B)
        if (threadIdx.x == 0) {
            double b = -1.0;
            int p = n;
            if (active)
                for (int c = m * per; c < (m + 1) * per; c++) {
                    const double v = __ldcg(&part[2 * c]);
                    const int vi = (int)__ldcg(&part[2 * c + 1]);
                    if (v > b || (v == b && vi < p)) {
                        b = v;
                        p = vi;
                    }
                }
            piv_row = p;
            piv_val = (active && p < n) ? __ldcg(&M.aug[(long long)p * W + k]) : 0.0;
            if (active && (p >= n || piv_val == 0.0)) {
                dead = true;
                if (rank == 0) err[m] = 1 + k;
            }
        }
        __syncthreads();
        const bool go = active && !dead;
        const int p = piv_row;
        if (go) {
            const double inv = 1.0 / piv_val;
            for (long long j = gtid; j < W; j += gstride) M.prow[j] = M.aug[(long long)p * W + j] * inv;
            for (long long i = gtid; i < n; i += gstride) {
                const long long src = (i == k) ? p : (i == p ? k : i);  // after exchanging rows k and p
                M.fcol[i] = (i == k) ? 0.0 : M.aug[src * W + k];
            }
        }
        grid.sync();
        // (C) row k <- scaled pivot row; row p <- old row k minus its multiple; others in place.
        // One warp per row: a row whose multiplier is zero keeps every entry (its pivot-column
        // entry is already zero), so the warp skips it whole.
        if (go) {
            const int wpc = blockDim.x >> 5, lane = threadIdx.x & 31;
            const long long gw = (long long)rank * wpc + (threadIdx.x >> 5), nw = (long long)per * wpc;
            for (long long i = gw; i < n; i += nw) {
                if (i == p && p != k) continue;  // handled together with row k
                if (i == k) {
                    double* rk = M.aug + (long long)k * W;
                    double* rp = M.aug + (long long)p * W;
                    const double fp = M.fcol[p];
                    for (long long j = lane; j < W; j += 32) {
                        const double pj = M.prow[j];
                        if (p != k) rp[j] = (j == k) ? 0.0 : rk[j] - fp * pj;
                        rk[j] = pj;
                    }
                    continue;
                }
                const double f = M.fcol[i];
                if (f == 0.0) continue;
                double* ri = M.aug + i * W;
                for (long long j = lane; j < W; j += 32) {
                    const double pj = M.prow[j];
                    if (j == k)
                        ri[j] = 0.0;
                    else if (pj != 0.0)
                        ri[j] -= f * pj;
                }
            }
        }
        grid.sync();
    }
}

// [0 | I] for every matrix: one CTA per row
__global__ void __launch_bounds__(256) k_gj_init(const GJMat* __restrict__ mats, const int2* __restrict__ rows) {
    const int2 it = rows[blockIdx.x];  // (matrix, row)
    const GJMat M = mats[it.x];
    const long long W = 2LL * M.n;
    double* a = M.aug + (long long)it.y * W;
    for (long long j = threadIdx.x; j < W; j += blockDim.x) a[j] = (j == M.n + it.y) ? 1.0 : 0.0;
}

// local matrices A_i (assembled 3x3 slots) into the left halves: slot t's (0,0) element goes to
// offset off[t] from the start of its own augmented matrix, whose row stride is 2 n
__global__ void k_dense_scatter(const double* __restrict__ slot, const long long* __restrict__ off,
                                const int* __restrict__ mat_of_slot, const GJMat* __restrict__ mats, long long nslot) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 9 * nslot) return;
    const long long q = t / 9;
    const int e = (int)(t - 9 * q);
    const GJMat M = mats[mat_of_slot[q]];
    M.aug[off[q] + (long long)(e / 3) * 2 * M.n + e % 3] = slot[9 * q + e];
}

// Exact local solve, owned rows only: z[own cell] = (A_i^{-1} R_i r)[own row], one warp per row
__global__ void __launch_bounds__(256) k_dense_apply(const SysTab* __restrict__ tab, const SubDesc* __restrict__ subs,
                                                     const int2* __restrict__ items) {
    const int2 it = items[blockIdx.x];  // (subdomain work item, first owned row of 8)
    const SubDesc& sd = subs[it.x];
    const SysTab& st = tab[sd.sys];
    const int out = st.ctl[C_APPLY_OUT];
    if (st.ctl[C_APPLY_IN] < 0) return;
    const int q = it.y + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (q >= 3 * sd.n_own) return;
    const int t = q / 3, comp = q - 3 * t;
    const int n3 = 3 * (sd.nf + sd.nc);
    const double* a = sd.dinv + (long long)(3 * sd.own_pos[t] + comp) * 2 * n3 + n3;
    double s = 0.0;
    for (int j = lane; j < n3; j += 32) s = fma(a[j], sd.y[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) st.ws[(long long)out * st.n3p + 3LL * sd.own_cell[t] + comp] = s;
}

}  // namespace

void launch_gj_init(const GJMat* mats, const int2* rows, int nrows, cudaStream_t st) {
    if (nrows > 0) k_gj_init<<<nrows, 256, 0, st>>>(mats, rows);
}

cudaError_t launch_gj_run(const GJMat* mats, int nmat, int nmax, double* part, int part_cap, int* err, int device,
                          cudaStream_t st) {
    if (nmat <= 0) return cudaSuccess;
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_batched, 256, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int cap = std::min(std::min(std::max(1, per_sm), 2) * std::max(1, sms), part_cap);
    if (cap < nmat) return cudaErrorInvalidValue;  // more matrices than co-resident CTAs
    const int per = cap / nmat;
    int grid = per * nmat;
    void* args[] = {(void*)&mats, (void*)&nmat, (void*)&nmax, (void*)&part, (void*)&err};
    return cudaLaunchCooperativeKernel((const void*)k_gj_batched, dim3(grid), dim3(256), args, 0, st);
}

void launch_dense_scatter(const double* slot, const long long* off, const int* mat_of_slot, const GJMat* mats,
                          long long nslot, cudaStream_t st) {
    if (nslot <= 0) return;
    k_dense_scatter<<<(unsigned)((9 * nslot + 255) / 256), 256, 0, st>>>(slot, off, mat_of_slot, mats, nslot);
}

void launch_dense_apply(const SysTab* tab, const SubDesc* subs, const int2* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_dense_apply<<<nitems, 256, 0, st>>>(tab, subs, items);
}

}  // namespace asm2
