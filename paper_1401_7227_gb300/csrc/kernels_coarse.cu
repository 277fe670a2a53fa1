// Classical coarse-grid corrections (Section 3, Eqs. 3.5-3.8), the comparators of the paper's
// boundary-conditioned method:
//   two-level:  z = B_AS^{-1} r + R_C^T A_C^{-1} R_C r                       (Eq. 3.5)
//   two-stage:  z = B_AS^{-1} r + R_C^T A_C^{-1} R_C (r - A B_AS^{-1} r)     (Eqs. 3.7-3.8)
// R_C sums the 3-vectors of each coarse box's cells, R_C^T copies a box's value to its cells and
// A_C = R_C A R_C^T (Eq. 3.6).  A_C is small (3 unknowns per coarse box), so it is inverted once
// per factorisation (Gauss-Jordan elimination with partial pivoting, FP64, kernels_dense.cu) and
// applied as a dense matrix-vector product.
#include <cuda_runtime.h>

#include <algorithm>

#include "asm2_internal.h"

namespace asm2 {
namespace {

// ------------------------------------------------------------------------------------------
// Setup: scatter the box-pair blocks into the augmented matrix [A_C | I] (n x 2n, row-major)
// ------------------------------------------------------------------------------------------
__global__ void k_coarse_init(long long n, double* __restrict__ aug) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 2 * n) return;
    const long long i = t / (2 * n), j = t - i * 2 * n;
    aug[t] = (j == n + i) ? 1.0 : 0.0;  // [0 | I]; the blocks of A_C are added next
}

__global__ void k_coarse_scatter(const long long* __restrict__ keys, const double* __restrict__ blocks, int nkeys,
                                 int nb, double* __restrict__ aug) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 9LL * nkeys) return;
    const long long q = t / 9;
    const int e = (int)(t - q * 9);
    const long long I = keys[q] / nb, J = keys[q] - (keys[q] / nb) * nb;
    const long long n = 3LL * nb;
    aug[(3 * I + e / 3) * 2 * n + 3 * J + e % 3] = blocks[9 * q + e];
}

// ------------------------------------------------------------------------------------------
// Apply (per system, gated by SysTab::cmode and an active apply)
// ------------------------------------------------------------------------------------------

// two-stage: w = r - A z (r = apply input, z = apply output of the local solves)
__global__ void __launch_bounds__(256) k_coarse_resid(const SysTab* __restrict__ tab, const RowItem* __restrict__ items) {
    const RowItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.cmode != 2) return;
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const int row = it.r0 + threadIdx.x;
    if (row >= st.n_cells) return;
    const double* __restrict__ r = st.ws + (long long)in * st.n3p;
    const double* __restrict__ z = st.ws + (long long)st.ctl[C_APPLY_OUT] * st.n3p;
    const long long rp = st.rows_pad;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < st.ell_w; w++) {
        const int c = st.ell_col[(long long)w * rp + row];
        const double x0 = z[3LL * c], x1 = z[3LL * c + 1], x2 = z[3LL * c + 2];
        const double* v = st.ell_val + (long long)w * 9 * rp + row;
        a0 += v[0] * x0 + v[rp] * x1 + v[2 * rp] * x2;
        a1 += v[3 * rp] * x0 + v[4 * rp] * x1 + v[5 * rp] * x2;
        a2 += v[6 * rp] * x0 + v[7 * rp] * x1 + v[8 * rp] * x2;
    }
    st.cw[3LL * row] = r[3LL * row] - a0;
    st.cw[3LL * row + 1] = r[3LL * row + 1] - a1;
    st.cw[3LL * row + 2] = r[3LL * row + 2] - a2;
}

// R_C: sum of the input over the cells of one coarse box (the apply input, or w for two-stage)
__global__ void __launch_bounds__(128) k_coarse_sum(const SysTab* __restrict__ tab, const BoxItem* __restrict__ items) {
    const BoxItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.cmode == 0) return;
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const double* __restrict__ x = st.cmode == 2 ? st.cw : st.ws + (long long)in * st.n3p;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int i = it.b0 + threadIdx.x; i < it.b1; i += blockDim.x) {
        const long long c = 3LL * it.cells[i];
        a0 += x[c];
        a1 += x[c + 1];
        a2 += x[c + 2];
    }
    __shared__ double red[3][128];
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
            red[2][threadIdx.x] += red[2][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) st.crc[3 * it.out + threadIdx.x] = red[threadIdx.x][0];
}

// y_C = A_C^{-1} (R_C x): one warp per row of the inverse (the right half of [I | A_C^{-1}])
__global__ void __launch_bounds__(256) k_coarse_gemv(const SysTab* __restrict__ tab, const RowItem* __restrict__ items) {
    const RowItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.cmode == 0 || st.ctl[C_APPLY_IN] < 0) return;
    const int n = 3 * st.cnb;
    const int row = it.r0 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;
    const double* a = st.caug + (long long)row * 2 * n + n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(a[j], st.crc[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) st.cyc[row] = s;
}

// R_C^T: z[cell] += y_C[box of cell]
__global__ void __launch_bounds__(VEC_THREADS) k_coarse_prolong(const SysTab* __restrict__ tab,
                                                                const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.cmode == 0 || st.ctl[C_APPLY_IN] < 0) return;
    double* z = st.ws + (long long)st.ctl[C_APPLY_OUT] * st.n3p;
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
        const long long e = e0 + i;
        if (e >= st.n3) break;
        const long long cell = e / 3;
        z[e] += st.cyc[3 * st.cbox[cell] + (int)(e - 3 * cell)];
    }
}

}  // namespace

cudaError_t launch_coarse_invert(const long long* keys, const double* blocks, int nkeys, int nb, double* aug,
                                 const GJMat* mat, double* part, int part_cap, int* err, int device, cudaStream_t st) {
    const long long n = 3LL * nb;
    const long long tot = n * 2 * n;
    k_coarse_init<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, aug);
    if (nkeys > 0) k_coarse_scatter<<<(unsigned)((9LL * nkeys + 255) / 256), 256, 0, st>>>(keys, blocks, nkeys, nb, aug);
    return launch_gj_run(mat, 1, (int)n, part, part_cap, err, device, st);
}

void launch_coarse_apply(const SysTab* tab, const RowItem* rows, int nrows, const BoxItem* boxes, int nboxes,
                         const RowItem* grows, int ngrows, const VecItem* vecs, int nvecs, bool two_stage,
                         cudaStream_t st) {
    if (nboxes <= 0) return;
    if (two_stage && nrows > 0) k_coarse_resid<<<nrows, 256, 0, st>>>(tab, rows);
    k_coarse_sum<<<nboxes, 128, 0, st>>>(tab, boxes);
    if (ngrows > 0) k_coarse_gemv<<<ngrows, 256, 0, st>>>(tab, grows);
    if (nvecs > 0) k_coarse_prolong<<<nvecs, VEC_THREADS, 0, st>>>(tab, vecs);
}

}  // namespace asm2
