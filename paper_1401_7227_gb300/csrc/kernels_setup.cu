// Setup kernels: ELL fill of A, far-box coarse matrix, assembly of the local matrices
// A_i = R_i A R_i^T (Eq. 3.4 with the R_i of Eq. 4.1; Eq. B.3), the level-scheduled block ILU(0)
// with column-sum compensation (Section 2; cf. Eq. A.7) and the packing of the factor streams.
#include <cuda_fp16.h>

#include "asm2_internal.h"

namespace asm2 {

namespace {

__device__ __forceinline__ double ell_at(const double* ell_val, int rows_pad, int loc, int e) {
    const int w = loc / rows_pad, r = loc - w * rows_pad;
    return ell_val[((long long)w * 9 + e) * rows_pad + r];
}

// BSR block e -> ELL slot loc = w * rows_pad + r
__global__ void k_ell_fill(const double* __restrict__ bsr, const int* __restrict__ loc, long long nnzb,
                           double* __restrict__ ell, int rows_pad) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnzb * 9) return;
    long long e = t / 9;
    int k = (int)(t - e * 9);
    int L = loc[e];
    int w = L / rows_pad, r = L - w * rows_pad;
    ell[((long long)w * 9 + k) * rows_pad + r] = bsr[t];
}

// C[J, J'] = sum of the blocks of A coupling far box J to far box J' (one CTA per C block)
__global__ void k_coarse(const int* __restrict__ cptr, const int* __restrict__ cloc,
                         const double* __restrict__ ell, int rows_pad, double* __restrict__ cval) {
    const int c = blockIdx.x;
    double acc[9];
#pragma unroll
    for (int e = 0; e < 9; e++) acc[e] = 0.0;
    for (int i = cptr[c] + threadIdx.x; i < cptr[c + 1]; i += blockDim.x) {
        const int L = cloc[i];
#pragma unroll
        for (int e = 0; e < 9; e++) acc[e] += ell_at(ell, rows_pad, L, e);
    }
    __shared__ double red[9][256];
#pragma unroll
    for (int e = 0; e < 9; e++) red[e][threadIdx.x] = acc[e];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int e = 0; e < 9; e++) red[e][threadIdx.x] += red[e][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 9) cval[(long long)c * 9 + threadIdx.x] = red[threadIdx.x][0];
}

// slot value = C block (far-far pairs) + signed sum of A blocks from the slot's list
__global__ void k_assemble(const int* __restrict__ aptr, const int* __restrict__ aloc, const int* __restrict__ acs,
                           const double* __restrict__ ell, int rows_pad, const double* __restrict__ cval,
                           double* __restrict__ slot, long long nslot) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nslot * 9) return;
    long long s = t / 9;
    int e = (int)(t - s * 9);
    double acc = 0.0;
    int c = acs[s];
    if (c >= 0) acc = cval[(long long)c * 9 + e];
    for (int i = aptr[s]; i < aptr[s + 1]; i++) {
        int L = aloc[i];
        if (L >= 0)
            acc += ell_at(ell, rows_pad, L, e);
        else
            acc -= ell_at(ell, rows_pad, ~L, e);
    }
    slot[t] = acc;
}

// 3x3 inverse by Gauss-Jordan elimination with partial pivoting; false on a zero pivot.
__device__ bool inverse3(const double* a, double* inv) {
    double m[3][6];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            m[r][c] = a[3 * r + c];
            m[r][3 + c] = (r == c) ? 1.0 : 0.0;
        }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        int p = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(m[r][c]) > fabs(m[p][c])) p = r;
        if (m[p][c] == 0.0) return false;
        if (p != c)
            for (int k = 0; k < 6; k++) {
                double t = m[c][k];
                m[c][k] = m[p][k];
                m[p][k] = t;
            }
        const double d = m[c][c];
        for (int k = 0; k < 6; k++) m[c][k] /= d;
        for (int r = 0; r < 3; r++) {
            if (r == c) continue;
            const double f = m[r][c];
            for (int k = 0; k < 6; k++) m[r][k] -= f * m[c][k];
        }
    }
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) inv[3 * r + c] = m[r][3 + c];
    return true;
}

// Right-looking block ILU(0) (+ colsum) in "pull" form, one CTA per subdomain.  Level by level:
// (A) every slot finalised at this level subtracts its (L, U) pairs in the order the
// right-looking update would apply them (compensations of dropped fill are pairs of the
// diagonal slots); (B) the level's pivots are inverted; (C) its L column blocks are scaled by
// D^{-1}.  All pairs reference slots finalised at lower levels.
__global__ void __launch_bounds__(256) k_factor(const FactDesc* __restrict__ fds, const int* __restrict__ ids,
                                                FactErr* err) {
    const FactDesc fd = fds[ids ? ids[blockIdx.x] : blockIdx.x];
    double* slot = fd.slot;
    for (int lv = 0; lv < fd.nlev; lv++) {
        for (int t = fd.tgt_lv[lv] + threadIdx.x; t < fd.tgt_lv[lv + 1]; t += blockDim.x) {
            double* s = slot + (long long)fd.tgt[t] * 9;
            double acc[9];
#pragma unroll
            for (int e = 0; e < 9; e++) acc[e] = s[e];
            for (int q = fd.pp[t]; q < fd.pp[t + 1]; q++) {
                const int2 pr = fd.pair[q];
                const double* L = slot + (long long)pr.x * 9;
                const double* U = slot + (long long)pr.y * 9;
                double l[9], u[9];
#pragma unroll
                for (int e = 0; e < 9; e++) {
                    l[e] = L[e];
                    u[e] = U[e];
                }
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        acc[3 * r + c] -= l[3 * r] * u[c] + l[3 * r + 1] * u[3 + c] + l[3 * r + 2] * u[6 + c];
            }
#pragma unroll
            for (int e = 0; e < 9; e++) s[e] = acc[e];
        }
        __syncthreads();
        for (int p = fd.lv_pos0[lv] + threadIdx.x; p < fd.lv_pos0[lv + 1]; p += blockDim.x) {
            double* d = slot + (long long)fd.diag_of_pos[p] * 9;
            double D[9], Di[9];
#pragma unroll
            for (int e = 0; e < 9; e++) D[e] = d[e];
            double* dp = fd.dpiv + (long long)fd.row_of_pos[p] * 9;
#pragma unroll
            for (int e = 0; e < 9; e++) dp[e] = D[e];
            if (!inverse3(D, Di)) {
                if (atomicCAS(&err->flag, 0, 1) == 0) {
                    err->sub = ids ? ids[blockIdx.x] : blockIdx.x;
                    err->row = fd.row_of_pos[p];
                }
#pragma unroll
                for (int e = 0; e < 9; e++) Di[e] = (e % 4 == 0) ? 1.0 : 0.0;
            }
#pragma unroll
            for (int e = 0; e < 9; e++) d[e] = Di[e];
        }
        __syncthreads();
        for (int t = fd.ls_lv[lv] + threadIdx.x; t < fd.ls_lv[lv + 1]; t += blockDim.x) {
            const int2 q = fd.ls[t];
            double* L = slot + (long long)q.x * 9;
            const double* Di = slot + (long long)q.y * 9;
            double a[9], di[9];
#pragma unroll
            for (int e = 0; e < 9; e++) {
                a[e] = L[e];
                di[e] = Di[e];
            }
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++)
                    L[3 * r + c] = a[3 * r] * di[c] + a[3 * r + 1] * di[3 + c] + a[3 * r + 2] * di[6 + c];
        }
        __syncthreads();
    }
}

// One thread per 3x3 block.  FP16 blocks are stored as 9 halves of v * 2^-e followed by e (int16),
// with e chosen so that the largest magnitude lands in [0.5, 1): U (~T) and D^{-1} (~1/T) then both
// keep FP16's full relative precision instead of overflowing or underflowing.
template <typename T>
__global__ void k_pack(const long long* __restrict__ off, const int* __restrict__ src, long long n,
                       unsigned char* __restrict__ base, const double* __restrict__ slot) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* v = slot + (long long)src[i] * 9;
    if constexpr (sizeof(T) == 2) {
        double mx = 0.0;
#pragma unroll
        for (int e = 0; e < 9; e++) mx = fmax(mx, fabs(v[e]));
        int ex = 0;
        if (mx > 0.0) ex = ilogb(mx) + 1;
        __half* dst = reinterpret_cast<__half*>(base + off[i]);
#pragma unroll
        for (int e = 0; e < 9; e++) dst[e] = __double2half(ldexp(v[e], -ex));
        reinterpret_cast<short*>(dst)[9] = (short)ex;
    } else {
        T* dst = reinterpret_cast<T*>(base + off[i]);
#pragma unroll
        for (int e = 0; e < 9; e++) dst[e] = (T)v[e];
    }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_ell_fill(const double* bsr_vals, const int* ell_loc, long long nnzb, double* ell_val, int rows_pad,
                     int, cudaStream_t st) {
    if (nnzb <= 0) return;
    k_ell_fill<<<blocks_for(nnzb * 9, 256), 256, 0, st>>>(bsr_vals, ell_loc, nnzb, ell_val, rows_pad);
}

void launch_coarse(const int* cptr, const int* cloc, const double* ell_val, int rows_pad, double* cval, int nc,
                   cudaStream_t st) {
    if (nc <= 0) return;
    k_coarse<<<nc, 256, 0, st>>>(cptr, cloc, ell_val, rows_pad, cval);
}

void launch_assemble(const int* aptr, const int* aloc, const int* acs, const double* ell_val, int rows_pad,
                     const double* cval, double* slot, long long nslot, cudaStream_t st) {
    if (nslot <= 0) return;
    k_assemble<<<blocks_for(nslot * 9, 256), 256, 0, st>>>(aptr, aloc, acs, ell_val, rows_pad, cval, slot, nslot);
}

void launch_factor(const FactDesc* fd, int nsub, FactErr* err, const int* sub_ids, cudaStream_t st) {
    if (nsub <= 0) return;
    k_factor<<<nsub, 256, 0, st>>>(fd, sub_ids, err);
}

void launch_pack(const long long* off, const int* src, long long n, int prec, unsigned char* stream_base,
                 const double* slot_base, cudaStream_t st) {
    if (n <= 0) return;
    unsigned g = blocks_for(n, 256);
    if (prec == 0)
        k_pack<double><<<g, 256, 0, st>>>(off, src, n, stream_base, slot_base);
    else if (prec == 1)
        k_pack<float><<<g, 256, 0, st>>>(off, src, n, stream_base, slot_base);
    else
        k_pack<__half><<<g, 256, 0, st>>>(off, src, n, stream_base, slot_base);
}

}  // namespace asm2
