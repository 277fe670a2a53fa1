// Setup kernels: ELL fill of A, far-box coarse matrix, assembly of the local matrices
// A_i = R_i A R_i^T (Eq. 3.4 with the R_i of Eq. 4.1; Eq. B.3), the level-scheduled block ILU(0)
// with column-sum compensation (Section 2; cf. Eq. A.7) and the packing of the factor streams.
#include <cuda_fp16.h>

#include "asm2_internal.h"

namespace asm2 {

namespace {


// ELL slot w of row r <- BSR block rp[r] + w (the w-th stored block of the row).  Threads run over
// (w, r) with r fastest, so the nine element planes are written with unit stride across a warp;
// each thread reads its block's 72 contiguous bytes.  Padding slots keep their zeros.
__global__ void k_ell_fill(const double* __restrict__ bsr, const int* __restrict__ rp, int n, int ell_w,
                           double* __restrict__ ell, int rows_pad) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ell_w * n) return;
    const int w = (int)(t / n), r = (int)(t - (long long)w * n);
    const int e = rp[r] + w;
    if (e >= rp[r + 1]) return;
    const double* b = bsr + 9LL * e;
    double v[9];
#pragma unroll
    for (int k = 0; k < 9; k++) v[k] = b[k];
#pragma unroll
    for (int k = 0; k < 9; k++) ell[((long long)w * 9 + k) * rows_pad + r] = v[k];
}

// C[J, J'] = sum of the blocks of A coupling far box J to far box J' (one CTA per C block); block
// lists hold BSR block indices into the array-of-blocks copy of A
__global__ void k_coarse(const int* __restrict__ cptr, const int* __restrict__ cloc,
                         const double* __restrict__ bsr, double* __restrict__ cval) {
    const int c = blockIdx.x;
    double acc[9];
#pragma unroll
    for (int e = 0; e < 9; e++) acc[e] = 0.0;
    for (int i = cptr[c] + threadIdx.x; i < cptr[c + 1]; i += blockDim.x) {
        const int L = cloc[i];
#pragma unroll
        for (int e = 0; e < 9; e++) acc[e] += bsr[9LL * L + e];
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
                           const double* __restrict__ bsr, const double* __restrict__ cval,
                           double* __restrict__ slot, long long nslot, int long_min) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nslot * 9) return;
    long long s = t / 9;
    int e = (int)(t - s * 9);
    const int i0 = aptr[s], i1 = aptr[s + 1];
    if (i1 - i0 >= long_min) return;  // a whole warp sums this one (k_assemble_long)
    double acc = 0.0;
    int c = acs[s];
    if (c >= 0) acc = cval[(long long)c * 9 + e];
    for (int i = i0; i < i1; i++) {
        int L = aloc[i];
        if (L >= 0)
            acc += bsr[9LL * L + e];
        else
            acc -= bsr[9LL * ~L + e];
    }
    slot[t] = acc;
}

// Slots with long lists (far-lump blocks: the box-pair block minus thousands of near-region
// couplings): one warp per slot, lanes over the list four entries at a time with the loads issued
// first, nine partial sums per lane combined by shuffles
__global__ void __launch_bounds__(256) k_assemble_long(const int* __restrict__ aptr, const int* __restrict__ aloc,
                                                       const int* __restrict__ acs, const double* __restrict__ bsr,
                                                       const double* __restrict__ cval,
                                                       double* __restrict__ slot, const int* __restrict__ long_slots,
                                                       int nlong) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= nlong) return;
    const int s = long_slots[w];
    const int i0 = aptr[s], i1 = aptr[s + 1];
    double acc[9];
#pragma unroll
    for (int e = 0; e < 9; e++) acc[e] = 0.0;
    constexpr int kU = 4;
    for (int b = i0 + lane; b < i1; b += 32 * kU) {
        int L[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) L[u] = b + 32 * u < i1 ? aloc[b + 32 * u] : 0x7fffffff;
#pragma unroll
        for (int u = 0; u < kU; u++) {
            if (L[u] == 0x7fffffff) continue;
            const int loc = L[u] >= 0 ? L[u] : ~L[u];
            const double sg = L[u] >= 0 ? 1.0 : -1.0;
#pragma unroll
            for (int e = 0; e < 9; e++) acc[e] = fma(sg, bsr[9LL * loc + e], acc[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < 9; e++)
        for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
    if (lane < 9) {
        double v = 0.0;
#pragma unroll
        for (int e = 0; e < 9; e++)
            if (e == lane) v = acc[e];
        const int c = acs[s];
        if (c >= 0) v += cval[(long long)c * 9 + lane];
        slot[(long long)s * 9 + lane] = v;
    }
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
        // one reciprocal per pivot column: FP64 division expands to many FP64-pipe instructions
        const double id = 1.0 / m[c][c];
        for (int k = 0; k < 6; k++) m[c][k] *= id;
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
// D^{-1}.  All pairs reference slots finalised at lower levels.  Four CTAs per SM (64 registers):
// the 512 subdomains of a 1M-cell grid run in one wave, and the extra warps fill the FP64 pipe's
// gaps (the 1M-cell re-factor 11.35 -> 10.51 ms against two CTAs per SM; three was slower).
__global__ void __launch_bounds__(256, 4) k_factor(const FactDesc* __restrict__ fds, const int* __restrict__ ids,
                                                FactErr* err) {
    const FactDesc fd = fds[ids ? ids[blockIdx.x] : blockIdx.x];
    double* slot = fd.slot;
    // nine lanes per 3x3 result (lane = 3 r + c within a group), three groups per warp: each FP64
    // instruction then serves three targets instead of one thread's nine elements
    const int lane = threadIdx.x & 31, grp = lane / 9, e9 = lane - 9 * grp, er = e9 / 3, ec = e9 - 3 * er;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const bool lane_on = grp < 3;
    for (int lv = 0; lv < fd.nlev; lv++) {
        for (int t0 = fd.tgt_lv[lv] + 3 * warp; t0 < fd.tgt_lv[lv + 1]; t0 += 3 * nwarp) {
            const int t = t0 + grp;
            if (!lane_on || t >= fd.tgt_lv[lv + 1]) continue;
            double* s = slot + (long long)fd.tgt[t] * 9;
            double acc = s[e9];
            // kP pairs at a time: their indices, then their blocks, are loaded before any arithmetic
            // (the pairs are subtracted in the same order as one at a time)
            constexpr int kP = 4;
            const int q1 = fd.pp[t + 1];
            for (int q0 = fd.pp[t]; q0 < q1; q0 += kP) {
                int2 pr[kP];
#pragma unroll
                for (int u = 0; u < kP; u++) pr[u] = q0 + u < q1 ? fd.pair[q0 + u] : make_int2(-1, -1);
                double l[kP][3], uu[kP][3];
#pragma unroll
                for (int u = 0; u < kP; u++) {
                    const bool on = pr[u].x >= 0;
                    const double* L = slot + (long long)(on ? pr[u].x : 0) * 9 + 3 * er;
                    const double* U = slot + (long long)(on ? pr[u].y : 0) * 9 + ec;
                    l[u][0] = L[0];
                    l[u][1] = L[1];
                    l[u][2] = L[2];
                    uu[u][0] = U[0];
                    uu[u][1] = U[3];
                    uu[u][2] = U[6];
                }
#pragma unroll
                for (int u = 0; u < kP; u++)
                    if (pr[u].x >= 0)  // three FMAs into the running value (not product, sum, subtract)
                        acc = fma(-l[u][2], uu[u][2], fma(-l[u][1], uu[u][1], fma(-l[u][0], uu[u][0], acc)));
            }
            s[e9] = acc;
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
        for (int t0 = fd.ls_lv[lv] + 3 * warp; t0 < fd.ls_lv[lv + 1]; t0 += 3 * nwarp) {
            const int t = t0 + grp;
            double v = 0.0;
            int2 q = make_int2(0, 0);
            const bool on = lane_on && t < fd.ls_lv[lv + 1];
            if (on) {
                q = fd.ls[t];
                const double* A = slot + (long long)q.x * 9 + 3 * er;
                const double* Di = slot + (long long)q.y * 9 + ec;
                v = A[0] * Di[0] + A[1] * Di[3] + A[2] * Di[6];
            }
            __syncwarp();  // every lane of the group has read its row of L before any writes
            if (on) slot[(long long)q.x * 9 + e9] = v;
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

void launch_ell_fill(const double* bsr_vals, const int* row_ptr, int n, int ell_w, double* ell_val, int rows_pad,
                     cudaStream_t st) {
    if (n <= 0 || ell_w <= 0) return;
    k_ell_fill<<<blocks_for((long long)ell_w * n, 256), 256, 0, st>>>(bsr_vals, row_ptr, n, ell_w, ell_val, rows_pad);
}

void launch_coarse(const int* cptr, const int* cloc, const double* bsr_val, double* cval, int nc,
                   cudaStream_t st) {
    if (nc <= 0) return;
    k_coarse<<<nc, 256, 0, st>>>(cptr, cloc, bsr_val, cval);
}

void launch_assemble(const int* aptr, const int* aloc, const int* acs, const double* bsr_val,
                     const double* cval, double* slot, long long nslot, cudaStream_t st, const int* long_slots,
                     int nlong) {
    if (nslot <= 0) return;
    const int long_min = long_slots ? kLongAssembly : 0x7fffffff;
    k_assemble<<<blocks_for(nslot * 9, 256), 256, 0, st>>>(aptr, aloc, acs, bsr_val, cval, slot, nslot,
                                                           long_min);
    if (long_slots && nlong > 0)
        k_assemble_long<<<(nlong + 7) / 8, 256, 0, st>>>(aptr, aloc, acs, bsr_val, cval, slot, long_slots,
                                                         nlong);
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
