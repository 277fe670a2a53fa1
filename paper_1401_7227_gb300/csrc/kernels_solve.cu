// Kernels of one Krylov step: far-box sums, the fused additive Schwarz apply
// (restriction -> forward sweep -> backward sweep -> owned-row scatter, Eqs. 4.2-4.5), the BSR
// SpMV, and the GMRES vector/state kernels (modified Gram-Schmidt Arnoldi with Givens rotations,
// Section 2).  Every kernel reads its system's control words, so systems at different points of
// their solve share the same launches.
#include <cuda_fp16.h>

#include <algorithm>
#include <cooperative_groups.h>

#include "asm2_internal.h"
#include "f64cvt.h"
#include "tma.h"

namespace asm2 {

namespace {

// residual values into a local vector's type; FP32 on the integer pipes (f64cvt.h)
template <typename T>
__device__ __forceinline__ T narrow(double v) {
    return (T)v;
}
template <>
__device__ __forceinline__ float narrow<float>(double v) {
    return f64_to_f32(v);
}

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Stored fine blocks: 9 FP32 values, or 9 FP16 values scaled by 2^-e followed by e (int16).
template <typename T>
struct FineBlock;
template <>
struct FineBlock<float> {
    static constexpr int bytes = 36;
    __device__ static __forceinline__ void load(const unsigned char* p, float* w) {
        const float* f = reinterpret_cast<const float*>(p);
#pragma unroll
        for (int e = 0; e < 9; e++) w[e] = f[e];
    }
};
template <>
struct FineBlock<__half> {
    static constexpr int bytes = 20;
    __device__ static __forceinline__ void load(const unsigned char* p, float* w) {
        const __half* h = reinterpret_cast<const __half*>(p);
        const float sc = ldexpf(1.0f, reinterpret_cast<const short*>(p)[9]);
#pragma unroll
        for (int e = 0; e < 9; e++) w[e] = __half2float(h[e]) * sc;
    }
};
template <>
struct FineBlock<double> {
    static constexpr int bytes = 72;
};

// a -= V x for one stored 3x3 block V (row-major) and a 3-vector x, as negated fused multiply-adds.
// FP32 blocks: 9 loads.  FP16 blocks (9 halves scaled by 2^-e, then e): 5 32-bit loads, the product
// of the unscaled block, then one multiply-add by 2^e per component (a power of two: exact).
template <typename TF>
__device__ __forceinline__ void block_mv_sub(const unsigned char* p, float x0, float x1, float x2, float& a0, float& a1,
                                             float& a2);
template <>
__device__ __forceinline__ void block_mv_sub<float>(const unsigned char* p, float x0, float x1, float x2, float& a0,
                                                    float& a1, float& a2) {
    const float* v = reinterpret_cast<const float*>(p);
    a0 = fmaf(-v[0], x0, fmaf(-v[1], x1, fmaf(-v[2], x2, a0)));
    a1 = fmaf(-v[3], x0, fmaf(-v[4], x1, fmaf(-v[5], x2, a1)));
    a2 = fmaf(-v[6], x0, fmaf(-v[7], x1, fmaf(-v[8], x2, a2)));
}
template <>
__device__ __forceinline__ void block_mv_sub<__half>(const unsigned char* p, float x0, float x1, float x2, float& a0,
                                                     float& a1, float& a2) {
    const unsigned* w = reinterpret_cast<const unsigned*>(p);
    const unsigned w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3], w4 = w[4];
    const float2 v01 = __half22float2(*reinterpret_cast<const __half2*>(&w0));
    const float2 v23 = __half22float2(*reinterpret_cast<const __half2*>(&w1));
    const float2 v45 = __half22float2(*reinterpret_cast<const __half2*>(&w2));
    const float2 v67 = __half22float2(*reinterpret_cast<const __half2*>(&w3));
    const float v8 = __half2float(__ushort_as_half((unsigned short)(w4 & 0xffffu)));
    const int ex = (int)(short)(w4 >> 16);
    const float sc = __int_as_float((127 + ex) << 23);  // 2^ex: |ex| is far below 126 for these factors
    const float t0 = fmaf(v01.x, x0, fmaf(v01.y, x1, v23.x * x2));
    const float t1 = fmaf(v23.y, x0, fmaf(v45.x, x1, v45.y * x2));
    const float t2 = fmaf(v67.x, x0, fmaf(v67.y, x1, v8 * x2));
    a0 = fmaf(-sc, t0, a0);
    a1 = fmaf(-sc, t1, a1);
    a2 = fmaf(-sc, t2, a2);
}

// ------------------------------------------------------------------------------------------
// gather sums of the apply input: far-box sums (kind 0) and, per subdomain, the sums of the
// near-region cells of each far box (kind 1); a far lump's restricted residual is their difference
// ------------------------------------------------------------------------------------------
// the 3-vector of one sum-list entry: a cell's entries of r, or a cell group's sum
__device__ __forceinline__ const double* sum_entry(const SysTab& st, const double* r, int e) {
    return e >= 0 ? r + 3LL * e : st.gsum + 3LL * ~e;
}

// Sums of the apply input over aligned 2x2x2 cell groups, thread per group, the group's cells in a
// fixed order (y, then x, then z): every list sum that covers whole groups reads these instead
__global__ void __launch_bounds__(256) k_groups(const SysTab* __restrict__ tab, const BoxItem* __restrict__ items) {
    const BoxItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const int G = it.b0 + threadIdx.x;
    if (G >= it.b1) return;
    const double* r = st.ws + (long long)in * st.n3p;
    const int ngz = (st.gnz + 1) >> 1, ngx = (st.gnx + 1) >> 1;
    const int gz = G % ngz, t = G / ngz, gx = t % ngx, gy = t / ngx;
    const int z0 = 2 * gz, x0 = 2 * gx, y0 = 2 * gy;
    const int z1 = min(z0 + 2, st.gnz), x1 = min(x0 + 2, st.gnx), y1 = min(y0 + 2, st.gny);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int y = y0; y < y1; y++)
        for (int x = x0; x < x1; x++)
            for (int z = z0; z < z1; z++) {
                const double* rc = r + 3LL * (z + (long long)st.gnz * (x + (long long)st.gnx * y));
                a0 += rc[0];
                a1 += rc[1];
                a2 += rc[2];
            }
    double* o = st.gsum + 3LL * G;
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
}

__global__ void __launch_bounds__(128) k_sums(const SysTab* __restrict__ tab, const BoxItem* __restrict__ items) {
    const BoxItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const double* r = st.ws + (long long)in * st.n3p;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 4
    for (int i = it.b0 + threadIdx.x; i < it.b1; i += blockDim.x) {
        const double* v = sum_entry(st, r, it.cells[i]);
        a0 += v[0];
        a1 += v[1];
        a2 += v[2];
    }
    __shared__ double red[3][128];
    red[0][threadIdx.x] = a0;
    red[1][threadIdx.x] = a1;
    red[2][threadIdx.x] = a2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
            red[2][threadIdx.x] += red[2][threadIdx.x + s];
        }
        __syncthreads();
    }
    double* out = it.kind == 0 ? st.boxsum : st.corr;
    if (threadIdx.x < 3) out[(long long)it.out * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// ------------------------------------------------------------------------------------------
// fused local solve of one subdomain (one CTA): y = R_i r; y = L^{-1} y; y = U^{-1} y;
// z[owned cells] = y[owned fine rows] (Eqs. 4.2-4.5).  Fine rows and lump rows live in separate
// local vectors (fine rows at the factor precision, lumps in FP64), in shared memory when they
// fit.  Levels are separated by CTA barriers.  Fine rows (<= 6 blocks) take one thread each;
// lump rows (up to ~70 blocks) take one warp each.
// ------------------------------------------------------------------------------------------
template <typename TF>
struct Compute {
    using T = float;  // fine rows of FP32/FP16 factors are applied in FP32
};
template <>
struct Compute<double> {
    using T = double;
};

template <typename TF>
__device__ __forceinline__ void load_fine(const unsigned char* p, typename Compute<TF>::T* w) {
    if constexpr (sizeof(TF) == 8) {
        const double* d = reinterpret_cast<const double*>(p);
#pragma unroll
        for (int e = 0; e < 9; e++) w[e] = d[e];
    } else {
        FineBlock<TF>::load(p, w);
    }
}

__device__ __forceinline__ void warp_sum3(double& a0, double& a1, double& a2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
}

// TMA bulk copies into a ring of shared-memory slots, completion tracked by mbarriers, with
// bounded waits (tma.h).
using tma::bulk_load;
using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait;

constexpr int kMaxSlots = 4;  // ring slots of the apply: a template argument, 2..kMaxSlots
constexpr int kRingHeader = 64;  // mbarriers

// One chunk of the forward (lower = true) or backward sweep, read from shared memory.  TL is the
// lump rows' storage and arithmetic type (double, or float with FP32/FP16 fine rows); ycf is the
// FP32 mirror of FP64 lump values that FP32 fine rows read (nullptr otherwise).
template <typename TF, typename TL>
__device__ __forceinline__ void sweep_chunk(const unsigned char* base, bool lower, typename Compute<TF>::T* yf,
                                            TL* yc, typename Compute<TF>::T* ycf) {
    using TC = typename Compute<TF>::T;
    constexpr int FB = FineBlock<TF>::bytes;
    const int4 h0 = reinterpret_cast<const int4*>(base)[0], h1 = reinterpret_cast<const int4*>(base)[1];
    const int f0 = h0.x, nf = h0.y, c0 = h0.z, nc = h0.w, ef = h1.x, ec = h1.y;
    const int lump_lg = (h1.z >> 8) & 15;
    const bool has_long = (h1.z & kChunkLongLumps) != 0;
    const unsigned char* p = base + 32;
    const int* fptr = reinterpret_cast<const int*>(p);
    p += align16(4 * (size_t)(nf + 1));
    const int* fcol = reinterpret_cast<const int*>(p);
    p += align16(4 * (size_t)ef);
    const unsigned char* fval = p;
    p += align16((size_t)FB * ef);
    const unsigned char* fdi = p;
    if (!lower) p += align16((size_t)FB * nf);
    const int* cptr = reinterpret_cast<const int*>(p);
    p += align16(4 * (size_t)(nc + 1));
    const int* ccol = reinterpret_cast<const int*>(p);
    p += align16(4 * (size_t)ec);
    const TL* cval = reinterpret_cast<const TL*>(p);
    p += align16(9 * sizeof(TL) * (size_t)ec);
    const TL* cdi = reinterpret_cast<const TL*>(p);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    if constexpr (sizeof(TL) == 4) {
        // FP32 lump rows (with FP32 or FP16-stored fine rows).  Both local vectors hold a row as
        // four floats (16 bytes, the last unused), so each operand is one vector load.  Every row
        // of the chunk, fine or lump, is one thread's, fine rows first.  A row's column indices
        // and then the operands they point at are loaded four entries at a time before any
        // arithmetic (a 7-point fine row has at most six entries).  Lump rows of more than
        // kLongLumpRow entries are summed by a whole warp after the loop.
        constexpr int kUnroll = 3;
        float4* yf4 = reinterpret_cast<float4*>(yf);
        float4* yc4 = reinterpret_cast<float4*>(yc);
        for (int q = tid; q < nf + nc; q += nt) {
            const bool fine = q < nf;
            const int i = fine ? q : q - nf;
            const int* ptr = fine ? fptr : cptr;
            const int e0 = ptr[i], e1 = ptr[i + 1];
            if (!fine && e1 - e0 > kLongLumpRow) continue;
            const int* col = fine ? fcol : ccol;
            float4* yo = fine ? yf4 + f0 + i : yc4 + c0 + i;
            // the row's own entry is subtracted from at the end, so its load overlaps the products
            const float4 own = *yo;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;  // - sum of the row's products
            // straight-line batches: a padded entry (past the row's end) reloads the row's last
            // entry and contributes zero, so no branch separates the loads of a batch
            const unsigned char* vbase =
                fine ? fval : reinterpret_cast<const unsigned char*>(cval);  // FP32 lumps: 36-byte blocks
            for (int eb = e0; eb < e1; eb += kUnroll) {
                const int last = e1 - 1;
                int cs[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; u++) cs[u] = col[min(eb + u, last)];
                float4 xs[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; u++) {
                    const int c = cs[u];
                    const float4 x = c >= 0 ? yf4[c] : yc4[~c];
                    const bool live = eb + u <= last;
                    xs[u] = make_float4(live ? x.x : 0.f, live ? x.y : 0.f, live ? x.z : 0.f, 0.f);
                }
                if (sizeof(TF) == 4 || fine) {
#pragma unroll
                    for (int u = 0; u < kUnroll; u++)
                        block_mv_sub<TF>(vbase + (size_t)FB * min(eb + u, last), xs[u].x, xs[u].y, xs[u].z, a0, a1, a2);
                } else {
#pragma unroll
                    for (int u = 0; u < kUnroll; u++)
                        block_mv_sub<float>(vbase + 36 * (size_t)min(eb + u, last), xs[u].x, xs[u].y, xs[u].z, a0, a1,
                                            a2);
                }
            }
            a0 += own.x;
            a1 += own.y;
            a2 += own.z;
            if (!lower) {  // z = D^{-1} a, as 0 - D^{-1} (-a)
                float b0 = 0.f, b1 = 0.f, b2 = 0.f;
                if (sizeof(TF) == 4 || fine)
                    block_mv_sub<TF>(fine ? fdi + (size_t)FB * i : reinterpret_cast<const unsigned char*>(cdi + 9 * i),
                                     -a0, -a1, -a2, b0, b1, b2);
                else
                    block_mv_sub<float>(reinterpret_cast<const unsigned char*>(cdi + 9 * i), -a0, -a1, -a2, b0, b1, b2);
                a0 = b0;
                a1 = b1;
                a2 = b2;
            }
            *yo = make_float4(a0, a1, a2, 0.f);
        }
        if (!has_long) return;
        // long lump rows: one warp each, lane = 8 k + s computing component k over the entries
        // s, s + 8, ..., kUnroll of them loaded at a time, combined by three shuffle adds
        const int k = lane >> 3, sl = lane & 7;
        const bool lane_on = lane < 24;
        for (int i = nwarp - 1 - warp; i < nc; i += nwarp) {
            const int e0 = cptr[i], e1 = cptr[i + 1];
            if (e1 - e0 <= kLongLumpRow) continue;
            float acc = 0.f;
            if (lane_on)
                for (int eb = e0 + sl; eb < e1; eb += 8 * kUnroll) {
                    float4 xs[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; u++) {
                        xs[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (eb + 8 * u < e1) {
                            const int c = ccol[eb + 8 * u];
                            xs[u] = c >= 0 ? yf4[c] : yc4[~c];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kUnroll; u++)
                        if (eb + 8 * u < e1) {
                            const float* v = cval + 9LL * (eb + 8 * u) + 3 * k;
                            acc = fmaf(v[0], xs[u].x, fmaf(v[1], xs[u].y, fmaf(v[2], xs[u].z, acc)));
                        }
                }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            float* yr = reinterpret_cast<float*>(yc4 + c0 + i);
            float b = 0.f;
            if (lane_on && sl == 0) b = yr[k] - acc;
            if (lower) {
                if (lane_on && sl == 0) yr[k] = b;
            } else {
                const float b0 = __shfl_sync(0xffffffffu, b, 0);
                const float b1 = __shfl_sync(0xffffffffu, b, 8);
                const float b2 = __shfl_sync(0xffffffffu, b, 16);
                if (lane_on && sl == 0) {
                    const float* d = cdi + 9LL * i + 3 * k;
                    yr[k] = fmaf(d[0], b0, fmaf(d[1], b1, d[2] * b2));
                }
            }
        }
        return;
    }
    if constexpr (sizeof(TC) == 8) {
        // FP64 fine rows: three lanes per row (one per output component), ten rows per warp, so that
        // each FP64 instruction carries three times the work of a thread-per-row loop
        const int r = lane / 3, k = lane - 3 * (lane / 3);
        for (int base = warp * 10; base < nf; base += nwarp * 10) {
            const int t = base + r;
            const bool on = lane < 30 && t < nf;
            double acc = 0.0;
            if (on) {
                const int f = f0 + t;
                acc = yf[3 * f + k];
                for (int e = fptr[t]; e < fptr[t + 1]; e++) {
                    const double* v = reinterpret_cast<const double*>(fval + (size_t)FB * e) + 3 * k;
                    const int c = fcol[e];
                    double x0, x1, x2;
                    if (c >= 0) {
                        x0 = yf[3 * c];
                        x1 = yf[3 * c + 1];
                        x2 = yf[3 * c + 2];
                    } else {
                        x0 = yc[3 * ~c];
                        x1 = yc[3 * ~c + 1];
                        x2 = yc[3 * ~c + 2];
                    }
                    acc -= fma(v[0], x0, fma(v[1], x1, v[2] * x2));
                }
            }
            if (lower) {
                if (on) yf[3 * (f0 + t) + k] = acc;
            } else {
                const int l0 = 3 * r;
                const double b0 = __shfl_sync(0xffffffffu, acc, l0 < 32 ? l0 : 0);
                const double b1 = __shfl_sync(0xffffffffu, acc, l0 + 1 < 32 ? l0 + 1 : 0);
                const double b2 = __shfl_sync(0xffffffffu, acc, l0 + 2 < 32 ? l0 + 2 : 0);
                if (on) {
                    const double* d = reinterpret_cast<const double*>(fdi + (size_t)FB * t) + 3 * k;
                    yf[3 * (f0 + t) + k] = fma(d[0], b0, fma(d[1], b1, d[2] * b2));
                }
            }
        }
    } else {
    // fine rows: one thread each; the blocks and x of up to kUnroll entries are loaded before any
    // arithmetic so that their shared-memory latencies overlap
    constexpr int kUnroll = 4;
    for (int t = tid; t < nf; t += nt) {
        const int f = f0 + t;
        TC a0 = yf[3 * f], a1 = yf[3 * f + 1], a2 = yf[3 * f + 2];
        const int e0 = fptr[t], e1 = fptr[t + 1];
        for (int eb = e0; eb < e1; eb += kUnroll) {
            TC xs[kUnroll][3];
            int cs[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; u++) cs[u] = eb + u < e1 ? fcol[eb + u] : f;
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                const int c = cs[u];
                if (c >= 0) {
                    xs[u][0] = yf[3 * c];
                    xs[u][1] = yf[3 * c + 1];
                    xs[u][2] = yf[3 * c + 2];
                } else {
                    const TC* src = ycf != nullptr ? ycf : reinterpret_cast<const TC*>(yc);
                    xs[u][0] = src[3 * ~c];
                    xs[u][1] = src[3 * ~c + 1];
                    xs[u][2] = src[3 * ~c + 2];
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; u++) {
                if (eb + u < e1) {
                    TC v[9];
                    load_fine<TF>(fval + (size_t)FB * (eb + u), v);
                    a0 -= v[0] * xs[u][0] + v[1] * xs[u][1] + v[2] * xs[u][2];
                    a1 -= v[3] * xs[u][0] + v[4] * xs[u][1] + v[5] * xs[u][2];
                    a2 -= v[6] * xs[u][0] + v[7] * xs[u][1] + v[8] * xs[u][2];
                }
            }
        }
        if (lower) {
            yf[3 * f] = a0;
            yf[3 * f + 1] = a1;
            yf[3 * f + 2] = a2;
        } else {
            TC d[9];
            load_fine<TF>(fdi + (size_t)FB * t, d);
            yf[3 * f] = d[0] * a0 + d[1] * a1 + d[2] * a2;
            yf[3 * f + 1] = d[3] * a0 + d[4] * a1 + d[5] * a2;
            yf[3 * f + 2] = d[6] * a0 + d[7] * a1 + d[8] * a2;
        }
    }
    }
    // Lump rows (TL = double: an FP64 warp instruction keeps an SM sub-partition's FP64 unit busy
    // for ~64 cycles whatever the number of active lanes, so lump work is packed into as few
    // instructions as the latency allows; the same packing serves TL = float):
    //  - short rows (<= kLongLumpRow blocks): 3 S lanes per row, lane = 3 s + k computing output
    //    component k over the entries s, s + S, ..., combined by log2(S) shuffle adds; 32 / (3 S)
    //    rows per warp.  S (1, 2, 4 or 8) is chosen per chunk by the host (header word 6);
    //  - long rows: one warp each, lane = 8 * k + s computing component k over the entries s, s+8,
    //    ..., combined by three shuffle adds.
    // Rows go to the warps from the last one (the first warps carry the fine rows of the chunk).
    constexpr int kLongRow = kLongLumpRow;
    {
        const int k = lane >> 3, sl = lane & 7;
        const bool lane_on = lane < 24;
        for (int i = nwarp - 1 - warp; i < nc; i += nwarp) {
            if (cptr[i + 1] - cptr[i] <= kLongRow) continue;
            TL acc = 0;
            if (lane_on)
                for (int e = cptr[i] + sl; e < cptr[i + 1]; e += 8) {
                    const TL* v = cval + 9LL * e + 3 * k;
                    const int c = ccol[e];
                    TL x0, x1, x2;
                    if (c >= 0) {
                        x0 = (TL)yf[3 * c];
                        x1 = (TL)yf[3 * c + 1];
                        x2 = (TL)yf[3 * c + 2];
                    } else {
                        x0 = yc[3 * ~c];
                        x1 = yc[3 * ~c + 1];
                        x2 = yc[3 * ~c + 2];
                    }
                    acc = fma(v[0], x0, fma(v[1], x1, fma(v[2], x2, acc)));
                }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const int c = c0 + i;
            TL b = 0;
            if (lane_on && sl == 0) b = yc[3 * c + k] - acc;
            if (lower) {
                if (lane_on && sl == 0) yc[3 * c + k] = b;
            } else {
                const TL b0 = __shfl_sync(0xffffffffu, b, 0);
                const TL b1 = __shfl_sync(0xffffffffu, b, 8);
                const TL b2 = __shfl_sync(0xffffffffu, b, 16);
                if (lane_on && sl == 0) {
                    const TL* d = cdi + 9LL * i + 3 * k;
                    const TL t = fma(d[0], b0, fma(d[1], b1, d[2] * b2));
                    yc[3 * c + k] = t;
                    if (ycf != nullptr) ycf[3 * c + k] = (TC)t;
                }
            }
        }
    }
    {
        const int S = 1 << lump_lg, lpr = 3 * S, rpw = 32 / lpr;
        const int r = lane / lpr, within = lane - r * lpr, sl = within / 3, k = within - 3 * sl;
        for (int base = (nwarp - 1 - warp) * rpw; base < nc; base += nwarp * rpw) {
            const int i = base + r;
            const bool on = r < rpw && i < nc && cptr[i + 1] - cptr[i] <= kLongRow;
            if (!__any_sync(0xffffffffu, on)) continue;
            TL acc = 0;
            if (on)
                for (int e = cptr[i] + sl; e < cptr[i + 1]; e += S) {
                    const TL* v = cval + 9LL * e + 3 * k;
                    const int c = ccol[e];
                    TL x0, x1, x2;
                    if (c >= 0) {
                        x0 = (TL)yf[3 * c];
                        x1 = (TL)yf[3 * c + 1];
                        x2 = (TL)yf[3 * c + 2];
                    } else {
                        x0 = yc[3 * ~c];
                        x1 = yc[3 * ~c + 1];
                        x2 = yc[3 * ~c + 2];
                    }
                    acc = fma(v[0], x0, fma(v[1], x1, fma(v[2], x2, acc)));
                }
            // slot 0 of each (row, component) collects the row's sum: sources stay inside the row
            for (int o = 3; o < lpr; o <<= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            const bool head = on && sl == 0;
            const int c = c0 + i;
            const TL b = head ? yc[3 * c + k] - acc : (TL)0;
            if (lower) {
                if (head) yc[3 * c + k] = b;
            } else {
                const int l0 = r * lpr;
                const TL b0 = __shfl_sync(0xffffffffu, b, l0 < 32 ? l0 : 0);
                const TL b1 = __shfl_sync(0xffffffffu, b, l0 + 1 < 32 ? l0 + 1 : 0);
                const TL b2 = __shfl_sync(0xffffffffu, b, l0 + 2 < 32 ? l0 + 2 : 0);
                if (head) {
                    const TL* d = cdi + 9LL * i + 3 * k;
                    const TL t = fma(d[0], b0, fma(d[1], b1, d[2] * b2));
                    yc[3 * c + k] = t;
                    if (ycf != nullptr) ycf[3 * c + k] = (TC)t;
                }
            }
        }
    }
}

// R_i r (Eqs. 4.1, B.2): fine entries copied from their cells (as TC), lump entries summed over
// the lump's cells in FP64 -- far lumps as the far box's sum minus its near-region cells, long
// lists by a whole warp -- and stored as TL.  The caller synchronises the CTA afterwards.
template <typename TC, typename TL>
__device__ __forceinline__ void restrict_local(const SysTab& st, const SubDesc& sd, const double* __restrict__ r,
                                               TC* yf, TL* yc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    // fine cells in batches of kB rows per thread: all cell indices, then all values, are in flight
    // together (two dependent global-load round trips per batch instead of per row)
    constexpr int kB = 4;
    for (int f0 = tid; f0 < sd.nf; f0 += kB * nt) {
        int cell[kB];
#pragma unroll
        for (int u = 0; u < kB; u++) cell[u] = f0 + u * nt < sd.nf ? sd.fcell[f0 + u * nt] : -1;
        double v[kB][3];
#pragma unroll
        for (int u = 0; u < kB; u++) {
            const double* rc = r + 3LL * (cell[u] >= 0 ? cell[u] : 0);
            v[u][0] = rc[0];
            v[u][1] = rc[1];
            v[u][2] = rc[2];
        }
#pragma unroll
        for (int u = 0; u < kB; u++)
            if (cell[u] >= 0) {
                const int f = f0 + u * nt;
                yf[3 * f] = narrow<TC>(v[u][0]);
                yf[3 * f + 1] = narrow<TC>(v[u][1]);
                yf[3 * f + 2] = narrow<TC>(v[u][2]);
            }
    }
    for (int c = tid; c < sd.nc; c += nt) {
        const int i0 = sd.rptr[c], i1 = sd.rptr[c + 1];
        if (i1 - i0 > 16) continue;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        const int b = sd.rbox[c];
        if (b >= 0) {
            a0 = st.boxsum[3 * b];
            a1 = st.boxsum[3 * b + 1];
            a2 = st.boxsum[3 * b + 2];
            const int k = sd.rcorr[c];
            if (k >= 0) {
                const double* q = st.corr + 3LL * (sd.corr0 + k);
                a0 -= q[0];
                a1 -= q[1];
                a2 -= q[2];
            }
        }
#pragma unroll 8
        for (int i = i0; i < i1; i++) {
            const double* rc = sum_entry(st, r, sd.rsrc[i]);
            a0 += rc[0];
            a1 += rc[1];
            a2 += rc[2];
        }
        yc[3 * c] = narrow<TL>(a0);
        yc[3 * c + 1] = narrow<TL>(a1);
        yc[3 * c + 2] = narrow<TL>(a2);
    }
    for (int k = warp; k < sd.n_long; k += nwarp) {
        const int c = sd.clong[k];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int i = sd.rptr[c] + lane; i < sd.rptr[c + 1]; i += 32) {
            const double* rc = sum_entry(st, r, sd.rsrc[i]);
            a0 += rc[0];
            a1 += rc[1];
            a2 += rc[2];
        }
        warp_sum3(a0, a1, a2);
        if (lane == 0) {
            yc[3 * c] = narrow<TL>(a0);
            yc[3 * c + 1] = narrow<TL>(a1);
            yc[3 * c + 2] = narrow<TL>(a2);
        }
    }
}

// R_i r (Eqs. 4.1, B.2) of every subdomain into its device-memory local vectors, in the layout of
// y_layout(): a fine row copies its cell's entries (rounded to the fine rows' compute type), a
// lump row sums its cells in FP64 -- a far lump as the far box's sum minus its near-region cells
// -- and is rounded to the lump type TL (with an FP32 mirror of FP64 lumps under FP32 fine rows;
// with FP32 lumps every row is four floats, the last zero).
// One thread per local row; items are (subdomain, first row of 256).
template <typename TC, typename TL>
__global__ void __launch_bounds__(256) k_restrict(const SysTab* __restrict__ tab, const SubDesc* __restrict__ subs,
                                                  const int2* __restrict__ items) {
    const int2 it = items[blockIdx.x];
    const SubDesc& sd = subs[it.x];
    const SysTab& st = tab[sd.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const double* __restrict__ r = st.ws + (long long)in * st.n3p;
    unsigned char* y = reinterpret_cast<unsigned char*>(sd.y);
    const int q = it.y + threadIdx.x;
    constexpr bool kRow16 = sizeof(TL) == 4;  // FP32 lumps: rows of four floats (16 bytes)
    if (q < sd.nf) {
        const double* rc = r + 3LL * sd.fcell[q];
        if constexpr (kRow16) {
            reinterpret_cast<float4*>(y + sd.y_fine)[q] =
                make_float4(f64_to_f32(rc[0]), f64_to_f32(rc[1]), f64_to_f32(rc[2]), 0.f);
        } else {
            TC* yf = reinterpret_cast<TC*>(y + sd.y_fine) + 3 * q;
            yf[0] = narrow<TC>(rc[0]);
            yf[1] = narrow<TC>(rc[1]);
            yf[2] = narrow<TC>(rc[2]);
        }
        return;
    }
    const int c = q - sd.nf;
    if (c >= sd.nc) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const int b = sd.rbox[c];
    if (b >= 0) {
        a0 = st.boxsum[3 * b];
        a1 = st.boxsum[3 * b + 1];
        a2 = st.boxsum[3 * b + 2];
        const int k = sd.rcorr[c];
        if (k >= 0) {
            const double* qc = st.corr + 3LL * (sd.corr0 + k);
            a0 -= qc[0];
            a1 -= qc[1];
            a2 -= qc[2];
        }
    }
    const int i0 = sd.rptr[c], i1 = sd.rptr[c + 1];
    for (int i = i0; i < i1; i += 4) {
        const double* src[4];
#pragma unroll
        for (int u = 0; u < 4; u++) src[u] = i + u < i1 ? sum_entry(st, r, sd.rsrc[i + u]) : nullptr;
        double v[4][3];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const double* rc = src[u] != nullptr ? src[u] : r;
            v[u][0] = rc[0];
            v[u][1] = rc[1];
            v[u][2] = rc[2];
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (src[u] != nullptr) {
                a0 += v[u][0];
                a1 += v[u][1];
                a2 += v[u][2];
            }
    }
    if constexpr (kRow16) {
        reinterpret_cast<float4*>(y)[c] = make_float4(f64_to_f32(a0), f64_to_f32(a1), f64_to_f32(a2), 0.f);
        return;
    }
    TL* yc = reinterpret_cast<TL*>(y) + 3 * c;
    yc[0] = narrow<TL>(a0);
    yc[1] = narrow<TL>(a1);
    yc[2] = narrow<TL>(a2);
    if constexpr (sizeof(TL) == 8 && sizeof(TC) == 4) {
        TC* ycf = reinterpret_cast<TC*>(y + sd.y_mirror) + 3 * c;
        ycf[0] = narrow<TC>(a0);
        ycf[1] = narrow<TC>(a1);
        ycf[2] = narrow<TC>(a2);
    }
}

// Fused local solve of one subdomain (one CTA): y = R_i r; y = L^{-1} y; y = U^{-1} y;
// z[owned cells] = y[owned fine rows] (Eqs. 4.2-4.5).  Thread 0 streams the factor chunks
// (front to back) into a ring of shared-memory slots with TMA bulk copies; all threads compute
// from shared memory, one chunk at a time, with a CTA barrier after each chunk (which also orders
// the wavefront levels).  Fine rows and lump rows live in separate local vectors (fine rows at the
// factor precision, lumps as TL: FP64, or FP32 with FP32/FP16 fine rows), in shared memory when
// they fit.
template <typename TF, typename TL, int YM, int SLOTS>
__global__ void __launch_bounds__(YM == Y_SMEM ? 256 : kApplyThreadsDev, YM == Y_SMEM ? 2 : 4)
    k_apply(const SysTab* __restrict__ tab, const SubDesc* __restrict__ subs) {
    using TC = typename Compute<TF>::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const SubDesc sd = subs[blockIdx.x];
    const SysTab& st = tab[sd.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const int out = st.ctl[C_APPLY_OUT];
    (void)in;
    double* __restrict__ z = st.ws + (long long)out * st.n3p;
    unsigned char* ring = smem_raw;
    const int cap = sd.chunk_cap, ring_bytes = SLOTS * cap;  // this subdomain's ring slots
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + ring_bytes);
    // local vectors (written by k_restrict in device memory): lumps (TL), fine rows (factor
    // precision) and, for FP64 lumps under FP32 fine rows, an FP32 mirror of the lumps, in the
    // layout of y_layout(); Y_SMEM copies all of them into shared memory, Y_LUMPS the lumps and the
    // mirror (as [lumps | mirror]), Y_DEVICE none
    constexpr bool kMirror = sizeof(TL) == 8 && sizeof(TC) == 4;
    unsigned char* ysm = smem_raw + ring_bytes + kRingHeader;
    unsigned char* ydev = reinterpret_cast<unsigned char*>(sd.y);
    unsigned char* yc_raw = YM == Y_DEVICE ? ydev : ysm;
    TL* yc = reinterpret_cast<TL*>(yc_raw);
    TC* yf = reinterpret_cast<TC*>((YM == Y_LUMPS ? ydev : yc_raw) + sd.y_fine);
    TC* ycf = !kMirror ? nullptr : reinterpret_cast<TC*>(yc_raw + (YM == Y_LUMPS ? sd.y_fine : sd.y_mirror));
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;

    if (tid == 0) {
        for (int k = 0; k < SLOTS; k++) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < SLOTS && k < sd.n_chunks; k++) {
            const int2 ch = sd.chunks[k];
            mbar_expect_tx(&bar[k], (unsigned)ch.y);
            bulk_load(ring + (size_t)k * cap, sd.stream + ch.x, (unsigned)ch.y, &bar[k]);
        }

    // the local vectors k_restrict wrote (overlaps the first chunk copies)
    if constexpr (YM != Y_DEVICE) {
        const int4* src = reinterpret_cast<const int4*>(ydev);
        int4* dst = reinterpret_cast<int4*>(ysm);
        const int n16 = (YM == Y_SMEM ? sd.y_bytes : sd.y_fine) >> 4;
        for (int i = tid; i < n16; i += nt) dst[i] = src[i];
        if (YM == Y_LUMPS && kMirror) {
            const int m16 = (sd.y_bytes - sd.y_mirror) >> 4;
            const int4* msrc = reinterpret_cast<const int4*>(ydev + sd.y_mirror);
            for (int i = tid; i < m16; i += nt) dst[n16 + i] = msrc[i];
        }
    }
    __syncthreads();

    // The copy that refills a slot is issued by lane 0 of a warp without rows in the chunk just
    // finished (fine rows fill warps from the first, lump rows from the last), so the next chunk's
    // rows are not held up behind it.  Both candidate issuers keep the next chunk's descriptor,
    // loaded one chunk ahead.
    // (With FP32 lump rows every row is one thread's, fine rows from thread 0 up and lump rows
    // after them, so the last warp issues every refill.)
    const bool issuer_fine = lane == 0 && warp == nwarp - 1,
               issuer_lump = sizeof(TL) == 4 ? issuer_fine : tid == 0;
    int2 next_ch = make_int2(0, 0);
    if ((issuer_fine || issuer_lump) && SLOTS < sd.n_chunks) next_ch = sd.chunks[SLOTS];
    for (int ci = 0; ci < sd.n_chunks; ci++) {
        const int slot = ci % SLOTS;
        // warp-uniform, so that the warp-collective code of the sweep runs on whole warps
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar[slot], (unsigned)(ci / SLOTS) & 1u, st.wait_limit));
        bool fine_chunk = false;
        if (ok) {
            const unsigned char* chunk = ring + (size_t)slot * cap;
            fine_chunk = reinterpret_cast<const int*>(chunk)[1] > 0;
            sweep_chunk<TF, TL>(chunk, ci < sd.n_fwd, yf, yc, ycf);
        }
        if (__syncthreads_or(!ok)) {
            // a copy did not land in time: report it, wait (bounded) for the copies still in
            // flight into this CTA's shared memory, and leave
            if (tid == 0) {
                atomicExch(st.dev_err, 7);
                const int last = min(sd.n_chunks, ci + SLOTS);
                for (int k = ci; k < last; k++) mbar_wait(&bar[k % SLOTS], (unsigned)(k / SLOTS) & 1u);
            }
            return;
        }
        if (ci + SLOTS < sd.n_chunks) {
            if (fine_chunk ? issuer_fine : issuer_lump) {
                mbar_expect_tx(&bar[slot], (unsigned)next_ch.y);
                bulk_load(ring + (size_t)slot * cap, sd.stream + next_ch.x, (unsigned)next_ch.y, &bar[slot]);
            }
            if ((issuer_fine || issuer_lump) && ci + SLOTS + 1 < sd.n_chunks) next_ch = sd.chunks[ci + SLOTS + 1];
        }
    }

    // P_i R_i^T: owned cells take this subdomain's solution; the lumps are discarded
    constexpr int RS = sizeof(TL) == 4 ? 4 : 3;  // floats per fine row (FP32 lumps: 16-byte rows)
    for (int t = tid; t < sd.n_own; t += nt) {
        const int f = sd.own_pos[t];
        const long long c = 3LL * sd.own_cell[t];
        z[c] = yf[RS * f];
        z[c + 1] = yf[RS * f + 1];
        z[c + 2] = yf[RS * f + 2];
    }
}

// Exact local solves: R_i r into the subdomain's FP64 local vector, fine indices then lump indices
// (the order of the dense A_i^{-1}); one CTA per subdomain
__global__ void __launch_bounds__(256) k_dense_restrict(const SysTab* __restrict__ tab, const SubDesc* __restrict__ subs) {
    const SubDesc& sd = subs[blockIdx.x];
    const SysTab& st = tab[sd.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    restrict_local<double, double>(st, sd, st.ws + (long long)in * st.n3p, sd.y, sd.y + 3 * sd.nf);
}

// ------------------------------------------------------------------------------------------
// SpMV y = A x or y = b - A x (ELL, one thread per block row, 3x3 blocks)
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_spmv(const SysTab* __restrict__ tab, const RowItem* __restrict__ items) {
    const RowItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    const int in = st.ctl[C_SPMV_IN];
    if (in < 0) return;
    const int row = it.r0 + threadIdx.x;
    if (row >= st.n_cells) return;
    const int out = st.ctl[C_SPMV_OUT];
    const int bs = st.ctl[C_SPMV_B];
    const double* __restrict__ x = st.ws + (long long)in * st.n3p;
    double* __restrict__ y = st.ws + (long long)out * st.n3p;
    const long long rp = st.rows_pad;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int w = 0; w < st.ell_w; w++) {
        const int c = st.ell_col[(long long)w * rp + row];
        const double x0 = x[3LL * c], x1 = x[3LL * c + 1], x2 = x[3LL * c + 2];
        const double* v = st.ell_val + (long long)w * 9 * rp + row;
        a0 += v[0] * x0 + v[rp] * x1 + v[2 * rp] * x2;
        a1 += v[3 * rp] * x0 + v[4 * rp] * x1 + v[5 * rp] * x2;
        a2 += v[6 * rp] * x0 + v[7 * rp] * x1 + v[8 * rp] * x2;
    }
    if (bs >= 0) {
        const double* b = st.ws + (long long)bs * st.n3p;
        a0 = b[3LL * row] - a0;
        a1 = b[3LL * row + 1] - a1;
        a2 = b[3LL * row + 2] - a2;
    }
    y[3LL * row] = a0;
    y[3LL * row + 1] = a1;
    y[3LL * row + 2] = a2;
}

// ------------------------------------------------------------------------------------------
// GMRES vector kernels.  A chunk is VEC_CHUNK elements of one system; reductions write one
// partial per chunk and the last chunk to arrive sums the partials in index order, so every
// result is independent of scheduling and of the other systems in the launch.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double* vec(const SysTab& st, int slot) { return st.ws + (long long)slot * st.n3p; }

__device__ __forceinline__ int zslot(const SysTab& st, int k) { return VV0 + st.m + 1 + k; }

// block sum of two values; result valid in thread 0.  The 256 partials go through shared memory
// and one warp reduces them (8 sequential adds + a 5-round tree): FP64 adds are scarce here, so
// this issues ~4x fewer of them than a shuffle tree in every warp.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double s0[VEC_THREADS], s1[VEC_THREADS];
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = 0.0, y = 0.0;
        for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) {
            x += s0[i];
            y += s1[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
        }
        a = x;
        b = y;
    }
    __syncthreads();
}

// Publish this chunk's partials; returns true in thread 0.. of the last chunk of its system,
// with (s0, s1) = the ordered total.
__device__ bool finish_reduction(const SysTab& st, int chunk, double& s0, double& s1) {
    __shared__ bool last;
    block_sum2(s0, s1);
    if (threadIdx.x == 0) {
        st.partial[2 * chunk] = s0;
        st.partial[2 * chunk + 1] = s1;
        __threadfence();
        const int prev = atomicAdd(&st.ctl[C_CNT_RED], 1);
        last = (prev == st.nchunk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < st.nchunk; i += blockDim.x) {
        a += __ldcg(&st.partial[2 * i]);
        b += __ldcg(&st.partial[2 * i + 1]);
    }
    block_sum2(a, b);
    s0 = a;
    s1 = b;
    if (threadIdx.x == 0) st.ctl[C_CNT_RED] = 0;
    return true;
}

__global__ void __launch_bounds__(VEC_THREADS) k_init(const SysTab* __restrict__ tab, const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.ctl[C_PHASE] != PH_INIT) return;
    double* x = vec(st, VX);
    const double* b = vec(st, VB);
    double* r = vec(st, VR);
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
        x[e0 + i] = 0.0;
        r[e0 + i] = b[e0 + i];
    }
}

// restart phase: u = V y (then u goes through B^{-1}), or x += Z y (flexible)
__global__ void __launch_bounds__(VEC_THREADS) k_prep(const SysTab* __restrict__ tab, const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.ctl[C_PHASE] != PH_RESTART) return;
    const int jend = st.ctl[C_JEND];
    const ScalLayout SL = ScalLayout::make(st.m);
    const double* yv = st.scal + SL.y;
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    double* dst = st.flexible ? vec(st, VX) : vec(st, VU);
    for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
        double acc = st.flexible ? dst[e0 + i] : 0.0;
        for (int k = 0; k < jend; k++) acc += yv[k] * vec(st, st.flexible ? zslot(st, k) : VV0 + k)[e0 + i];
        dst[e0 + i] = acc;
    }
}

// restart phase (non-flexible): x += z
__global__ void __launch_bounds__(VEC_THREADS) k_post(const SysTab* __restrict__ tab, const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.ctl[C_PHASE] != PH_RESTART || st.flexible) return;
    double* x = vec(st, VX);
    const double* z = vec(st, VZ);
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) x[e0 + i] += z[e0 + i];
}

// MGS step k of Arnoldi column j: w -= h_{k-1,j} v_{k-1} (k >= 1), then h_{k,j} = (w, v_k)
// (k <= j) or h_{j+1,j} = ||w|| (k = j + 1).  k = 0 also gives ||w|| before orthogonalisation.
// Restart/init systems compute beta = ||r|| at k = 0.
__global__ void __launch_bounds__(VEC_THREADS) k_mgs(const SysTab* __restrict__ tab, const VecItem* __restrict__ items,
                                                     int k) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.krylov != 0) return;
    const int ph = st.ctl[C_PHASE];
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    const ScalLayout SL = ScalLayout::make(st.m);
    double s0 = 0.0, s1 = 0.0;
    if (ph == PH_ARNOLDI) {
        const int j = st.ctl[C_J];
        if (k > j + 1) return;
        double* w = vec(st, VW);
        if (k >= 1) {
            const double h = st.scal[SL.H + (k - 1) * st.m + j];
            const double* v = vec(st, VV0 + k - 1);
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) w[e0 + i] -= h * v[e0 + i];
        }
        if (k <= j) {
            const double* v = vec(st, VV0 + k);
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
                const double a = w[e0 + i];
                s0 += a * v[e0 + i];
                s1 += a * a;
            }
        } else {
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
                const double a = w[e0 + i];
                s0 += a * a;
            }
        }
        if (!finish_reduction(st, it.chunk, s0, s1)) return;
        if (threadIdx.x == 0) {
            if (k <= j) {
                st.scal[SL.H + k * st.m + j] = s0;
                if (k == 0) st.scal[SL.w0] = sqrt(s1);
            } else {
                const double hn = sqrt(s0);
                st.scal[SL.hn] = hn;
                st.scal[SL.H + (j + 1) * st.m + j] = hn;
            }
        }
    } else if (ph == PH_RESTART || ph == PH_INIT) {
        if (k != 0) return;
        const double* r = vec(st, VR);
        for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
            const double a = r[e0 + i];
            s0 += a * a;
        }
        if (!finish_reduction(st, it.chunk, s0, s1)) return;
        if (threadIdx.x == 0) st.scal[SL.beta] = sqrt(s0);
    }
}

__device__ void set_slots(const SysTab& st, int ph, int j) {
    int* c = st.ctl;
    if (ph == PH_ARNOLDI) {
        c[C_APPLY_IN] = VV0 + j;
        c[C_APPLY_OUT] = st.flexible ? zslot(st, j) : VZ;
        c[C_SPMV_IN] = c[C_APPLY_OUT];
        c[C_SPMV_OUT] = VW;
        c[C_SPMV_B] = -1;
    } else if (ph == PH_RESTART) {
        c[C_APPLY_IN] = st.flexible ? -1 : VU;
        c[C_APPLY_OUT] = VZ;
        c[C_SPMV_IN] = VX;
        c[C_SPMV_OUT] = VR;
        c[C_SPMV_B] = VB;
    } else {
        c[C_APPLY_IN] = -1;
        c[C_SPMV_IN] = -1;
    }
}

// Givens rotation of column j and the GMRES state machine of one system (one thread).
__device__ void step_state(const SysTab& st, int ph) {
    const ScalLayout SL = ScalLayout::make(st.m);
    const int m = st.m;
    int* c = st.ctl;
    double* s = st.scal;
    double* H = s + SL.H;
    if (ph == PH_ARNOLDI) {
        const int j = c[C_J];
        for (int k = 0; k < j; k++) {
            const double a = H[k * m + j], b = H[(k + 1) * m + j];
            H[k * m + j] = s[SL.cs + k] * a + s[SL.sn + k] * b;
            H[(k + 1) * m + j] = -s[SL.sn + k] * a + s[SL.cs + k] * b;
        }
        const double a = H[j * m + j], b = H[(j + 1) * m + j];
        const double rr = hypot(a, b);
        double cs = 1.0, sn = 0.0;
        if (rr != 0.0) {
            cs = a / rr;
            sn = b / rr;
        }
        s[SL.cs + j] = cs;
        s[SL.sn + j] = sn;
        H[j * m + j] = cs * a + sn * b;
        H[(j + 1) * m + j] = 0.0;
        const double gj = s[SL.g + j];
        s[SL.g + j + 1] = -sn * gj;
        s[SL.g + j] = cs * gj;
        c[C_ITERS] += 1;
        const bool breakdown = s[SL.hn] <= 1e-14 * s[SL.w0];
        if (breakdown) c[C_BREAKDOWN] = 1;
        const bool small = fabs(s[SL.g + j + 1]) <= s[SL.tol] * s[SL.bnorm];
        if (small || breakdown || c[C_ITERS] >= c[C_MAXIT] || j + 1 == m) {
            const int jend = j + 1;
            c[C_JEND] = jend;
            for (int k = jend - 1; k >= 0; k--) {
                double acc = s[SL.g + k];
                for (int l = k + 1; l < jend; l++) acc -= H[k * m + l] * s[SL.y + l];
                s[SL.y + k] = acc / H[k * m + k];
            }
            c[C_PHASE] = PH_RESTART;
            set_slots(st, PH_RESTART, 0);
        } else {
            c[C_J] = j + 1;
            set_slots(st, PH_ARNOLDI, j + 1);
        }
        return;
    }
    const double beta = s[SL.beta];
    if (ph == PH_INIT) {
        s[SL.bnorm] = beta;
        if (beta == 0.0) {
            c[C_CONVERGED] = 1;
            c[C_STATUS] = 0;
            c[C_PHASE] = PH_DONE;
            set_slots(st, PH_DONE, 0);
            return;
        }
    } else {
        c[C_RESTARTS] += 1;
    }
    const double rel = beta / s[SL.bnorm];
    if (rel <= s[SL.tol]) {
        c[C_CONVERGED] = 1;
        c[C_STATUS] = 0;
        c[C_PHASE] = PH_DONE;
        set_slots(st, PH_DONE, 0);
    } else if (c[C_ITERS] >= c[C_MAXIT] || beta == 0.0) {
        c[C_STATUS] = 4;  // ASM_ERR_NOT_CONVERGED
        c[C_PHASE] = PH_DONE;
        set_slots(st, PH_DONE, 0);
    } else {
        for (int k = 0; k <= m; k++) s[SL.g + k] = 0.0;
        s[SL.g] = beta;
        c[C_J] = 0;
        c[C_PHASE] = PH_ARNOLDI;
        set_slots(st, PH_ARNOLDI, 0);
    }
}


// End of a step: vector scaling (v_{j+1} = w / h_{j+1,j}, or v_0 = r / beta), then the last chunk
// of each system applies the Givens rotations and moves its state machine.
__global__ void __launch_bounds__(VEC_THREADS) k_finish(const SysTab* __restrict__ tab,
                                                        const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    const int ph = st.ctl[C_PHASE];
    if (ph == PH_DONE || st.krylov != 0) return;
    const ScalLayout SL = ScalLayout::make(st.m);
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    if (ph == PH_ARNOLDI) {
        const int j = st.ctl[C_J];
        const double hn = st.scal[SL.hn];
        if (hn > 0.0) {
            const double inv = 1.0 / hn;
            const double* w = vec(st, VW);
            double* v = vec(st, VV0 + j + 1);
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) v[e0 + i] = w[e0 + i] * inv;
        }
    } else {
        const double beta = st.scal[SL.beta];
        if (beta > 0.0) {
            const double inv = 1.0 / beta;
            const double* r = vec(st, VR);
            double* v = vec(st, VV0);
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) v[e0 + i] = r[e0 + i] * inv;
        }
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st.ctl[C_CNT_FIN], 1) == st.nchunk - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    st.ctl[C_CNT_FIN] = 0;
    step_state(st, ph);
}

// ------------------------------------------------------------------------------------------
// ORTHOMIN(k) (Section 2): the new direction p = B^{-1} r, q = A p is A-orthogonalised against the
// k most recent directions (newest first, each projection on the q already updated), then
// alpha = (r, q) / (q, q), x += alpha p, r -= alpha q.  The directions sit in a ring of k + 1
// slots: P_s = VV0 + s, Q_s = VV0 + k + 1 + s.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int om_p(const SysTab& st, int s) { return VV0 + s; }
__device__ __forceinline__ int om_q(const SysTab& st, int s) { return VV0 + st.m + 1 + s; }

__device__ void om_set_slots(const SysTab& st, int ph) {
    int* c = st.ctl;
    if (ph == PH_OM) {
        const int s = c[C_OM_SLOT];
        c[C_APPLY_IN] = VR;
        c[C_APPLY_OUT] = om_p(st, s);
        c[C_SPMV_IN] = om_p(st, s);
        c[C_SPMV_OUT] = om_q(st, s);
        c[C_SPMV_B] = -1;
    } else if (ph == PH_OM_FINAL) {
        c[C_APPLY_IN] = -1;
        c[C_SPMV_IN] = VX;
        c[C_SPMV_OUT] = VW;
        c[C_SPMV_B] = VB;
    } else {
        c[C_APPLY_IN] = -1;
        c[C_SPMV_IN] = -1;
    }
}

// ORTHOMIN state machine of one system (one thread).  nrm = ||r|| (initial and after an update)
// or ||b - A x|| (final).
__device__ void om_state(const SysTab& st, int ph, double nrm) {
    const ScalLayout SL = ScalLayout::make(st.m);
    int* c = st.ctl;
    double* s = st.scal;
    int next = PH_OM;
    if (ph == PH_INIT) {
        s[SL.bnorm] = nrm;
        s[SL.beta] = nrm;
        if (nrm == 0.0) {
            c[C_CONVERGED] = 1;
            c[C_STATUS] = 0;
            next = PH_DONE;
        } else {
            c[C_OM_STORED] = 0;
            c[C_OM_SLOT] = 0;
        }
    } else if (ph == PH_OM) {
        c[C_ITERS] += 1;
        if (c[C_OM_STORED] < st.m) c[C_OM_STORED] += 1;
        if (nrm <= s[SL.tol] * s[SL.bnorm] || c[C_ITERS] >= c[C_MAXIT])
            next = PH_OM_FINAL;
        else
            c[C_OM_SLOT] = (c[C_OM_SLOT] + 1) % (st.m + 1);
    } else {  // PH_OM_FINAL
        s[SL.beta] = nrm;
        const bool conv = nrm <= s[SL.tol] * s[SL.bnorm];
        c[C_CONVERGED] = conv ? 1 : 0;
        c[C_STATUS] = conv ? 0 : 4;  // ASM_ERR_NOT_CONVERGED
        next = PH_DONE;
    }
    c[C_PHASE] = next;
    om_set_slots(st, next);
}

// Pass l of a direction step: l >= 1 first applies projection l (p -= beta_l P_os, q -= beta_l Q_os,
// os = the l-th most recent stored direction); then either the next coefficient
// beta_{l+1} = (q, Q_os') / (Q_os', Q_os') or, after the last projection, (q, q) and (r, q).
__global__ void __launch_bounds__(VEC_THREADS) k_om(const SysTab* __restrict__ tab, const VecItem* __restrict__ items,
                                                    int l) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.krylov != 1) return;
    const int ph = st.ctl[C_PHASE];
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    const ScalLayout SL = ScalLayout::make(st.m);
    double s0 = 0.0, s1 = 0.0;
    if (ph == PH_OM) {
        const int stored = st.ctl[C_OM_STORED];
        if (l > stored) return;
        const int K1 = st.m + 1, slot = st.ctl[C_OM_SLOT];
        double* p = vec(st, om_p(st, slot));
        double* q = vec(st, om_q(st, slot));
        if (l >= 1) {
            const int os = (slot - l + K1) % K1;
            const double beta = st.scal[SL.om_beta + l - 1];
            const double* po = vec(st, om_p(st, os));
            const double* qo = vec(st, om_q(st, os));
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
                p[e0 + i] -= beta * po[e0 + i];
                q[e0 + i] -= beta * qo[e0 + i];
            }
        }
        if (l < stored) {
            const double* qo = vec(st, om_q(st, (slot - l - 1 + K1) % K1));
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) s0 += q[e0 + i] * qo[e0 + i];
        } else {
            const double* r = vec(st, VR);
            for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
                const double a = q[e0 + i];
                s0 += a * a;
                s1 += r[e0 + i] * a;
            }
        }
        if (!finish_reduction(st, it.chunk, s0, s1)) return;
        if (threadIdx.x == 0) {
            if (l < stored) {
                const int on = (slot - l - 1 + K1) % K1;
                st.scal[SL.om_beta + l] = s0 / st.scal[SL.om_qq + on];
            } else {
                st.scal[SL.om_qq + slot] = s0;
                st.scal[SL.om_alpha] = s0 != 0.0 ? s1 / s0 : 0.0;
            }
        }
    } else if (ph == PH_INIT || ph == PH_OM_FINAL) {
        if (l != 0) return;
        const double* r = vec(st, ph == PH_INIT ? VR : VW);
        for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
            const double a = r[e0 + i];
            s0 += a * a;
        }
        if (!finish_reduction(st, it.chunk, s0, s1)) return;
        if (threadIdx.x == 0) om_state(st, ph, sqrt(s0));
    }
}

// x += alpha p, r -= alpha q and ||r||; a direction with (q, q) = 0 ends the iteration instead.
__global__ void __launch_bounds__(VEC_THREADS) k_om_update(const SysTab* __restrict__ tab,
                                                           const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    if (st.krylov != 1 || st.ctl[C_PHASE] != PH_OM) return;
    const ScalLayout SL = ScalLayout::make(st.m);
    const int slot = st.ctl[C_OM_SLOT];
    const bool dead = st.scal[SL.om_qq + slot] == 0.0;
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    double s0 = 0.0, s1 = 0.0;
    if (!dead) {
        const double alpha = st.scal[SL.om_alpha];
        const double* p = vec(st, om_p(st, slot));
        const double* q = vec(st, om_q(st, slot));
        double* x = vec(st, VX);
        double* r = vec(st, VR);
        for (int i = threadIdx.x; i < VEC_CHUNK; i += blockDim.x) {
            x[e0 + i] += alpha * p[e0 + i];
            const double a = r[e0 + i] - alpha * q[e0 + i];
            r[e0 + i] = a;
            s0 += a * a;
        }
    }
    if (!finish_reduction(st, it.chunk, s0, s1)) return;
    if (threadIdx.x != 0) return;
    if (dead) {
        st.ctl[C_PHASE] = PH_OM_FINAL;
        om_set_slots(st, PH_OM_FINAL);
    } else {
        om_state(st, PH_OM, sqrt(s0));
    }
}

// The whole orthogonalisation of one step of one system in one cooperative launch: modified
// Gram-Schmidt with one grid-wide barrier per projection instead of one launch.  Each CTA keeps a
// single partial per projection (grid-stride over the elements), and every CTA reduces the G
// partials in the same fixed order, so the result is deterministic for a given grid size.
// w stays in L2 between projections, so each basis vector is streamed from HBM about once.
__device__ __forceinline__ void grid_total(const double* part, int G, double& s0, double& s1) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) {
        a += __ldcg(&part[2 * i]);
        b += __ldcg(&part[2 * i + 1]);
    }
    block_sum2(a, b);
    __shared__ double bc[2];
    if (threadIdx.x == 0) {
        bc[0] = a;
        bc[1] = b;
    }
    __syncthreads();
    s0 = bc[0];
    s1 = bc[1];
    __syncthreads();
}

__global__ void __launch_bounds__(VEC_THREADS, 2) k_ortho_coop(const SysTab* __restrict__ tab, double* __restrict__ part2) {
    constexpr int kU = 4;
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const SysTab& st = tab[0];
    const int ph = st.ctl[C_PHASE];
    if (ph == PH_DONE) return;
    const ScalLayout SL = ScalLayout::make(st.m);
    const int m = st.m;
    const int G = gridDim.x;
    const long long n = st.n3p;
    const long long stride = (long long)G * blockDim.x;
    const long long e_begin = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double* w = vec(st, VW);
    if (ph == PH_ARNOLDI) {
        const int j = st.ctl[C_J];
        double hprev = 0.0, w0 = 0.0, hn = 0.0;
        // Operands of the current group of kU elements; the next group's loads are issued before
        // the current group is computed.  The first group of pass k + 1 needs nothing from the
        // barrier that ends pass k (its w is this thread's own result), so its loads are issued
        // before that barrier.
        double A[kU], B[kU], C[kU];
        {
            const double* v0 = vec(st, VV0);
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const long long e = e_begin + u * stride;
                A[u] = e < n ? w[e] : 0.0;
                B[u] = 0.0;
                C[u] = e < n ? v0[e] : 0.0;
            }
        }
        for (int k = 0; k <= j + 1; k++) {
            double* part = part2 + (size_t)(k & 1) * 2 * G;
            double s0 = 0.0, s1 = 0.0;
            // kU partial sums per thread, combined in a fixed order
            double p0[kU], p1[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) p0[u] = p1[u] = 0.0;
            const double* vp = k > 0 ? vec(st, VV0 + k - 1) : nullptr;
            const double* vk = k <= j ? vec(st, VV0 + k) : nullptr;
            for (long long e0 = e_begin; e0 < n; e0 += kU * stride) {
                const long long e1 = e0 + kU * stride;
                double An[kU], Bn[kU], Cn[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const long long e = e1 + u * stride;
                    const bool in = e < n;
                    An[u] = in ? w[e] : 0.0;
                    Bn[u] = in && vp ? vp[e] : 0.0;
                    Cn[u] = in && vk ? vk[e] : 0.0;
                }
                if (k == 0) {  // (w, v_0) and (w, w)
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        p0[u] = fma(A[u], C[u], p0[u]);
                        p1[u] = fma(A[u], A[u], p1[u]);
                    }
                } else {  // w -= h_{k-1} v_{k-1}, then (w, v_k), or (w, w) after the last projection
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        const long long e = e0 + u * stride;
                        const double x = fma(-hprev, B[u], A[u]);
                        if (e < n) w[e] = x;
                        p0[u] = fma(x, vk ? C[u] : x, p0[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    A[u] = An[u];
                    B[u] = Bn[u];
                    C[u] = Cn[u];
                }
            }
            if (k <= j) {  // the first group of pass k + 1
                const double* vn = k + 1 <= j ? vec(st, VV0 + k + 1) : nullptr;
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const long long e = e_begin + u * stride;
                    const bool in = e < n;
                    A[u] = in ? w[e] : 0.0;
                    B[u] = in ? vk[e] : 0.0;
                    C[u] = in && vn ? vn[e] : 0.0;
                }
            }
            s0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
            s1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
            block_sum2(s0, s1);
            if (threadIdx.x == 0) {
                part[2 * blockIdx.x] = s0;
                part[2 * blockIdx.x + 1] = s1;
            }
            grid.sync();
            double t0, t1;
            grid_total(part, G, t0, t1);
            if (k <= j) {
                hprev = t0;
                if (k == 0) w0 = sqrt(t1);
                if (blockIdx.x == 0 && threadIdx.x == 0) st.scal[SL.H + k * m + j] = t0;
            } else {
                hn = sqrt(t0);
            }
        }
        if (hn > 0.0) {
            const double inv = 1.0 / hn;
            double* v = vec(st, VV0 + j + 1);
            for (long long e0 = e_begin; e0 < n; e0 += kU * stride) {
                double a[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) a[u] = e0 + u * stride < n ? w[e0 + u * stride] : 0.0;
#pragma unroll
                for (int u = 0; u < kU; u++)
                    if (e0 + u * stride < n) v[e0 + u * stride] = a[u] * inv;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st.scal[SL.w0] = w0;
            st.scal[SL.hn] = hn;
            st.scal[SL.H + (j + 1) * m + j] = hn;
            step_state(st, ph);
        }
    } else {
        const double* r = vec(st, VR);
        double s0 = 0.0, s1 = 0.0;
        for (long long e = e_begin; e < n; e += stride) s0 = fma(r[e], r[e], s0);
        block_sum2(s0, s1);
        if (threadIdx.x == 0) {
            part2[2 * blockIdx.x] = s0;
            part2[2 * blockIdx.x + 1] = s1;
        }
        grid.sync();
        double t0, t1;
        grid_total(part2, G, t0, t1);
        const double beta = sqrt(t0);
        if (beta > 0.0) {
            const double inv = 1.0 / beta;
            double* v = vec(st, VV0);
            for (long long e = e_begin; e < n; e += stride) v[e] = r[e] * inv;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st.scal[SL.beta] = beta;
            step_state(st, ph);
        }
    }
}

}  // namespace

void launch_boxsum(const SysTab* tab, const BoxItem* items, int nitems, int ngroup, cudaStream_t st) {
    if (ngroup > 0) k_groups<<<ngroup, 256, 0, st>>>(tab, items);
    if (nitems > ngroup) k_sums<<<nitems - ngroup, 128, 0, st>>>(tab, items + ngroup);
}

size_t apply_smem_bytes(int nf, int nc, int prec, bool lump32) { return y_layout(nf, nc, prec, lump32).total; }

size_t apply_ring_bytes(int slots, int chunk) { return (size_t)slots * chunk + kRingHeader; }

size_t apply_lump_bytes(int nc, int prec, bool lump32) { return y_layout(0, nc, prec, lump32).lump_part; }

ApplyConfig apply_local_vectors(int nsub, int all_bytes, int lump_bytes, int smem_slots, int chunk, int sm_smem,
                                int sms, int force) {
    const long long ring_all = (long long)apply_ring_bytes(smem_slots, chunk) + 1024,
                    ring2 = (long long)apply_ring_bytes(2, chunk) + 1024;
    const long long fit_all = all_bytes > 0 ? std::min<long long>(2, sm_smem / (all_bytes + ring_all)) : 0;
    const bool lumps_fit = lump_bytes > 0 && 4 * (lump_bytes + ring2) <= sm_smem;
    const ApplyConfig all{Y_SMEM, all_bytes, smem_slots, chunk}, lumps{Y_LUMPS, lump_bytes, 2, chunk},
        dev{Y_DEVICE, 0, 2, chunk};
    if (force == Y_SMEM + 1) return fit_all >= 1 ? all : dev;
    if (force == Y_LUMPS + 1) return lumps_fit ? lumps : dev;
    if (force == Y_DEVICE + 1) return dev;
    if (fit_all >= 1 && (long long)nsub <= fit_all * sms) return all;
    return lumps_fit ? lumps : dev;
}

namespace {
template <typename TF, typename TL, int YM, int SLOTS>
void launch_apply_t(const SysTab* tab, const SubDesc* subs, int nsub, int smem, cudaStream_t st, int* occ) {
    static int configured = -1;
    if (configured < smem) {
        cudaFuncSetAttribute(k_apply<TF, TL, YM, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        configured = smem;
    }
    const int threads = YM == Y_SMEM ? 256 : kApplyThreadsDev;
    if (occ != nullptr) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_apply<TF, TL, YM, SLOTS>, threads, smem) != cudaSuccess)
            *occ = 0;
        return;
    }
    k_apply<TF, TL, YM, SLOTS><<<nsub, threads, smem, st>>>(tab, subs);
}
template <typename TF, typename TL, int YM>
void launch_apply_s(const SysTab* tab, const SubDesc* subs, int nsub, int smem, int slots, cudaStream_t st, int* occ) {
    if (slots == 2)
        launch_apply_t<TF, TL, YM, 2>(tab, subs, nsub, smem, st, occ);
    else if (slots == 3)
        launch_apply_t<TF, TL, YM, 3>(tab, subs, nsub, smem, st, occ);
    else
        launch_apply_t<TF, TL, YM, 4>(tab, subs, nsub, smem, st, occ);
}
template <typename TF, typename TL>
void launch_apply_p(const SysTab* tab, const SubDesc* subs, int nsub, ApplyConfig cfg, int slots, cudaStream_t st,
                    int* occ) {
    const int ring = (int)apply_ring_bytes(slots, cfg.chunk);
    if (cfg.ymode == Y_SMEM)
        launch_apply_s<TF, TL, Y_SMEM>(tab, subs, nsub, ring + cfg.smem, slots, st, occ);
    else if (cfg.ymode == Y_LUMPS)
        launch_apply_s<TF, TL, Y_LUMPS>(tab, subs, nsub, ring + cfg.smem, slots, st, occ);
    else
        launch_apply_s<TF, TL, Y_DEVICE>(tab, subs, nsub, ring, slots, st, occ);
}
// the k_apply instance of (prec, lump32, cfg): launched, or (occ != nullptr) its resident CTAs per SM
void apply_dispatch(const SysTab* tab, const SubDesc* subs, int nsub, int prec, bool lump32, ApplyConfig cfg,
                    cudaStream_t st, int* occ) {
    const int slots = cfg.slots < 2 ? 2 : (cfg.slots > kMaxSlots ? kMaxSlots : cfg.slots);
    if (prec == 0)
        launch_apply_p<double, double>(tab, subs, nsub, cfg, slots, st, occ);
    else if (prec == 1 && lump32)
        launch_apply_p<float, float>(tab, subs, nsub, cfg, slots, st, occ);
    else if (prec == 1)
        launch_apply_p<float, double>(tab, subs, nsub, cfg, slots, st, occ);
    else if (lump32)
        launch_apply_p<__half, float>(tab, subs, nsub, cfg, slots, st, occ);
    else
        launch_apply_p<__half, double>(tab, subs, nsub, cfg, slots, st, occ);
}
}  // namespace

void launch_apply(const SysTab* tab, const SubDesc* subs, int nsub, int prec, bool lump32, ApplyConfig cfg,
                  cudaStream_t st) {
    if (nsub > 0) apply_dispatch(tab, subs, nsub, prec, lump32, cfg, st, nullptr);
}

int apply_ctas_per_sm(int prec, bool lump32, ApplyConfig cfg) {
    int occ = 0;
    apply_dispatch(nullptr, nullptr, 0, prec, lump32, cfg, nullptr, &occ);
    return occ;
}

void launch_restrict(const SysTab* tab, const SubDesc* subs, const int2* items, int nitems, int prec, bool lump32,
                     cudaStream_t st) {
    if (nitems <= 0) return;
    if (prec == 0)
        k_restrict<double, double><<<nitems, 256, 0, st>>>(tab, subs, items);
    else if (lump32)
        k_restrict<float, float><<<nitems, 256, 0, st>>>(tab, subs, items);
    else
        k_restrict<float, double><<<nitems, 256, 0, st>>>(tab, subs, items);
}

void launch_dense_restrict(const SysTab* tab, const SubDesc* subs, int nsub, cudaStream_t st) {
    if (nsub > 0) k_dense_restrict<<<nsub, 256, 0, st>>>(tab, subs);
}

void launch_spmv(const SysTab* tab, const RowItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_spmv<<<nitems, 256, 0, st>>>(tab, items);
}

void launch_init(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_init<<<nitems, VEC_THREADS, 0, st>>>(tab, items);
}
void launch_prep(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_prep<<<nitems, VEC_THREADS, 0, st>>>(tab, items);
}
void launch_post(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_post<<<nitems, VEC_THREADS, 0, st>>>(tab, items);
}
void launch_mgs(const SysTab* tab, const VecItem* items, int nitems, int k, cudaStream_t st) {
    if (nitems > 0) k_mgs<<<nitems, VEC_THREADS, 0, st>>>(tab, items, k);
}
int ortho_coop_grid(int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ortho_coop, VEC_THREADS, 0) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    // two CTAs per SM: enough loads in flight, few partials to reduce and cheap grid barriers
    return std::min(per_sm, 2) * sms;
}

cudaError_t launch_ortho_coop(const SysTab* tab, double* part2, int grid, cudaStream_t st) {
    void* args[] = {(void*)&tab, (void*)&part2};
    return cudaLaunchCooperativeKernel((const void*)k_ortho_coop, dim3(grid), dim3(VEC_THREADS), args, 0, st);
}

void launch_om(const SysTab* tab, const VecItem* items, int nitems, int l, cudaStream_t st) {
    if (nitems > 0) k_om<<<nitems, VEC_THREADS, 0, st>>>(tab, items, l);
}
void launch_om_update(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_om_update<<<nitems, VEC_THREADS, 0, st>>>(tab, items);
}

void launch_finish(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_finish<<<nitems, VEC_THREADS, 0, st>>>(tab, items);
}

}  // namespace asm2
