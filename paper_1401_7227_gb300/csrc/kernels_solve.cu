// The preconditioner apply of one Krylov step: cell-group and far-box sums, the restriction into
// the local vectors, the fused ILU(0) sweeps of every subdomain (forward sweep -> backward sweep
// -> owned-row scatter, Eqs. 4.2-4.5), and the restriction of the exact local solves.  Every
// kernel reads its system's control words, so systems at different points of their solve share
// the same launches.  The SpMV and the Krylov vector kernels are in kernels_krylov.cu.
#include <cuda_fp16.h>

#include <algorithm>

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
// fixed order (y, then x, then z): every list sum that covers whole groups reads these instead.
// With FP32 local vectors it also writes each cell's entries rounded to FP32 (r32, 16 bytes per
// cell), once per cell, for the restriction's fine rows to copy.
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
                const long long cell = z + (long long)st.gnz * (x + (long long)st.gnx * y);
                const double* rc = r + 3LL * cell;
                const double v0 = rc[0], v1 = rc[1], v2 = rc[2];
                a0 += v0;
                a1 += v1;
                a2 += v2;
                if (st.r32 != nullptr) st.r32[cell] = make_float4(f64_to_f32(v0), f64_to_f32(v1), f64_to_f32(v2), 0.f);
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
                    acc = fma(-v[2], x2, fma(-v[1], x1, fma(-v[0], x0, acc)));  // one FMA per product
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
        if constexpr (kRow16) {
            float4* yf4 = reinterpret_cast<float4*>(y + sd.y_fine) + q;
            if (st.r32 != nullptr) {  // rounded once per cell by k_groups
                *yf4 = st.r32[sd.fcell[q]];
            } else {
                const double* rc = r + 3LL * sd.fcell[q];
                *yf4 = make_float4(f64_to_f32(rc[0]), f64_to_f32(rc[1]), f64_to_f32(rc[2]), 0.f);
            }
        } else {
            const double* rc = r + 3LL * sd.fcell[q];
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

}  // namespace

void launch_boxsum(const SysTab* tab, const BoxItem* items, int nitems, int ngroup, cudaStream_t st) {
    if (ngroup > 0) k_groups<<<ngroup, 256, 0, st>>>(tab, items);
    if (nitems > ngroup) k_sums<<<nitems - ngroup, 128, 0, st>>>(tab, items + ngroup);
}

size_t apply_smem_bytes(int nf, int nc, int prec, bool lump32) { return y_layout(nf, nc, prec, lump32).total; }

size_t apply_ring_bytes(int slots, int chunk) { return (size_t)slots * chunk + kRingHeader; }

size_t apply_lump_bytes(int nc, int prec, bool lump32) { return y_layout(0, nc, prec, lump32).lump_part; }

ApplyConfig apply_local_vectors(int nsub, int all_bytes, int lump_bytes, int smem_slots, int chunk, int sm_smem,
                                int sms, int force, int other_slots) {
    const long long ring_all = (long long)apply_ring_bytes(smem_slots, chunk) + 1024,
                    ring_o = (long long)apply_ring_bytes(other_slots, chunk) + 1024;
    const long long fit_all = all_bytes > 0 ? std::min<long long>(2, sm_smem / (all_bytes + ring_all)) : 0;
    const bool lumps_fit = lump_bytes > 0 && 4 * (lump_bytes + ring_o) <= sm_smem;
    const ApplyConfig all{Y_SMEM, all_bytes, smem_slots, chunk}, lumps{Y_LUMPS, lump_bytes, other_slots, chunk},
        dev{Y_DEVICE, 0, other_slots, chunk};
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

}  // namespace asm2
