// Kernels of one Krylov step: far-box sums, the fused additive Schwarz apply
// (restriction -> forward sweep -> backward sweep -> owned-row scatter, Eqs. 4.2-4.5), the BSR
// SpMV, and the GMRES vector/state kernels (modified Gram-Schmidt Arnoldi with Givens rotations,
// Section 2).  Every kernel reads its system's control words, so systems at different points of
// their solve share the same launches.
#include <cuda_fp16.h>

#include "asm2_internal.h"

namespace asm2 {

namespace {

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
__device__ __forceinline__ float ldf(const T* p);
template <>
__device__ __forceinline__ float ldf<float>(const float* p) {
    return *p;
}
template <>
__device__ __forceinline__ float ldf<__half>(const __half* p) {
    return __half2float(*p);
}

// ------------------------------------------------------------------------------------------
// far-box sums of the apply input: boxsum[b] = sum over the cells of far box b
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_boxsum(const SysTab* __restrict__ tab, const BoxItem* __restrict__ items) {
    const BoxItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const double* r = st.ws + (long long)in * st.n3p;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int i = it.b0 + threadIdx.x; i < it.b1; i += blockDim.x) {
        const long long c = (long long)it.bcell[i] * 3;
        a0 += r[c];
        a1 += r[c + 1];
        a2 += r[c + 2];
    }
    __shared__ double red[3][256];
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
    if (threadIdx.x < 3) st.boxsum[(long long)it.box * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// ------------------------------------------------------------------------------------------
// fused local solve of one subdomain (one CTA): y = R_i r; y = L^{-1} y; y = U^{-1} y;
// z[owned cells] = y[owned positions].  Levels are separated by CTA barriers.
// ------------------------------------------------------------------------------------------
template <typename TF>
__global__ void __launch_bounds__(256) k_apply(const SysTab* __restrict__ tab, const SubDesc* __restrict__ subs) {
    const SubDesc sd = subs[blockIdx.x];
    const SysTab& st = tab[sd.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const int out = st.ctl[C_APPLY_OUT];
    const double* __restrict__ r = st.ws + (long long)in * st.n3p;
    double* __restrict__ z = st.ws + (long long)out * st.n3p;
    double* __restrict__ y = sd.y;
    const int tid = threadIdx.x, nt = blockDim.x;

    // restriction R_i r: fine rows copy, lumps sum (far lumps: box sum minus the near region)
    for (int p = tid; p < sd.n; p += nt) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        const int b = sd.rbox[p];
        if (b >= 0) {
            a0 = st.boxsum[3 * b];
            a1 = st.boxsum[3 * b + 1];
            a2 = st.boxsum[3 * b + 2];
        }
        for (int i = sd.rptr[p]; i < sd.rptr[p + 1]; i++) {
            const int c = sd.rsrc[i];
            if (c >= 0) {
                const double* rc = r + 3LL * c;
                a0 += rc[0];
                a1 += rc[1];
                a2 += rc[2];
            } else {
                const double* rc = r + 3LL * (~c);
                a0 -= rc[0];
                a1 -= rc[1];
                a2 -= rc[2];
            }
        }
        y[3 * p] = a0;
        y[3 * p + 1] = a1;
        y[3 * p + 2] = a2;
    }
    __syncthreads();

    // forward sweep: y_p -= sum_k L_pk y_k, level by level
    for (int lv = 0; lv < sd.nlev; lv++) {
        const LevelInfo L = sd.lv[lv];
        const unsigned char* seg = sd.stream + L.fwd_off;
        const int* fptr = reinterpret_cast<const int*>(seg);
        size_t o = align16(4 * (size_t)(L.nf + 1));
        const int* fcol = reinterpret_cast<const int*>(seg + o);
        o += align16(4 * (size_t)L.eLf);
        const TF* fval = reinterpret_cast<const TF*>(seg + o);
        o += align16(sizeof(TF) * 9 * (size_t)L.eLf);
        const int* cptr = reinterpret_cast<const int*>(seg + o);
        o += align16(4 * (size_t)(L.nc + 1));
        const int* ccol = reinterpret_cast<const int*>(seg + o);
        o += align16(4 * (size_t)L.eLc);
        const double* cval = reinterpret_cast<const double*>(seg + o);
        for (int t = tid; t < L.nf + L.nc; t += nt) {
            if (t < L.nf) {
                const int pos = L.pos0 + t;
                if constexpr (sizeof(TF) == 8) {
                    double a0 = y[3 * pos], a1 = y[3 * pos + 1], a2 = y[3 * pos + 2];
                    for (int e = fptr[t]; e < fptr[t + 1]; e++) {
                        const double* v = reinterpret_cast<const double*>(fval) + 9LL * e;
                        const int c = fcol[e];
                        const double x0 = y[3 * c], x1 = y[3 * c + 1], x2 = y[3 * c + 2];
                        a0 -= v[0] * x0 + v[1] * x1 + v[2] * x2;
                        a1 -= v[3] * x0 + v[4] * x1 + v[5] * x2;
                        a2 -= v[6] * x0 + v[7] * x1 + v[8] * x2;
                    }
                    y[3 * pos] = a0;
                    y[3 * pos + 1] = a1;
                    y[3 * pos + 2] = a2;
                } else {
                    float a0 = (float)y[3 * pos], a1 = (float)y[3 * pos + 1], a2 = (float)y[3 * pos + 2];
                    for (int e = fptr[t]; e < fptr[t + 1]; e++) {
                        const TF* v = fval + 9LL * e;
                        const int c = fcol[e];
                        const float x0 = (float)y[3 * c], x1 = (float)y[3 * c + 1], x2 = (float)y[3 * c + 2];
                        a0 -= ldf(v) * x0 + ldf(v + 1) * x1 + ldf(v + 2) * x2;
                        a1 -= ldf(v + 3) * x0 + ldf(v + 4) * x1 + ldf(v + 5) * x2;
                        a2 -= ldf(v + 6) * x0 + ldf(v + 7) * x1 + ldf(v + 8) * x2;
                    }
                    y[3 * pos] = a0;
                    y[3 * pos + 1] = a1;
                    y[3 * pos + 2] = a2;
                }
            } else {
                const int i = t - L.nf;
                const int pos = L.pos0 + t;
                double a0 = y[3 * pos], a1 = y[3 * pos + 1], a2 = y[3 * pos + 2];
                for (int e = cptr[i]; e < cptr[i + 1]; e++) {
                    const double* v = cval + 9LL * e;
                    const int c = ccol[e];
                    const double x0 = y[3 * c], x1 = y[3 * c + 1], x2 = y[3 * c + 2];
                    a0 -= v[0] * x0 + v[1] * x1 + v[2] * x2;
                    a1 -= v[3] * x0 + v[4] * x1 + v[5] * x2;
                    a2 -= v[6] * x0 + v[7] * x1 + v[8] * x2;
                }
                y[3 * pos] = a0;
                y[3 * pos + 1] = a1;
                y[3 * pos + 2] = a2;
            }
        }
        __syncthreads();
    }

    // backward sweep: y_p = D_p^{-1} (y_p - sum_q U_pq y_q), levels in reverse
    for (int lv = sd.nlev - 1; lv >= 0; lv--) {
        const LevelInfo L = sd.lv[lv];
        const unsigned char* seg = sd.stream + L.bwd_off;
        const int* fptr = reinterpret_cast<const int*>(seg);
        size_t o = align16(4 * (size_t)(L.nf + 1));
        const int* fcol = reinterpret_cast<const int*>(seg + o);
        o += align16(4 * (size_t)L.eUf);
        const TF* fval = reinterpret_cast<const TF*>(seg + o);
        o += align16(sizeof(TF) * 9 * (size_t)L.eUf);
        const TF* fdi = reinterpret_cast<const TF*>(seg + o);
        o += align16(sizeof(TF) * 9 * (size_t)L.nf);
        const int* cptr = reinterpret_cast<const int*>(seg + o);
        o += align16(4 * (size_t)(L.nc + 1));
        const int* ccol = reinterpret_cast<const int*>(seg + o);
        o += align16(4 * (size_t)L.eUc);
        const double* cval = reinterpret_cast<const double*>(seg + o);
        o += align16(8 * 9 * (size_t)L.eUc);
        const double* cdi = reinterpret_cast<const double*>(seg + o);
        for (int t = tid; t < L.nf + L.nc; t += nt) {
            if (t < L.nf) {
                const int pos = L.pos0 + t;
                if constexpr (sizeof(TF) == 8) {
                    double a0 = y[3 * pos], a1 = y[3 * pos + 1], a2 = y[3 * pos + 2];
                    for (int e = fptr[t]; e < fptr[t + 1]; e++) {
                        const double* v = reinterpret_cast<const double*>(fval) + 9LL * e;
                        const int c = fcol[e];
                        const double x0 = y[3 * c], x1 = y[3 * c + 1], x2 = y[3 * c + 2];
                        a0 -= v[0] * x0 + v[1] * x1 + v[2] * x2;
                        a1 -= v[3] * x0 + v[4] * x1 + v[5] * x2;
                        a2 -= v[6] * x0 + v[7] * x1 + v[8] * x2;
                    }
                    const double* d = reinterpret_cast<const double*>(fdi) + 9LL * t;
                    y[3 * pos] = d[0] * a0 + d[1] * a1 + d[2] * a2;
                    y[3 * pos + 1] = d[3] * a0 + d[4] * a1 + d[5] * a2;
                    y[3 * pos + 2] = d[6] * a0 + d[7] * a1 + d[8] * a2;
                } else {
                    float a0 = (float)y[3 * pos], a1 = (float)y[3 * pos + 1], a2 = (float)y[3 * pos + 2];
                    for (int e = fptr[t]; e < fptr[t + 1]; e++) {
                        const TF* v = fval + 9LL * e;
                        const int c = fcol[e];
                        const float x0 = (float)y[3 * c], x1 = (float)y[3 * c + 1], x2 = (float)y[3 * c + 2];
                        a0 -= ldf(v) * x0 + ldf(v + 1) * x1 + ldf(v + 2) * x2;
                        a1 -= ldf(v + 3) * x0 + ldf(v + 4) * x1 + ldf(v + 5) * x2;
                        a2 -= ldf(v + 6) * x0 + ldf(v + 7) * x1 + ldf(v + 8) * x2;
                    }
                    const TF* d = fdi + 9LL * t;
                    y[3 * pos] = ldf(d) * a0 + ldf(d + 1) * a1 + ldf(d + 2) * a2;
                    y[3 * pos + 1] = ldf(d + 3) * a0 + ldf(d + 4) * a1 + ldf(d + 5) * a2;
                    y[3 * pos + 2] = ldf(d + 6) * a0 + ldf(d + 7) * a1 + ldf(d + 8) * a2;
                }
            } else {
                const int i = t - L.nf;
                const int pos = L.pos0 + t;
                double a0 = y[3 * pos], a1 = y[3 * pos + 1], a2 = y[3 * pos + 2];
                for (int e = cptr[i]; e < cptr[i + 1]; e++) {
                    const double* v = cval + 9LL * e;
                    const int c = ccol[e];
                    const double x0 = y[3 * c], x1 = y[3 * c + 1], x2 = y[3 * c + 2];
                    a0 -= v[0] * x0 + v[1] * x1 + v[2] * x2;
                    a1 -= v[3] * x0 + v[4] * x1 + v[5] * x2;
                    a2 -= v[6] * x0 + v[7] * x1 + v[8] * x2;
                }
                const double* d = cdi + 9LL * i;
                y[3 * pos] = d[0] * a0 + d[1] * a1 + d[2] * a2;
                y[3 * pos + 1] = d[3] * a0 + d[4] * a1 + d[5] * a2;
                y[3 * pos + 2] = d[6] * a0 + d[7] * a1 + d[8] * a2;
            }
        }
        __syncthreads();
    }

    // P_i R_i^T: owned cells take this subdomain's solution; the lumps are discarded
    for (int t = tid; t < sd.n_own; t += nt) {
        const int p = sd.own_pos[t];
        const long long c = 3LL * sd.own_cell[t];
        z[c] = y[3 * p];
        z[c + 1] = y[3 * p + 1];
        z[c + 2] = y[3 * p + 2];
    }
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

// block sum of two values; result valid in thread 0
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double s0[32], s1[32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s0[w] = a;
        s1[w] = b;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        a = l < nw ? s0[l] : 0.0;
        b = l < nw ? s1[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
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

// End of a step: vector scaling (v_{j+1} = w / h_{j+1,j}, or v_0 = r / beta), then the last chunk
// of each system applies the Givens rotations and moves its state machine.
__global__ void __launch_bounds__(VEC_THREADS) k_finish(const SysTab* __restrict__ tab,
                                                        const VecItem* __restrict__ items) {
    const VecItem it = items[blockIdx.x];
    const SysTab& st = tab[it.sys];
    const int ph = st.ctl[C_PHASE];
    if (ph == PH_DONE) return;
    const ScalLayout SL = ScalLayout::make(st.m);
    const long long e0 = (long long)it.chunk * VEC_CHUNK;
    const int m = st.m;
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

}  // namespace

void launch_boxsum(const SysTab* tab, const BoxItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_boxsum<<<nitems, 256, 0, st>>>(tab, items);
}

void launch_apply(const SysTab* tab, const SubDesc* subs, int nsub, int prec, cudaStream_t st) {
    if (nsub <= 0) return;
    if (prec == 0)
        k_apply<double><<<nsub, 256, 0, st>>>(tab, subs);
    else if (prec == 1)
        k_apply<float><<<nsub, 256, 0, st>>>(tab, subs);
    else
        k_apply<__half><<<nsub, 256, 0, st>>>(tab, subs);
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
void launch_finish(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st) {
    if (nitems > 0) k_finish<<<nitems, VEC_THREADS, 0, st>>>(tab, items);
}

}  // namespace asm2
