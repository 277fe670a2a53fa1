// The Krylov side of one step: the BSR SpMV and the GMRES / ORTHOMIN vector and state kernels
// (modified Gram-Schmidt Arnoldi with Givens rotations, and ORTHOMIN(k) projections, Section 2).
// Every kernel reads its system's control words, so systems at different points of their solve
// share the same launches.
#include <algorithm>
#include <cooperative_groups.h>

#include "asm2_internal.h"

namespace asm2 {

namespace {

// ------------------------------------------------------------------------------------------
// SpMV y = A x or y = b - A x (ELL, one thread per block row, 3x3 blocks); four CTAs per SM
// (64 registers) hide the gathers of x better than three at 80 registers
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_spmv(const SysTab* __restrict__ tab, const RowItem* __restrict__ items) {
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
        // one FMA per product into the running sums: an FP64 instruction costs a warp ~64 cycles
        // here, and a separate product-then-add form would take four per three products
        a0 = fma(v[2 * rp], x2, fma(v[rp], x1, fma(v[0], x0, a0)));
        a1 = fma(v[5 * rp], x2, fma(v[4 * rp], x1, fma(v[3 * rp], x0, a1)));
        a2 = fma(v[8 * rp], x2, fma(v[7 * rp], x1, fma(v[6 * rp], x0, a2)));
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

// single-value forms of block_sum2 / grid_total (the same summation order for that value)
__device__ __forceinline__ void block_sum1(double& a) {
    __shared__ double s0[VEC_THREADS];
    s0[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        double x = 0.0;
        for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) x += s0[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        a = x;
    }
    __syncthreads();
}
__device__ __forceinline__ double grid_total1(const double* part, int G) {
    double a = 0.0;
    for (int i = threadIdx.x; i < G; i += blockDim.x) a += __ldcg(&part[i]);
    block_sum1(a);
    __shared__ double bc;
    if (threadIdx.x == 0) bc = a;
    __syncthreads();
    const double t = bc;
    __syncthreads();
    return t;
}

// Classical Gram-Schmidt for step j (asm_options.ortho = ASM_ORTHO_CGS): every coefficient
// h_i = (w, v_i), i = 0..j, and (w, w) from the same w, one sweep per dot and one grid reduction
// for all of them; then w' = w - sum_i h_i v_i (i in order) in one sweep, stored in w, and its norm
// from a second grid reduction.  Two grid barriers per step instead of MGS's j + 2; the rounding
// differs from MGS.  Partials: part2[i G + b] for value i of CTA b, the norm's after them.  The
// caller scales w' into v_{j+1}.  j + 2 <= kCgsMax.
__device__ void cgs_project(const SysTab& st, double* part2, cooperative_groups::grid_group& grid, int j,
                            const ScalLayout& SL, double& w0, double& hn) {
    constexpr int kU = 4;
    const int G = gridDim.x, nv = j + 2, m = st.m;
    const long long n = st.n3p;
    const long long stride = (long long)G * blockDim.x;
    const long long e_begin = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double* w = vec(st, VW);
    // kD dots per sweep over w (vector i of the sweep: v_{i0 + i}, or w itself for the norm);
    // each thread keeps one partial per dot and element slot
    constexpr int kD = 4;
    __shared__ double red[kD][VEC_THREADS];
    for (int i0 = 0; i0 < nv; i0 += kD) {
        const double* vs[kD];
#pragma unroll
        for (int d = 0; d < kD; d++) {
            const int i = i0 + d;
            vs[d] = i <= j ? vec(st, VV0 + i) : (i == j + 1 ? w : nullptr);
        }
        double p[kD][2];
#pragma unroll
        for (int d = 0; d < kD; d++) p[d][0] = p[d][1] = 0.0;
        double a[2], b[kD][2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const long long e = e_begin + u * stride;
            a[u] = e < n ? w[e] : 0.0;
#pragma unroll
            for (int d = 0; d < kD; d++) b[d][u] = e < n && vs[d] ? vs[d][e] : 0.0;
        }
        for (long long e0 = e_begin; e0 < n; e0 += 2 * stride) {
            double an[2], bn[kD][2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const long long e = e0 + (2 + u) * stride;
                an[u] = e < n ? w[e] : 0.0;
#pragma unroll
                for (int d = 0; d < kD; d++) bn[d][u] = e < n && vs[d] ? vs[d][e] : 0.0;
            }
#pragma unroll
            for (int d = 0; d < kD; d++)
                if (vs[d] != nullptr)
#pragma unroll
                    for (int u = 0; u < 2; u++) p[d][u] = fma(a[u], b[d][u], p[d][u]);
#pragma unroll
            for (int u = 0; u < 2; u++) {
                a[u] = an[u];
#pragma unroll
                for (int d = 0; d < kD; d++) b[d][u] = bn[d][u];
            }
        }
        // the kD block sums: warp d adds column d (eight entries per lane, then five shuffles)
#pragma unroll
        for (int d = 0; d < kD; d++) red[d][threadIdx.x] = p[d][0] + p[d][1];
        __syncthreads();
        const int wd = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (wd < kD) {
            double x = 0.0;
            for (int t = lane; t < (int)blockDim.x; t += 32) x += red[wd][t];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0 && i0 + wd < nv) part2[(size_t)(i0 + wd) * G + blockIdx.x] = x;
        }
        __syncthreads();
    }
    grid.sync();
    // the nv totals in every CTA: eight threads per value over its G partials (index order within
    // each thread, then three butterfly adds), 32 values per round
    __shared__ double htot[kCgsMax];
    for (int base = 0; base < nv; base += 32) {
        const int i = base + (int)(threadIdx.x >> 3), q = threadIdx.x & 7;
        double a = 0.0;
        if (i < nv) {
            const double* pi = part2 + (size_t)i * G;
            int c = q;
            for (; c + 24 < G; c += 32) {
                const double l0 = __ldcg(&pi[c]), l1 = __ldcg(&pi[c + 8]), l2 = __ldcg(&pi[c + 16]), l3 = __ldcg(&pi[c + 24]);
                a += l0;
                a += l1;
                a += l2;
                a += l3;
            }
            for (; c < G; c += 8) a += __ldcg(&pi[c]);
        }
        a += __shfl_xor_sync(0xffffffffu, a, 4);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        if (q == 0 && i < nv) htot[i] = a;
    }
    __syncthreads();
    w0 = sqrt(htot[j + 1]);
    double p[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) p[u] = 0.0;
    for (long long e0 = e_begin; e0 < n; e0 += kU * stride) {
        double x[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) x[u] = e0 + u * stride < n ? w[e0 + u * stride] : 0.0;
        // kV basis vectors at a time: all their loads are issued before their multiply-adds (which
        // keep the order i = 0..j), so that enough loads are in flight to stream V from memory
        constexpr int kV = 4;
        int i = 0;
        for (; i + kV <= j + 1; i += kV) {
            double b[kV][kU];
#pragma unroll
            for (int d = 0; d < kV; d++) {
                const double* vi = vec(st, VV0 + i + d);
#pragma unroll
                for (int u = 0; u < kU; u++) b[d][u] = e0 + u * stride < n ? vi[e0 + u * stride] : 0.0;
            }
#pragma unroll
            for (int d = 0; d < kV; d++) {
                const double h = htot[i + d];
#pragma unroll
                for (int u = 0; u < kU; u++) x[u] = fma(-h, b[d][u], x[u]);
            }
        }
        for (; i <= j; i++) {
            const double h = htot[i];
            const double* vi = vec(st, VV0 + i);
            double b[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) b[u] = e0 + u * stride < n ? vi[e0 + u * stride] : 0.0;
#pragma unroll
            for (int u = 0; u < kU; u++) x[u] = fma(-h, b[u], x[u]);
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            if (e0 + u * stride < n) w[e0 + u * stride] = x[u];
            p[u] = fma(x[u], x[u], p[u]);
        }
    }
    double sum = (p[0] + p[1]) + (p[2] + p[3]);
    block_sum1(sum);
    double* pn = part2 + (size_t)nv * G;
    if (threadIdx.x == 0) pn[blockIdx.x] = sum;
    grid.sync();
    hn = sqrt(grid_total1(pn, G));
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int i = 0; i <= j; i++) st.scal[SL.H + i * m + j] = htot[i];
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
        if (st.ortho == 1) {
            cgs_project(st, part2, grid, j, SL, w0, hn);
        } else {
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
                double t0, t1 = 0.0;
                if (k == 0) {  // (w, v_0) and (w, w)
                    s1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
                    block_sum2(s0, s1);
                    if (threadIdx.x == 0) {
                        part[2 * blockIdx.x] = s0;
                        part[2 * blockIdx.x + 1] = s1;
                    }
                    grid.sync();
                    grid_total(part, G, t0, t1);
                } else {  // one sum: half the FP64 adds of the two reductions (same order for s0)
                    block_sum1(s0);
                    if (threadIdx.x == 0) part[blockIdx.x] = s0;
                    grid.sync();
                    t0 = grid_total1(part, G);
                }
                if (k <= j) {
                    hprev = t0;
                    if (k == 0) w0 = sqrt(t1);
                    if (blockIdx.x == 0 && threadIdx.x == 0) st.scal[SL.H + k * m + j] = t0;
                } else {
                    hn = sqrt(t0);
                }
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
