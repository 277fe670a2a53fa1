// Nested factorisation (Appendix A) as the local solver of local problems without lumps: each
// subdomain's A_i is hepta-banded on its box of bx * by * bz cells (local cell p = z + bz (x + bx y)),
// A = D + L1 + U1 + L2 + U2 + L3 + U3, and
//   B = (P + L3)(I + P^{-1} U3),  P = (T + L2)(I + T^{-1} U2),  T = (G + L1)(I + G^{-1} U1)
// with G block diagonal, G = D - L1 G^{-1} U1 (Eq. A.6), with colsum also minus the block column sums
// of L2 T^{-1} U2 and L3 P^{-1} U3 (Eq. A.7).
//
// Both the factorisation and the solve are sequential along the cells of a subdomain: every line
// depends on the previous line of its plane, every plane on the previous plane.  So one warp takes
// one subdomain.  In the factorisation its lanes share the 3x3 block algebra (lane 3 r + c holds
// element (r, c) of a block) and the independent per-cell products.  The apply streams one packet
// per line -- G^{-1}, G^{-1} L1, G^{-1} U1, their two-step products, L2, L3, U3, U2 of the line's
// cells, packed after the factorisation -- through a shared-memory ring of 2-4 slots by bulk copies,
// ahead of the line being solved.  The products that do not depend on the line recurrences run on
// all lanes; the two recurrences of T^{-1}, with one level of recursive doubling, run from shared
// memory on one lane (FP32) or three (FP64, one row each: an FP64 instruction costs the same for one
// lane as for 32).
#include <cuda_runtime.h>

#include <algorithm>

#include "asm2_internal.h"
#include "tma.h"

namespace asm2 {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- the factorisation: 3x3 blocks held one element per lane (lanes 0..8; others carry zeros) ----

// Each cell's seven band blocks D, L1, U1, L2, U2, L3, U3 (zero where the neighbour is missing),
// gathered from the assembled slots into the compute type before the sequential factorisation,
// so that its operand loads need no index and can be issued early.
enum { BD_D = 0, BD_L1, BD_U1, BD_L2, BD_U2, BD_L3, BD_U3, BD_N };

template <typename TC>
__global__ void __launch_bounds__(128) k_nf_gather(const NFDesc* __restrict__ descs) {
    const NFDesc& d = descs[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // (cell, band)
    if (t >= BD_N * d.n) return;
    const int sl = d.bands[t];
    TC* o = static_cast<TC*>(d.fband) + 9LL * t;
    for (int e = 0; e < 9; e++) o[e] = sl >= 0 ? (TC)d.slot[9LL * sl + e] : TC(0);
}

// a * b for blocks held per lane
template <typename TC>
__device__ __forceinline__ TC bmul(TC a, TC b, int lane) {
    const int r = lane < 9 ? lane / 3 : 0, c = lane < 9 ? lane - 3 * (lane / 3) : 0;
    const TC a0 = __shfl_sync(kFull, a, 3 * r), a1 = __shfl_sync(kFull, a, 3 * r + 1), a2 = __shfl_sync(kFull, a, 3 * r + 2);
    const TC b0 = __shfl_sync(kFull, b, c), b1 = __shfl_sync(kFull, b, 3 + c), b2 = __shfl_sync(kFull, b, 6 + c);
    return lane < 9 ? a0 * b0 + a1 * b1 + a2 * b2 : TC(0);
}

// Inverse of a block held per lane by cofactors: lane 3 r + c gets C_cr / det, with the cofactor
// C_ij = a_{i+1,j+1} a_{i+2,j+2} - a_{i+1,j+2} a_{i+2,j+1} (indices mod 3) and det = sum_k a_0k C_0k.
// Twelve dependent operations instead of the ~60 of an elimination on one lane (a dependent FP64
// operation costs ~100 cycles here).  false (on every lane) when det = 0.
template <typename TC>
__device__ __forceinline__ bool binv(TC a, TC& inv, int lane) {
    const int r = lane < 9 ? lane / 3 : 0, c = lane < 9 ? lane - 3 * (lane / 3) : 0;
    const int i1 = c == 2 ? 0 : c + 1, i2 = c == 0 ? 2 : c - 1, j1 = r == 2 ? 0 : r + 1, j2 = r == 0 ? 2 : r - 1;
    const TC p = __shfl_sync(kFull, a, 3 * i1 + j1), q = __shfl_sync(kFull, a, 3 * i2 + j2);
    const TC u = __shfl_sync(kFull, a, 3 * i1 + j2), v = __shfl_sync(kFull, a, 3 * i2 + j1);
    const TC cof = p * q - u * v;                       // C_cr
    const TC term = __shfl_sync(kFull, a, r) * cof;     // lanes 3 r (c = 0): a_0r C_0r
    const TC det = __shfl_sync(kFull, term, 0) + __shfl_sync(kFull, term, 3) + __shfl_sync(kFull, term, 6);
    if (det == TC(0)) return false;
    inv = lane < 9 ? cof / det : TC(0);
    return true;
}

template <typename TC>
struct NFView {
    const NFDesc& d;
    TC* nk;  // N_p = G_p^{-1} U1_p ([9 n]), then K_p = L1_{p+1} G_p^{-1} ([9 n])
    __device__ const TC* band(int k, int p) const { return static_cast<const TC*>(d.fband) + 9LL * (BD_N * p + k); }
    __device__ const double* gi(int p) const { return d.gi + 9LL * p; }
    __device__ const TC* N(int p) const { return nk + 9LL * p; }
    __device__ const TC* K(int p) const { return nk + 9LL * (d.n + p); }
};

// element `lane` of a block (lanes 9..31: zero)
template <typename TC, typename TS>
__device__ __forceinline__ TC ld(const TS* p, int lane) { return lane < 9 ? (TC)p[lane] : TC(0); }

// W = u T^{-1} on the line starting at cell q0: W (G + L1)(I + G^{-1} U1) = u (rows of blocks).
// With N_q = G_q^{-1} U1_q and K_q = L1_{q+1} G_q^{-1} (formed once per line after its G), each
// sequential step is one block product:
//   forward   v_q = u_q - v_{q-1} N_{q-1}            (v (I + G^{-1} U1) = u)
//   backward  W_q = v_q G_q^{-1} - W_{q+1} K_q       (W (G + L1) = v; v_q G_q^{-1} on all lanes first)
// The operands come from device memory (L2) at ~400 cycles, against ~50 cycles of arithmetic per
// FP32 step, so the chains take them kRowG steps at a time into one of two register buffers, the
// next group's loads issued before the current group is computed.  An FP64 step takes ~300 cycles,
// so four steps cover the load latency, and the smaller buffers keep k_nf_factor<double> free of
// register spills (eight: 255 registers and 92 bytes spilled; four: 233 registers, none, and the
// FP64 re-factor 12% faster at 1M cells).
template <typename TC>
__device__ void line_row_solve(const NFView<TC>& v, int q0, const TC* u, TC* vtmp, TC* W, int lane) {
    constexpr int kRowG = sizeof(TC) == 8 ? 4 : 8;
    const int bz = v.d.bz;
    {
        TC a[2][kRowG], b[2][kRowG];  // u_q, N_{q-1}
        TC prev = 0;
#define NF_LOAD_F(h, gs)                                                            \
    _Pragma("unroll") for (int i = 0; i < kRowG; i++) {                             \
        const int q = (gs) + i;                                                     \
        a[h][i] = q < bz ? ld<TC>(u + 9 * q, lane) : TC(0);                         \
        b[h][i] = q > 0 && q < bz ? ld<TC>(v.N(q0 + q - 1), lane) : TC(0);          \
    }
        NF_LOAD_F(0, 0)
        for (int g0 = 0; g0 < bz; g0 += 2 * kRowG) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int gs = g0 + h * kRowG;
                if (gs < bz) {
                    if (gs + kRowG < bz) {
                        if (h == 0) {
                            NF_LOAD_F(1, gs + kRowG)
                        } else {
                            NF_LOAD_F(0, gs + kRowG)
                        }
                    }
#pragma unroll
                    for (int i = 0; i < kRowG; i++) {
                        const int q = gs + i;
                        if (q < bz) {
                            TC x = a[h][i];
                            if (q > 0) x -= bmul(prev, b[h][i], lane);
                            if (lane < 9) vtmp[9 * q + lane] = x;
                            prev = x;
                        }
                    }
                }
            }
        }
#undef NF_LOAD_F
    }
    __syncwarp();
    // v_q G_q^{-1}, one block element per lane, kB elements' loads in flight per lane
    constexpr int kB = 4;
    for (int t0 = lane; t0 < 9 * bz; t0 += 32 * kB) {
        TC av[kB][3], gv[kB][3];
#pragma unroll
        for (int j = 0; j < kB; j++) {
            const int t = t0 + 32 * j, q = t / 9, e = t - 9 * q, r = e / 3, k = e - 3 * r;
            const bool in = t < 9 * bz;
            const TC* a = vtmp + 9 * (in ? q : 0);
            const double* g = v.gi(q0 + (in ? q : 0));
#pragma unroll
            for (int m = 0; m < 3; m++) {
                av[j][m] = a[3 * r + m];
                gv[j][m] = (TC)g[3 * m + k];
            }
        }
#pragma unroll
        for (int j = 0; j < kB; j++)
            if (t0 + 32 * j < 9 * bz) W[t0 + 32 * j] = av[j][0] * gv[j][0] + av[j][1] * gv[j][1] + av[j][2] * gv[j][2];
    }
    __syncwarp();
    {
        TC a[2][kRowG], b[2][kRowG];  // (v G^{-1})_q, K_q, for q = bz - 1 - (step)
        TC next = 0;
#define NF_LOAD_B(h, gs)                                                            \
    _Pragma("unroll") for (int i = 0; i < kRowG; i++) {                             \
        const int q = bz - 1 - ((gs) + i);                                          \
        a[h][i] = q >= 0 ? ld<TC>(W + 9 * q, lane) : TC(0);                         \
        b[h][i] = q >= 0 && q < bz - 1 ? ld<TC>(v.K(q0 + q), lane) : TC(0);         \
    }
        NF_LOAD_B(0, 0)
        for (int g0 = 0; g0 < bz; g0 += 2 * kRowG) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int gs = g0 + h * kRowG;
                if (gs < bz) {
                    if (gs + kRowG < bz) {
                        if (h == 0) {
                            NF_LOAD_B(1, gs + kRowG)
                        } else {
                            NF_LOAD_B(0, gs + kRowG)
                        }
                    }
#pragma unroll
                    for (int i = 0; i < kRowG; i++) {
                        const int q = bz - 1 - (gs + i);
                        if (q >= 0) {
                            TC x = a[h][i];
                            if (q < bz - 1) x -= bmul(next, b[h][i], lane);
                            if (lane < 9) W[9 * q + lane] = x;
                            next = x;
                        }
                    }
                }
            }
        }
#undef NF_LOAD_B
    }
    __syncwarp();
}

// Independent block operations over n cells, one block element per lane and step (all 32 lanes):
// dst_c = src_c - A_c B_c (SUB), dst_c = A_c B_c, or dst_c = src_c (no product); src, A, B give
// each cell's block (src may be null: zero)
template <bool SUB, typename TC, typename FS, typename FA, typename FB>
__device__ __forceinline__ void blocks(TC* dst, int n, FS src, FA A, FB B, int lane) {
    for (int t = lane; t < 9 * n; t += 32) {
        const int c = t / 9, e = t - 9 * c, r = e / 3, k = e - 3 * r;
        const TC* a = A(c);
        const TC* b = B(c);
        const TC* s0 = src(c);
        TC v = 0;
        if (a && b) v = a[3 * r] * b[k] + a[3 * r + 1] * b[3 + k] + a[3 * r + 2] * b[6 + k];
        if (SUB) v = (s0 ? s0[e] : TC(0)) - v;
        dst[9 * c + e] = v;
    }
    __syncwarp();
}

// W = u P^{-1} on the plane starting at c0 (rows of blocks); scratch: vb (9 S), x, y, vt (9 bz each)
template <typename TC>
__device__ void plane_row_solve(const NFView<TC>& v, int c0, const TC* u, TC* vb, TC* x, TC* y, TC* vt, TC* W,
                                int lane) {
    const int bz = v.d.bz, bx = v.d.bx;
    const auto none = [](int) -> const TC* { return nullptr; };
    for (int l = 0; l < bx; l++) {  // vb (I + T^{-1} U2) = u: vb_l = u_l - (vb_{l-1} T_{l-1}^{-1}) U2_{l-1}
        const int cl = l * bz;
        if (l > 0) {
            line_row_solve(v, c0 + cl - bz, vb + 9 * (cl - bz), vt, x, lane);
            blocks<true>(vb + 9 * cl, bz, [&](int q) { return u + 9 * (cl + q); }, [&](int q) { return x + 9 * q; },
                         [&](int q) { return v.band(BD_U2, c0 + cl - bz + q); }, lane);
        } else {
            blocks<true>(vb, bz, [&](int q) { return u + 9 * q; }, none, none, lane);
        }
    }
    for (int l = bx - 1; l >= 0; l--) {  // W (T + L2) = vb: W_l = (vb_l - W_{l+1} L2_{l+1}) T_l^{-1}
        const int cl = l * bz;
        if (l < bx - 1)
            blocks<true>(y, bz, [&](int q) { return vb + 9 * (cl + q); }, [&](int q) { return W + 9 * (cl + bz + q); },
                         [&](int q) { return v.band(BD_L2, c0 + cl + bz + q); }, lane);
        else
            blocks<true>(y, bz, [&](int q) { return vb + 9 * (cl + q); }, none, none, lane);
        line_row_solve(v, c0 + cl, y, vt, W + 9 * cl, lane);
    }
}

// Factorisation in the compute type TC: G and G^{-1} (stored in FP64) of every cell, plane by
// plane, line by line, cell by cell
template <typename TC>
__global__ void __launch_bounds__(128) k_nf_factor(const NFDesc* __restrict__ descs, int ndesc, FactErr* err) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= ndesc) return;
    const NFDesc d = descs[w];  // by value: its fields stay in registers across the stores
    const int bz = d.bz, bx = d.bx, by = d.by, S = bz * bx;
    // scratch: cs3 (9 S), u (9 S), W (9 S), vb (9 S), x, y, vt, cs2 (9 bz each), N and K (9 n each)
    TC* cs3 = reinterpret_cast<TC*>(d.work);
    const NFView<TC> v{d, cs3 + 36 * S + 36 * bz};
    TC* u = cs3 + 9 * S;
    TC* W = u + 9 * S;
    TC* vb = W + 9 * S;
    TC* x = vb + 9 * S;
    TC* y = x + 9 * bz;
    TC* vt = y + 9 * bz;
    TC* cs2 = vt + 9 * bz;
    for (int j = 0; j < by; j++) {
        const int c0 = j * S;
        const bool plane_term = d.colsum && j > 0;
        const auto none = [](int) -> const TC* { return nullptr; };
        if (plane_term) {  // block column sums of L3 P_{j-1}^{-1} U3 on plane j
            blocks<true>(u, S, [&](int c) { return v.band(BD_L3, c0 + c); }, none, none, lane);
            plane_row_solve(v, c0 - S, u, vb, x, y, vt, W, lane);
            blocks<false>(cs3, S, none, [&](int c) { return W + 9 * c; }, [&](int c) { return v.band(BD_U3, c0 - S + c); },
                          lane);
        }
        for (int l = 0; l < bx; l++) {
            const int q0 = c0 + l * bz;
            const bool line_term = d.colsum && l > 0;
            if (line_term) {  // block column sums of L2 T_{l-1}^{-1} U2 on line l
                blocks<true>(u, bz, [&](int q) { return v.band(BD_L2, q0 + q); }, none, none, lane);
                line_row_solve(v, q0 - bz, u, vt, W, lane);
                blocks<false>(cs2, bz, none, [&](int q) { return W + 9 * q; },
                              [&](int q) { return v.band(BD_U2, q0 - bz + q); }, lane);
            }
            // G_p = D_p - L1_p G_{p-1}^{-1} U1_{p-1} - (line and plane column sums); the previous
            // cell's G^{-1} stays in a register, the next cell's operands load early
            TC gprev = 0;
            TC nd = ld<TC>(v.band(BD_D, q0), lane), nl1 = 0, nu1 = 0;
            TC nc2 = line_term ? ld<TC>(cs2, lane) : TC(0), nc3 = plane_term ? ld<TC>(cs3 + 9 * l * bz, lane) : TC(0);
            for (int q = 0; q < bz; q++) {
                const int p = q0 + q;
                const TC cd = nd, cl1 = nl1, cu1 = nu1, cc2 = nc2, cc3 = nc3;
                if (q + 1 < bz) {
                    nd = ld<TC>(v.band(BD_D, p + 1), lane);
                    nl1 = ld<TC>(v.band(BD_L1, p + 1), lane);
                    nu1 = ld<TC>(v.band(BD_U1, p), lane);
                    if (line_term) nc2 = ld<TC>(cs2 + 9 * (q + 1), lane);
                    if (plane_term) nc3 = ld<TC>(cs3 + 9 * (l * bz + q + 1), lane);
                }
                TC g = cd;
                if (q > 0) g -= bmul(bmul(cl1, gprev, lane), cu1, lane);
                g -= cc2;
                g -= cc3;
                if (lane < 9) d.g[9LL * p + lane] = (double)g;
                TC gi;
                if (!binv(g, gi, lane)) {
                    if (lane == 0 && atomicCAS(&err->flag, 0, 1) == 0) {
                        err->sub = d.sub;
                        err->row = p;
                    }
                    return;  // the whole warp leaves together (binv's result is warp-uniform)
                }
                if (lane < 9) d.gi[9LL * p + lane] = (double)gi;
                gprev = gi;
            }
            __syncwarp();
            // N_q = G_q^{-1} U1_q and K_q = L1_{q+1} G_q^{-1} of this line, for its row-vector solves
            TC* nline = v.nk + 9LL * q0;
            TC* kline = v.nk + 9LL * (d.n + q0);
            for (int t = lane; t < 9 * bz; t += 32) {
                const int q = t / 9, e = t - 9 * q, r = e / 3, k = e - 3 * r;
                const double* g = v.gi(q0 + q);
                const TC* u1 = v.band(BD_U1, q0 + q);
                nline[t] = (TC)g[3 * r] * u1[k] + (TC)g[3 * r + 1] * u1[3 + k] + (TC)g[3 * r + 2] * u1[6 + k];
                TC kv = 0;
                if (q + 1 < bz) {
                    const TC* l1 = v.band(BD_L1, q0 + q + 1);
                    kv = l1[3 * r] * (TC)g[k] + l1[3 * r + 1] * (TC)g[3 + k] + l1[3 * r + 2] * (TC)g[6 + k];
                }
                kline[t] = kv;
            }
            __syncwarp();
        }
    }
}

// ---- the apply ---------------------------------------------------------------------------------

// fields of a line packet, each bz blocks, field after field.  A line solve copies only the fields
// it reads into a ring slot of SL_FIELDS fields: G^{-1}, M, N, P, Q always (slot fields 0-4),
// then L2 and L3 on a forward line of a forward plane, L2 and U3 on a forward line of a backward
// plane, U2 on a backward line (slot fields 5, 6).
enum { PK_GI = 0, PK_M, PK_N, PK_P, PK_Q, PK_L2, PK_L3, PK_U3, PK_U2, PK_FIELDS };
enum { SL_X = 5, SL_Y = 6, SL_FIELDS = 7 };

// Layout of the compute type: a 3x3 block is 3 rows of RS values (row r at r RS), a cell's
// 3-vector takes VS values in shared memory.  FP32 pads both to 4, so that a row or a vector is one
// 16-byte access; FP64 keeps them dense (its packets are twice as large already).
template <typename T>
struct Lay {
    static constexpr int RS = 3, VS = 3;
};
template <>
struct Lay<float> {
    static constexpr int RS = 4, VS = 4;
};

__device__ __forceinline__ void ld3(const float* p, float& a, float& b, float& c) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = v.x;
    b = v.y;
    c = v.z;
}
__device__ __forceinline__ void ld3(const double* p, double& a, double& b, double& c) {
    a = p[0];
    b = p[1];
    c = p[2];
}
__device__ __forceinline__ void st3(float* p, float a, float b, float c) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, 0.f);
}
__device__ __forceinline__ void st3(double* p, double a, double b, double c) {
    p[0] = a;
    p[1] = b;
    p[2] = c;
}

// y -= a x for a 3x3 block a and 3-vectors, one fused chain per row
template <typename T>
__device__ __forceinline__ void sub_mv(const T* a, T x0, T x1, T x2, T& y0, T& y1, T& y2) {
    constexpr int RS = Lay<T>::RS;
    T a0, a1, a2;
    ld3(a, a0, a1, a2);
    y0 = fma(-a2, x2, fma(-a1, x1, fma(-a0, x0, y0)));
    ld3(a + RS, a0, a1, a2);
    y1 = fma(-a2, x2, fma(-a1, x1, fma(-a0, x0, y1)));
    ld3(a + 2 * RS, a0, a1, a2);
    y2 = fma(-a2, x2, fma(-a1, x1, fma(-a0, x0, y2)));
}

// packets of every line, one thread per cell: G^{-1}, M = G^{-1} L1 (the forward recurrence of
// (G + L1) s = u is s_q = G_q^{-1} u_q - M_q s_{q-1}), N = G^{-1} U1 (the backward recurrence of
// (I + G^{-1} U1) w = s is w_q = s_q - N_q w_{q+1}), the two-step products P_q = M_q M_{q-1} and
// Q_q = N_q N_{q+1}, and the blocks L2, U2, L3, U3 (zero where the neighbour is missing); products
// in FP64, stored in the compute type (row padding stays zero)
// bytes of one field of a line packet: bz blocks, rounded up to 16 bytes (a bulk-copy unit)
template <typename T>
__host__ __device__ __forceinline__ size_t field_bytes(int bz) {
    return ((size_t)9 * Lay<T>::RS / 3 * sizeof(T) * bz + 15) & ~(size_t)15;
}

template <typename T>
__global__ void __launch_bounds__(128) k_nf_pack(const NFDesc* __restrict__ descs) {
    constexpr int RS = Lay<T>::RS, BS = 3 * RS;
    const NFDesc& d = descs[blockIdx.y];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.n) return;
    const int bz = d.bz, line = p / bz, q = p - line * bz;
    T* pk = reinterpret_cast<T*>(static_cast<unsigned char*>(d.pack) + (size_t)line * d.line_bytes);
    const auto band = [&](int k) -> const double* {
        const int s = d.bands[7 * p + k];
        return s >= 0 ? d.slot + 9LL * s : nullptr;
    };
    const auto put = [&](int f, const double* b) {
        T* o = pk + (size_t)f * (field_bytes<T>(bz) / sizeof(T)) + (size_t)q * BS;
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) o[r * RS + c] = b ? (T)b[3 * r + c] : T(0);
    };
    const auto mul = [](const double* a, const double* b, double* c) {
        for (int r = 0; r < 3; r++)
            for (int k = 0; k < 3; k++) c[3 * r + k] = a[3 * r] * b[k] + a[3 * r + 1] * b[3 + k] + a[3 * r + 2] * b[6 + k];
    };
    // G^{-1} L1 (k = 1) or G^{-1} U1 (k = 2) of cell pp; false where that band block is missing
    const auto gib = [&](int pp, int k, double* out) {
        const int sl = d.bands[7 * pp + k];
        if (sl < 0) return false;
        mul(d.gi + 9LL * pp, d.slot + 9LL * sl, out);
        return true;
    };
    double m[9], m2[9], pq[9];
    put(PK_GI, d.gi + 9LL * p);
    const bool hm = gib(p, 1, m);
    put(PK_M, hm ? m : nullptr);
    put(PK_P, hm && q > 0 && gib(p - 1, 1, m2) ? (mul(m, m2, pq), pq) : nullptr);
    const bool hn = gib(p, 2, m);
    put(PK_N, hn ? m : nullptr);
    put(PK_Q, hn && q + 1 < bz && gib(p + 1, 2, m2) ? (mul(m, m2, pq), pq) : nullptr);
    put(PK_L2, band(3));
    put(PK_U2, band(4));
    put(PK_L3, band(5));
    put(PK_U3, band(6));
}

// The line solves of one apply, in order: forward planes j = 0 .. by-1, then backward planes
// j = by-2 .. 0; in each plane the forward lines l = 0 .. bx-1 of (T + L2) z = t, then the
// backward lines l = bx-2 .. 0 of (I + T^{-1} U2) o = z.  P counts the plane passes, i the line
// solves of the pass; next() advances without divisions.
struct LineStep {
    int P = 0, i = 0, j = 0, l = 0;
    bool fwd_plane = true, fwd_line = true, plane_first = true, plane_done = false;
    __device__ __forceinline__ void set(int bx, int by) {
        fwd_plane = P < by;
        j = fwd_plane ? P : 2 * by - 2 - P;
        fwd_line = i < bx;
        l = fwd_line ? i : 2 * bx - 2 - i;
        plane_first = i == 0;
        plane_done = i == 2 * bx - 2;
    }
    __device__ __forceinline__ void next(int bx, int by) {
        if (++i == 2 * bx - 1) {
            i = 0;
            ++P;
        }
        set(bx, by);
    }
};

__host__ __device__ size_t nf_rline_bytes(int bz) { return ((size_t)24 * bz + 32 + 15) & ~(size_t)15; }

// bytes of a plane vector (VS values per cell, rounded up to 16)
template <typename T>
__host__ __device__ __forceinline__ size_t nf_plane_bytes(int S) {
    return ((size_t)Lay<T>::VS * S * sizeof(T) + 15) & ~(size_t)15;
}

// z[owned cells of plane j] = x_j (held in pv)
template <typename T>
__device__ __forceinline__ void write_owned(const NFDesc& d, int j, const T* pv, double* z, int lane) {
    constexpr int VS = Lay<T>::VS;
    if (j < d.own_lo[1] || j >= d.own_hi[1]) return;
    const int wx = d.own_hi[0] - d.own_lo[0], wz = d.own_hi[2] - d.own_lo[2];
    for (int t = lane; t < wx * wz; t += 32) {
        const int x = d.own_lo[0] + t / wz, zz = d.own_lo[2] + t % wz;
        const long long cell = d.c0 + zz + (long long)d.gnz * (x + (long long)d.gnx * j);
        const T* v = pv + VS * (x * d.bz + zz);
        z[3 * cell] = (double)v[0];
        z[3 * cell + 1] = (double)v[1];
        z[3 * cell + 2] = (double)v[2];
    }
}

// One chain step x <- c + A x for a 3x3 block A (three float4 rows) and 3-vectors, one fused
// chain per row
__device__ __forceinline__ void chain_step(const float4* a, float4 c, float& x0, float& x1, float& x2) {
    const float n0 = fmaf(a[0].z, x2, fmaf(a[0].y, x1, fmaf(a[0].x, x0, c.x)));
    const float n1 = fmaf(a[1].z, x2, fmaf(a[1].y, x1, fmaf(a[1].x, x0, c.y)));
    const float n2 = fmaf(a[2].z, x2, fmaf(a[2].y, x1, fmaf(a[2].x, x0, c.z)));
    x0 = n0;
    x1 = n1;
    x2 = n2;
}

// x_q = c_q + A_q x_{q-d} for q = q0, q0 + d, ... (d = +-2; the x before q0 is zero), in place
// in cb, on one lane (FP32).  Four steps make a group whose operands are loaded first.
__device__ __forceinline__ void chain(const float* A, float* cb, int q0, int d, int count) {
    const float4* Av = reinterpret_cast<const float4*>(A);
    float4* cv = reinterpret_cast<float4*>(cb);
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    int i = 0;
    for (; i + 4 <= count; i += 4) {
        float4 a[12], c[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int q = q0 + d * (i + u);
            a[3 * u] = Av[3 * q];
            a[3 * u + 1] = Av[3 * q + 1];
            a[3 * u + 2] = Av[3 * q + 2];
            c[u] = cv[q];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            chain_step(a + 3 * u, c[u], x0, x1, x2);
            c[u] = make_float4(x0, x1, x2, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) cv[q0 + d * (i + u)] = c[u];
    }
    for (; i < count; i++) {
        const int q = q0 + d * i;
        const float4 a[3] = {Av[3 * q], Av[3 * q + 1], Av[3 * q + 2]};
        chain_step(a, cv[q], x0, x1, x2);
        cv[q] = make_float4(x0, x1, x2, 0.f);
    }
}

// The same on three lanes (FP64: lane r takes row r, the state goes round by shuffles; an FP64
// instruction costs the same for one lane as for 32)
__device__ __forceinline__ void chain(const double* A, double* cb, int q0, int d, int count, int lane) {
    constexpr unsigned kRow = 0x7u;
    double x = 0.0;
    for (int i = 0; i < count; i++) {
        const int q = q0 + d * i;
        const double* a = A + 9 * q + 3 * lane;
        const double a0 = a[0], a1 = a[1], a2 = a[2], c = cb[3 * q + lane];
        const double x0 = __shfl_sync(kRow, x, 0), x1 = __shfl_sync(kRow, x, 1), x2 = __shfl_sync(kRow, x, 2);
        x = fma(a2, x2, fma(a1, x1, fma(a0, x0, c)));
        cb[3 * q + lane] = x;
    }
}

// T^{-1} of one line, c = G^{-1} u given in cb: s_q = c_q - M_q s_{q-1} (s_{-1} = 0), then
// w_q = s_q - N_q w_{q+1} (w_bz = 0), with one level of recursive doubling: the sequential chains
// visit every other cell,
//   s_q = (c_q - M_q c_{q-1}) + P_q s_{q-2},  P_q = M_q M_{q-1}    (q odd)
//   w_q = (s_q - N_q s_{q+1}) + Q_q w_{q+2},  Q_q = N_q N_{q+1}    (chain cells q = bz-2, bz-4, ...)
// and the cells in between follow from their neighbours on all lanes, each lane finishing the
// cells next to its own (three passes over the line besides the two chains).  On return o_q = w_q
// (forward line) or o_q -= w_q (backward line).  Called by the whole warp.
template <typename T>
__device__ __forceinline__ void line_solve(const T* M, const T* N, const T* P, const T* Q, T* cb, T* o, int bz,
                                           bool fwd_line, int lane) {
    constexpr int BS = 3 * Lay<T>::RS, VS = Lay<T>::VS;
    // y_q - B_q x_{q'} for cells of cb (a missing q' contributes nothing)
    const auto sub = [&](const T* B, int q, int qx, T& y0, T& y1, T& y2) {
        if (qx < 0 || qx >= bz) return;
        T x0, x1, x2;
        ld3(cb + VS * qx, x0, x1, x2);
        sub_mv(B + BS * q, x0, x1, x2, y0, y1, y2);
    };
    // odd q: c_q - M_q c_{q-1}
    for (int q = 1 + 2 * lane; q < bz; q += 64) {
        T y0, y1, y2;
        ld3(cb + VS * q, y0, y1, y2);
        sub(M, q, q - 1, y0, y1, y2);
        st3(cb + VS * q, y0, y1, y2);
    }
    __syncwarp();
    if constexpr (sizeof(T) == 4) {
        if (lane == 0) chain(P, cb, 1, 2, bz / 2);
    } else {
        if (lane < 3) chain(P, cb, 1, 2, bz / 2, lane);
    }
    __syncwarp();
    // chain cells q = bz-2-2i: t_q = s_q - N_q s_{q+1}, the even one of q and q + 1 first finished
    // as s_e = c_e - M_e s_{e-1} (it is this lane's: bz even, e = q; bz odd, e = q + 1)
    for (int i = lane;; i += 32) {
        const int q = bz - 2 - 2 * i;
        if (q < 0) break;
        T s0, s1, s2, n0, n1, n2;
        ld3(cb + VS * q, s0, s1, s2);
        ld3(cb + VS * (q + 1), n0, n1, n2);
        if ((q & 1) == 0) {
            sub(M, q, q - 1, s0, s1, s2);  // s_q
        } else {
            sub_mv(M + BS * (q + 1), s0, s1, s2, n0, n1, n2);  // s_{q+1} = c_{q+1} - M_{q+1} s_q
            st3(cb + VS * (q + 1), n0, n1, n2);
        }
        sub_mv(N + BS * q, n0, n1, n2, s0, s1, s2);
        st3(cb + VS * q, s0, s1, s2);
    }
    __syncwarp();
    if constexpr (sizeof(T) == 4) {
        if (lane == 0) chain(Q, cb, bz - 2, -2, bz / 2);
    } else {
        if (lane < 3) chain(Q, cb, bz - 2, -2, bz / 2, lane);
    }
    __syncwarp();
    // the other cells q = bz-1-2i: w_q = s_q - N_q w_{q+1} (w_bz = 0); this lane then writes the
    // output of q and of the chain cell q - 1 below it
    const auto out = [&](int q, T w0, T w1, T w2) {
        if (!fwd_line) {
            T a0, a1, a2;
            ld3(o + VS * q, a0, a1, a2);
            w0 = a0 - w0;
            w1 = a1 - w1;
            w2 = a2 - w2;
        }
        st3(o + VS * q, w0, w1, w2);
    };
    for (int i = lane;; i += 32) {
        const int q = bz - 1 - 2 * i;
        if (q < 0) break;
        T w0, w1, w2;
        ld3(cb + VS * q, w0, w1, w2);
        sub(N, q, q + 1, w0, w1, w2);
        out(q, w0, w1, w2);
        if (q > 0) {
            ld3(cb + VS * (q - 1), w0, w1, w2);
            out(q - 1, w0, w1, w2);
        }
    }
}

// B_i^{-1} R_i r for one subdomain per CTA (one warp), owned cells written to the apply output.
// Shared memory: SLOTS + 1 mbarriers (16 bytes each) | SLOTS packet slots | SLOTS slots for the
// line's part of r (FP64) | plane vector pv [VS S] | y_j of a backward plane [VS S] | line vector
// cb [VS bz].  pv holds, in turn, y_{j-1} and z / o of plane j during the forward planes, then
// x_{j+1} and z / o of plane j during the backward ones: every line reads the previous plane's
// value of a line before it overwrites it.  y_j goes to device memory (yv, one plane every
// nf_plane_bytes) when its forward plane is done, and comes back by a bulk copy issued at the start
// of its backward plane.
template <typename T, int SLOTS>
__global__ void __launch_bounds__(32) k_nf_apply(const SysTab* __restrict__ tab, const NFDesc* __restrict__ descs) {
    constexpr int BS = 3 * Lay<T>::RS, VS = Lay<T>::VS;
    extern __shared__ __align__(16) unsigned char nf_smem[];
    const NFDesc d = descs[blockIdx.x];  // by value: its fields stay in registers across the stores
    const SysTab& st = tab[d.sys];
    const int in = st.ctl[C_APPLY_IN];
    if (in < 0) return;
    const double* __restrict__ r = st.ws + (long long)in * st.n3p;
    double* __restrict__ z = st.ws + (long long)st.ctl[C_APPLY_OUT] * st.n3p;
    const int lane = threadIdx.x;
    const int bx = d.bx, by = d.by, bz = d.bz, S = bx * bz;
    const unsigned fb = (unsigned)field_bytes<T>(bz);
    const size_t LB = (size_t)d.line_bytes, SB = (size_t)SL_FIELDS * fb, RB = nf_rline_bytes(bz),
                 PB = nf_plane_bytes<T>(S);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(nf_smem);  // 2 words apart
    unsigned long long* ybar = bar + 2 * SLOTS;
    unsigned char* const pk_base = nf_smem + 16 * (SLOTS + 1);
    unsigned char* const r_base = pk_base + SLOTS * SB;
    T* pv = reinterpret_cast<T*>(r_base + SLOTS * RB);
    T* yb = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(pv) + PB);
    T* cb = reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(yb) + PB);
    unsigned char* yv = static_cast<unsigned char*>(d.yv);
    const int K = (2 * by - 1) * (2 * bx - 1);
    const size_t fe = fb / sizeof(T);

    // the grid cell of a line's first cell; the line's cells follow it (z is the fastest index)
    const auto cell0_of = [&](const LineStep& s) {
        return d.c0 + (long long)d.gnz * (s.l + (long long)d.gnx * s.j);
    };
    // packet of a line solve into slot b, plus the line's part of r for a forward line of a forward
    // plane (the copy starts at the 16-byte boundary at or below it: one leading double when the
    // cell is odd); only the fields the line solve reads
    const auto issue = [&](const LineStep& s, int b) {
        unsigned rbytes = 0;
        const unsigned char* rsrc = nullptr;
        if (s.fwd_plane && s.fwd_line) {
            const long long c0 = cell0_of(s);
            const long long a = (24 * c0) & ~15LL, e = (24 * (c0 + bz) + 15) & ~15LL;
            rbytes = (unsigned)(e - a);
            rsrc = reinterpret_cast<const unsigned char*>(r) + a;
        }
        // (packet field, slot field, count) of each copy
        int f[3][3] = {{PK_GI, 0, PK_Q + 1}, {0, 0, 0}, {0, 0, 0}};
        if (!s.fwd_line) {
            f[1][0] = PK_U2, f[1][1] = SL_X, f[1][2] = 1;
        } else if (s.fwd_plane) {
            f[1][0] = PK_L2, f[1][1] = SL_X, f[1][2] = 2;  // L2, L3
        } else {
            f[1][0] = PK_L2, f[1][1] = SL_X, f[1][2] = 1;
            f[2][0] = PK_U3, f[2][1] = SL_Y, f[2][2] = 1;
        }
        if (f[1][2] > 0 && f[1][0] == f[0][0] + f[0][2] && f[1][1] == f[0][1] + f[0][2]) {
            f[0][2] += f[1][2];  // adjacent in the packet and in the slot: one copy
            f[1][2] = 0;
        }
        unsigned tx = rbytes;
        for (int i = 0; i < 3; i++) tx += (unsigned)f[i][2] * fb;
        tma::mbar_expect_tx(&bar[2 * b], tx);
        const unsigned char* src = static_cast<const unsigned char*>(d.pack) + (size_t)(s.j * bx + s.l) * LB;
        for (int i = 0; i < 3; i++)
            if (f[i][2] > 0)
                tma::bulk_load(pk_base + b * SB + (size_t)f[i][1] * fb, src + (size_t)f[i][0] * fb,
                               (unsigned)f[i][2] * fb, &bar[2 * b]);
        if (rbytes) tma::bulk_load(r_base + b * RB, rsrc, rbytes, &bar[2 * b]);
    };

    LineStep nx, s;  // the next line solve to issue, the one in progress
    nx.set(bx, by);
    s.set(bx, by);
    int ni = 0, bi = 0;  // line solves issued, slot of the next issue
    if (lane == 0) {
        for (int b = 0; b <= SLOTS; b++) tma::mbar_init(&bar[2 * b], 1);
        tma::fence_mbar_init();
    }
    __syncwarp();
    for (; ni < SLOTS - 1 && ni < K; ni++) {
        if (lane == 0) issue(nx, bi);
        nx.next(bx, by);
        bi = bi + 1 == SLOTS ? 0 : bi + 1;
    }
    bool ypend = false;
    // a wait that expired: report it, wait (bounded) for the copies still in flight, and leave
    const auto fail = [&](int k) {
        if (lane == 0) {
            atomicExch(st.dev_err, 7);
            for (int k2 = k; k2 < ni; k2++) tma::mbar_wait(&bar[2 * (k2 % SLOTS)], (unsigned)(k2 / SLOTS) & 1u);
            if (ypend) tma::mbar_wait(ybar, (unsigned)(by - 2 - s.j) & 1u);
        }
    };
    int bc = 0;
    unsigned ph = 0;  // slot and barrier phase of the line solve in progress
    for (int k = 0; k < K; k++) {
        // line solve k + SLOTS - 1 goes into the slot that line solve k - 1 has finished with
        if (ni < K) {
            if (lane == 0) issue(nx, bi);
            nx.next(bx, by);
            bi = bi + 1 == SLOTS ? 0 : bi + 1;
            ni++;
        }
        if (s.plane_first && !s.fwd_plane) {  // y_j of this backward plane, needed when it is done
            if (lane == 0) {
                tma::mbar_expect_tx(ybar, (unsigned)PB);
                tma::bulk_load(yb, yv + (size_t)s.j * PB, (unsigned)PB, ybar);
            }
            ypend = true;
        }
        const bool ok = tma::mbar_wait(&bar[2 * bc], ph, st.wait_limit);
        if (!__all_sync(kFull, ok)) {
            fail(k);
            return;
        }
        const T* pk = reinterpret_cast<const T*>(pk_base + bc * SB);
        const auto blk = [&](int f, int q) { return pk + f * fe + (size_t)q * BS; };
        T* pl = pv + (size_t)VS * s.l * bz;  // this line's part of the plane vector
        // c = G^{-1} u, u the line's right-hand side:
        //   forward line of a forward plane:   u = r - L3 y_{j-1} - L2 z_{l-1}
        //   forward line of a backward plane:  u = U3 x_{j+1} - L2 z_{l-1}
        //   backward line:                     u = U2 o_{l+1}
        // (a product that is added goes through sub_mv with the vector negated, which is exact)
        const double* rl = reinterpret_cast<const double*>(r_base + bc * RB) + (cell0_of(s) & 1);
        for (int q = lane; q < bz; q += 32) {
            T u0 = 0, u1 = 0, u2 = 0, x0, x1, x2;
            const T* cur = pl + VS * q;
            if (s.fwd_line) {
                if (s.fwd_plane) {
                    u0 = (T)rl[3 * q];
                    u1 = (T)rl[3 * q + 1];
                    u2 = (T)rl[3 * q + 2];
                    if (s.j > 0) {
                        ld3(cur, x0, x1, x2);
                        sub_mv(blk(SL_Y, q), x0, x1, x2, u0, u1, u2);  // L3
                    }
                } else {
                    ld3(cur, x0, x1, x2);
                    sub_mv(blk(SL_Y, q), -x0, -x1, -x2, u0, u1, u2);  // U3
                }
                if (s.l > 0) {
                    ld3(cur - VS * bz, x0, x1, x2);
                    sub_mv(blk(SL_X, q), x0, x1, x2, u0, u1, u2);  // L2
                }
            } else {
                ld3(cur + VS * bz, x0, x1, x2);
                sub_mv(blk(SL_X, q), -x0, -x1, -x2, u0, u1, u2);  // U2
            }
            T c0 = 0, c1 = 0, c2 = 0;
            sub_mv(blk(PK_GI, q), -u0, -u1, -u2, c0, c1, c2);
            st3(cb + VS * q, c0, c1, c2);
        }
        __syncwarp();
        line_solve(blk(PK_M, 0), blk(PK_N, 0), blk(PK_P, 0), blk(PK_Q, 0), cb, pl, bz, s.fwd_line, lane);
        __syncwarp();
        if (s.plane_done) {  // pv = P_j^{-1} t
            if (s.fwd_plane) {
                if (s.j < by - 1) {  // y_j to device memory, ordered before its later bulk copy back
                    T* yj = reinterpret_cast<T*>(yv + (size_t)s.j * PB);
                    for (int e = lane; e < VS * S; e += 32) yj[e] = pv[e];
                    asm volatile("fence.proxy.async;" ::: "memory");
                } else {
                    write_owned(d, s.j, pv, z, lane);  // x_{by-1} = y_{by-1}
                }
            } else {
                const bool yok = tma::mbar_wait(ybar, (unsigned)(by - 2 - s.j) & 1u, st.wait_limit);
                if (!__all_sync(kFull, yok)) {
                    fail(k + 1);
                    return;
                }
                ypend = false;
                for (int e = lane; e < VS * S; e += 32) pv[e] = yb[e] - pv[e];  // x_j = y_j - pv
                __syncwarp();
                write_owned(d, s.j, pv, z, lane);
            }
            __syncwarp();
        }
        s.next(bx, by);
        if (++bc == SLOTS) {
            bc = 0;
            ph ^= 1u;
        }
    }
}

template <typename T, int SLOTS>
void nf_apply_t(const SysTab* tab, const NFDesc* descs, int ndesc, size_t smem, cudaStream_t st) {
    cudaFuncSetAttribute(k_nf_apply<T, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_nf_apply<T, SLOTS><<<ndesc, 32, smem, st>>>(tab, descs);
}

template <typename T>
void nf_apply_s(const SysTab* tab, const NFDesc* descs, int ndesc, int slots, size_t smem, cudaStream_t st) {
    if (slots >= 4)
        nf_apply_t<T, 4>(tab, descs, ndesc, smem, st);
    else if (slots == 3)
        nf_apply_t<T, 3>(tab, descs, ndesc, smem, st);
    else
        nf_apply_t<T, 2>(tab, descs, ndesc, smem, st);
}

}  // namespace

size_t nf_line_bytes(int bz, int prec) {
    return PK_FIELDS * (prec == 0 ? field_bytes<double>(bz) : field_bytes<float>(bz));
}

size_t nf_plane_bytes(int S, int prec) { return prec == 0 ? nf_plane_bytes<double>(S) : nf_plane_bytes<float>(S); }

size_t nf_apply_smem(int bx, int bz, int prec, int slots) {
    const size_t t = prec == 0 ? 8 : 4, vs = prec == 0 ? 3 : 4;
    const size_t fb = prec == 0 ? field_bytes<double>(bz) : field_bytes<float>(bz);
    return 16 * (size_t)(slots + 1) + slots * (SL_FIELDS * fb + nf_rline_bytes(bz)) +
           2 * nf_plane_bytes(bx * bz, prec) + vs * (size_t)bz * t;
}

size_t nf_work_doubles(int bx, int by, int bz) {
    return 36 * ((size_t)bx * bz + (size_t)bz) + 18 * (size_t)bx * by * bz;
}

void launch_nf_factor(const NFDesc* descs, int ndesc, int nmax, int prec, FactErr* err, cudaStream_t st) {
    if (ndesc <= 0) return;
    const dim3 ggrid((unsigned)((BD_N * nmax + 127) / 128), (unsigned)ndesc);
    const dim3 grid((unsigned)((nmax + 127) / 128), (unsigned)ndesc);
    if (prec == 0) {
        k_nf_gather<double><<<ggrid, 128, 0, st>>>(descs);
        k_nf_factor<double><<<(ndesc + 3) / 4, 128, 0, st>>>(descs, ndesc, err);
        k_nf_pack<double><<<grid, 128, 0, st>>>(descs);
    } else {
        k_nf_gather<float><<<ggrid, 128, 0, st>>>(descs);
        k_nf_factor<float><<<(ndesc + 3) / 4, 128, 0, st>>>(descs, ndesc, err);
        k_nf_pack<float><<<grid, 128, 0, st>>>(descs);
    }
}

void launch_nf_apply(const SysTab* tab, const NFDesc* descs, int ndesc, int prec, int slots, size_t smem,
                     cudaStream_t st) {
    if (ndesc <= 0) return;
    if (prec == 0)
        nf_apply_s<double>(tab, descs, ndesc, slots, smem, st);
    else
        nf_apply_s<float>(tab, descs, ndesc, slots, smem, st);
}

int nf_apply_slots(int ndesc, int bx_max, int bz_max, int prec, int sm_smem, int sms, int dev_smem) {
    // the deepest ring with which every CTA of the launch is resident at once; else the shallowest
    // that fits a CTA at all
    const long long per_sm = (ndesc + std::max(1, sms) - 1) / std::max(1, sms);
    for (int s = 4; s >= 2; s--) {
        const size_t b = nf_apply_smem(bx_max, bz_max, prec, s);
        if (b <= (size_t)dev_smem && per_sm * (long long)(b + 1024) <= (long long)sm_smem) return s;
    }
    return 2;
}

}  // namespace asm2
