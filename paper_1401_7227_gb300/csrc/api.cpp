// C-ABI of libasm2 (include/asm2.h): handle state, device memory, factorisation and the batched
// Krylov driver.  It covers:
//   - the set-up of A and of the boundary-conditioned subdomains (Section 4, Eq. 4.1);
//   - the local factorisations (Section 2, block ILU(0) with column sums; Section 5, exact;
//     Appendix A, nested factorisation);
//   - GMRES(m) and ORTHOMIN(k) right-preconditioned by the additive Schwarz apply (Section 2,
//     Eqs. 4.2-4.5);
//   - the classical coarse corrections (Section 3);
//   - the continuous-batching server.
// All arithmetic of the method runs in the CUDA kernels; the host only moves data, builds the
// symbolic structure and sequences launches.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "asm2.h"
#include "asm2_internal.h"
#include "symbolic.h"

using namespace asm2;

namespace {

struct CudaFail {
    int status;
};

inline void ck(cudaError_t e) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw CudaFail{e == cudaErrorMemoryAllocation ? ASM_ERR_OOM : ASM_ERR_CUDA};
    }
}

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    void alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        ck(cudaMalloc(&p, b));
        bytes = b;
    }
    void zero(cudaStream_t st) { ck(cudaMemsetAsync(p, 0, bytes, st)); }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
    template <class T>
    void upload(const std::vector<T>& v, cudaStream_t st) {
        alloc(v.size() * sizeof(T));
        if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    }
    // as upload, but keeps the allocation when it is large enough (tables rebuilt often: no
    // cudaFree, which would wait for the device, and no cudaMalloc)
    template <class T>
    void upload_reuse(const std::vector<T>& v, cudaStream_t st) {
        const size_t need = std::max<size_t>(16, v.size() * sizeof(T));
        if (!p || bytes < need) alloc(need + need / 2);
        if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    }
};

}  // namespace

struct asm_ctx {
    asm_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int prec = 0;
    int flexible = 0;
    bool lump32 = false;  // lump rows of the ILU factors stored and applied in FP32 (FP32/FP16 fine rows)
    std::string server_skey;  // serving: structure key of the request this system was built for
    // grid / matrix
    int nx = 0, ny = 0, nz = 0, N = 0;
    bool has_grid = false, has_matrix = false, has_partition = false;
    Pattern pat;
    int nnzb = 0;
    DBuf d_ell_val, d_ell_col, d_ell_loc, d_bsr_rp;
    DBuf d_bsr_val;  // A's values as 3x3 blocks in BSR order (assembly reads whole blocks from here)
    // partition / symbolic
    Geom geom;
    std::shared_ptr<SysSym> sym;
    bool sym_valid = false;
    bool factored = false;
    // device preconditioner data
    DBuf d_bcell, d_cptr, d_cloc, d_cval, d_boxsum;
    DBuf d_slot, d_dpiv, d_aptr, d_aloc, d_acs, d_along;
    int n_along = 0;  // slots whose assembly lists are summed by a warp each
    DBuf d_fp;  // factor program arrays (one allocation, see upload_factor_program)
    DBuf d_stream, d_pk_off_f, d_pk_src_f, d_pk_off_c, d_pk_src_c;
    DBuf d_lv, d_rlists, d_y, d_corr_cells, d_corr, d_dev_err, d_gsum, d_r32;
    int n_group_items = 0;  // box_items[0 .. n_group_items): the cell-group sums (kind 2)
    int apply_smem = 0;       // shared memory for all local vectors of the largest subdomain (0: none)
    int apply_smem_need = 0;  // the same before the fit test of choose_ring()
    int apply_lump_smem = 0;  // shared memory for its lump vector and the FP32 mirror
    int apply_slots = 3; // factor-stream ring slots of the apply
    int chunk_cap = kStreamChunkMin;  // largest stream-chunk capacity of the subdomains (ring slot bytes)
    int sm_smem = 0, n_sms = 1, dev_smem = 0;  // shared memory per SM / per CTA (opt-in), SM count
    int chunk_force = 0;  // stream-chunk capacity asked for (bytes; 0: per-subdomain rule)
    int slots_force = 0;  // ring slots asked for with all local vectors in shared memory (0: rule)
    DBuf d_factdesc, d_subdesc_single, d_ritems1;
    int n_ritems1 = 0;
    DBuf d_err;
    std::vector<FactDesc> fact_desc;
    std::vector<SubDesc> sub_desc;   // sys = 0
    std::vector<double> sub_cost;    // estimated apply time of each subdomain (launch order)
    std::vector<BoxItem> box_items;  // sys = 0
    std::vector<long long> slot_base, stream_base, row_base;
    std::vector<long long> y_base;  // doubles: each subdomain's local vectors when not in shared memory
    long long pk_nf = 0, pk_nc = 0, total_slots = 0;
    // Krylov workspace
    int ws_m = -1, ws_flex = -1;
    long long n3p = 0;
    int nchunk = 0;
    DBuf d_ws, d_scal, d_ctl, d_partial;
    SysTab tab{};
    DBuf d_tab1, d_vec1, d_row1, d_box1;
    int n_vec1 = 0, n_row1 = 0;
    // profiling
    bool profiling = false;
    bool no_coop = false;  // per-kernel orthogonalisation path instead of the cooperative one
    int apply_place = 0;  // 0 automatic, else ApplyY + 1 (asm_set_tuning ASM_TUNE_APPLY_SMEM)
    bool no_autotune = false;  // asm_set_tuning ASM_TUNE_AUTOTUNE = 0
    bool no_graphs = false;    // asm_set_tuning ASM_TUNE_GRAPHS = 0
    long long wait_limit = 1LL << 22;  // asm_set_tuning ASM_TUNE_WAIT_LIMIT (polls per chunk wait)
    int tuned_ymode = -1;      // placement the online tuner chose for single-system solves (-1: none)
    ApplyConfig last_solve_apply{-1, 0, 0, 0};  // apply configuration of the last solve this handle was in
    asm_profile_info prof{};
    // exact local solves (local_solver = ASM_LOCAL_EXACT): [A_i | I] inverted in place per subdomain
    DBuf d_daug, d_dprow, d_dfcol, d_dmats, d_dinit, d_doff, d_dmat_of_slot, d_dpart, d_derr, d_ditems1;
    std::vector<long long> daug_base;            // offset of each subdomain's augmented matrix
    std::vector<std::vector<int>> drow_of_q;     // local row of each dense block row (error location)
    int n_dinit = 0, n_ditems1 = 0, dpart_cap = 0, dmax3 = 0;
    // nested factorisation (ASM_LOCAL_NF_COLSUM / ASM_LOCAL_NF): band tables, G, G^{-1}, scratch
    DBuf d_nfint, d_nfval, d_nfdesc1, d_nfpack, d_nfy, d_nfband;
    size_t nf_smem = 0;                            // shared memory of the apply launch
    int nf_slots = 2, nf_bx_max = 0, nf_bz_max = 0;  // its ring depth; the largest line and plane
    std::vector<NFDesc> nf_desc;                   // sys = 0
    std::vector<std::vector<int>> nf_row_of_cell;  // local row of each box cell (error location)
    std::vector<long long> nf_g_off;               // offset of each subdomain's G in d_nfval
    // classical coarse-grid correction (Eqs. 3.5-3.8)
    int coarse_mode = 0;
    int coarse_c[3] = {0, 0, 0};  // {0,0,0}: partition boxes
    bool coarse_valid = false;    // coarse structure built for the current grid, partition, pattern
    int cnb = 0, cnkeys = 0, cpart_cap = 0;
    DBuf d_cbox, d_ccells, d_ckptr, d_ckloc, d_ckeys, d_cblk, d_caug, d_cprow, d_cfcol, d_cpart, d_cerr, d_crc, d_cyc,
        d_cw, d_cbox_items1, d_cgrow1, d_cmat;
    std::vector<BoxItem> cbox_items;   // sys = 0: cells of each coarse box
    std::vector<RowItem> cgrow_items;  // sys = 0: 8 rows of A_C^{-1} each
    // diagnostics
    int err_sub = -1, err_row = -1;
    double setup_ms = 0, factor_ms = 0;
    std::string last_error;
};

namespace {

bool is_nf(const asm_ctx* h) {
    return h->opt.local_solver == ASM_LOCAL_NF_COLSUM || h->opt.local_solver == ASM_LOCAL_NF;
}

int guard(asm_ctx* h, const std::function<int()>& f) {
    try {
        if (h) ck(cudaSetDevice(h->device));
        return f();
    } catch (const CudaFail& e) {
        return e.status;
    } catch (const std::bad_alloc&) {
        return ASM_ERR_OOM;
    } catch (const std::exception&) {  // other host resources: vector growth, thread creation
        return ASM_ERR_OOM;
    }
}

void sync(asm_ctx* h) { ck(cudaStreamSynchronize(h->stream)); }

// copy between caller memory (host or device) and device memory, in stream order
void copy_in(asm_ctx* h, void* dst, const void* src, size_t bytes, int on_device) {
    ck(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
}
void copy_out(asm_ctx* h, void* dst, const void* src, size_t bytes, int on_device) {
    ck(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
}

void fill_ell(asm_ctx* h, const double* vals, int on_device) {
    const size_t vb = (size_t)h->nnzb * 9 * sizeof(double);
    if (h->d_bsr_val.bytes < vb) h->d_bsr_val.alloc(vb);
    copy_in(h, h->d_bsr_val.p, vals, vb, on_device);
    launch_ell_fill(h->d_bsr_val.as<double>(), h->d_bsr_rp.as<int>(), h->N, h->pat.ell_w, h->d_ell_val.as<double>(),
                    h->pat.rows_pad, h->stream);
    ck(cudaGetLastError());
    if (!on_device) sync(h);
}

// BSR block index of an ELL location w * rows_pad + r (slot w of row r holds block rp[r] + w); the
// sign encoding of subtracted blocks (~) is kept
int bsr_of_loc(const Pattern& P, int loc) {
    const bool neg = loc < 0;
    const int L = neg ? ~loc : loc;
    const int w = L / P.rows_pad, r = L - w * P.rows_pad;
    const int e = P.rp[r] + w;
    return neg ? ~e : e;
}
std::vector<int> bsr_of_locs(const Pattern& P, const std::vector<int>& locs) {
    std::vector<int> out(locs.size());
    for (size_t i = 0; i < locs.size(); i++) out[i] = bsr_of_loc(P, locs[i]);
    return out;
}

// Exact-local-solve work items of an ordered subdomain list: (item index, first of 8 owned rows)
std::vector<int2> dense_items(const std::vector<SubDesc>& sd) {
    std::vector<int2> it;
    for (int i = 0; i < (int)sd.size(); i++)
        for (int q = 0; q < 3 * sd[i].n_own; q += 8) it.push_back(make_int2(i, q));
    return it;
}

// Work items of the restriction: (subdomain, first local row) per 256 rows (fine rows, then lumps)
std::vector<int2> restrict_items(const std::vector<SubDesc>& sd) {
    std::vector<int2> it;
    for (int i = 0; i < (int)sd.size(); i++)
        for (int q = 0; q < sd[i].nf + sd[i].nc; q += 256) it.push_back(make_int2(i, q));
    return it;
}

// Subdomain work items of several systems, most expensive first (the order of the CTAs of the
// apply launch; every CTA writes only its own subdomain's owned rows, so the order does not
// change any result)
std::vector<SubDesc> longest_first(const std::vector<asm_ctx*>& hs) {
    std::vector<std::pair<double, SubDesc>> v;
    for (int k = 0; k < (int)hs.size(); k++)
        for (size_t i = 0; i < hs[k]->sub_desc.size(); i++) {
            SubDesc d = hs[k]->sub_desc[i];
            d.sys = k;
            v.emplace_back(i < hs[k]->sub_cost.size() ? hs[k]->sub_cost[i] : 0.0, d);
        }
    std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<SubDesc> out;
    out.reserve(v.size());
    for (auto& e : v) out.push_back(e.second);
    return out;
}

// Upload the symbolic structure and build the per-subdomain descriptors.
// Exact local solves: per subdomain an augmented [A_i | I] (3n x 6n) in fine-index-then-lump-index
// order, the scatter offsets of the assembled slots into it, and the Gauss-Jordan descriptors.
void upload_dense(asm_ctx* h, cudaStream_t st) {
    const SysSym& S = *h->sym;
    const int K = (int)S.subs.size();
    h->daug_base.assign(K + 1, 0);
    h->drow_of_q.assign(K, {});
    std::vector<long long> pbase(K + 1, 0), fbase(K + 1, 0);
    int nmax3 = 0;
    for (int s = 0; s < K; s++) {
        const SubSym& o = S.subs[s];
        if (o.n > 4096) throw CudaFail{ASM_ERR_INVALID_ARG};
        const long long n3 = 3LL * o.n;
        h->daug_base[s + 1] = h->daug_base[s] + n3 * 2 * n3;
        pbase[s + 1] = pbase[s] + 2 * n3;
        fbase[s + 1] = fbase[s] + n3;
        nmax3 = std::max(nmax3, (int)n3);
    }
    h->dmax3 = nmax3;
    h->d_daug.alloc((size_t)h->daug_base[K] * sizeof(double));
    h->d_dprow.alloc((size_t)pbase[K] * sizeof(double));
    h->d_dfcol.alloc((size_t)fbase[K] * sizeof(double));
    std::vector<GJMat> mats(K);
    std::vector<int2> init;
    std::vector<long long> off;
    std::vector<int> mat_of_slot;
    off.reserve(h->total_slots);
    mat_of_slot.reserve(h->total_slots);
    for (int s = 0; s < K; s++) {
        const SubSym& o = S.subs[s];
        const int n3 = 3 * o.n;
        mats[s] = GJMat{h->d_daug.as<double>() + h->daug_base[s], n3, h->d_dprow.as<double>() + pbase[s],
                        h->d_dfcol.as<double>() + fbase[s]};
        for (int r = 0; r < n3; r++) init.push_back(make_int2(s, r));
        std::vector<int> q(o.n);
        h->drow_of_q[s].assign(o.n, 0);
        for (int p = 0; p < o.n; p++) {
            q[p] = p < o.nf ? o.fidx_of_row[p] : o.nf + o.cidx_of_row[p];
            h->drow_of_q[s][q[p]] = p;
        }
        // offset of the slot's (0,0) element within its own augmented matrix (row stride 2 n3); the
        // scatter adds rows 0..2 and columns 0..2, all inside the left half
        for (int p = 0; p < o.n; p++)
            for (int t = o.prp[p]; t < o.prp[p + 1]; t++) {
                const long long o0 = 3LL * q[p] * 2 * n3 + 3LL * q[o.pci[t]];
                if (q[p] < 0 || q[p] >= o.n || q[o.pci[t]] < 0 || q[o.pci[t]] >= o.n ||
                    o0 + 2LL * 2 * n3 + 2 >= (long long)n3 * 2 * n3)
                    throw CudaFail{ASM_ERR_INVALID_ARG};
                off.push_back(o0);
                mat_of_slot.push_back(s);
            }
        h->sub_desc[s].dinv = h->d_daug.as<double>() + h->daug_base[s];
    }
    if ((long long)off.size() != h->total_slots) throw CudaFail{ASM_ERR_INVALID_ARG};
    h->d_dmats.upload(mats, st);
    h->d_dinit.upload(init, st);
    h->n_dinit = (int)init.size();
    h->d_doff.upload(off, st);
    h->d_dmat_of_slot.upload(mat_of_slot, st);
    int sms = 0;
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->dpart_cap = 4 * std::max(1, sms);
    h->d_dpart.alloc((size_t)2 * h->dpart_cap * sizeof(double));
    h->d_derr.alloc((size_t)std::max(1, K) * sizeof(int));
    sync(h);
}

// Nested factorisation: every local problem must be a box of fine cells (no lumps), whose A_i is
// then hepta-banded in the box order p = z + bz (x + bx y) (Appendix A, Eq. A.1).  Per subdomain:
// the slot of each band block of each cell, the cells, the owned cells, and G / G^{-1} / scratch.
void upload_nf(asm_ctx* h, cudaStream_t st) {
    const SysSym& S = *h->sym;
    const Geom& g = S.g;
    const int K = (int)S.subs.size();
    struct Part {
        int bx, by, bz, n, c0;
        int lo[3], olo[3], ohi[3];
        size_t bands;                         // int offset
        long long g, gi, work, pack, yv, band;  // double / byte offsets
    };
    std::vector<Part> parts(K);
    std::vector<int> ints;
    long long nval = 0, npack = 0, ny = 0, nband = 0;
    h->nf_smem = 0;
    h->nf_bx_max = h->nf_bz_max = 0;
    h->nf_row_of_cell.assign(K, {});
    h->nf_g_off.assign(K, 0);
    for (int s = 0; s < K; s++) {
        const SubSym& o = S.subs[s];
        if (o.n != o.nf) {
            h->last_error = "nested factorisation needs local problems without lumps (near_width 0, far mode none)";
            throw CudaFail{ASM_ERR_INVALID_ARG};
        }
        int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {-1, -1, -1};
        std::vector<int> xyz(3 * (size_t)o.n);
        for (int p = 0; p < o.n; p++) {
            const int c = o.cells_of_row[o.cells_of_row_ptr[p]];
            const int v[3] = {(c / g.nz) % g.nx, c / (g.nz * g.nx), c % g.nz};  // x, y, z
            for (int d = 0; d < 3; d++) {
                xyz[3 * p + d] = v[d];
                lo[d] = std::min(lo[d], v[d]);
                hi[d] = std::max(hi[d], v[d]);
            }
        }
        Part& P = parts[s];
        P.bx = hi[0] - lo[0] + 1;
        P.by = hi[1] - lo[1] + 1;
        P.bz = hi[2] - lo[2] + 1;
        P.n = o.n;
        if ((long long)P.bx * P.by * P.bz != o.n) {
            h->last_error = "nested factorisation: a fine set is not a box";
            throw CudaFail{ASM_ERR_INVALID_ARG};
        }
        std::vector<int> nat(o.n), cell(o.n), bands(7 * (size_t)o.n, -1);
        h->nf_row_of_cell[s].assign(o.n, 0);
        for (int p = 0; p < o.n; p++) {
            nat[p] = (xyz[3 * p + 2] - lo[2]) + P.bz * ((xyz[3 * p] - lo[0]) + P.bx * (xyz[3 * p + 1] - lo[1]));
            cell[nat[p]] = o.cells_of_row[o.cells_of_row_ptr[p]];
            h->nf_row_of_cell[s][nat[p]] = p;
        }
        for (int p = 0; p < o.n; p++) {
            const int a = nat[p];
            for (int t = o.prp[p]; t < o.prp[p + 1]; t++) {
                const int q = o.pci[t];
                // the band follows from the box coordinates: neighbours in z are L1/U1, in x L2/U2,
                // in y L3/U3 (an index offset alone is ambiguous when bz or bx is 1)
                const int dx = xyz[3 * q] - xyz[3 * p], dy = xyz[3 * q + 1] - xyz[3 * p + 1],
                          dz = xyz[3 * q + 2] - xyz[3 * p + 2];
                int k = -1;
                if (dx == 0 && dy == 0 && dz >= -1 && dz <= 1)
                    k = dz == 0 ? 0 : dz < 0 ? 1 : 2;
                else if (dz == 0 && dy == 0 && (dx == -1 || dx == 1))
                    k = dx < 0 ? 3 : 4;
                else if (dz == 0 && dx == 0 && (dy == -1 || dy == 1))
                    k = dy < 0 ? 5 : 6;
                if (k < 0 || bands[7 * (size_t)a + k] >= 0) {
                    h->last_error = "nested factorisation: a local matrix is not hepta-banded on its box";
                    throw CudaFail{ASM_ERR_PATTERN};
                }
                bands[7 * (size_t)a + k] = t;
            }
            if (bands[7 * (size_t)a] < 0) throw CudaFail{ASM_ERR_PATTERN};
        }
        // the owned cells form a box: its local bounds, checked against the owned-cell list
        for (int d = 0; d < 3; d++) {
            P.lo[d] = lo[d];
            P.olo[d] = INT32_MAX;
            P.ohi[d] = -1;
        }
        for (const int c : o.own_cell) {
            const int v[3] = {(c / g.nz) % g.nx - lo[0], c / (g.nz * g.nx) - lo[1], c % g.nz - lo[2]};
            for (int d = 0; d < 3; d++) {
                P.olo[d] = std::min(P.olo[d], v[d]);
                P.ohi[d] = std::max(P.ohi[d], v[d] + 1);
            }
        }
        if ((long long)(P.ohi[0] - P.olo[0]) * (P.ohi[1] - P.olo[1]) * (P.ohi[2] - P.olo[2]) != (long long)o.own_cell.size())
            throw CudaFail{ASM_ERR_INVALID_ARG};
        P.c0 = cell[0];
        P.bands = ints.size();
        ints.insert(ints.end(), bands.begin(), bands.end());
        P.g = nval;
        P.gi = P.g + 9LL * o.n;
        P.work = P.gi + 9LL * o.n;
        nval = P.work + (long long)nf_work_doubles(P.bx, P.by, P.bz);
        h->nf_g_off[s] = P.g;
        const size_t lb = nf_line_bytes(P.bz, h->prec);
        P.pack = npack;
        npack += (long long)(lb * (size_t)P.bx * P.by + 255) / 256 * 256;
        P.band = nband;
        nband += (63LL * o.n * (h->prec == 0 ? 8 : 4) + 255) / 256 * 256;
        P.yv = ny;
        ny += ((long long)nf_plane_bytes(P.bx * P.bz, h->prec) * P.by + 255) / 256 * 256;
        h->nf_bx_max = std::max(h->nf_bx_max, P.bx);
        h->nf_bz_max = std::max(h->nf_bz_max, P.bz);
    }
    int dev_smem = 0, sm_smem = 0, sms = 0;
    ck(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    ck(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->nf_slots = nf_apply_slots(K, h->nf_bx_max, h->nf_bz_max, h->prec, sm_smem, sms, dev_smem);
    h->nf_smem = nf_apply_smem(h->nf_bx_max, h->nf_bz_max, h->prec, h->nf_slots);
    if (h->nf_smem > (size_t)dev_smem) {
        h->last_error = "nested factorisation: a line of the fine boxes is too long for the apply's shared memory";
        throw CudaFail{ASM_ERR_INVALID_ARG};
    }
    h->d_nfint.upload(ints, st);
    h->d_nfval.alloc((size_t)std::max<long long>(1, nval) * sizeof(double));
    h->d_nfpack.alloc((size_t)std::max<long long>(256, npack));
    h->d_nfpack.zero(st);
    h->d_nfy.alloc((size_t)std::max<long long>(256, ny));
    h->d_nfband.alloc((size_t)std::max<long long>(256, nband));
    h->nf_desc.assign(K, NFDesc{});
    const int* ib = h->d_nfint.as<int>();
    double* vb = h->d_nfval.as<double>();
    for (int s = 0; s < K; s++) {
        const Part& P = parts[s];
        NFDesc& d = h->nf_desc[s];
        d.sys = 0;
        d.sub = s;
        d.bx = P.bx;
        d.by = P.by;
        d.bz = P.bz;
        d.n = P.n;
        d.colsum = h->opt.local_solver == ASM_LOCAL_NF_COLSUM ? 1 : 0;
        d.c0 = P.c0;
        d.gnz = g.nz;
        d.gnx = g.nx;
        for (int k = 0; k < 3; k++) {
            d.own_lo[k] = P.olo[k];
            d.own_hi[k] = P.ohi[k];
        }
        d.line_bytes = (int)nf_line_bytes(P.bz, h->prec);
        d.slot = h->d_slot.as<double>() + 9 * h->slot_base[s];
        d.bands = ib + P.bands;
        d.g = vb + P.g;
        d.gi = vb + P.gi;
        d.work = vb + P.work;
        d.pack = h->d_nfpack.as<unsigned char>() + P.pack;
        d.yv = h->d_nfy.as<unsigned char>() + P.yv;
        d.fband = h->d_nfband.as<unsigned char>() + P.band;
    }
    h->d_nfdesc1.upload(h->nf_desc, st);
    sync(h);
}

// Ring slots of the apply with the lump vector or no local vector in shared memory: the number
// asked for (asm_set_tuning ASM_TUNE_APPLY_SLOTS), else 2.
int other_slots(const asm_ctx* h) { return h->slots_force > 0 ? h->slots_force : 2; }

// Ring slots of the apply with all local vectors in shared memory: the number asked for
// (asm_set_tuning ASM_TUNE_APPLY_SLOTS), else as many as keep two CTAs per SM (shared memory per
// SM minus 1 KB per CTA), else 4 with one CTA per SM.  That placement is off (apply_smem = 0)
// when the local vectors and the ring do not fit one CTA's shared memory.
void choose_ring(asm_ctx* h) {
    h->apply_smem = h->apply_smem_need;
    h->apply_slots = 4;
    if (h->slots_force > 0) {
        h->apply_slots = h->slots_force;
    } else {
        for (int sl = 4; sl >= 2; sl--)
            if (2 * ((size_t)h->apply_smem + apply_ring_bytes(sl, h->chunk_cap) + 1024) <= (size_t)h->sm_smem) {
                h->apply_slots = sl;
                break;
            }
    }
    if ((size_t)h->apply_smem + apply_ring_bytes(h->apply_slots, h->chunk_cap) > (size_t)h->dev_smem - 1024) {
        h->apply_smem = 0;
        h->apply_slots = h->slots_force > 0 ? h->slots_force : 3;
    }
}

void upload_symbolic(asm_ctx* h) {
    SysSym& S = *h->sym;
    cudaStream_t st = h->stream;
    const int K = (int)S.subs.size();
    h->slot_base.assign(K + 1, 0);
    h->stream_base.assign(K + 1, 0);
    h->row_base.assign(K + 1, 0);
    std::vector<long long> aloc_base(K + 1, 0), fp_base(K + 1, 0), rl_base(K + 1, 0), lv_base(K + 1, 0);
    long long npf = 0, npc = 0;
    for (int s = 0; s < K; s++) {
        const SubSym& o = S.subs[s];
        h->slot_base[s + 1] = h->slot_base[s] + o.nslot;
        h->stream_base[s + 1] = h->stream_base[s] + (long long)((o.stream.size() + 255) / 256 * 256);
        h->row_base[s + 1] = h->row_base[s] + o.n;
        aloc_base[s + 1] = aloc_base[s] + (long long)o.aloc.size();
        // factor program ints: lv_pos0, diag_of_pos, row_of_pos, tgt_lv, tgt, pp, ls_lv, pair, ls
        long long fpi = (long long)o.lv_pos0.size() + o.diag_of_pos.size() + o.row_of_pos.size() + o.tgt_lv.size() +
                        o.tgt.size() + o.pp.size() + o.ls_lv.size();
        fpi = (fpi + 1) / 2 * 2;
        fpi += (long long)o.pair.size() + (long long)o.ls.size();
        fp_base[s + 1] = fp_base[s] + fpi;
        long long rli = (long long)o.fcell.size() + o.rptr.size() + o.rsrc.size() + o.rbox.size() + o.rcorr.size() +
                        o.clong.size() + o.own_pos.size() + o.own_cell.size() + 2LL * o.chunk_off.size();
        rl_base[s + 1] = rl_base[s] + (rli + 1) / 2 * 2;  // even: each block starts 8-byte aligned
        lv_base[s + 1] = lv_base[s] + o.nlev;
        npf += (long long)o.pk_off_f.size();
        npc += (long long)o.pk_off_c.size();
    }
    h->total_slots = h->slot_base[K];
    if (h->total_slots >= (1LL << 31) / 9 || aloc_base[K] >= (1LL << 31)) throw CudaFail{ASM_ERR_INVALID_ARG};
    h->d_slot.alloc((size_t)h->total_slots * 9 * sizeof(double));
    h->d_dpiv.alloc((size_t)h->row_base[K] * 9 * sizeof(double));
    // local vectors of the apply in device memory: the same layout as in shared memory
    // (FP64 lumps, fine rows at the factor precision, an FP32 lump mirror), 16-byte aligned
    h->y_base.assign(K + 1, 0);
    for (int s = 0; s < K; s++) {
        const SubSym& o = S.subs[s];
        const long long bytes = std::max<long long>((long long)apply_smem_bytes(o.nf, o.n - o.nf, S.prec, S.lump32), 24LL * o.n);
        h->y_base[s + 1] = h->y_base[s] + (bytes + 15) / 16 * 2;
    }
    h->d_y.alloc((size_t)h->y_base[K] * sizeof(double));
    // assembly lists (global offsets)
    {
        std::vector<int> aptr;
        aptr.reserve(h->total_slots + 1);
        std::vector<int> acs, along;
        acs.reserve(h->total_slots);
        for (int s = 0; s < K; s++) {
            const SubSym& o = S.subs[s];
            for (int t = 0; t < o.nslot; t++) {
                aptr.push_back((int)(aloc_base[s] + o.aptr[t]));
                acs.push_back(o.acs[t]);
                if (o.aptr[t + 1] - o.aptr[t] >= kLongAssembly) along.push_back((int)(h->slot_base[s] + t));
            }
        }
        aptr.push_back((int)aloc_base[K]);
        h->d_aptr.upload(aptr, st);
        h->d_acs.upload(acs, st);
        h->d_along.upload(along, st);
        h->n_along = (int)along.size();
        h->d_aloc.alloc((size_t)aloc_base[K] * 4);
        for (int s = 0; s < K; s++)
            if (!S.subs[s].aloc.empty()) {
                const std::vector<int> a = bsr_of_locs(h->pat, S.subs[s].aloc);
                ck(cudaMemcpyAsync(h->d_aloc.as<int>() + aloc_base[s], a.data(), a.size() * 4, cudaMemcpyHostToDevice,
                                   st));
            }
        sync(h);
    }
    // factor program
    h->d_fp.alloc((size_t)fp_base[K] * 4);
    h->fact_desc.assign(K, FactDesc{});
    {
        std::vector<int> buf;
        for (int s = 0; s < K; s++) {
            const SubSym& o = S.subs[s];
            buf.clear();
            int* base = h->d_fp.as<int>() + fp_base[s];
            FactDesc& fd = h->fact_desc[s];
            fd.sys = 0;
            fd.nlev = o.nlev;
            fd.n = o.n;
            fd.slot = h->d_slot.as<double>() + h->slot_base[s] * 9;
            fd.dpiv = h->d_dpiv.as<double>() + h->row_base[s] * 9;
            auto put = [&](const std::vector<int>& v) {
                const int* p = base + buf.size();
                buf.insert(buf.end(), v.begin(), v.end());
                return p;
            };
            fd.lv_pos0 = put(o.lv_pos0);
            fd.diag_of_pos = put(o.diag_of_pos);
            fd.row_of_pos = put(o.row_of_pos);
            fd.tgt_lv = put(o.tgt_lv);
            fd.tgt = put(o.tgt);
            fd.pp = put(o.pp);
            fd.ls_lv = put(o.ls_lv);
            if (buf.size() % 2) buf.push_back(0);
            fd.pair = reinterpret_cast<const int2*>(put(o.pair));
            fd.ls = reinterpret_cast<const int2*>(put(o.ls));
            // a copy from pageable host memory returns once the source is staged: buf may be
            // reused at once, and no stream sync per subdomain is needed
            ck(cudaMemcpyAsync(base, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice, st));
        }
        h->d_factdesc.upload(h->fact_desc, st);
    }
    // streams + pack lists + level tables + restriction lists
    h->d_stream.alloc((size_t)h->stream_base[K]);
    h->d_rlists.alloc((size_t)std::max<long long>(2, rl_base[K]) * 4);
    std::vector<BoxItem> corr_items;
    std::vector<int> corr_cells;
    int corr_base = 0;
    std::vector<long long> offf, offc;
    std::vector<int> srcf, srcc;
    offf.reserve(npf);
    srcf.reserve(npf);
    offc.reserve(npc);
    srcc.reserve(npc);
    h->sub_desc.assign(K, SubDesc{});
    h->sub_cost.assign(K, 0.0);
    h->apply_smem = 0;
    h->apply_smem_need = 0;
    h->apply_lump_smem = 0;
    h->chunk_cap = kStreamChunkMin;
    h->tuned_ymode = -1;
    for (int s = 0; s < K; s++) {
        const SubSym& o = S.subs[s];
        if (!o.stream.empty())
            ck(cudaMemcpyAsync(h->d_stream.as<unsigned char>() + h->stream_base[s], o.stream.data(), o.stream.size(),
                               cudaMemcpyHostToDevice, st));
        for (size_t i = 0; i < o.pk_off_f.size(); i++) {
            offf.push_back(h->stream_base[s] + o.pk_off_f[i]);
            srcf.push_back((int)(h->slot_base[s] + o.pk_src_f[i]));
        }
        for (size_t i = 0; i < o.pk_off_c.size(); i++) {
            offc.push_back(h->stream_base[s] + o.pk_off_c[i]);
            srcc.push_back((int)(h->slot_base[s] + o.pk_src_c[i]));
        }
        std::vector<int> rl;
        rl.reserve(rl_base[s + 1] - rl_base[s]);
        int* base = h->d_rlists.as<int>() + rl_base[s];
        SubDesc& sd = h->sub_desc[s];
        auto put = [&](const std::vector<int>& v) {
            const int* p = base + rl.size();
            rl.insert(rl.end(), v.begin(), v.end());
            return p;
        };
        sd.sys = 0;
        sd.nf = o.nf;
        sd.nc = o.n - o.nf;
        sd.n_chunks = (int)o.chunk_off.size();
        sd.n_fwd = o.n_fwd_chunks;
        // a chunk costs about one barrier-bounded step; lump-only chunks (FP64 rows) about 2.3
        for (size_t i = 0; i < o.chunk_off.size(); i++) {
            int hdr_nf = 0;
            std::memcpy(&hdr_nf, o.stream.data() + o.chunk_off[i] + 4, sizeof(int));
            h->sub_cost[s] += hdr_nf == 0 ? 2.3 : 1.0;
        }
        sd.n_own = (int)o.own_pos.size();
        sd.n_long = (int)o.clong.size();
        sd.corr0 = corr_base;
        sd.chunk_cap = o.chunk_cap;
        h->chunk_cap = std::max(h->chunk_cap, o.chunk_cap);
        sd.stream = h->d_stream.as<unsigned char>() + h->stream_base[s];
        sd.y = h->d_y.as<double>() + h->y_base[s];
        {
            const YLayout L = y_layout(o.nf, o.n - o.nf, S.prec, S.lump32);
            sd.y_fine = (int)L.fine;
            sd.y_mirror = (int)L.mirror;
            sd.y_bytes = (int)L.total;
        }
        {
            // the chunk table goes first: base is 8-byte aligned, so the int2 entries are too
            std::vector<int> ch;
            for (size_t i = 0; i < o.chunk_off.size(); i++) {
                ch.push_back((int)o.chunk_off[i]);
                ch.push_back(o.chunk_bytes[i]);
            }
            sd.chunks = reinterpret_cast<const int2*>(put(ch));
        }
        sd.fcell = put(o.fcell);
        sd.rptr = put(o.rptr);
        sd.rsrc = put(o.rsrc);
        sd.rbox = put(o.rbox);
        sd.rcorr = put(o.rcorr);
        sd.clong = put(o.clong);
        sd.own_pos = put(o.own_pos);
        sd.own_cell = put(o.own_cell);
        h->apply_smem_need = std::max<int>(h->apply_smem_need, (int)apply_smem_bytes(o.nf, o.n - o.nf, S.prec, S.lump32));
        h->apply_lump_smem = std::max<int>(h->apply_lump_smem, (int)apply_lump_bytes(o.n - o.nf, S.prec, S.lump32));
        for (size_t k = 0; k + 1 < o.corr_ptr.size(); k++)
            corr_items.push_back(BoxItem{0, corr_base + (int)k, (int)corr_cells.size() + o.corr_ptr[k],
                                         (int)corr_cells.size() + o.corr_ptr[k + 1], 1, 0, nullptr});
        corr_cells.insert(corr_cells.end(), o.corr_cells.begin(), o.corr_cells.end());
        corr_base += (int)o.corr_ptr.size() - 1;
        if (!rl.empty()) ck(cudaMemcpyAsync(base, rl.data(), rl.size() * 4, cudaMemcpyHostToDevice, st));
    }
    if (h->opt.local_solver == ASM_LOCAL_EXACT) upload_dense(h, st);
    if (is_nf(h)) upload_nf(h, st);
    h->pk_nf = (long long)offf.size();
    h->pk_nc = (long long)offc.size();
    h->d_pk_off_f.upload(offf, st);
    h->d_pk_src_f.upload(srcf, st);
    h->d_pk_off_c.upload(offc, st);
    h->d_pk_src_c.upload(srcc, st);
    // cell-group sums (when any sum list may use them), far boxes, their near-region corrections,
    // and the coarse matrix
    h->box_items.clear();
    h->n_group_items = 0;
    bool sum_lists = S.g.far_mode != 0;
    for (const SubSym& o : S.subs) sum_lists = sum_lists || !o.rsrc.empty();
    if (sum_lists) {
        const int ng = n_groups(S.g);
        h->d_gsum.alloc((size_t)ng * 3 * sizeof(double));
        // FP32 local vectors: k_groups also rounds every cell's entries once, for the fine rows
        if (h->lump32) h->d_r32.alloc((size_t)h->N * 4 * sizeof(float));
        for (int g0 = 0; g0 < ng; g0 += 256) h->box_items.push_back(BoxItem{0, 0, g0, std::min(ng, g0 + 256), 2, 0, nullptr});
        h->n_group_items = (int)h->box_items.size();
    } else {
        h->d_gsum.alloc(16);
    }
    if (S.g.far_mode != 0) {
        h->d_bcell.upload(S.bsum, st);
        h->d_cptr.upload(S.cptr, st);
        h->d_cloc.upload(bsr_of_locs(h->pat, S.cloc), st);
        h->d_cval.alloc((size_t)std::max(1, S.nC) * 9 * sizeof(double));
        h->d_boxsum.alloc((size_t)std::max(1, S.nboxes) * 3 * sizeof(double));
        for (int b = 0; b < S.nboxes; b++)
            h->box_items.push_back(BoxItem{0, b, S.bsum_ptr[b], S.bsum_ptr[b + 1], 0, 0, h->d_bcell.as<int>()});
    } else {
        h->d_cval.alloc(16);
        h->d_boxsum.alloc(16);
    }
    h->d_corr_cells.upload(corr_cells, st);
    h->d_corr.alloc((size_t)std::max(1, corr_base) * 3 * sizeof(double));
    for (BoxItem& it : corr_items) {
        it.cells = h->d_corr_cells.as<int>();
        h->box_items.push_back(it);
    }
    ck(cudaDeviceGetAttribute(&h->dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    ck(cudaDeviceGetAttribute(&h->sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
    ck(cudaDeviceGetAttribute(&h->n_sms, cudaDevAttrMultiProcessorCount, h->device));
    choose_ring(h);
    // most expensive subdomains first: the CTAs of the last wave are then the short ones
    {
        const std::vector<SubDesc> ordered = longest_first({h});
        h->d_subdesc_single.upload(ordered, st);
        const std::vector<int2> di = dense_items(ordered);
        h->d_ditems1.upload(di, st);
        h->n_ditems1 = (int)di.size();
        const std::vector<int2> ri = restrict_items(ordered);
        h->d_ritems1.upload(ri, st);
        h->n_ritems1 = (int)ri.size();
    }
    h->d_err.alloc(sizeof(FactErr));
    sync(h);
}

// Krylov workspace and the single-system tables
void ensure_workspace(asm_ctx* h) {
    const int m = std::max(1, h->opt.restart);
    const bool om = h->opt.krylov == ASM_KRYLOV_ORTHOMIN;
    const int flex = om ? 2 : h->flexible;  // ORTHOMIN keeps its own slot layout
    if (h->ws_m == m && h->ws_flex == flex && h->d_ws.p) return;
    const long long n3 = 3LL * h->N;
    h->n3p = (n3 + VEC_CHUNK - 1) / VEC_CHUNK * VEC_CHUNK;
    h->nchunk = (int)(h->n3p / VEC_CHUNK);
    // GMRES: V_0..V_m (+ Z_0..Z_{m-1} when flexible); ORTHOMIN: P_0..P_k, Q_0..Q_k
    const int nslots = om ? VV0 + 2 * (m + 1) : VV0 + m + 1 + (flex ? m : 0);
    h->d_ws.alloc((size_t)nslots * h->n3p * sizeof(double));
    h->d_ws.zero(h->stream);
    const ScalLayout SL = ScalLayout::make(m);
    h->d_scal.alloc((size_t)SL.n * sizeof(double));
    h->d_scal.zero(h->stream);
    h->d_ctl.alloc(C_NCTL * sizeof(int));
    h->d_ctl.zero(h->stream);
    // chunk partials; the cooperative Gram-Schmidt's per-CTA partials (classical: kCgsMax values per
    // CTA, at most two CTAs per SM)
    h->d_partial.alloc(std::max<size_t>((size_t)4 * std::max(h->nchunk, 4096), (size_t)kCgsMax * 2 * 1024) *
                       sizeof(double));
    h->ws_m = m;
    h->ws_flex = flex;
    SysTab& t = h->tab;
    t.ws = h->d_ws.as<double>();
    t.n3p = h->n3p;
    t.n3 = (int)n3;
    t.n_cells = h->N;
    t.m = m;
    t.flexible = om ? 0 : flex;
    t.krylov = om ? 1 : 0;
    t.ortho = om ? 0 : h->opt.ortho;
    t.nchunk = h->nchunk;
    t.scal = h->d_scal.as<double>();
    t.ctl = h->d_ctl.as<int>();
    t.partial = h->d_partial.as<double>();
    t.ell_val = h->d_ell_val.as<double>();
    t.ell_col = h->d_ell_col.as<int>();
    t.ell_w = h->pat.ell_w;
    t.rows_pad = h->pat.rows_pad;
    t.boxsum = h->d_boxsum.as<double>();
    t.corr = h->d_corr.p ? h->d_corr.as<double>() : h->d_boxsum.as<double>();
    t.gsum = h->d_gsum.p ? h->d_gsum.as<double>() : h->d_boxsum.as<double>();
    t.r32 = h->n_group_items > 0 && h->lump32 && h->d_r32.p ? h->d_r32.as<float4>() : nullptr;
    t.gnx = h->geom.nx;
    t.gny = h->geom.ny;
    t.gnz = h->geom.nz;
    if (!h->d_dev_err.p) {
        h->d_dev_err.alloc(16);
        h->d_dev_err.zero(h->stream);
    }
    t.dev_err = h->d_dev_err.as<int>();
    t.wait_limit = h->wait_limit;
    const bool coarse = h->coarse_mode != 0 && h->coarse_valid;
    t.cmode = coarse ? h->coarse_mode : 0;
    t.cnb = coarse ? h->cnb : 0;
    t.cbox = coarse ? h->d_cbox.as<int>() : nullptr;
    t.caug = coarse ? h->d_caug.as<double>() : nullptr;
    t.crc = coarse ? h->d_crc.as<double>() : nullptr;
    t.cyc = coarse ? h->d_cyc.as<double>() : nullptr;
    t.cw = coarse && h->coarse_mode == 2 ? h->d_cw.as<double>() : nullptr;
    std::vector<SysTab> tabs{t};
    h->d_tab1.upload(tabs, h->stream);
    std::vector<VecItem> vi;
    for (int c = 0; c < h->nchunk; c++) vi.push_back(VecItem{0, c});
    h->d_vec1.upload(vi, h->stream);
    h->n_vec1 = (int)vi.size();
    std::vector<RowItem> ri;
    for (int r = 0; r < h->N; r += 256) ri.push_back(RowItem{0, r});
    h->d_row1.upload(ri, h->stream);
    h->n_row1 = (int)ri.size();
    h->d_box1.upload(h->box_items, h->stream);
    if (coarse) {
        h->d_cbox_items1.upload(h->cbox_items, h->stream);
        h->d_cgrow1.upload(h->cgrow_items, h->stream);
    }
    sync(h);
}

// device status word: nonzero after a bounded wait of a kernel expired; read and clear
bool take_dev_err(asm_ctx* h) {
    if (!h->d_dev_err.p) return false;
    int e = 0;
    ck(cudaMemcpyAsync(&e, h->d_dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    sync(h);
    if (e) h->d_dev_err.zero(h->stream);
    return e != 0;
}

void set_ctl(asm_ctx* h, int apply_in, int apply_out, int spmv_in, int spmv_out, int spmv_b) {
    int c[C_NCTL];
    std::memset(c, 0, sizeof(c));
    c[C_PHASE] = PH_DONE;
    c[C_APPLY_IN] = apply_in;
    c[C_APPLY_OUT] = apply_out;
    c[C_SPMV_IN] = spmv_in;
    c[C_SPMV_OUT] = spmv_out;
    c[C_SPMV_B] = spmv_b;
    ck(cudaMemcpyAsync(h->d_ctl.p, c, sizeof(c), cudaMemcpyHostToDevice, h->stream));
    sync(h);
}

}  // namespace

// Coarse boxes of the classical correction for the current grid and partition: cell -> box, the
// cells of each box, and the box pairs of A's blocks (with their ELL locations) for A_C.
int coarse_box_count(const asm_ctx* h, const int* c) {
    if (c[0] == 0) return h->geom.px * h->geom.py * h->geom.pz;
    return ((h->nx + c[0] - 1) / c[0]) * ((h->ny + c[1] - 1) / c[1]) * ((h->nz + c[2] - 1) / c[2]);
}

void coarse_build(asm_ctx* h) {
    const Geom& g = h->geom;
    const int N = h->N;
    const int* c = h->coarse_c;
    const int nb = coarse_box_count(h, c);
    std::vector<int> box(N);
    auto part = [](int n, int p, int x) {  // part t of n cells is [n t / p, n (t + 1) / p)
        int t = (int)(((long long)x * p) / n);
        while (t + 1 < p && (long long)n * (t + 1) / p <= x) t++;
        while (t > 0 && (long long)n * t / p > x) t--;
        return t;
    };
    const int nbx = c[0] ? (h->nx + c[0] - 1) / c[0] : 0, nbz = c[0] ? (h->nz + c[2] - 1) / c[2] : 0;
    for (int y = 0; y < h->ny; y++)
        for (int x = 0; x < h->nx; x++)
            for (int z = 0; z < h->nz; z++) {
                const int cell = z + h->nz * (x + h->nx * y);
                box[cell] = c[0] == 0 ? part(h->nz, g.pz, z) + g.pz * (part(h->nx, g.px, x) + g.px * part(h->ny, g.py, y))
                                      : z / c[2] + nbz * (x / c[0] + nbx * (y / c[1]));
            }
    std::vector<int> bptr(nb + 1, 0), cells(N);
    for (int a = 0; a < N; a++) bptr[box[a] + 1]++;
    for (int b = 0; b < nb; b++) bptr[b + 1] += bptr[b];
    {
        std::vector<int> fill(bptr.begin(), bptr.end() - 1);
        for (int a = 0; a < N; a++) cells[fill[box[a]]++] = a;
    }
    std::vector<std::pair<long long, int>> kv;
    kv.reserve(h->pat.ci.size());
    for (int a = 0; a < N; a++)
        for (int e = h->pat.rp[a]; e < h->pat.rp[a + 1]; e++)
            kv.push_back({(long long)box[a] * nb + box[h->pat.ci[e]], e});
    std::sort(kv.begin(), kv.end());
    std::vector<int> kptr, kloc(kv.size());
    std::vector<long long> keys;
    for (size_t i = 0; i < kv.size(); i++) {
        if (i == 0 || kv[i].first != kv[i - 1].first) {
            kptr.push_back((int)i);
            keys.push_back(kv[i].first);
        }
        kloc[i] = kv[i].second;
    }
    kptr.push_back((int)kv.size());
    cudaStream_t st = h->stream;
    h->cnb = nb;
    h->cnkeys = (int)keys.size();
    h->d_cbox.upload(box, st);
    h->d_ccells.upload(cells, st);
    h->d_ckptr.upload(kptr, st);
    h->d_ckloc.upload(kloc, st);
    h->d_ckeys.upload(keys, st);
    const long long n = 3LL * nb;
    h->d_cblk.alloc((size_t)std::max(1, h->cnkeys) * 9 * sizeof(double));
    h->d_caug.alloc((size_t)(n * 2 * n) * sizeof(double));
    h->d_cprow.alloc((size_t)(2 * n) * sizeof(double));
    h->d_cfcol.alloc((size_t)n * sizeof(double));
    int sms = 0;
    ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    h->cpart_cap = 4 * std::max(1, sms);
    h->d_cpart.alloc((size_t)2 * h->cpart_cap * sizeof(double));
    h->d_cerr.alloc(sizeof(int));
    {
        std::vector<GJMat> m{GJMat{h->d_caug.as<double>(), (int)n, h->d_cprow.as<double>(), h->d_cfcol.as<double>()}};
        h->d_cmat.upload(m, st);
    }
    h->d_crc.alloc((size_t)n * sizeof(double));
    h->d_cyc.alloc((size_t)n * sizeof(double));
    if (h->coarse_mode == 2)
        h->d_cw.alloc((size_t)3 * N * sizeof(double));
    else
        h->d_cw.release();
    h->cbox_items.clear();
    for (int b = 0; b < nb; b++)
        h->cbox_items.push_back(BoxItem{0, b, bptr[b], bptr[b + 1], 0, 0, h->d_ccells.as<int>()});
    h->cgrow_items.clear();
    for (long long r0 = 0; r0 < n; r0 += 8) h->cgrow_items.push_back(RowItem{0, (int)r0});
    sync(h);
    h->coarse_valid = true;
    h->ws_m = -1;  // the system table takes the new coarse buffers
}

// A_C = R_C A R_C^T from the current values, inverted in place; ZERO_PIVOT for a singular A_C
int coarse_numeric(asm_ctx* h) {
    launch_coarse(h->d_ckptr.as<int>(), h->d_ckloc.as<int>(), h->d_bsr_val.as<double>(),
                  h->d_cblk.as<double>(), h->cnkeys, h->stream);
    h->d_cerr.zero(h->stream);
    ck(launch_coarse_invert(h->d_ckeys.as<long long>(), h->d_cblk.as<double>(), h->cnkeys, h->cnb,
                            h->d_caug.as<double>(), h->d_cmat.as<GJMat>(), h->d_cpart.as<double>(), h->cpart_cap,
                            h->d_cerr.as<int>(), h->device, h->stream));
    ck(cudaGetLastError());
    int err = 0;
    ck(cudaMemcpyAsync(&err, h->d_cerr.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    sync(h);
    h->prof.kernel_launches += 4;
    if (err != 0) {
        h->err_sub = -1;
        h->err_row = (err - 1) / 3;
        return ASM_ERR_ZERO_PIVOT;
    }
    return ASM_OK;
}

// Device assembly, factorisation and packing of the current symbolic structure.
int factor_numeric(asm_ctx* h) {
    SysSym& S = *h->sym;
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0));
    ck(cudaEventCreate(&e1));
    ck(cudaEventRecord(e0, h->stream));
    if (S.g.far_mode != 0)
        launch_coarse(h->d_cptr.as<int>(), h->d_cloc.as<int>(), h->d_bsr_val.as<double>(),
                      h->d_cval.as<double>(), S.nC, h->stream);
    launch_assemble(h->d_aptr.as<int>(), h->d_aloc.as<int>(), h->d_acs.as<int>(), h->d_bsr_val.as<double>(),
                    h->d_cval.as<double>(), h->d_slot.as<double>(), h->total_slots, h->stream, h->d_along.as<int>(),
                    h->n_along);
    h->d_err.zero(h->stream);
    const bool exact = h->opt.local_solver == ASM_LOCAL_EXACT;
    if (exact) {
        const int K = (int)S.subs.size();
        launch_gj_init(h->d_dmats.as<GJMat>(), h->d_dinit.as<int2>(), h->n_dinit, h->stream);
        launch_dense_scatter(h->d_slot.as<double>(), h->d_doff.as<long long>(), h->d_dmat_of_slot.as<int>(),
                             h->d_dmats.as<GJMat>(), h->total_slots, h->stream);
        h->d_derr.zero(h->stream);
        ck(launch_gj_run(h->d_dmats.as<GJMat>(), K, h->dmax3, h->d_dpart.as<double>(), h->dpart_cap,
                         h->d_derr.as<int>(), h->device, h->stream));
    } else if (is_nf(h)) {
        int nmax = 0;
        for (const NFDesc& d : h->nf_desc) nmax = std::max(nmax, d.n);
        launch_nf_factor(h->d_nfdesc1.as<NFDesc>(), (int)h->nf_desc.size(), nmax, h->prec, h->d_err.as<FactErr>(),
                         h->stream);
    } else {
        launch_factor(h->d_factdesc.as<FactDesc>(), (int)S.subs.size(), h->d_err.as<FactErr>(), nullptr, h->stream);
        launch_pack(h->d_pk_off_f.as<long long>(), h->d_pk_src_f.as<int>(), h->pk_nf, h->prec,
                    h->d_stream.as<unsigned char>(), h->d_slot.as<double>(), h->stream);
        launch_pack(h->d_pk_off_c.as<long long>(), h->d_pk_src_c.as<int>(), h->pk_nc, h->lump32 ? 1 : 0,
                    h->d_stream.as<unsigned char>(), h->d_slot.as<double>(), h->stream);
    }
    ck(cudaGetLastError());
    ck(cudaEventRecord(e1, h->stream));
    FactErr fe;
    ck(cudaMemcpyAsync(&fe, h->d_err.p, sizeof(fe), cudaMemcpyDeviceToHost, h->stream));
    std::vector<int> derr;
    if (exact) {
        derr.assign(S.subs.size(), 0);
        ck(cudaMemcpyAsync(derr.data(), h->d_derr.p, derr.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    }
    sync(h);
    for (size_t s = 0; s < derr.size(); s++)
        if (derr[s] != 0) {  // the first singular local matrix, its local block row
            fe.flag = 1;
            fe.sub = (int)s;
            fe.row = h->drow_of_q[s][(derr[s] - 1) / 3];
            break;
        }
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->factor_ms = ms;
    h->prof.factor_ms += ms;
    h->prof.kernel_launches += 5;
    if (fe.flag && is_nf(h) && fe.sub >= 0 && fe.sub < (int)h->nf_row_of_cell.size() && fe.row >= 0 &&
        fe.row < (int)h->nf_row_of_cell[fe.sub].size())
        fe.row = h->nf_row_of_cell[fe.sub][fe.row];  // box cell -> local row
    if (fe.flag) {
        h->err_sub = fe.sub;
        h->err_row = fe.row;
        h->factored = false;
        return ASM_ERR_ZERO_PIVOT;
    }
    if (h->coarse_mode != 0) {
        if (!h->coarse_valid) coarse_build(h);
        const int cs = coarse_numeric(h);
        if (cs != ASM_OK) {
            h->factored = false;
            return cs;
        }
    }
    h->factored = true;
    return ASM_OK;
}

// ---------------------------------------------------------------------------------------------
// Batch driver: all systems advance together; each kernel reads each system's own state.
// ---------------------------------------------------------------------------------------------
namespace {

struct Batch {
    std::vector<asm_ctx*> hs;
    DBuf d_tab, d_vec, d_row, d_box, d_sub, d_gather, d_ritems;
    int nritems = 0;
    int nvec = 0, nrow = 0, nbox = 0, nsub = 0, prec = 0, slots = 3, chunk = kStreamChunkMin;
    int ngroup = 0;  // d_box[0 .. ngroup): every system's cell-group sum items
    bool lump32 = false;
    ApplyConfig apply{Y_DEVICE, 0, 2, kStreamChunkMin};
    int all_bytes = 0, lump_bytes = 0;  // largest subdomain's shared-memory needs (placements)
    DBuf d_dense;           // exact local solves: (subdomain item, first owned row of 8)
    int ndense = 0;
    bool exact = false;     // every system of the batch has exact local solves
    DBuf d_nf;              // nested factorisation: every system's subdomains
    int nnf = 0;
    size_t nf_smem = 0;
    int nf_slots = 2;
    bool nf = false;        // every system of the batch has nested-factorisation local solves
    DBuf d_cbox, d_cgrow;   // coarse-correction work items of the systems that have one
    int ncbox = 0, ncgrow = 0;
    bool two_stage = false;
    int coop_grid = 0;  // > 0: single system, orthogonalisation in one cooperative launch
    bool has_init = false;  // a system may be in its initial phase (serving: systems join mid-flight)
    std::vector<int> host_ctl;
    int* pinned = nullptr;
    size_t pinned_cap = 0;
    ~Batch() {
        if (pinned) cudaFreeHost(pinned);
    }
};

void build_batch(Batch& B, cudaStream_t st) {
    std::vector<SysTab> tabs;
    std::vector<VecItem> vi;
    std::vector<RowItem> ri;
    std::vector<BoxItem> bi;
    std::vector<SubDesc> sd;
    for (int k = 0; k < (int)B.hs.size(); k++) {
        asm_ctx* h = B.hs[k];
        tabs.push_back(h->tab);
        for (int c = 0; c < h->nchunk; c++) vi.push_back(VecItem{k, c});
        for (int r = 0; r < h->N; r += 256) ri.push_back(RowItem{k, r});
        for (int j = 0; j < h->n_group_items; j++) {
            BoxItem b = h->box_items[j];
            b.sys = k;
            bi.push_back(b);
        }
    }
    B.ngroup = (int)bi.size();
    for (int k = 0; k < (int)B.hs.size(); k++) {
        const asm_ctx* h = B.hs[k];
        for (size_t j = h->n_group_items; j < h->box_items.size(); j++) {
            BoxItem b = h->box_items[j];
            b.sys = k;
            bi.push_back(b);
        }
    }
    sd = longest_first(B.hs);
    B.exact = !B.hs.empty() && B.hs[0]->opt.local_solver == ASM_LOCAL_EXACT;
    B.nf = !B.hs.empty() && is_nf(B.hs[0]);
    if (B.nf) {
        std::vector<NFDesc> nd;
        int bxm = 0, bzm = 0;
        for (int k = 0; k < (int)B.hs.size(); k++) {
            bxm = std::max(bxm, B.hs[k]->nf_bx_max);
            bzm = std::max(bzm, B.hs[k]->nf_bz_max);
            for (NFDesc d : B.hs[k]->nf_desc) {
                d.sys = k;
                nd.push_back(d);
            }
        }
        std::stable_sort(nd.begin(), nd.end(), [](const NFDesc& a, const NFDesc& b) { return a.n > b.n; });
        B.d_nf.upload_reuse(nd, st);
        B.nnf = (int)nd.size();
        asm_ctx* h0 = B.hs[0];
        int dev_smem = 0;
        ck(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h0->device));
        B.nf_slots = nf_apply_slots(B.nnf, bxm, bzm, B.hs[0]->prec, h0->sm_smem, h0->n_sms, dev_smem);
        B.nf_smem = nf_apply_smem(bxm, bzm, B.hs[0]->prec, B.nf_slots);
    }
    if (B.exact) {
        const std::vector<int2> di = dense_items(sd);
        B.d_dense.upload_reuse(di, st);
        B.ndense = (int)di.size();
    }
    std::vector<BoxItem> cb;
    std::vector<RowItem> cg;
    B.two_stage = false;
    for (int k = 0; k < (int)B.hs.size(); k++) {
        asm_ctx* h = B.hs[k];
        if (h->coarse_mode == 0 || !h->coarse_valid) continue;
        for (BoxItem b : h->cbox_items) {
            b.sys = k;
            cb.push_back(b);
        }
        for (RowItem r : h->cgrow_items) {
            r.sys = k;
            cg.push_back(r);
        }
        B.two_stage = B.two_stage || h->coarse_mode == 2;
    }
    B.d_cbox.upload_reuse(cb, st);
    B.d_cgrow.upload_reuse(cg, st);
    B.ncbox = (int)cb.size();
    B.ncgrow = (int)cg.size();
    B.d_tab.upload_reuse(tabs, st);
    B.d_vec.upload_reuse(vi, st);
    B.d_row.upload_reuse(ri, st);
    B.d_box.upload_reuse(bi, st);
    B.d_sub.upload_reuse(sd, st);
    {
        const std::vector<int2> ri = restrict_items(sd);
        B.d_ritems.upload_reuse(ri, st);
        B.nritems = (int)ri.size();
    }
    B.nvec = (int)vi.size();
    B.nrow = (int)ri.size();
    B.nbox = (int)bi.size();
    B.nsub = (int)sd.size();
    // pinned control words: grown, never shrunk (pinning host memory is slow)
    const size_t npin = std::max<size_t>(1, B.hs.size());
    if (!B.pinned || B.pinned_cap < npin) {
        if (B.pinned) cudaFreeHost(B.pinned);
        B.pinned = nullptr;
        B.pinned_cap = npin + npin / 2;
        ck(cudaMallocHost((void**)&B.pinned, sizeof(int) * C_NCTL * B.pinned_cap));
    }
    // kernel variants shared by the whole batch
    B.prec = B.hs.empty() ? 0 : B.hs[0]->prec;
    B.lump32 = !B.hs.empty() && B.hs[0]->lump32;
    int all_bytes = 0, lump_bytes = 0;
    bool all_ok = !B.hs.empty();
    for (asm_ctx* h : B.hs) {
        all_bytes = std::max(all_bytes, h->apply_smem);
        lump_bytes = std::max(lump_bytes, h->apply_lump_smem);
        all_ok = all_ok && h->apply_smem > 0;
    }
    if (!all_ok) all_bytes = 0;
    B.all_bytes = all_bytes;
    B.lump_bytes = lump_bytes;
    B.slots = 4;
    B.chunk = kStreamChunkMin;
    for (asm_ctx* h : B.hs) {
        B.slots = std::min(B.slots, h->apply_slots);
        B.chunk = std::max(B.chunk, h->chunk_cap);
    }
    if (!B.hs.empty())
        B.apply = apply_local_vectors(B.nsub, all_bytes, lump_bytes, B.slots, B.chunk, B.hs[0]->sm_smem,
                                      B.hs[0]->n_sms, B.hs[0]->apply_place, other_slots(B.hs[0]));
}

// events bracketing the launch groups of one step: [prep | apply | post | spmv | mgs+finish]
struct StepEvents {
    cudaEvent_t e[6] = {};
    bool live = false;
    void create() {
        for (auto& x : e) ck(cudaEventCreate(&x));
        live = true;
    }
    ~StepEvents() {
        if (live)
            for (auto& x : e) cudaEventDestroy(x);
    }
};

// The placements of the apply's local vectors that fit this batch, for the online tuner (one entry
// when a placement was asked for).  Every placement gives the same bits, so the tuner may try them
// on the solve's own first steps.
std::vector<ApplyConfig> apply_candidates(const Batch& B) {
    std::vector<ApplyConfig> c;
    if (B.hs.empty() || B.exact || B.nf) return c;
    const asm_ctx* h = B.hs[0];
    if (h->apply_place != 0) return {B.apply};
    for (int force : {Y_SMEM + 1, Y_LUMPS + 1, Y_DEVICE + 1}) {
        const ApplyConfig a =
            apply_local_vectors(B.nsub, B.all_bytes, B.lump_bytes, B.slots, B.chunk, h->sm_smem, h->n_sms, force,
                                other_slots(h));
        if (a.ymode == force - 1) c.push_back(a);
    }
    return c;
}

// kernels launched by launch_local_solves
int local_solve_launches(const Batch& B) { return B.nf ? 1 : 2; }

// the local solves of one apply: R_i r and the fused ILU sweeps, or R_i r and the owned rows of
// A_i^{-1} R_i r, or the nested-factorisation sweeps
void launch_local_solves(Batch& B, const SysTab* tab, cudaStream_t st) {
    if (B.nf) {
        launch_nf_apply(tab, B.d_nf.as<NFDesc>(), B.nnf, B.prec, B.nf_slots, B.nf_smem, st);
    } else if (B.exact) {
        launch_dense_restrict(tab, B.d_sub.as<SubDesc>(), B.nsub, st);
        launch_dense_apply(tab, B.d_sub.as<SubDesc>(), B.d_dense.as<int2>(), B.ndense, st);
    } else {
        launch_restrict(tab, B.d_sub.as<SubDesc>(), B.d_ritems.as<int2>(), B.nritems, B.prec, B.lump32, st);
        launch_apply(tab, B.d_sub.as<SubDesc>(), B.nsub, B.prec, B.lump32, B.apply, st);
    }
}

void launch_step(Batch& B, int kmax, cudaStream_t st, StepEvents* ev) {
    const SysTab* tab = B.d_tab.as<SysTab>();
    const VecItem* vi = B.d_vec.as<VecItem>();
    if (ev) ck(cudaEventRecord(ev->e[0], st));
    if (B.has_init) launch_init(tab, vi, B.nvec, st);
    launch_prep(tab, vi, B.nvec, st);
    if (ev) ck(cudaEventRecord(ev->e[1], st));
    launch_boxsum(tab, B.d_box.as<BoxItem>(), B.nbox, B.ngroup, st);
    launch_local_solves(B, tab, st);
    launch_coarse_apply(tab, B.d_row.as<RowItem>(), B.nrow, B.d_cbox.as<BoxItem>(), B.ncbox, B.d_cgrow.as<RowItem>(),
                        B.ncgrow, vi, B.nvec, B.two_stage, st);
    if (ev) ck(cudaEventRecord(ev->e[2], st));
    launch_post(tab, vi, B.nvec, st);
    if (ev) ck(cudaEventRecord(ev->e[3], st));
    launch_spmv(tab, B.d_row.as<RowItem>(), B.nrow, st);
    if (ev) ck(cudaEventRecord(ev->e[4], st));
    long long n = 4 + local_solve_launches(B);
    if (B.coop_grid > 0) {
        ck(launch_ortho_coop(tab, B.hs[0]->d_partial.as<double>(), B.coop_grid, st));
        n += 1;
    } else {
        for (int k = 0; k <= kmax; k++) launch_mgs(tab, vi, B.nvec, k, st);
        launch_finish(tab, vi, B.nvec, st);
        n += kmax + 2;
    }
    if (ev) ck(cudaEventRecord(ev->e[5], st));
    ck(cudaGetLastError());
    for (asm_ctx* h : B.hs) h->prof.kernel_launches += n;
}

// One ORTHOMIN step of every system: [apply | mat-vec | projections 0..kmax + update], with the
// events at the same places as a GMRES step (the prep and post groups are empty)
void launch_step_om(Batch& B, int kmax, cudaStream_t st, StepEvents* ev) {
    const SysTab* tab = B.d_tab.as<SysTab>();
    const VecItem* vi = B.d_vec.as<VecItem>();
    if (ev) ck(cudaEventRecord(ev->e[0], st));
    if (B.has_init) launch_init(tab, vi, B.nvec, st);
    if (ev) ck(cudaEventRecord(ev->e[1], st));
    launch_boxsum(tab, B.d_box.as<BoxItem>(), B.nbox, B.ngroup, st);
    launch_local_solves(B, tab, st);
    launch_coarse_apply(tab, B.d_row.as<RowItem>(), B.nrow, B.d_cbox.as<BoxItem>(), B.ncbox, B.d_cgrow.as<RowItem>(),
                        B.ncgrow, vi, B.nvec, B.two_stage, st);
    if (ev) {
        ck(cudaEventRecord(ev->e[2], st));
        ck(cudaEventRecord(ev->e[3], st));
    }
    launch_spmv(tab, B.d_row.as<RowItem>(), B.nrow, st);
    if (ev) ck(cudaEventRecord(ev->e[4], st));
    for (int l = 0; l <= kmax; l++) launch_om(tab, vi, B.nvec, l, st);
    launch_om_update(tab, vi, B.nvec, st);
    if (ev) ck(cudaEventRecord(ev->e[5], st));
    ck(cudaGetLastError());
    for (asm_ctx* h : B.hs) h->prof.kernel_launches += 3 + local_solve_launches(B) + kmax + 1;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, a, b));
    return ms;
}

void read_ctl(Batch& B, cudaStream_t st) {
    for (size_t k = 0; k < B.hs.size(); k++)
        ck(cudaMemcpyAsync(B.pinned + k * C_NCTL, B.hs[k]->d_ctl.p, sizeof(int) * C_NCTL, cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
}

// b into slot VB, control words (initial phase) and tolerance of one system
void begin_solve(asm_ctx* h, const double* b, int on_device, double rtol, int max_iter) {
    ensure_workspace(h);
    const ScalLayout SL = ScalLayout::make(h->ws_m);
    copy_in(h, h->d_ws.as<double>() + (long long)VB * h->n3p, b, sizeof(double) * 3 * (size_t)h->N, on_device);
    int c[C_NCTL];
    std::memset(c, 0, sizeof(c));
    c[C_PHASE] = PH_INIT;
    c[C_APPLY_IN] = -1;
    c[C_SPMV_IN] = -1;
    c[C_MAXIT] = max_iter;
    c[C_STATUS] = ASM_ERR_NOT_CONVERGED;
    ck(cudaMemcpyAsync(h->d_ctl.p, c, sizeof(c), cudaMemcpyHostToDevice, h->stream));
    double tol = rtol;
    ck(cudaMemcpyAsync(h->d_scal.as<double>() + SL.tol, &tol, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    ck(cudaStreamSynchronize(h->stream));
}

// x and the result of a finished (or abandoned) system; c = its control words
int harvest(asm_ctx* h, const int* c, double* x, int on_device, asm_solve_info* info) {
    const ScalLayout SL = ScalLayout::make(h->ws_m);
    double sc[2];
    ck(cudaMemcpyAsync(sc, h->d_scal.as<double>() + SL.bnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    copy_out(h, x, h->d_ws.as<double>() + (long long)VX * h->n3p, sizeof(double) * 3 * (size_t)h->N, on_device);
    ck(cudaStreamSynchronize(h->stream));
    int status = c[C_PHASE] == PH_DONE ? c[C_STATUS] : ASM_ERR_NOT_CONVERGED;
    if (take_dev_err(h)) status = ASM_ERR_TIMEOUT;
    if (info) {
        info->iterations = c[C_ITERS];
        info->restarts = c[C_RESTARTS];
        info->converged = c[C_CONVERGED];
        info->status = status;
        info->rel_residual = sc[0] > 0 ? sc[1] / sc[0] : 0.0;
    }
    return status;
}

// GMRES(m) or ORTHOMIN(k) (every system of the batch uses the same method)
int run_krylov(std::vector<asm_ctx*>& hs, const double* const* b, double* const* x, double rtol, int max_iter,
              int on_device, asm_solve_info* infos) {
    cudaStream_t st = hs[0]->stream;
    Batch B;
    B.hs = hs;
    for (size_t k = 0; k < hs.size(); k++) begin_solve(hs[k], b[k], on_device, rtol, max_iter);
    build_batch(B, st);
    const bool om = hs[0]->opt.krylov == ASM_KRYLOV_ORTHOMIN;
    if (hs.size() == 1 && !hs[0]->no_coop && !om) B.coop_grid = ortho_coop_grid(hs[0]->device);
    {
        // initial step: x = 0, r = b, beta = ||b||
        const SysTab* tab = B.d_tab.as<SysTab>();
        const VecItem* vi = B.d_vec.as<VecItem>();
        launch_init(tab, vi, B.nvec, st);
        if (om) {
            launch_om(tab, vi, B.nvec, 0, st);
        } else if (B.coop_grid > 0) {
            ck(launch_ortho_coop(tab, hs[0]->d_partial.as<double>(), B.coop_grid, st));
        } else {
            launch_mgs(tab, vi, B.nvec, 0, st);
            launch_finish(tab, vi, B.nvec, st);
        }
        ck(cudaGetLastError());
        for (asm_ctx* h : hs) h->prof.kernel_launches += (B.coop_grid > 0 || om) ? 2 : 3;
    }
    const bool prof = hs[0]->profiling;
    // online tuner: the first apply steps try each placement of the local vectors (one round to
    // warm up, one timed); the fastest is kept (and remembered for this handle's next solves)
    std::vector<ApplyConfig> cand;
    if (!hs[0]->no_autotune) cand = apply_candidates(B);
    int tune_total = cand.size() > 1 ? 2 * (int)cand.size() : 0;
    if (hs.size() == 1 && hs[0]->tuned_ymode >= 0)
        for (const ApplyConfig& a : cand)
            if (a.ymode == hs[0]->tuned_ymode) {
                B.apply = a;
                tune_total = 0;
            }
    std::vector<float> tune_ms(cand.size(), 0.0f);
    int tune_next = 0, tune_at = -1;
    for (asm_ctx* h : hs) h->last_solve_apply = B.apply;
    StepEvents ev;
    if (prof || tune_total > 0) ev.create();
    // CUDA graphs for batches: the launch sequence of a step depends only on the number of
    // projections, so each is captured once (after one plain run) and replayed
    bool graphs_ok = hs.size() > 1 && B.coop_grid == 0 && !prof && st != nullptr && !hs[0]->no_graphs;
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, long long> graph_launches;
    std::set<int> seen;
    auto plain_step = [&](int kmax, StepEvents* e) {
        if (om)
            launch_step_om(B, kmax, st, e);
        else
            launch_step(B, kmax, st, e);
    };
    bool pending = false;
    int pending_applies = 0;
    const int guard_steps = 4 * max_iter + 64;
    for (int step = 0; step < guard_steps; step++) {
        read_ctl(B, st);
        if (pending) {
            asm_profile_info& P = hs[0]->prof;
            P.ortho_ms += elapsed(ev.e[0], ev.e[1]) + elapsed(ev.e[2], ev.e[3]) + elapsed(ev.e[4], ev.e[5]);
            P.apply_ms += elapsed(ev.e[1], ev.e[2]);
            P.spmv_ms += elapsed(ev.e[3], ev.e[4]);
            P.apply_launches += pending_applies;
            pending = false;
        }
        if (tune_at >= 0) {
            if (tune_at >= (int)cand.size()) tune_ms[tune_at - cand.size()] = elapsed(ev.e[1], ev.e[2]);
            tune_at = -1;
            if (tune_next == tune_total) {
                int best = 0;
                for (size_t k = 1; k < cand.size(); k++)
                    if (tune_ms[k] < tune_ms[best]) best = (int)k;
                B.apply = cand[best];
                if (hs.size() == 1) hs[0]->tuned_ymode = B.apply.ymode;
                for (asm_ctx* h : hs) h->last_solve_apply = B.apply;
            }
        }
        int kmax = -1;
        bool any = false;
        for (size_t k = 0; k < hs.size(); k++) {
            const int* c = B.pinned + k * C_NCTL;
            if (c[C_PHASE] == PH_DONE) continue;
            any = true;
            if (c[C_PHASE] == PH_ARNOLDI) kmax = std::max(kmax, c[C_J] + 1);
            else if (c[C_PHASE] == PH_OM) kmax = std::max(kmax, c[C_OM_STORED]);
            else kmax = std::max(kmax, 0);
        }
        if (!any) break;
        pending_applies = 0;
        for (size_t k = 0; k < hs.size(); k++) {
            const int* c = B.pinned + k * C_NCTL;
            if (c[C_APPLY_IN] >= 0 && c[C_PHASE] != PH_DONE) pending_applies++;
        }
        if (tune_next < tune_total && pending_applies > 0) {
            B.apply = cand[tune_next % cand.size()];
            tune_at = tune_next++;
            plain_step(kmax, &ev);
            pending = prof;
        } else if (graphs_ok && tune_next >= tune_total) {
            auto it = graphs.find(kmax);
            if (it == graphs.end() && seen.count(kmax)) {
                // capture this step's launch sequence (its kernels were all launched once before)
                const long long before = hs[0]->prof.kernel_launches;
                cudaGraph_t g = nullptr;
                cudaGraphExec_t ex = nullptr;
                bool okc = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (okc) {
                    try {
                        plain_step(kmax, nullptr);
                    } catch (const CudaFail&) {
                        okc = false;
                    }
                    okc = cudaStreamEndCapture(st, &g) == cudaSuccess && okc;
                }
                if (okc) okc = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
                for (asm_ctx* h : hs) h->prof.kernel_launches -= hs[0]->prof.kernel_launches - before;
                if (okc) {
                    it = graphs.emplace(kmax, ex).first;
                    graph_launches[kmax] = hs[0]->prof.kernel_launches - before;
                } else {
                    cudaGetLastError();
                    if (ex) cudaGraphExecDestroy(ex);
                    graphs_ok = false;
                }
            }
            if (it != graphs.end()) {
                ck(cudaGraphLaunch(it->second, st));
                for (asm_ctx* h : hs) h->prof.kernel_launches += graph_launches[kmax];
            } else {
                plain_step(kmax, nullptr);
                seen.insert(kmax);
            }
        } else {
            plain_step(kmax, prof ? &ev : nullptr);
            pending = prof;
        }
    }
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    read_ctl(B, st);
    int worst = ASM_OK;
    for (size_t k = 0; k < hs.size(); k++) {
        const int status = harvest(hs[k], B.pinned + k * C_NCTL, x[k], on_device, infos ? &infos[k] : nullptr);
        if (status == ASM_ERR_TIMEOUT)
            worst = ASM_ERR_TIMEOUT;
        else if (status != ASM_OK && worst != ASM_ERR_TIMEOUT)
            worst = status;
    }
    return worst;
}

}  // namespace

int handle_matrix_view(asm_ctx* h, MatrixView* out) {
    if (!h || !out) return ASM_ERR_INVALID_ARG;
    if (!h->has_matrix) return ASM_ERR_STATE;
    out->ell_val = h->d_ell_val.as<double>();
    out->ell_col = h->d_ell_col.as<int>();
    out->ell_w = h->pat.ell_w;
    out->rows_pad = h->pat.rows_pad;
    out->n_cells = h->N;
    out->device = h->device;
    out->stream = h->stream;
    return ASM_OK;
}


// ---------------------------------------------------------------------------------------------
// Serving loop: requests of any grid size join the running batch between Krylov steps
// ---------------------------------------------------------------------------------------------
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace {

size_t ctx_device_bytes(const asm_ctx* h) {
    const DBuf* bufs[] = {&h->d_ell_val, &h->d_ell_col, &h->d_ell_loc, &h->d_bsr_rp, &h->d_bsr_val, &h->d_bcell,
                          &h->d_cptr, &h->d_cloc, &h->d_cval, &h->d_boxsum, &h->d_slot, &h->d_dpiv, &h->d_aptr,
                          &h->d_aloc, &h->d_acs, &h->d_along, &h->d_fp, &h->d_stream, &h->d_pk_off_f, &h->d_pk_src_f,
                          &h->d_pk_off_c, &h->d_pk_src_c, &h->d_lv, &h->d_rlists, &h->d_y, &h->d_corr_cells,
                          &h->d_corr, &h->d_dev_err, &h->d_gsum, &h->d_r32, &h->d_factdesc, &h->d_subdesc_single,
                          &h->d_err, &h->d_ws,
                          &h->d_scal, &h->d_ctl, &h->d_partial, &h->d_tab1, &h->d_vec1, &h->d_row1, &h->d_box1,
                          // exact local solves, nested factorisation, classical coarse correction
                          &h->d_daug, &h->d_dprow, &h->d_dfcol, &h->d_dmats, &h->d_dinit, &h->d_doff,
                          &h->d_dmat_of_slot, &h->d_dpart, &h->d_derr, &h->d_ditems1, &h->d_ritems1, &h->d_nfint, &h->d_nfval,
                          &h->d_nfdesc1, &h->d_nfpack, &h->d_nfy, &h->d_nfband, &h->d_cbox, &h->d_ccells, &h->d_ckptr,
                          &h->d_ckloc, &h->d_ckeys, &h->d_cblk, &h->d_caug, &h->d_cprow, &h->d_cfcol, &h->d_cpart,
                          &h->d_cerr, &h->d_crc, &h->d_cyc, &h->d_cw, &h->d_cbox_items1, &h->d_cgrow1, &h->d_cmat};
    size_t b = 0;
    for (const DBuf* d : bufs) b += d->bytes;
    return b;
}

// symbolic structure of one (grid, partition, pattern): built once on a worker thread
struct SymEntry {
    Pattern pat;
    std::shared_ptr<SysSym> sym;
    bool ready = false;
    std::string err;
    int status = ASM_ERR_INVALID_ARG;  // the requests' status when err is set
};

struct Req {
    long long ticket = 0;
    asm_request in{};
    std::vector<double> b;
    std::string skey;
    asm_ctx* h = nullptr;
    int state = 0;  // 0 pending, 1 active, 2 done
    std::vector<double> x;
    asm_solve_info info{};
};

unsigned long long fnv1a(const void* p, size_t n, unsigned long long h) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; i++) {
        h ^= c[i];
        h *= 1099511628211ULL;
    }
    return h;
}

}  // namespace

struct asm_server {
    asm_server_options opt{};
    cudaStream_t stream = nullptr;
    size_t budget = 0, resident = 0;
    long long next_ticket = 1;
    std::deque<Req*> pending;
    std::vector<Req*> active;
    std::unordered_map<long long, Req*> by_ticket;
    std::map<long long, asm_ctx*> idle;  // factored systems kept for matrix reuse (keyless ones under
                                         // negative keys: reusable by structure only)
    long long next_keyless = -2;
    std::list<long long> lru;            // idle keys, least recently used first
    std::map<long long, bool> key_busy;
    Batch batch;
    bool dirty = true;
    // symbolic cache + worker
    std::mutex mu;
    std::condition_variable cv;
    std::map<std::string, SymEntry> syms;
    std::deque<std::pair<std::string, Req*>> jobs;
    bool quit = false;
    std::thread worker;
    asm_server_stats st{};
};

namespace {

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void sym_worker(asm_server* S) {
    for (;;) {
        std::string key;
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->quit || !S->jobs.empty(); });
            if (S->quit) return;
            key = S->jobs.front().first;
            r = S->jobs.front().second;
            S->jobs.pop_front();
        }
        SymEntry e;
        const asm_request& q = r->in;
        const auto t0 = std::chrono::steady_clock::now();
        try {  // an exception must not leave the thread: host memory or threads ran out
            e.err = build_pattern(q.n_cells, q.row_ptr, q.col_idx, q.nnzb, e.pat);
            if (e.err.empty()) {
                Geom g;
                g.nx = q.nx;
                g.ny = q.ny;
                g.nz = q.nz;
                g.px = q.px;
                g.py = q.py;
                g.pz = q.pz;
                g.ov = q.overlap;
                g.nw = q.near_width;
                for (int d = 0; d < 3; d++) {
                    g.cn[d] = q.near_width > 0 ? q.c_near[d] : 1;
                    g.cf[d] = q.far_mode == ASM_FAR_BOXES ? q.c_far[d] : 1;
                }
                g.far_mode = q.far_mode;
                e.sym = std::make_shared<SysSym>();
                e.err = build_symbolic(g, e.pat, S->opt.precision, S->opt.lump_precision == ASM_LUMP_FP32 ? 1 : 0, 1, *e.sym, 0);
            }
        } catch (const std::exception& ex) {
            e.sym.reset();
            e.err = std::string("host resources: ") + ex.what();
            e.status = ASM_ERR_OOM;
        }
        e.ready = true;
        std::lock_guard<std::mutex> lk(S->mu);
        S->st.analysis_ms += ms_since(t0);
        S->syms[key] = std::move(e);
    }
}

std::string structure_key(const asm_request& q, int prec) {
    unsigned long long hsh = 1469598103934665603ULL;
    hsh = fnv1a(q.row_ptr, sizeof(int) * ((size_t)q.n_cells + 1), hsh);
    hsh = fnv1a(q.col_idx, sizeof(int) * (size_t)q.nnzb, hsh);
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%d,%d,%d|%d,%d,%d|%d,%d|%d,%d,%d|%d|%d,%d,%d|%d|%llx", q.nx, q.ny, q.nz, q.px, q.py,
                  q.pz, q.overlap, q.near_width, q.c_near[0], q.c_near[1], q.c_near[2], q.far_mode, q.c_far[0],
                  q.c_far[1], q.c_far[2], prec, hsh);
    return buf;
}

void evict_idle(asm_server* S, size_t need) {
    while (S->resident + need > S->budget && !S->lru.empty()) {
        const long long key = S->lru.front();
        S->lru.pop_front();
        asm_ctx* h = S->idle[key];
        S->idle.erase(key);
        S->resident -= ctx_device_bytes(h);
        asm_destroy(h);
        S->st.evictions++;
    }
}

// New system for a request whose structure is ready: matrix, shared symbolic, numeric factor.
int build_ctx(asm_server* S, Req* r, const SymEntry& e, asm_ctx** out) {
    asm_options o;
    asm_default_options(&o);
    o.precision = S->opt.precision;
    o.restart = S->opt.restart;
    o.device = S->opt.device;
    o.lump_precision = S->opt.lump_precision;
    asm_ctx* h = nullptr;
    int st = asm_create(&h, &o, S->stream);
    if (st) return st;
    const asm_request& q = r->in;
    st = guard(h, [&]() -> int {
        asm_set_grid(h, q.nx, q.ny, q.nz);
        h->pat = e.pat;
        h->nnzb = q.nnzb;
        h->d_ell_val.alloc((size_t)h->pat.ell_w * 9 * h->pat.rows_pad * sizeof(double));
        h->d_ell_val.zero(h->stream);
        h->d_ell_col.upload(h->pat.ell_col, h->stream);
        h->d_ell_loc.upload(h->pat.ell_loc, h->stream);
        h->d_bsr_rp.upload(h->pat.rp, h->stream);
        fill_ell(h, q.vals, 0);
        h->has_matrix = true;
        const int cf[3] = {q.c_far[0], q.c_far[1], q.c_far[2]};
        int s2 = asm_set_partition_boxes(h, q.px, q.py, q.pz, q.overlap, q.near_width, q.c_near, q.far_mode, cf);
        if (s2) return s2;
        h->sym = e.sym;
        upload_symbolic(h);
        h->sym_valid = true;
        h->ws_m = -1;
        const auto tf = std::chrono::steady_clock::now();
        const int fs = factor_numeric(h);
        S->st.build_factor_ms += ms_since(tf);
        return fs;
    });
    if (st) {
        asm_destroy(h);
        return st;
    }
    *out = h;
    return ASM_OK;
}

// An idle system whose structure key is skey (least recently used first), taken out of the idle
// set; nullptr if there is none.
asm_ctx* take_idle_structure(asm_server* S, const std::string& skey) {
    for (auto it = S->lru.begin(); it != S->lru.end(); ++it) {
        asm_ctx* h = S->idle[*it];
        if (h->server_skey != skey) continue;
        S->idle.erase(*it);
        S->lru.erase(it);
        return h;
    }
    return nullptr;
}

// A system already on the device takes a request's matrix: new values, re-assembly and
// re-factorisation (Section 4: the coarsened matrices are rebuilt for new values, the structure
// is not), without any allocation or structure upload.
int rekey_ctx(asm_ctx* h, const Req* r) {
    return guard(h, [&]() -> int {
        fill_ell(h, r->in.vals, 0);
        return factor_numeric(h);
    });
}

void admit(asm_server* S) {
    for (auto it = S->pending.begin(); it != S->pending.end();) {
        Req* r = *it;
        if (S->opt.max_active > 0 && (int)S->active.size() >= S->opt.max_active) break;
        const long long key = r->in.matrix_key;
        asm_ctx* h = nullptr;
        bool fresh = false;  // a newly built system (a reused one is already counted as resident)
        if (key >= 0 && S->key_busy[key]) {  // same matrix in flight: wait for it
            ++it;
            continue;
        }
        if (!(key >= 0 && S->idle.count(key)) && r->skey.empty()) r->skey = structure_key(r->in, S->opt.precision);
        if (key >= 0 && S->idle.count(key)) {  // repeated matrix: factors already on the device
            h = S->idle[key];
            S->idle.erase(key);
            S->lru.remove(key);
            S->st.reuse_hits++;
        } else if (!r->skey.empty() && (h = take_idle_structure(S, r->skey)) != nullptr) {
            // a new matrix of a structure an idle system already holds on the device
            const auto t0 = std::chrono::steady_clock::now();
            const int st = rekey_ctx(h, r);
            S->st.rekey_ms += ms_since(t0);
            if (st) {
                S->resident -= ctx_device_bytes(h);
                asm_destroy(h);
                r->info.status = st;
                r->state = 2;
                it = S->pending.erase(it);
                continue;
            }
            S->st.structure_reuses++;
        } else {
            SymEntry* e = nullptr;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                auto f = S->syms.find(r->skey);
                if (f == S->syms.end()) {
                    S->syms[r->skey] = SymEntry();
                    S->jobs.push_back({r->skey, r});
                    S->cv.notify_one();
                    S->st.structure_builds++;
                } else if (f->second.ready) {
                    e = &f->second;
                }
            }
            if (!e) {  // structure being analysed on the worker thread
                ++it;
                continue;
            }
            if (!e->err.empty()) {
                r->info.status = e->status;
                r->state = 2;
                it = S->pending.erase(it);
                continue;
            }
            const size_t need = (size_t)r->in.n_cells * 6144;  // ~6 KB per cell resident (FP32 factors, m = 30)
            evict_idle(S, need);
            if (S->resident + need > S->budget && !S->active.empty()) {
                ++it;  // no memory now: wait for systems to finish
                continue;
            }
            const auto t0 = std::chrono::steady_clock::now();
            const int st = build_ctx(S, r, *e, &h);
            S->st.build_ms += ms_since(t0);
            if (st) {
                r->info.status = st;
                r->state = 2;
                it = S->pending.erase(it);
                continue;
            }
            fresh = true;
            h->server_skey = r->skey;
        }
        const int st = guard(h, [&]() -> int {
            begin_solve(h, r->b.data(), 0, r->in.rtol, r->in.max_iter);
            return ASM_OK;
        });
        if (st) {
            r->info.status = st;
            r->state = 2;
            asm_destroy(h);
            it = S->pending.erase(it);
            continue;
        }
        r->h = h;
        r->state = 1;
        if (fresh) S->resident += ctx_device_bytes(h);
        if (key >= 0) S->key_busy[key] = true;
        S->active.push_back(r);
        S->dirty = true;
        it = S->pending.erase(it);
        S->st.admitted++;
    }
}

void retire(asm_server* S, Req* r, const int* c) {
    const auto t0 = std::chrono::steady_clock::now();
    asm_ctx* h = r->h;
    r->x.resize(3 * (size_t)h->N);
    guard(h, [&]() -> int {
        harvest(h, c, r->x.data(), 0, &r->info);
        return ASM_OK;
    });
    r->state = 2;
    r->h = nullptr;
    long long key = r->in.matrix_key;
    if (key >= 0) S->key_busy[key] = false;
    if (S->opt.max_cached > 0) {
        // kept on the device: a later request with the same matrix key reuses the factors, one with
        // the same structure the allocations and the structure (keyless systems under negative
        // keys, reusable by structure only)
        if (key < 0) key = S->next_keyless--;
        S->idle[key] = h;
        S->lru.push_back(key);
        while ((int)S->idle.size() > S->opt.max_cached) {
            const long long k0 = S->lru.front();
            S->lru.pop_front();
            S->resident -= ctx_device_bytes(S->idle[k0]);
            asm_destroy(S->idle[k0]);
            S->idle.erase(k0);
            S->st.evictions++;
        }
    } else {
        S->resident -= ctx_device_bytes(h);
        asm_destroy(h);
    }
    S->st.retire_ms += ms_since(t0);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

void asm_default_options(asm_options* opt) {
    if (!opt) return;
    opt->precision = ASM_PREC_FP64;
    opt->krylov = ASM_KRYLOV_GMRES;
    opt->restart = 30;
    opt->local_solver = ASM_LOCAL_BILU0_COLSUM;
    opt->flexible = -1;
    opt->device = 0;
    opt->lump_precision = ASM_LUMP_FP32;
    opt->ortho = ASM_ORTHO_MGS;
}

const char* asm_error_string(int s) {
    switch (s) {
        case ASM_OK: return "ok";
        case ASM_ERR_INVALID_ARG: return "invalid argument";
        case ASM_ERR_PATTERN: return "block pattern not structurally symmetric or missing a diagonal block";
        case ASM_ERR_ZERO_PIVOT: return "singular 3x3 pivot in a local factorisation";
        case ASM_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case ASM_ERR_OOM: return "out of memory";
        case ASM_ERR_CUDA: return "CUDA runtime error";
        case ASM_ERR_TIMEOUT: return "bounded device wait expired";
        case ASM_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

int asm_create(asm_handle* out, const asm_options* opt, void* cuda_stream) {
    if (!out) return ASM_ERR_INVALID_ARG;
    *out = nullptr;
    asm_options o;
    asm_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < 0 || o.precision > 2 || o.krylov < 0 || o.krylov > 1 || o.restart < 1 || o.restart > 512 ||
        o.local_solver < 0 || o.local_solver > 4 || o.flexible < -1 || o.flexible > 1 || o.lump_precision < 0 ||
        o.lump_precision > 1 || o.ortho < 0 || o.ortho > 1 ||
        (o.ortho == ASM_ORTHO_CGS && o.restart > kCgsMax - 2) ||
        (o.local_solver == ASM_LOCAL_EXACT && o.precision != ASM_PREC_FP64) ||
        (o.local_solver >= ASM_LOCAL_NF_COLSUM && o.precision == ASM_PREC_FP16S))
        return ASM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    if (o.device < 0 || o.device >= ndev) return ASM_ERR_INVALID_ARG;
    asm_ctx* h = new (std::nothrow) asm_ctx();
    if (!h) return ASM_ERR_OOM;
    h->opt = o;
    h->device = o.device;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->prec = o.precision;
    h->lump32 = o.precision != ASM_PREC_FP64 && o.lump_precision == ASM_LUMP_FP32;
    h->flexible = o.flexible >= 0 ? o.flexible : (o.precision == ASM_PREC_FP64 ? 0 : 1);
    // loads the no-allocation residual's module and kernel now, so that its calls allocate nothing
    int st = guard(h, [&] { return asm2::noalloc_prepare(h->device); });
    if (st) {
        delete h;
        return st;
    }
    *out = h;
    return ASM_OK;
}

int asm_destroy(asm_handle h) {
    if (!h) return ASM_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    delete h;
    return ASM_OK;
}

int asm_set_grid(asm_handle h, int nx, int ny, int nz) {
    if (!h || nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 27)) return ASM_ERR_INVALID_ARG;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->N = nx * ny * nz;
    h->has_grid = true;
    h->has_matrix = false;
    h->sym_valid = false;
    h->factored = false;
    return ASM_OK;
}

int asm_set_matrix_bsr(asm_handle h, int n_cells, int nnzb, const int* row_ptr, const int* col_idx,
                       const double* vals, int on_device) {
    if (!h || !row_ptr || !col_idx || !vals) return ASM_ERR_INVALID_ARG;
    if (!h->has_grid) return ASM_ERR_STATE;
    if (n_cells != h->N || nnzb < n_cells) return ASM_ERR_INVALID_ARG;
    return guard(h, [&]() -> int {
        Pattern P;
        std::string e = build_pattern(n_cells, row_ptr, col_idx, nnzb, P);
        if (!e.empty()) {
            h->last_error = e;
            return e.rfind("pattern", 0) == 0 ? ASM_ERR_PATTERN : ASM_ERR_INVALID_ARG;
        }
        h->pat = std::move(P);
        h->nnzb = nnzb;
        h->d_ell_val.alloc((size_t)h->pat.ell_w * 9 * h->pat.rows_pad * sizeof(double));
        h->d_ell_val.zero(h->stream);
        h->d_ell_col.upload(h->pat.ell_col, h->stream);
        h->d_ell_loc.upload(h->pat.ell_loc, h->stream);
        h->d_bsr_rp.upload(h->pat.rp, h->stream);
        fill_ell(h, vals, on_device);
        sync(h);
        h->has_matrix = true;
        h->sym_valid = false;
        h->factored = false;
        h->ws_m = -1;
        return ASM_OK;
    });
}

int asm_update_values(asm_handle h, const double* vals, int on_device) {
    if (!h || !vals) return ASM_ERR_INVALID_ARG;
    if (!h->has_matrix) return ASM_ERR_STATE;
    return guard(h, [&]() -> int {
        fill_ell(h, vals, on_device);
        sync(h);
        h->factored = false;
        return ASM_OK;
    });
}

int asm_set_partition_boxes(asm_handle h, int px, int py, int pz, int overlap, int near_width, const int* c_near,
                            int far_mode, const int* c_far) {
    if (!h) return ASM_ERR_INVALID_ARG;
    if (!h->has_grid) return ASM_ERR_STATE;
    if (px < 1 || py < 1 || pz < 1 || px > h->nx || py > h->ny || pz > h->nz || overlap < 0 || near_width < 0 ||
        far_mode < 0 || far_mode > 2)
        return ASM_ERR_INVALID_ARG;
    Geom g;
    g.nx = h->nx;
    g.ny = h->ny;
    g.nz = h->nz;
    g.px = px;
    g.py = py;
    g.pz = pz;
    g.ov = overlap;
    g.nw = near_width;
    if (near_width > 0) {
        if (!c_near || c_near[0] < 1 || c_near[1] < 1 || c_near[2] < 1) return ASM_ERR_INVALID_ARG;
        for (int d = 0; d < 3; d++) g.cn[d] = c_near[d];
    }
    g.far_mode = far_mode;
    if (far_mode == ASM_FAR_BOXES) {
        if (!c_far || c_far[0] < 1 || c_far[1] < 1 || c_far[2] < 1) return ASM_ERR_INVALID_ARG;
        for (int d = 0; d < 3; d++) g.cf[d] = c_far[d];
    }
    h->geom = g;
    h->has_partition = true;
    h->sym_valid = false;
    h->factored = false;
    return ASM_OK;
}

int asm_set_coarse_correction(asm_handle h, int mode, const int* c_box) {
    if (!h) return ASM_ERR_INVALID_ARG;
    if (mode < ASM_COARSE_NONE || mode > ASM_COARSE_TWO_STAGE) return ASM_ERR_INVALID_ARG;
    int c[3] = {0, 0, 0};
    if (c_box && (c_box[0] != 0 || c_box[1] != 0 || c_box[2] != 0)) {
        if (c_box[0] < 1 || c_box[1] < 1 || c_box[2] < 1) return ASM_ERR_INVALID_ARG;
        for (int d = 0; d < 3; d++) c[d] = c_box[d];
    }
    if (mode != ASM_COARSE_NONE) {
        if (!h->has_grid || (c[0] == 0 && !h->has_partition)) return ASM_ERR_STATE;
        if (coarse_box_count(h, c) > 1024) return ASM_ERR_INVALID_ARG;
    }
    h->coarse_mode = mode;
    for (int d = 0; d < 3; d++) h->coarse_c[d] = c[d];
    h->coarse_valid = false;
    h->factored = false;
    h->ws_m = -1;
    return ASM_OK;
}

int asm_factor(asm_handle h) {
    if (!h) return ASM_ERR_INVALID_ARG;
    if (!h->has_matrix || !h->has_partition) return ASM_ERR_STATE;
    return guard(h, [&]() -> int {
        h->err_sub = h->err_row = -1;
        if (!h->sym_valid) {
            auto t0 = std::chrono::steady_clock::now();
            h->sym = std::make_shared<SysSym>();
            std::string e = build_symbolic(h->geom, h->pat, h->prec, h->lump32 ? 1 : 0,
                                           h->opt.local_solver == ASM_LOCAL_BILU0_COLSUM ? 1 : 0,
                                           *h->sym, 0, h->chunk_force);
            if (!e.empty()) {
                h->last_error = e;
                h->sym.reset();
                return e.find("pattern") != std::string::npos ? ASM_ERR_PATTERN : ASM_ERR_INVALID_ARG;
            }
            upload_symbolic(h);
            h->sym_valid = true;
            h->coarse_valid = false;
            h->ws_m = -1;
            h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        return factor_numeric(h);
    });
}

// the placement of a single-system apply: `place` as ASM_TUNE_APPLY_SMEM stores it (0 automatic)
ApplyConfig single_apply_config(const asm_ctx* h, int place) {
    return apply_local_vectors((int)h->sub_desc.size(), h->apply_smem, h->apply_lump_smem, h->apply_slots,
                               h->chunk_cap, h->sm_smem, h->n_sms, place, other_slots(h));
}

// R_i r and the fused ILU sweeps of every subdomain (after k_sums), single-system tables
void launch_ilu_local_solves(asm_ctx* h, const ApplyConfig& cfg) {
    launch_restrict(h->d_tab1.as<SysTab>(), h->d_subdesc_single.as<SubDesc>(), h->d_ritems1.as<int2>(), h->n_ritems1,
                    h->prec, h->lump32, h->stream);
    launch_apply(h->d_tab1.as<SysTab>(), h->d_subdesc_single.as<SubDesc>(), (int)h->sub_desc.size(), h->prec,
                 h->lump32, cfg, h->stream);
}

int asm_apply_precond(asm_handle h, const double* r, double* z, int on_device) {
    if (!h || !r || !z) return ASM_ERR_INVALID_ARG;
    if (!h->factored) return ASM_ERR_STATE;
    return guard(h, [&]() -> int {
        ensure_workspace(h);
        const size_t bytes = sizeof(double) * 3 * (size_t)h->N;
        double* in = h->d_ws.as<double>() + (long long)VU * h->n3p;
        double* out = h->d_ws.as<double>() + (long long)VZ * h->n3p;
        copy_in(h, in, r, bytes, on_device);
        set_ctl(h, VU, VZ, -1, -1, -1);
        launch_boxsum(h->d_tab1.as<SysTab>(), h->d_box1.as<BoxItem>(), (int)h->box_items.size(), h->n_group_items,
                      h->stream);
        if (is_nf(h)) {
            launch_nf_apply(h->d_tab1.as<SysTab>(), h->d_nfdesc1.as<NFDesc>(), (int)h->nf_desc.size(), h->prec,
                            h->nf_slots, h->nf_smem, h->stream);
        } else if (h->opt.local_solver == ASM_LOCAL_EXACT) {
            launch_dense_restrict(h->d_tab1.as<SysTab>(), h->d_subdesc_single.as<SubDesc>(), (int)h->sub_desc.size(),
                                  h->stream);
            launch_dense_apply(h->d_tab1.as<SysTab>(), h->d_subdesc_single.as<SubDesc>(), h->d_ditems1.as<int2>(),
                               h->n_ditems1, h->stream);
        } else {
            launch_ilu_local_solves(h, single_apply_config(h, h->apply_place));
        }
        if (h->tab.cmode != 0)
            launch_coarse_apply(h->d_tab1.as<SysTab>(), h->d_row1.as<RowItem>(), h->n_row1,
                                h->d_cbox_items1.as<BoxItem>(), (int)h->cbox_items.size(), h->d_cgrow1.as<RowItem>(),
                                (int)h->cgrow_items.size(), h->d_vec1.as<VecItem>(), h->n_vec1, h->tab.cmode == 2,
                                h->stream);
        ck(cudaGetLastError());
        h->prof.kernel_launches += is_nf(h) ? 2 : 3;
        copy_out(h, z, out, bytes, on_device);
        sync(h);
        return take_dev_err(h) ? ASM_ERR_TIMEOUT : ASM_OK;
    });
}

int asm_tune_tiling(asm_handle h, int reps, asm_tiling_report* out) {
    if (!h || !out || reps < 1) return ASM_ERR_INVALID_ARG;
    if (!h->factored) return ASM_ERR_STATE;
    if (is_nf(h) || h->opt.local_solver == ASM_LOCAL_EXACT) return ASM_ERR_INVALID_ARG;
    *out = asm_tiling_report{};
    return guard(h, [&]() -> int {
        struct Ev {
            cudaEvent_t e = nullptr;
            ~Ev() {
                if (e) cudaEventDestroy(e);
            }
        } ev0, ev1;
        ck(cudaEventCreate(&ev0.e));
        ck(cudaEventCreate(&ev1.e));
        cudaEvent_t e0 = ev0.e, e1 = ev1.e;
        // median time of one apply (box sums, restriction, sweeps) in placement `place`
        auto time_apply = [&](int place) -> double {
            ensure_workspace(h);
            set_ctl(h, VU, VZ, -1, -1, -1);
            const ApplyConfig cfg = single_apply_config(h, place);
            std::vector<float> t;
            for (int k = 0; k < reps + 2; k++) {
                ck(cudaEventRecord(e0, h->stream));
                launch_boxsum(h->d_tab1.as<SysTab>(), h->d_box1.as<BoxItem>(), (int)h->box_items.size(), h->n_group_items,
                      h->stream);
                launch_ilu_local_solves(h, cfg);
                ck(cudaEventRecord(e1, h->stream));
                ck(cudaEventSynchronize(e1));
                float ms = 0.0f;
                ck(cudaEventElapsedTime(&ms, e0, e1));
                if (k >= 2) t.push_back(ms);
            }
            ck(cudaGetLastError());
            std::sort(t.begin(), t.end());
            return t[t.size() / 2];
        };
        auto rebuild = [&](int chunk_bytes) -> int {
            if (h->chunk_force == chunk_bytes && h->sym_valid) return ASM_OK;
            h->chunk_force = chunk_bytes;
            h->sym_valid = false;
            h->factored = false;
            return asm_factor(h);
        };
        const int place0 = h->apply_place, slots0 = h->slots_force, chunk0 = h->chunk_force;
        const bool autotune0 = h->no_autotune;
        // the default configuration first
        h->slots_force = 0;
        int stt = rebuild(0);
        if (stt != ASM_OK) return stt;
        out->rule_ms = time_apply(0);
        std::vector<std::vector<int>> seen;
        for (int kb : {0, 8, 12, 16, 20, 24}) {
            h->slots_force = 0;
            stt = rebuild(kb * 1024);
            if (stt != ASM_OK) return stt;
            std::vector<int> caps;
            long long chunks = 0;
            for (const SubSym& o : h->sym->subs) {
                caps.push_back(o.chunk_cap);
                chunks += (long long)o.chunk_off.size();
            }
            if (std::find(seen.begin(), seen.end(), caps) != seen.end()) continue;
            seen.push_back(caps);
            struct Cand {
                int place, slots;
            };
            std::vector<Cand> cands;
            for (int place : {Y_SMEM + 1, Y_LUMPS + 1, Y_DEVICE + 1})
                for (int sl = 2; sl <= 4; sl++) cands.push_back({place, sl});
            for (const Cand& c : cands) {
                if (out->n >= ASM_TILING_MAX) break;
                h->slots_force = c.slots;
                choose_ring(h);
                const ApplyConfig cfg = single_apply_config(h, c.place);
                if (cfg.ymode != c.place - 1) continue;  // does not fit
                asm_tiling_entry& e = out->e[out->n];
                e.chunk_kb = kb;
                e.chunk_max_kb = h->chunk_cap / 1024;
                e.chunks = chunks;
                e.placement = cfg.ymode == Y_SMEM ? 3 : (cfg.ymode == Y_LUMPS ? 2 : 0);
                e.slots = cfg.slots;
                e.ctas_per_sm = apply_ctas_per_sm(h->prec, h->lump32, cfg);
                e.apply_ms = time_apply(c.place);
                out->n++;
            }
        }
        if (out->n == 0) {
            h->apply_place = place0;
            h->slots_force = slots0;
            h->no_autotune = autotune0;
            stt = rebuild(chunk0);
            return stt != ASM_OK ? stt : ASM_ERR_INVALID_ARG;
        }
        for (int k = 1; k < out->n; k++)
            if (out->e[k].apply_ms < out->e[out->best].apply_ms) out->best = k;
        const asm_tiling_entry& b = out->e[out->best];
        h->slots_force = b.slots;
        stt = rebuild(b.chunk_kb * 1024);
        if (stt != ASM_OK) return stt;
        choose_ring(h);
        h->apply_place = b.placement == 3 ? Y_SMEM + 1 : (b.placement == 2 ? Y_LUMPS + 1 : Y_DEVICE + 1);
        h->no_autotune = true;
        h->tuned_ymode = -1;
        return ASM_OK;
    });
}

int asm_spmv(asm_handle h, const double* x, double* y, int on_device) {
    if (!h || !x || !y) return ASM_ERR_INVALID_ARG;
    if (!h->has_matrix) return ASM_ERR_STATE;
    return guard(h, [&]() -> int {
        if (!h->sym_valid) {
            // SpMV needs only A; give it a workspace without a preconditioner
            h->box_items.clear();
            h->n_group_items = 0;
            if (!h->d_boxsum.p) h->d_boxsum.alloc(16);
        }
        ensure_workspace(h);
        const size_t bytes = sizeof(double) * 3 * (size_t)h->N;
        double* in = h->d_ws.as<double>() + (long long)VU * h->n3p;
        double* out = h->d_ws.as<double>() + (long long)VZ * h->n3p;
        copy_in(h, in, x, bytes, on_device);
        set_ctl(h, -1, -1, VU, VZ, -1);
        launch_spmv(h->d_tab1.as<SysTab>(), h->d_row1.as<RowItem>(), h->n_row1, h->stream);
        ck(cudaGetLastError());
        h->prof.kernel_launches += 1;
        copy_out(h, y, out, bytes, on_device);
        sync(h);
        return ASM_OK;
    });
}

int asm_solve(asm_handle h, const double* b, double* x, double rtol, int max_iter, int on_device,
              asm_solve_info* info) {
    if (!h || !b || !x || !(rtol >= 0.0) || max_iter < 1) return ASM_ERR_INVALID_ARG;
    if (!h->factored) return ASM_ERR_STATE;
    return guard(h, [&]() -> int {
        std::vector<asm_ctx*> hs{h};
        const double* bs[1] = {b};
        double* xs[1] = {x};
        return run_krylov(hs, bs, xs, rtol, max_iter, on_device, info);
    });
}

int asm_solve_batch(asm_handle* hs, int n, const double* const* b, double* const* x, double rtol, int max_iter,
                    int on_device, asm_solve_info* infos) {
    if (!hs || n < 1 || !b || !x || !(rtol >= 0.0) || max_iter < 1) return ASM_ERR_INVALID_ARG;
    std::vector<asm_ctx*> v;
    try {
        v.assign(hs, hs + n);
    } catch (const std::exception&) {
        return ASM_ERR_OOM;
    }
    for (asm_ctx* h : v) {
        if (!h) return ASM_ERR_INVALID_ARG;
        if (!h->factored) return ASM_ERR_STATE;
        if (h->device != v[0]->device || h->stream != v[0]->stream || h->prec != v[0]->prec ||
            h->lump32 != v[0]->lump32 ||
            h->opt.krylov != v[0]->opt.krylov ||
            (h->opt.local_solver == ASM_LOCAL_EXACT) != (v[0]->opt.local_solver == ASM_LOCAL_EXACT) ||
            is_nf(h) != is_nf(v[0]))
            return ASM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; i++)
        for (int k = i + 1; k < n; k++)
            if (v[i] == v[k]) return ASM_ERR_INVALID_ARG;
    return guard(v[0], [&]() -> int { return run_krylov(v, b, x, rtol, max_iter, on_device, infos); });
}

int asm_tune_tiling_batch(asm_handle* hs, int n, const double* const* b, double* const* x, double rtol, int max_iter,
                          int on_device, asm_tiling_report* out) {
    if (!hs || n < 1 || !b || !x || !out || !(rtol >= 0.0) || max_iter < 1) return ASM_ERR_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        if (!hs[i]) return ASM_ERR_INVALID_ARG;
        if (!hs[i]->factored) return ASM_ERR_STATE;
        if (is_nf(hs[i]) || hs[i]->opt.local_solver == ASM_LOCAL_EXACT) return ASM_ERR_INVALID_ARG;
    }
    *out = asm_tiling_report{};
    asm_ctx* h0 = hs[0];
    return guard(h0, [&]() -> int {
        struct Ev {
            cudaEvent_t e = nullptr;
            ~Ev() {
                if (e) cudaEventDestroy(e);
            }
        } ev0, ev1;
        ck(cudaEventCreate(&ev0.e));
        ck(cudaEventCreate(&ev1.e));
        auto set_all = [&](int chunk_bytes) -> int {
            for (int i = 0; i < n; i++) {
                asm_ctx* h = hs[i];
                if (h->chunk_force == chunk_bytes && h->sym_valid && h->factored) continue;
                h->chunk_force = chunk_bytes;
                h->sym_valid = false;
                h->factored = false;
                const int stt = asm_factor(h);
                if (stt != ASM_OK) return stt;
            }
            return ASM_OK;
        };
        // one warm batched solve (its first steps run the online placement tuner), one timed
        auto time_solve = [&]() -> double {
            int stt = asm_solve_batch(hs, n, b, x, rtol, max_iter, on_device, nullptr);
            if (stt != ASM_OK && stt != ASM_ERR_NOT_CONVERGED) throw CudaFail{stt};
            ck(cudaEventRecord(ev0.e, h0->stream));
            stt = asm_solve_batch(hs, n, b, x, rtol, max_iter, on_device, nullptr);
            if (stt != ASM_OK && stt != ASM_ERR_NOT_CONVERGED) throw CudaFail{stt};
            ck(cudaEventRecord(ev1.e, h0->stream));
            ck(cudaEventSynchronize(ev1.e));
            float ms = 0.0f;
            ck(cudaEventElapsedTime(&ms, ev0.e, ev1.e));
            return ms;
        };
        std::vector<std::vector<int>> seen;
        for (int kb : {0, 8, 12, 16, 20, 24}) {
            int stt = set_all(kb * 1024);
            if (stt != ASM_OK) return stt;
            std::vector<int> caps;
            long long chunks = 0;
            int cmax = 0;
            for (int i = 0; i < n; i++) {
                for (const SubSym& o : hs[i]->sym->subs) {
                    caps.push_back(o.chunk_cap);
                    chunks += (long long)o.chunk_off.size();
                }
                cmax = std::max(cmax, hs[i]->chunk_cap);
            }
            if (std::find(seen.begin(), seen.end(), caps) != seen.end()) continue;
            seen.push_back(caps);
            if (out->n >= ASM_TILING_MAX) break;
            const double ms = time_solve();
            if (kb == 0) out->rule_ms = ms;
            asm_tiling_entry& e = out->e[out->n];
            const ApplyConfig& a = h0->last_solve_apply;
            e.chunk_kb = kb;
            e.chunk_max_kb = cmax / 1024;
            e.chunks = chunks;
            e.placement = a.ymode == Y_SMEM ? 3 : (a.ymode == Y_LUMPS ? 2 : 0);
            e.slots = a.slots;
            e.ctas_per_sm = apply_ctas_per_sm(h0->prec, h0->lump32, a);
            e.apply_ms = ms;
            out->n++;
        }
        for (int k = 1; k < out->n; k++)
            if (out->e[k].apply_ms < out->e[out->best].apply_ms) out->best = k;
        return set_all(out->e[out->best].chunk_kb * 1024);
    });
}

int asm_get_stats(asm_handle h, asm_stats* st) {
    if (!h || !st) return ASM_ERR_INVALID_ARG;
    std::memset(st, 0, sizeof(*st));
    st->n_cells = h->N;
    st->matrix_bytes = (long long)h->nnzb * (72 + 4);
    if (h->sym) {
        const SysSym& S = *h->sym;
        st->n_sub = (int)S.subs.size();
        st->local_rows = S.total_rows;
        st->max_local_rows = S.max_n;
        st->max_levels = S.max_lev;
        st->local_blocks = S.total_slots;
        long long fb = 0, ib = 0;
        for (const SubSym& o : S.subs) {
            fb += (long long)o.stream.size();
            ib += o.apply_index_bytes;
        }
        st->factor_bytes = fb;
        st->apply_index_bytes = ib;
        const long long wf = S.prec == 0 ? 8 : (S.prec == 1 ? 4 : 2), wl = S.lump32 ? 4 : 8;
        long long ab = 48LL * h->N;
        for (const SubSym& o : S.subs)
            for (int p = 0; p < o.n; p++) {
                const long long w = p < o.nf ? wf : wl;
                const long long ne = o.prp[p + 1] - o.prp[p] - 1;
                ab += ne * (9 * w + 4) + 9 * w;
            }
        st->alg_apply_bytes = ab;
    }
    st->setup_ms = h->setup_ms;
    st->factor_ms = h->factor_ms;
    if (h->sym && h->sym_valid && !is_nf(h) && h->opt.local_solver != ASM_LOCAL_EXACT) {
        st->chunk_max_kb = h->chunk_cap / 1024;
        for (const SubSym& o : h->sym->subs) st->stream_chunks += (long long)o.chunk_off.size();
        const int place = h->apply_place != 0 ? h->apply_place : (h->tuned_ymode >= 0 ? h->tuned_ymode + 1 : 0);
        const ApplyConfig cfg = single_apply_config(h, place);
        st->apply_placement = cfg.ymode == Y_SMEM ? 3 : (cfg.ymode == Y_LUMPS ? 2 : 0);
        st->apply_slots = cfg.slots;
        const ApplyConfig& l = h->last_solve_apply;
        st->last_solve_placement = l.ymode < 0 ? -1 : (l.ymode == Y_SMEM ? 3 : (l.ymode == Y_LUMPS ? 2 : 0));
        st->last_solve_slots = l.ymode < 0 ? 0 : l.slots;
        st->last_solve_chunk_kb = l.ymode < 0 ? 0 : l.chunk / 1024;
    }
    return ASM_OK;
}

int asm_set_tuning(asm_handle h, int key, int value) {
    if (!h || value < 0) return ASM_ERR_INVALID_ARG;
    if (key == ASM_TUNE_APPLY_SMEM) {
        if (value > 3) return ASM_ERR_INVALID_ARG;
        static const int place[4] = {Y_DEVICE + 1, 0, Y_LUMPS + 1, Y_SMEM + 1};
        h->apply_place = place[value];
        h->tuned_ymode = -1;
    } else if (key == ASM_TUNE_AUTOTUNE) {
        if (value > 1) return ASM_ERR_INVALID_ARG;
        h->no_autotune = value == 0;
        h->tuned_ymode = -1;
    } else if (key == ASM_TUNE_GRAPHS) {
        if (value > 1) return ASM_ERR_INVALID_ARG;
        h->no_graphs = value == 0;
    } else if (key == ASM_TUNE_COOP_ORTHO) {
        if (value > 1) return ASM_ERR_INVALID_ARG;
        h->no_coop = value == 0;
    } else if (key == ASM_TUNE_CHUNK_KB) {
        if (value != 0 && (value % 4 != 0 || value * 1024 < kStreamChunkMin || value * 1024 > kStreamChunkMax))
            return ASM_ERR_INVALID_ARG;
        if (h->chunk_force != value * 1024) {
            h->chunk_force = value * 1024;
            h->sym_valid = false;
            h->factored = false;
        }
    } else if (key == ASM_TUNE_APPLY_SLOTS) {
        if (value != 0 && (value < 2 || value > 4)) return ASM_ERR_INVALID_ARG;
        h->slots_force = value;
        h->tuned_ymode = -1;
        if (h->sym_valid && h->sm_smem > 0) choose_ring(h);
    } else if (key == ASM_TUNE_WAIT_LIMIT) {
        if (value > 30) return ASM_ERR_INVALID_ARG;
        h->wait_limit = value == 0 ? 0 : 1LL << value;
        h->tab.wait_limit = h->wait_limit;
        if (h->d_tab1.p)  // the single-system table already on the device
            return guard(h, [&] {
                ck(cudaMemcpyAsync(h->d_tab1.p, &h->tab, sizeof(SysTab), cudaMemcpyHostToDevice, h->stream));
                sync(h);
                return ASM_OK;
            });
    } else {
        return ASM_ERR_INVALID_ARG;
    }
    return ASM_OK;
}

int asm_set_profiling(asm_handle h, int enable) {
    if (!h) return ASM_ERR_INVALID_ARG;
    h->profiling = enable != 0;
    return ASM_OK;
}

int asm_get_profile(asm_handle h, asm_profile_info* p) {
    if (!h || !p) return ASM_ERR_INVALID_ARG;
    *p = h->prof;
    return ASM_OK;
}

int asm_reset_profile(asm_handle h) {
    if (!h) return ASM_ERR_INVALID_ARG;
    h->prof = asm_profile_info{};
    return ASM_OK;
}

int asm_get_error_location(asm_handle h, int* sub, int* row) {
    if (!h) return ASM_ERR_INVALID_ARG;
    if (sub) *sub = h->err_sub;
    if (row) *row = h->err_row;
    return ASM_OK;
}

int asm_get_local_info(asm_handle h, int s, int* n, int* nnzb, int* counts, int* n_levels) {
    if (!h || !h->sym_valid || s < 0 || s >= (int)h->sym->subs.size()) return ASM_ERR_INVALID_ARG;
    const SubSym& o = h->sym->subs[s];
    if (n) *n = o.n;
    if (nnzb) *nnzb = o.nslot;
    if (counts) {
        counts[0] = o.nf;
        counts[1] = o.nn;
        counts[2] = o.nfar;
    }
    if (n_levels) *n_levels = o.nlev;
    return ASM_OK;
}

int asm_get_local_map(asm_handle h, int s, int* map) {
    if (!h || !map || !h->sym_valid || s < 0 || s >= (int)h->sym->subs.size()) return ASM_ERR_INVALID_ARG;
    try {
        std::vector<int> m;
        local_map(*h->sym, s, m);
        std::memcpy(map, m.data(), m.size() * sizeof(int));
    } catch (const std::exception&) {
        return ASM_ERR_OOM;
    }
    return ASM_OK;
}

int asm_get_local_matrix(asm_handle h, int s, int* row_ptr, int* col_idx, double* vals) {
    if (!h || !h->sym_valid || s < 0 || s >= (int)h->sym->subs.size()) return ASM_ERR_INVALID_ARG;
    const SubSym& o = h->sym->subs[s];
    if (row_ptr) std::memcpy(row_ptr, o.prp.data(), o.prp.size() * sizeof(int));
    if (col_idx) std::memcpy(col_idx, o.pci.data(), o.pci.size() * sizeof(int));
    if (!vals) return ASM_OK;
    return guard(h, [&]() -> int {
        // re-assemble this subdomain's slots into a scratch buffer (the live slots hold factors)
        DBuf tmp;
        tmp.alloc((size_t)o.nslot * 9 * sizeof(double));
        std::vector<int> aptr(o.aptr.begin(), o.aptr.end());
        DBuf dap, dal, dac;
        dap.upload(aptr, h->stream);
        dal.upload(bsr_of_locs(h->pat, o.aloc), h->stream);
        dac.upload(o.acs, h->stream);
        if (h->sym->g.far_mode != 0)
            launch_coarse(h->d_cptr.as<int>(), h->d_cloc.as<int>(), h->d_bsr_val.as<double>(),
                          h->d_cval.as<double>(), h->sym->nC, h->stream);
        launch_assemble(dap.as<int>(), dal.as<int>(), dac.as<int>(), h->d_bsr_val.as<double>(),
                        h->d_cval.as<double>(), tmp.as<double>(), o.nslot, h->stream);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(vals, tmp.p, (size_t)o.nslot * 9 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        sync(h);
        return ASM_OK;
    });
}

int asm_get_local_factors(asm_handle h, int s, double* lu, double* dpiv) {
    if (!h || !h->sym_valid || s < 0 || s >= (int)h->sym->subs.size()) return ASM_ERR_INVALID_ARG;
    if (h->opt.local_solver == ASM_LOCAL_EXACT) return ASM_ERR_INVALID_ARG;  // no ILU factors
    if (is_nf(h) && lu) return ASM_ERR_INVALID_ARG;                          // G blocks only
    if (!h->factored) return ASM_ERR_STATE;
    const SubSym& o = h->sym->subs[s];
    if (is_nf(h)) {
        if (!dpiv) return ASM_OK;
        return guard(h, [&]() -> int {  // G of every box cell, by local row
            std::vector<double> G(9 * (size_t)o.n);
            ck(cudaMemcpyAsync(G.data(), h->d_nfval.as<double>() + h->nf_g_off[s], G.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
            sync(h);
            for (int c = 0; c < o.n; c++)
                std::memcpy(dpiv + 9 * (size_t)h->nf_row_of_cell[s][c], G.data() + 9 * (size_t)c, 9 * sizeof(double));
            return ASM_OK;
        });
    }
    return guard(h, [&]() -> int {
        if (lu)
            ck(cudaMemcpyAsync(lu, h->d_slot.as<double>() + h->slot_base[s] * 9, (size_t)o.nslot * 9 * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
        if (dpiv)
            ck(cudaMemcpyAsync(dpiv, h->d_dpiv.as<double>() + h->row_base[s] * 9, (size_t)o.n * 9 * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
        sync(h);
        return ASM_OK;
    });
}


void asm_server_default_options(asm_server_options* o) {
    if (!o) return;
    o->precision = ASM_PREC_FP32;
    o->restart = 30;
    o->device = 0;
    o->max_active = 64;
    o->max_cached = 16;
    o->hbm_budget = 0;
    o->lump_precision = ASM_LUMP_FP32;
}

int asm_server_create(asm_server_handle* out, const asm_server_options* opt, void* cuda_stream) {
    if (!out) return ASM_ERR_INVALID_ARG;
    *out = nullptr;
    asm_server_options o;
    asm_server_default_options(&o);
    if (opt) o = *opt;
    if (o.precision < 0 || o.precision > 2 || o.restart < 1 || o.restart > 512 || o.max_active < 0 || o.max_cached < 0 ||
        o.hbm_budget < 0 || o.lump_precision < 0 || o.lump_precision > 1)
        return ASM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {  // no driver or no device, as in asm_create
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    if (o.device < 0 || o.device >= ndev) return ASM_ERR_INVALID_ARG;
    if (cudaSetDevice(o.device) != cudaSuccess) {
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    asm_server* S = new (std::nothrow) asm_server();
    if (!S) return ASM_ERR_OOM;
    S->opt = o;
    S->stream = static_cast<cudaStream_t>(cuda_stream);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return ASM_ERR_CUDA;
    }
    S->budget = o.hbm_budget > 0 ? (size_t)o.hbm_budget : (size_t)(0.85 * (double)fr);
    try {
        S->worker = std::thread(sym_worker, S);
    } catch (const std::exception&) {
        delete S;
        return ASM_ERR_OOM;
    }
    *out = S;
    return ASM_OK;
}

int asm_server_submit(asm_server_handle S, const asm_request* q, long long* ticket) {
    if (!S || !q || !ticket || !q->b || !q->row_ptr || !q->col_idx || !q->vals) return ASM_ERR_INVALID_ARG;
    if (q->nx < 1 || q->ny < 1 || q->nz < 1 || (long long)q->nx * q->ny * q->nz != q->n_cells || q->nnzb < q->n_cells ||
        !(q->rtol >= 0.0) || q->max_iter < 1 || q->px < 1 || q->py < 1 || q->pz < 1 || q->px > q->nx ||
        q->py > q->ny || q->pz > q->nz)
        return ASM_ERR_INVALID_ARG;
    // what asm_set_grid and asm_set_partition_boxes refuse, refused before the analysis thread
    // builds the structure from the request
    if (q->n_cells > (1 << 27) || q->overlap < 0 || q->near_width < 0 || q->far_mode < ASM_FAR_NONE ||
        q->far_mode > ASM_FAR_BOXES)
        return ASM_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if ((q->near_width > 0 && q->c_near[d] < 1) || (q->far_mode == ASM_FAR_BOXES && q->c_far[d] < 1))
            return ASM_ERR_INVALID_ARG;
    Req* r = new (std::nothrow) Req();
    if (!r) return ASM_ERR_OOM;
    r->ticket = S->next_ticket;
    r->in = *q;
    r->in.b = nullptr;
    try {  // host memory: on failure nothing of the request stays queued
        r->b.assign(q->b, q->b + 3 * (size_t)q->n_cells);
        S->by_ticket[r->ticket] = r;
        S->pending.push_back(r);
    } catch (const std::exception&) {
        S->by_ticket.erase(r->ticket);
        delete r;
        return ASM_ERR_OOM;
    }
    S->next_ticket++;
    S->st.submitted++;
    *ticket = r->ticket;
    return ASM_OK;
}

int asm_server_progress(asm_server_handle S, int max_steps, int* n_active, int* n_pending) {
    if (!S || max_steps < 0) return ASM_ERR_INVALID_ARG;
    if (cudaSetDevice(S->opt.device) != cudaSuccess) {
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    S->st.progress_calls++;
    try {
        const auto ta = std::chrono::steady_clock::now();
        admit(S);
        S->st.admit_ms += ms_since(ta);
        for (int step = 0; step < max_steps && !S->active.empty(); step++) {
            const auto ts = std::chrono::steady_clock::now();
            const double retire0 = S->st.retire_ms, admit0 = S->st.admit_ms;
            if (S->dirty) {
                S->batch.hs.clear();
                for (Req* r : S->active) S->batch.hs.push_back(r->h);
                build_batch(S->batch, S->stream);
                S->batch.has_init = true;
                S->dirty = false;
            }
            read_ctl(S->batch, S->stream);
            int kmax = -1;
            std::vector<Req*> keep;
            for (size_t k = 0; k < S->active.size(); k++) {
                const int* c = S->batch.pinned + k * C_NCTL;
                if (c[C_PHASE] == PH_DONE) {
                    retire(S, S->active[k], c);
                    S->st.completed++;
                    S->dirty = true;
                    continue;
                }
                keep.push_back(S->active[k]);
                kmax = std::max(kmax, c[C_PHASE] == PH_ARNOLDI ? c[C_J] + 1 : 0);
            }
            if (S->dirty) {  // membership changed: retired systems leave, waiting ones join
                S->active.swap(keep);
                const auto ti = std::chrono::steady_clock::now();
                admit(S);
                S->st.admit_ms += ms_since(ti);
                if (S->active.empty()) break;
                S->batch.hs.clear();
                for (Req* r : S->active) S->batch.hs.push_back(r->h);
                build_batch(S->batch, S->stream);
                S->batch.has_init = true;
                S->dirty = false;
                read_ctl(S->batch, S->stream);
                kmax = -1;
                for (size_t k = 0; k < S->active.size(); k++) {
                    const int* c = S->batch.pinned + k * C_NCTL;
                    if (c[C_PHASE] != PH_DONE) kmax = std::max(kmax, c[C_PHASE] == PH_ARNOLDI ? c[C_J] + 1 : 0);
                }
            }
            launch_step(S->batch, kmax, S->stream, nullptr);
            S->st.steps++;
            S->st.step_ms += ms_since(ts) - (S->st.retire_ms - retire0) - (S->st.admit_ms - admit0);
        }
    } catch (const CudaFail& e) {
        return e.status;
    } catch (const std::bad_alloc&) {
        return ASM_ERR_OOM;
    } catch (const std::exception&) {
        return ASM_ERR_OOM;
    }
    if (n_active) *n_active = (int)S->active.size();
    if (n_pending) *n_pending = (int)S->pending.size();
    S->st.resident_bytes = (long long)S->resident;
    return ASM_OK;
}

int asm_server_result(asm_server_handle S, long long ticket, double* x, asm_solve_info* info) {
    if (!S) return ASM_ERR_INVALID_ARG;
    auto f = S->by_ticket.find(ticket);
    if (f == S->by_ticket.end()) return ASM_ERR_INVALID_ARG;
    Req* r = f->second;
    if (r->state != 2) return ASM_ERR_STATE;
    if (x && !r->x.empty()) std::memcpy(x, r->x.data(), r->x.size() * sizeof(double));
    if (info) *info = r->info;
    const int st = r->info.status;
    S->by_ticket.erase(f);
    delete r;
    return st == ASM_OK || st == ASM_ERR_NOT_CONVERGED ? ASM_OK : st;
}

int asm_server_get_stats(asm_server_handle S, asm_server_stats* out) {
    if (!S || !out) return ASM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);  // the analysis thread adds to analysis_ms
    S->st.resident_bytes = (long long)S->resident;
    S->st.budget_bytes = (long long)S->budget;
    S->st.active = (int)S->active.size();
    S->st.pending = (int)S->pending.size();
    *out = S->st;
    return ASM_OK;
}

int asm_server_destroy(asm_server_handle S) {
    if (!S) return ASM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->quit = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->opt.device);
    for (Req* r : S->active)
        if (r->h) asm_destroy(r->h);
    for (auto& kv : S->idle) asm_destroy(kv.second);
    for (auto& kv : S->by_ticket) delete kv.second;
    delete S;
    return ASM_OK;
}

}  // extern "C"
