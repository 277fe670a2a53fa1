// Test-only host shim: runs the library's symbolic analysis (symbolic.cpp) on the CPU, without a
// GPU, and hands its lists to the CPU tests.  The tests check them against the oracle (local maps,
// patterns, the assembled A_i = R_i A R_i^T of Eq. 4.1) and against the rules the sweeps rely on
// (wavefront levels, stream chunks, the pack map).  Not part of the library.
#include <cstring>
#include <string>
#include <vector>

#include "symbolic.h"

using namespace asm2;

namespace {

struct Handle {
    Pattern pat;
    SysSym sym;
};

template <class T>
long long put(const std::vector<T>& v, void* out) {
    if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(T));
    return (long long)v.size();
}

// ELL location (w * rows_pad + r, ~ for a subtracted block) -> BSR block index (same sign code)
std::vector<int> to_bsr(const Pattern& P, const std::vector<int>& locs) {
    std::vector<int> out(locs.size());
    for (size_t i = 0; i < locs.size(); i++) {
        const bool neg = locs[i] < 0;
        const int L = neg ? ~locs[i] : locs[i];
        const int w = L / P.rows_pad, r = L - w * P.rows_pad;
        out[i] = neg ? ~(P.rp[r] + w) : P.rp[r] + w;
    }
    return out;
}

}  // namespace

extern "C" {

// geo = {nx, ny, nz, px, py, pz, ov, near_width, cn[3], far_mode, cf[3]}; lump32: lump-row
// factors in FP32 (FP32/FP16 fine rows only); chunk_force: stream-chunk capacity in bytes (0: the
// per-subdomain rule); NULL on error (message in err)
void* hs_create(const int* geo, int n, int nnzb, const int* rp, const int* ci, int prec, int lump32, int colsum,
                char* err, int errlen, int chunk_force) {
    Geom g;
    g.nx = geo[0];
    g.ny = geo[1];
    g.nz = geo[2];
    g.px = geo[3];
    g.py = geo[4];
    g.pz = geo[5];
    g.ov = geo[6];
    g.nw = geo[7];
    for (int d = 0; d < 3; d++) g.cn[d] = geo[8 + d];
    g.far_mode = geo[11];
    for (int d = 0; d < 3; d++) g.cf[d] = geo[12 + d];
    Handle* h = new Handle();
    std::string e = build_pattern(n, rp, ci, nnzb, h->pat);
    if (e.empty()) e = build_symbolic(g, h->pat, prec, lump32, colsum, h->sym, 0, chunk_force);
    if (!e.empty()) {
        std::strncpy(err, e.c_str(), (size_t)errlen - 1);
        err[errlen - 1] = 0;
        delete h;
        return nullptr;
    }
    return h;
}

void hs_destroy(void* p) { delete static_cast<Handle*>(p); }

// build_pattern alone: "" or its error message (for the input checks of asm_set_matrix_bsr)
int hs_check_pattern(int n, int nnzb, const int* rp, const int* ci, char* err, int errlen) {
    Pattern P;
    const std::string e = build_pattern(n, rp, ci, nnzb, P);
    std::strncpy(err, e.c_str(), (size_t)errlen - 1);
    err[errlen - 1] = 0;
    return e.empty() ? 0 : 1;
}

// copies the list `what` of subdomain s (s = -1: of the system) into out (if not NULL); returns
// its length, or -1 for an unknown name.  int32 lists unless noted: chunk_off int64, stream bytes.
long long hs_get(void* p, int s, const char* what, void* out) {
    const Handle& h = *static_cast<Handle*>(p);
    const std::string w = what;
    if (s < 0) {
        if (w == "n_sub") return put(std::vector<int>{(int)h.sym.subs.size()}, out);
        if (w == "cptr") return put(h.sym.cptr, out);
        if (w == "cloc") return put(to_bsr(h.pat, h.sym.cloc), out);
        if (w == "ell_shape") return put(std::vector<int>{h.pat.ell_w, h.pat.rows_pad}, out);
        if (w == "ell_loc") return put(h.pat.ell_loc, out);
        if (w == "ell_col") return put(h.pat.ell_col, out);
        if (w == "bsum_ptr") return put(h.sym.bsum_ptr, out);
        if (w == "bsum") return put(h.sym.bsum, out);
        return -1;
    }
    const SubSym& o = h.sym.subs[s];
    if (w == "info") return put(std::vector<int>{o.n, o.nf, o.nn, o.nfar, o.nslot, o.nlev, o.chunk_cap, o.n_fwd_chunks}, out);
    if (w == "map") {
        std::vector<int> m;
        local_map(h.sym, s, m);
        return put(m, out);
    }
    if (w == "prp") return put(o.prp, out);
    if (w == "pci") return put(o.pci, out);
    if (w == "pdiag") return put(o.pdiag, out);
    if (w == "aptr") return put(o.aptr, out);
    if (w == "aloc") return put(to_bsr(h.pat, o.aloc), out);
    if (w == "acs") return put(o.acs, out);
    if (w == "row_of_pos") return put(o.row_of_pos, out);
    if (w == "lv_pos0") return put(o.lv_pos0, out);
    if (w == "fidx_of_row") return put(o.fidx_of_row, out);
    if (w == "cidx_of_row") return put(o.cidx_of_row, out);
    if (w == "chunk_off") return put(o.chunk_off, out);
    if (w == "chunk_bytes") return put(o.chunk_bytes, out);
    if (w == "stream") return put(o.stream, out);
    if (w == "pk_off_f") return put(o.pk_off_f, out);
    if (w == "pk_src_f") return put(o.pk_src_f, out);
    if (w == "pk_off_c") return put(o.pk_off_c, out);
    if (w == "pk_src_c") return put(o.pk_src_c, out);
    if (w == "rptr") return put(o.rptr, out);
    if (w == "rsrc") return put(o.rsrc, out);
    if (w == "rbox") return put(o.rbox, out);
    if (w == "rcorr") return put(o.rcorr, out);
    if (w == "corr_ptr") return put(o.corr_ptr, out);
    if (w == "corr_cells") return put(o.corr_cells, out);
    return -1;
}

}  // extern "C"
