// Host symbolic analysis (see symbolic.h).
//
// Geometry (Section 4, Eq. 4.1, Figs. 2-3): subdomain s owns a box of the px*py*pz partition;
// its fine set F is that box grown by `ov` cells; near lumps are the cn-sized aligned boxes that
// meet the ring of width nw around F, minus F; far lumps are the far boxes minus F and the near
// lumps.  Local rows: fine cells by cell index, then near lumps, then far lumps, by box index.
//
// Only the near region N = F + near-lump cells is enumerated per subdomain, so the analysis costs
// O(|N|) per subdomain instead of O(N_cells).  A far-far block of A_s = R_s A R_s^T (Eq. 3.4) is
// the block of the global far-box matrix C (all couplings between two far boxes) minus the
// couplings that touch N; every other block is a short signed list of blocks of A.
#include "symbolic.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <thread>
#include <unordered_map>

namespace asm2 {

namespace {

inline int split_lo(int n, int p, int t) { return (int)((long long)n * t / p); }
// lump rows whose restriction list is longer than this are summed by a whole warp
constexpr int kLongList = 16;
// largest factor-stream chunk (one shared-memory ring slot of the apply)
inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Box {
    int lo[3], hi[3];  // x, y, z; half-open
    bool empty() const { return lo[0] >= hi[0] || lo[1] >= hi[1] || lo[2] >= hi[2]; }
    bool has(int x, int y, int z) const {
        return x >= lo[0] && x < hi[0] && y >= lo[1] && y < hi[1] && z >= lo[2] && z < hi[2];
    }
};

Box owned_box(const Geom& g, int s) {
    const int tz = s % g.pz, tx = (s / g.pz) % g.px, ty = s / (g.pz * g.px);
    Box b;
    b.lo[0] = split_lo(g.nx, g.px, tx);
    b.hi[0] = split_lo(g.nx, g.px, tx + 1);
    b.lo[1] = split_lo(g.ny, g.py, ty);
    b.hi[1] = split_lo(g.ny, g.py, ty + 1);
    b.lo[2] = split_lo(g.nz, g.pz, tz);
    b.hi[2] = split_lo(g.nz, g.pz, tz + 1);
    return b;
}

Box grow(const Geom& g, Box b, int w) {
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; d++) {
        b.lo[d] = std::max(0, b.lo[d] - w);
        b.hi[d] = std::min(n[d], b.hi[d] + w);
    }
    return b;
}

Box meet(const Box& a, const Box& b) {
    Box r;
    for (int d = 0; d < 3; d++) {
        r.lo[d] = std::max(a.lo[d], b.lo[d]);
        r.hi[d] = std::min(a.hi[d], b.hi[d]);
    }
    return r;
}

bool inside(const Box& a, const Box& b) {  // a within b (a non-empty)
    for (int d = 0; d < 3; d++)
        if (a.lo[d] < b.lo[d] || a.hi[d] > b.hi[d]) return false;
    return true;
}

inline int cell_of(const Geom& g, int x, int y, int z) { return z + g.nz * (x + g.nx * y); }

// cells of group G inside the grid
int group_size(const Geom& g, int G) {
    const int gz = G % group_dims(g.nz), t = G / group_dims(g.nz), gx = t % group_dims(g.nx), gy = t / group_dims(g.nx);
    return std::min(2, g.nx - 2 * gx) * std::min(2, g.ny - 2 * gy) * std::min(2, g.nz - 2 * gz);
}

// Appends the sum list of a set of distinct cells to out: every group whose cells in the grid all
// belong to the set becomes one entry ~G, at the place of its first cell in `cells`; the other
// cells stay, in their order.  cnt / done: scratch of n_groups(g) entries, zero on entry and exit.
void append_sum_list(const Geom& g, const int* cells, int n, std::vector<int>& out, std::vector<int>& cnt,
                     std::vector<char>& done) {
    for (int i = 0; i < n; i++) cnt[cell_group(g, cells[i])]++;
    for (int i = 0; i < n; i++) {
        const int G = cell_group(g, cells[i]);
        if (cnt[G] == group_size(g, G)) {
            if (!done[G]) out.push_back(~G);
            done[G] = 1;
        } else {
            out.push_back(cells[i]);
        }
    }
    for (int i = 0; i < n; i++) {
        const int G = cell_group(g, cells[i]);
        cnt[G] = 0;
        done[G] = 0;
    }
}

struct Tup {
    int p, q, v;  // kind: 0 plus (v = ELL loc), 1 minus (v = ELL loc), 2 coarse (v = C slot)
    int kind;
    bool operator<(const Tup& o) const { return p != o.p ? p < o.p : q < o.q; }
};

int find_in(const int* b, const int* e, int q) {
    const int* it = std::lower_bound(b, e, q);
    return (it != e && *it == q) ? (int)(it - b) : -1;
}

struct Ctx {
    const Geom& g;
    const Pattern& A;
    const SysSym& S;
    int prec, colsum;
    std::vector<long long> ckey;  // sorted unique far-box pair keys of C
};

std::string build_sub(const Ctx& X, int s, SubSym& o) {
    const Geom& g = X.g;
    const Pattern& A = X.A;
    const SysSym& S = X.S;
    const bool far = g.far_mode != 0;

    const Box own = owned_box(g, s);
    const Box F = grow(g, own, g.ov);
    const Box outer = grow(g, F, g.nw);
    Box G = F;
    if (g.nw > 0) {
        const int n[3] = {g.nx, g.ny, g.nz};
        for (int d = 0; d < 3; d++) {
            G.lo[d] = (outer.lo[d] / g.cn[d]) * g.cn[d];
            G.hi[d] = std::min(n[d], ((outer.hi[d] + g.cn[d] - 1) / g.cn[d]) * g.cn[d]);
        }
    }
    const int gx = G.hi[0] - G.lo[0], gy = G.hi[1] - G.lo[1], gz = G.hi[2] - G.lo[2];
    std::vector<int> gmap((size_t)gx * gy * gz, -1);
    auto gidx = [&](int x, int y, int z) { return (size_t)(z - G.lo[2]) + (size_t)gz * ((x - G.lo[0]) + (size_t)gx * (y - G.lo[1])); };

    // fine cells, ascending cell index
    std::vector<int> rowcells_ptr(1, 0), rowcells;
    int idx = 0;
    for (int y = F.lo[1]; y < F.hi[1]; y++)
        for (int x = F.lo[0]; x < F.hi[0]; x++)
            for (int z = F.lo[2]; z < F.hi[2]; z++) {
                gmap[gidx(x, y, z)] = idx++;
                rowcells.push_back(cell_of(g, x, y, z));
                rowcells_ptr.push_back((int)rowcells.size());
            }
    o.nf = idx;
    // near lumps: aligned boxes meeting the ring outer \ F, in box-index order
    if (g.nw > 0) {
        const int cx = g.cn[0], cy = g.cn[1], cz = g.cn[2];
        for (int by = G.lo[1] / cy; by * cy < G.hi[1]; by++)
            for (int bx = G.lo[0] / cx; bx * cx < G.hi[0]; bx++)
                for (int bz = G.lo[2] / cz; bz * cz < G.hi[2]; bz++) {
                    Box B = {{bx * cx, by * cy, bz * cz},
                             {std::min(g.nx, (bx + 1) * cx), std::min(g.ny, (by + 1) * cy), std::min(g.nz, (bz + 1) * cz)}};
                    Box I = meet(B, outer);
                    if (I.empty() || inside(I, F)) continue;
                    for (int y = B.lo[1]; y < B.hi[1]; y++)
                        for (int x = B.lo[0]; x < B.hi[0]; x++)
                            for (int z = B.lo[2]; z < B.hi[2]; z++)
                                if (!F.has(x, y, z)) {
                                    gmap[gidx(x, y, z)] = idx;
                                    rowcells.push_back(cell_of(g, x, y, z));
                                }
                    rowcells_ptr.push_back((int)rowcells.size());
                    idx++;
                }
    }
    o.nn = idx - o.nf;
    const int nN = idx;  // rows of the near region
    // far lumps: boxes with cells outside the near region
    std::vector<int> flump;
    std::vector<int> far_box_of_row;
    std::vector<std::vector<int>> corr;  // cells of box J inside the near region
    if (far) {
        flump.assign(S.nboxes, -1);
        std::vector<int> cntN(S.nboxes, 0);
        for (int c : rowcells) cntN[S.farbox[c]]++;
        for (int J = 0; J < S.nboxes; J++)
            if (S.bptr[J + 1] - S.bptr[J] > cntN[J]) {
                flump[J] = idx++;
                far_box_of_row.push_back(J);
            }
        corr.resize(S.nboxes);
        for (int c : rowcells)
            if (flump[S.farbox[c]] >= 0) corr[S.farbox[c]].push_back(c);
        for (auto& v : corr) std::sort(v.begin(), v.end());
    }
    o.nfar = idx - nN;
    o.n = idx;
    const int n = o.n;
    auto lmap = [&](int c) -> int {
        const int z = c % g.nz, x = (c / g.nz) % g.nx, y = c / (g.nz * g.nx);
        if (G.has(x, y, z)) {
            int v = gmap[gidx(x, y, z)];
            if (v >= 0) return v;
        }
        return far ? flump[S.farbox[c]] : -1;
    };

    // entries of A_s
    std::vector<Tup> T;
    T.reserve((size_t)rowcells.size() * 10);
    std::unordered_map<long long, int> cntE2;
    const long long NB = S.nboxes;
    for (int p = 0; p < nN; p++) {
        for (int t = rowcells_ptr[p]; t < rowcells_ptr[p + 1]; t++) {
            const int a = rowcells[t];
            for (int e = A.rp[a]; e < A.rp[a + 1]; e++) {
                const int b = A.ci[e];
                const int q = lmap(b);
                const bool bN = q >= 0 && q < nN;
                int e2 = -1;
                if (q >= 0) {
                    T.push_back({p, q, A.ell_loc[e], 0});
                    if (!bN) {
                        e2 = A.find(b, a);
                        if (e2 < 0) return "pattern not structurally symmetric";
                        T.push_back({q, p, A.ell_loc[e2], 0});
                    }
                }
                if (far) {
                    const int Ja = S.farbox[a], Jb = S.farbox[b];
                    if (flump[Ja] >= 0 && flump[Jb] >= 0) {
                        T.push_back({flump[Ja], flump[Jb], A.ell_loc[e], 1});
                        cntE2[Ja * NB + Jb]++;
                        if (!bN) {
                            if (e2 < 0) e2 = A.find(b, a);
                            if (e2 < 0) return "pattern not structurally symmetric";
                            T.push_back({flump[Jb], flump[Ja], A.ell_loc[e2], 1});
                            cntE2[Jb * NB + Ja]++;
                        }
                    }
                }
            }
        }
    }
    if (far) {
        for (int c = 0; c < S.nC; c++) {
            const long long key = X.ckey[c];
            const int J = (int)(key / NB), Jp = (int)(key % NB);
            if (flump[J] < 0 || flump[Jp] < 0) continue;
            auto it = cntE2.find(key);
            const int e2 = it == cntE2.end() ? 0 : it->second;
            if (S.cptr[c + 1] - S.cptr[c] > e2) T.push_back({flump[J], flump[Jp], c, 2});
        }
    }
    std::stable_sort(T.begin(), T.end());

    // slots
    o.prp.assign(n + 1, 0);
    o.aptr.assign(1, 0);
    for (size_t i = 0; i < T.size();) {
        size_t j = i;
        bool has_c = false, has_minus = false;
        int cs = -1;
        while (j < T.size() && T[j].p == T[i].p && T[j].q == T[i].q) {
            if (T[j].kind == 2) {
                has_c = true;
                cs = T[j].v;
            }
            if (T[j].kind == 1) has_minus = true;
            j++;
        }
        if (!has_minus || has_c) {
            o.pci.push_back(T[i].q);
            o.prp[T[i].p + 1]++;
            o.acs.push_back(cs);
            for (size_t k = i; k < j; k++) {
                if (T[k].kind == 0) o.aloc.push_back(T[k].v);
                if (T[k].kind == 1) o.aloc.push_back(~T[k].v);
            }
            o.aptr.push_back((int)o.aloc.size());
        }
        i = j;
    }
    for (int p = 0; p < n; p++) o.prp[p + 1] += o.prp[p];
    o.nslot = (int)o.pci.size();
    o.pdiag.assign(n, -1);
    for (int p = 0; p < n; p++) {
        o.pdiag[p] = find_in(o.pci.data() + o.prp[p], o.pci.data() + o.prp[p + 1], p);
        if (o.pdiag[p] < 0) return "local matrix without a diagonal block";
        o.pdiag[p] += o.prp[p];
    }
    auto slot = [&](int p, int q) -> int {
        int k = find_in(o.pci.data() + o.prp[p], o.pci.data() + o.prp[p + 1], q);
        return k < 0 ? -1 : o.prp[p] + k;
    };
    for (int p = 0; p < n; p++)
        for (int t = o.prp[p]; t < o.prp[p + 1]; t++)
            if (slot(o.pci[t], p) < 0) return "local pattern not structurally symmetric";

    // Wavefront levels of the DAG of L (the same sets, reversed, serve U), every row at the earliest
    // level its dependencies allow: the lump rows then run in the same levels as the fine
    // rows they follow instead of after the last of them, which shortens the chain of levels (and
    // of CTA barriers) by about a fifth at 1M cells.  Any level assignment that respects the DAG
    // gives the same arithmetic.
    std::vector<int> level(n, 0);
    int nlev = 0;
    for (int p = 0; p < n; p++) {
        int l = 0;
        for (int t = o.prp[p]; t < o.pdiag[p]; t++) l = std::max(l, level[o.pci[t]] + 1);
        level[p] = l;
        nlev = std::max(nlev, l + 1);
    }
    if (n == 0) nlev = 0;
    o.nlev = nlev;
    std::vector<int> cntf(nlev, 0), cntc(nlev, 0);
    for (int p = 0; p < n; p++) (p < o.nf ? cntf : cntc)[level[p]]++;
    o.lv_pos0.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; l++) o.lv_pos0[l + 1] = o.lv_pos0[l] + cntf[l] + cntc[l];
    o.row_of_pos.assign(n, 0);
    o.pos_of_row.assign(n, 0);
    {
        std::vector<int> nf_fill(nlev, 0), nc_fill(nlev, 0);
        for (int p = 0; p < n; p++) {
            const int l = level[p];
            const int pos = p < o.nf ? o.lv_pos0[l] + nf_fill[l]++ : o.lv_pos0[l] + cntf[l] + nc_fill[l]++;
            o.row_of_pos[pos] = p;
            o.pos_of_row[p] = pos;
        }
    }

    // factorisation program: the right-looking loop of block ILU(0), recorded as pairs per target
    std::vector<int> npair(o.nslot, 0);
    for (int pass = 0; pass < 2; pass++) {
        std::vector<int> fill;
        if (pass == 1) {
            o.pp.clear();
        }
        std::vector<int> start(o.nslot + 1, 0);
        if (pass == 1) {
            for (int t = 0; t < o.nslot; t++) start[t + 1] = start[t] + npair[t];
            o.pair.assign(2 * (size_t)start[o.nslot], 0);
            fill.assign(o.nslot, 0);
        }
        for (int k = 0; k < n; k++) {
            for (int tq = o.pdiag[k] + 1; tq < o.prp[k + 1]; tq++) {
                const int q = o.pci[tq];
                for (int tp = o.pdiag[k] + 1; tp < o.prp[k + 1]; tp++) {
                    const int p = o.pci[tp];
                    int tgt = slot(p, q);
                    if (tgt < 0) {
                        if (!X.colsum) continue;
                        tgt = o.pdiag[q];
                    }
                    if (pass == 0) {
                        npair[tgt]++;
                    } else {
                        const size_t w = (size_t)start[tgt] + fill[tgt]++;
                        o.pair[2 * w] = slot(p, k);
                        o.pair[2 * w + 1] = tq;
                    }
                }
            }
        }
        if (pass == 1) {
            // group targets by the level of the pivot that finalises them
            std::vector<int> slot_row(o.nslot);
            for (int p = 0; p < n; p++)
                for (int t = o.prp[p]; t < o.prp[p + 1]; t++) slot_row[t] = p;
            std::vector<std::vector<int>> by_lev(nlev);
            for (int t = 0; t < o.nslot; t++)
                if (npair[t] > 0) by_lev[level[std::min(slot_row[t], o.pci[t])]].push_back(t);
            std::vector<int> pair2;
            o.tgt_lv.assign(1, 0);
            o.pp.assign(1, 0);
            o.tgt.clear();
            for (int l = 0; l < nlev; l++) {
                for (int t : by_lev[l]) {
                    o.tgt.push_back(t);
                    for (int q = start[t]; q < start[t + 1]; q++) {
                        pair2.push_back(o.pair[2 * (size_t)q]);
                        pair2.push_back(o.pair[2 * (size_t)q + 1]);
                    }
                    o.pp.push_back((int)(pair2.size() / 2));
                }
                o.tgt_lv.push_back((int)o.tgt.size());
            }
            o.pair.swap(pair2);
        }
    }
    o.ls_lv.assign(1, 0);
    o.ls.clear();
    for (int l = 0; l < nlev; l++) {
        for (int pos = o.lv_pos0[l]; pos < o.lv_pos0[l + 1]; pos++) {
            const int k = o.row_of_pos[pos];
            for (int tp = o.pdiag[k] + 1; tp < o.prp[k + 1]; tp++) {
                o.ls.push_back(slot(o.pci[tp], k));
                o.ls.push_back(o.pdiag[k]);
            }
        }
        o.ls_lv.push_back((int)(o.ls.size() / 2));
    }
    o.diag_of_pos.assign(n, 0);
    for (int pos = 0; pos < n; pos++) o.diag_of_pos[pos] = o.pdiag[o.row_of_pos[pos]];

    // fine and lump rows get separate index spaces (fine index / lump index, both in level order),
    // so the apply can keep them in separate local vectors of their own precision
    o.fidx_of_row.assign(n, -1);
    o.cidx_of_row.assign(n, -1);
    {
        int nfi = 0, nci = 0;
        for (int pos = 0; pos < n; pos++) {
            const int p = o.row_of_pos[pos];
            if (p < o.nf)
                o.fidx_of_row[p] = nfi++;
            else
                o.cidx_of_row[p] = nci++;
        }
    }
    // restriction: fine rows copy one cell; lump rows sum their cells (far lumps: box sum minus the
    // near-region cells of the box)
    o.fcell.assign(o.nf, 0);
    for (int p = 0; p < o.nf; p++) o.fcell[o.fidx_of_row[p]] = rowcells[rowcells_ptr[p]];
    const int nc = n - o.nf;
    std::vector<int> row_of_c(nc);
    for (int p = o.nf; p < n; p++) row_of_c[o.cidx_of_row[p]] = p;
    // near lumps: their cells; far lumps: box sum minus the sum of the box's near-region cells,
    // the latter gathered by a separate pass over corr_cells
    o.rptr.assign(1, 0);
    o.rsrc.clear();
    o.rbox.assign(nc, -1);
    o.rcorr.assign(nc, -1);
    o.clong.clear();
    o.corr_ptr.assign(1, 0);
    o.corr_cells.clear();
    static thread_local std::vector<int> gcnt;
    static thread_local std::vector<char> gdone;
    gcnt.assign(n_groups(g), 0);
    gdone.assign(n_groups(g), 0);
    for (int c = 0; c < nc; c++) {
        const int p = row_of_c[c];
        if (p < nN) {
            append_sum_list(g, rowcells.data() + rowcells_ptr[p], rowcells_ptr[p + 1] - rowcells_ptr[p], o.rsrc, gcnt,
                            gdone);
        } else {
            const int J = far_box_of_row[p - nN];
            o.rbox[c] = J;
            if (!corr[J].empty()) {
                o.rcorr[c] = (int)o.corr_ptr.size() - 1;
                append_sum_list(g, corr[J].data(), (int)corr[J].size(), o.corr_cells, gcnt, gdone);
                o.corr_ptr.push_back((int)o.corr_cells.size());
            }
        }
        o.rptr.push_back((int)o.rsrc.size());
        if (o.rptr[c + 1] - o.rptr[c] > kLongList) o.clong.push_back(c);
    }
    o.own_pos.clear();
    o.own_cell.clear();
    for (int y = own.lo[1]; y < own.hi[1]; y++)
        for (int x = own.lo[0]; x < own.hi[0]; x++)
            for (int z = own.lo[2]; z < own.hi[2]; z++) {
                o.own_cell.push_back(cell_of(g, x, y, z));
                o.own_pos.push_back(o.fidx_of_row[gmap[gidx(x, y, z)]]);
            }
    o.apply_index_bytes = 4LL * ((long long)o.fcell.size() + (long long)o.rptr.size() + (long long)o.rsrc.size() + 2LL * nc +
                                 (long long)o.clong.size() + 2LL * o.own_pos.size() + (long long)o.corr_cells.size() +
                                 (long long)o.corr_ptr.size());
    o.cells_of_row_ptr = rowcells_ptr;
    o.cells_of_row = rowcells;
    for (int J : far_box_of_row) o.cells_of_row.push_back(-1 - J);  // far rows: -1 - box

    // Factor stream: self-contained chunks of at most o.chunk_cap, each holding rows of one wavefront
    // level (fine rows at the factor precision, lump rows in FP64 or FP32): all forward chunks in level
    // order, then all backward chunks in reverse level order -- the order the apply consumes them,
    // so the stream is read front to back.  Chunk layout (every array 16-byte aligned):
    //   header int[8] = {f0, nf, c0, nc, nef, nec, flags, bytes}; flags: bit 0 = last chunk of
    //   the level, bits 8..11 = log2 of the short lump rows' entry slots
    //   fptr[nf+1] fcol[nef] fval[nef blocks] (fdinv[nf blocks]) cptr[nc+1] ccol[nec] cval[nec] (cdinv[nc])
    // Columns: fine index (>= 0) or ~lump index.
    const size_t fbb = X.prec == 0 ? 72 : (X.prec == 1 ? 36 : 20);  // FP64 / FP32 / FP16 + exponent
    const size_t lbb = X.S.lump32 ? 36 : 72;                            // lump rows: FP32 / FP64
    struct Piece {
        int lv, pos_f, nf, pos_c, nc;
        bool fwd, last;
    };
    std::vector<Piece> pieces;
    auto nl = [&](int p) { return o.pdiag[p] - o.prp[p]; };
    auto nu = [&](int p) { return o.prp[p + 1] - o.pdiag[p] - 1; };
    auto chunk_bytes = [&](int nf_, int ef, int nc_, int ec, bool fwd) {
        size_t b = 32 + al16(4 * (size_t)(nf_ + 1)) + al16(4 * (size_t)ef) + al16(fbb * ef) + al16(4 * (size_t)(nc_ + 1)) +
                   al16(4 * (size_t)ec) + al16(lbb * (size_t)ec);
        if (!fwd) b += al16(fbb * nf_) + al16(lbb * (size_t)nc_);
        return b;
    };
    // chunk capacity: the largest fine level (forward or backward part) and the longest single lump
    // row in one chunk, rounded up to 4 KB, within [kStreamChunkMin, kStreamChunkMax] (fewer chunks
    // mean fewer barriers in the apply; larger ring slots mean fewer CTAs per SM, so small
    // subdomains keep the smallest capacity).  A capacity asked for (the tiling tuner's) replaces
    // the level term; every single row must still fit.
    {
        size_t big = 0, one = 0;
        for (int l = 0; l < nlev; l++)
            for (int pass = 0; pass < 2; pass++) {
                int ef = 0;
                for (int pos = o.lv_pos0[l]; pos < o.lv_pos0[l] + cntf[l]; pos++) {
                    const int e = pass == 0 ? nl(o.row_of_pos[pos]) : nu(o.row_of_pos[pos]);
                    ef += e;
                    one = std::max(one, chunk_bytes(1, e, 0, 0, pass == 0) + 256);
                }
                big = std::max(big, chunk_bytes(cntf[l], ef, 0, 0, pass == 0) + 256);
            }
        for (int p = o.nf; p < n; p++)
            for (int pass = 0; pass < 2; pass++) {
                const size_t b = chunk_bytes(0, 0, 1, pass == 0 ? nl(p) : nu(p), pass == 0);
                big = std::max(big, b);
                one = std::max(one, b);
            }
        if (X.S.chunk_force > 0) big = std::max(one, (size_t)X.S.chunk_force);
        const size_t cap = (big + 4095) / 4096 * 4096;
        o.chunk_cap = (int)std::min<size_t>(asm2::kStreamChunkMax, std::max<size_t>(asm2::kStreamChunkMin, cap));
    }
    const size_t kChunkBytes = (size_t)o.chunk_cap;
    for (int pass = 0; pass < 2; pass++) {
        const bool fwd = pass == 0;
        for (int li = 0; li < nlev; li++) {
            const int l = fwd ? li : nlev - 1 - li;
            const int p0 = o.lv_pos0[l], pf_end = o.lv_pos0[l] + cntf[l], pc_end = o.lv_pos0[l + 1];
            int pf = p0, pc = pf_end;
            while (pf < pf_end || pc < pc_end) {
                Piece pc_{l, pf, 0, pc, 0, fwd, false};
                int ef = 0, ec = 0;
                while (pf < pf_end) {
                    const int p = o.row_of_pos[pf];
                    const int e = fwd ? nl(p) : nu(p);
                    if (chunk_bytes(pc_.nf + 1, ef + e, 0, 0, fwd) > kChunkBytes - 256) break;
                    ef += e;
                    pc_.nf++;
                    pf++;
                }
                if (pf == pf_end) {
                    while (pc < pc_end) {
                        const int p = o.row_of_pos[pc];
                        const int e = fwd ? nl(p) : nu(p);
                        if (chunk_bytes(pc_.nf, ef, pc_.nc + 1, ec + e, fwd) > kChunkBytes) break;
                        ec += e;
                        pc_.nc++;
                        pc++;
                    }
                }
                if (pc_.nf == 0 && pc_.nc == 0) return "a single row does not fit in a stream chunk";
                pc_.last = pf == pf_end && pc == pc_end;
                pieces.push_back(pc_);
            }
        }
    }
    // fine index / lump index of the first row of each position range
    std::vector<int> fidx_pos(n + 1, 0), cidx_pos(n + 1, 0);
    for (int pos = 0; pos < n; pos++) {
        const int p = o.row_of_pos[pos];
        fidx_pos[pos + 1] = fidx_pos[pos] + (p < o.nf ? 1 : 0);
        cidx_pos[pos + 1] = cidx_pos[pos] + (p < o.nf ? 0 : 1);
    }
    size_t total = 0;
    o.chunk_off.clear();
    o.chunk_bytes.clear();
    o.n_fwd_chunks = 0;
    for (const Piece& pc_ : pieces) {
        int ef = 0, ec = 0;
        for (int k = 0; k < pc_.nf; k++) ef += pc_.fwd ? nl(o.row_of_pos[pc_.pos_f + k]) : nu(o.row_of_pos[pc_.pos_f + k]);
        for (int k = 0; k < pc_.nc; k++) ec += pc_.fwd ? nl(o.row_of_pos[pc_.pos_c + k]) : nu(o.row_of_pos[pc_.pos_c + k]);
        const size_t bytes = chunk_bytes(pc_.nf, ef, pc_.nc, ec, pc_.fwd);
        o.chunk_off.push_back((long long)total);
        o.chunk_bytes.push_back((int)bytes);
        if (pc_.fwd) o.n_fwd_chunks++;
        total += bytes;
    }
    o.stream.assign(total, 0);
    o.pk_off_f.clear();
    o.pk_off_c.clear();
    o.pk_src_f.clear();
    o.pk_src_c.clear();
    auto put_rows = [&](size_t& w, int pos_b, int cnt, bool lower, size_t bb, bool with_dinv, bool fine_group) {
        int* ptr = reinterpret_cast<int*>(o.stream.data() + w);
        int ne = 0;
        ptr[0] = 0;
        for (int k = 0; k < cnt; k++) {
            const int p = o.row_of_pos[pos_b + k];
            ne += lower ? nl(p) : nu(p);
            ptr[k + 1] = ne;
        }
        w += al16(4 * (size_t)(cnt + 1));
        int* col = reinterpret_cast<int*>(o.stream.data() + w);
        size_t vw = w + al16(4 * (size_t)ne);
        int e = 0;
        for (int k = 0; k < cnt; k++) {
            const int p = o.row_of_pos[pos_b + k];
            const int tb = lower ? o.prp[p] : o.pdiag[p] + 1, te = lower ? o.pdiag[p] : o.prp[p + 1];
            for (int t = tb; t < te; t++, e++) {
                const int q = o.pci[t];
                col[e] = q < o.nf ? o.fidx_of_row[q] : ~o.cidx_of_row[q];
                (fine_group ? o.pk_off_f : o.pk_off_c).push_back((long long)(vw + bb * e));
                (fine_group ? o.pk_src_f : o.pk_src_c).push_back(t);
            }
        }
        w = vw + al16(bb * ne);
        if (with_dinv) {
            for (int k = 0; k < cnt; k++) {
                (fine_group ? o.pk_off_f : o.pk_off_c).push_back((long long)(w + bb * k));
                (fine_group ? o.pk_src_f : o.pk_src_c).push_back(o.diag_of_pos[pos_b + k]);
            }
            w += al16(bb * (size_t)cnt);
        }
        return ne;
    };
    // Entry slots of the short lump rows of a chunk.  A row split over S slots costs
    // 3 ceil(len / S) FMAs plus log2(S) shuffle-adds per lane, and 32 / (3 S) rows share a warp;
    // groups of rows go to warps 7, 6, ..., so groups g and g + 4 share an SM sub-partition, whose
    // FP64 pipe issues one warp instruction at a time.  S minimises the FP64 instructions of the
    // busiest sub-partition (the sweep is latency-bound: these instructions are its critical path).
    auto lump_slots_log2 = [&](const Piece& pc_) {
        int rows = 0, len = 0;
        for (int k = 0; k < pc_.nc; k++) {
            const int p = o.row_of_pos[pc_.pos_c + k];
            const int e = pc_.fwd ? nl(p) : nu(p);
            if (e <= asm2::kLongLumpRow) {
                rows++;
                len = std::max(len, e);
            }
        }
        int best = 0;
        long long best_cost = -1;
        for (int lg = 0; lg <= 3; lg++) {
            const int S = 1 << lg, rpw = 32 / (3 * S);
            const long long groups = (rows + rpw - 1) / rpw, per_smsp = (groups + 3) / 4;
            const long long cost = per_smsp * (3LL * ((len + S - 1) / S) + lg);
            if (best_cost < 0 || cost < best_cost) {
                best_cost = cost;
                best = lg;
            }
        }
        return best;
    };
    for (size_t i = 0; i < pieces.size(); i++) {
        const Piece& pc_ = pieces[i];
        size_t w = (size_t)o.chunk_off[i];
        int* hdr = reinterpret_cast<int*>(o.stream.data() + w);
        w += 32;
        const int ef = put_rows(w, pc_.pos_f, pc_.nf, pc_.fwd, fbb, !pc_.fwd, true);
        const int ec = put_rows(w, pc_.pos_c, pc_.nc, pc_.fwd, lbb, !pc_.fwd, false);
        hdr[0] = fidx_pos[pc_.pos_f];
        hdr[1] = pc_.nf;
        hdr[2] = cidx_pos[pc_.pos_c];
        hdr[3] = pc_.nc;
        hdr[4] = ef;
        hdr[5] = ec;
        bool has_long = false;
        for (int k = 0; k < pc_.nc; k++) {
            const int p = o.row_of_pos[pc_.pos_c + k];
            has_long = has_long || (pc_.fwd ? nl(p) : nu(p)) > asm2::kLongLumpRow;
        }
        hdr[6] = (pc_.last ? 1 : 0) | (lump_slots_log2(pc_) << 8) | (has_long ? asm2::kChunkLongLumps : 0);
        hdr[7] = o.chunk_bytes[i];
        if (w != (size_t)o.chunk_off[i] + (size_t)o.chunk_bytes[i]) return "stream chunk layout mismatch";
    }
    o.lv.clear();
    return "";
}

}  // namespace

int Pattern::find(int r, int c) const {
    const int* b = ci.data() + rp[r];
    const int* e = ci.data() + rp[r + 1];
    int k = find_in(b, e, c);
    return k < 0 ? -1 : rp[r] + k;
}

std::string build_pattern(int n, const int* rp, const int* ci, int nnzb, Pattern& P) {
    if (n < 1 || nnzb < n) return "bad sizes";
    if (rp[0] != 0 || rp[n] != nnzb) return "row_ptr does not span col_idx";
    // all of row_ptr first: a row that ends past nnzb must not be read
    for (int r = 0; r < n; r++)
        if (rp[r + 1] < rp[r] || rp[r + 1] > nnzb) return "row_ptr not monotone";
    P.n = n;
    P.rp.assign(rp, rp + n + 1);
    P.ci.assign(ci, ci + nnzb);
    int w = 0;
    for (int r = 0; r < n; r++) {
        w = std::max(w, rp[r + 1] - rp[r]);
        bool diag = false;
        for (int e = rp[r]; e < rp[r + 1]; e++) {
            if (ci[e] < 0 || ci[e] >= n) return "column index out of range";
            if (e > rp[r] && ci[e] <= ci[e - 1]) return "columns not strictly ascending in a row";
            if (ci[e] == r) diag = true;
        }
        if (!diag) return "pattern: missing diagonal block";
    }
    for (int r = 0; r < n; r++)
        for (int e = rp[r]; e < rp[r + 1]; e++)
            if (P.find(ci[e], r) < 0) return "pattern: not structurally symmetric";
    P.ell_w = w;
    P.rows_pad = (n + 63) / 64 * 64;
    // ELL locations w * rows_pad + r are int (the kernels index the values in 64 bits)
    if ((long long)w * P.rows_pad > (long long)INT_MAX) return "too large: the longest row times the rows";
    P.ell_loc.assign(nnzb, 0);
    P.ell_col.assign((size_t)w * P.rows_pad, 0);
    for (int r = 0; r < P.rows_pad; r++)
        for (int k = 0; k < w; k++) P.ell_col[(size_t)k * P.rows_pad + r] = r < n ? r : 0;
    for (int r = 0; r < n; r++)
        for (int e = rp[r]; e < rp[r + 1]; e++) {
            const int k = e - rp[r];
            P.ell_loc[e] = k * P.rows_pad + r;
            P.ell_col[(size_t)k * P.rows_pad + r] = ci[e];
        }
    return "";
}

std::string build_symbolic(const Geom& g, const Pattern& A, int prec, int lump32, int colsum, SysSym& S,
                           int threads, int chunk_force) {
    const int N = g.n_cells();
    if (A.n != N) return "matrix size does not match the grid";
    if (chunk_force != 0 &&
        (chunk_force % 4096 != 0 || chunk_force < asm2::kStreamChunkMin || chunk_force > asm2::kStreamChunkMax))
        return "stream chunk capacity out of range";
    S = SysSym();
    S.g = g;
    S.prec = prec;
    S.lump32 = prec != 0 && lump32 ? 1 : 0;
    S.colsum = colsum;
    S.chunk_force = chunk_force;
    const int K = g.n_sub();
    if (g.far_mode != 0) {
        S.farbox.assign(N, 0);
        std::vector<int> tx(g.nx), ty(g.ny), tz(g.nz);
        if (g.far_mode == 1) {
            for (int t = 0; t < g.px; t++)
                for (int i = split_lo(g.nx, g.px, t); i < split_lo(g.nx, g.px, t + 1); i++) tx[i] = t;
            for (int t = 0; t < g.py; t++)
                for (int i = split_lo(g.ny, g.py, t); i < split_lo(g.ny, g.py, t + 1); i++) ty[i] = t;
            for (int t = 0; t < g.pz; t++)
                for (int i = split_lo(g.nz, g.pz, t); i < split_lo(g.nz, g.pz, t + 1); i++) tz[i] = t;
            S.nboxes = K;
            for (int y = 0; y < g.ny; y++)
                for (int x = 0; x < g.nx; x++)
                    for (int z = 0; z < g.nz; z++) S.farbox[cell_of(g, x, y, z)] = tz[z] + g.pz * (tx[x] + g.px * ty[y]);
        } else {
            const int nbx = (g.nx + g.cf[0] - 1) / g.cf[0], nby = (g.ny + g.cf[1] - 1) / g.cf[1],
                      nbz = (g.nz + g.cf[2] - 1) / g.cf[2];
            S.nboxes = nbx * nby * nbz;
            for (int y = 0; y < g.ny; y++)
                for (int x = 0; x < g.nx; x++)
                    for (int z = 0; z < g.nz; z++)
                        S.farbox[cell_of(g, x, y, z)] = z / g.cf[2] + nbz * (x / g.cf[0] + nbx * (y / g.cf[1]));
        }
        S.bptr.assign(S.nboxes + 1, 0);
        for (int c = 0; c < N; c++) S.bptr[S.farbox[c] + 1]++;
        for (int b = 0; b < S.nboxes; b++) S.bptr[b + 1] += S.bptr[b];
        S.bcell.assign(N, 0);
        {
            std::vector<int> fill(S.bptr.begin(), S.bptr.end() - 1);
            for (int c = 0; c < N; c++) S.bcell[fill[S.farbox[c]]++] = c;
        }
        {
            std::vector<int> cnt(n_groups(g), 0);
            std::vector<char> done(n_groups(g), 0);
            S.bsum_ptr.assign(1, 0);
            S.bsum.clear();
            for (int b = 0; b < S.nboxes; b++) {
                append_sum_list(g, S.bcell.data() + S.bptr[b], S.bptr[b + 1] - S.bptr[b], S.bsum, cnt, done);
                S.bsum_ptr.push_back((int)S.bsum.size());
            }
        }
    }
    Ctx X{g, A, S, prec, colsum, {}};
    if (g.far_mode != 0) {
        const long long NB = S.nboxes;
        std::vector<std::pair<long long, int>> kv;
        kv.reserve(A.ci.size());
        for (int a = 0; a < N; a++)
            for (int e = A.rp[a]; e < A.rp[a + 1]; e++) kv.push_back({S.farbox[a] * NB + S.farbox[A.ci[e]], e});
        std::sort(kv.begin(), kv.end());
        S.cptr.assign(1, 0);
        S.cloc.resize(kv.size());
        for (size_t i = 0; i < kv.size(); i++) {
            if (i > 0 && kv[i].first != kv[i - 1].first) {
                S.cptr.push_back((int)i);
            }
            if (i == 0 || kv[i].first != kv[i - 1].first) X.ckey.push_back(kv[i].first);
            S.cloc[i] = A.ell_loc[kv[i].second];
        }
        S.cptr.push_back((int)kv.size());
        S.nC = (int)X.ckey.size();
    }
    S.subs.resize(K);
    std::vector<std::string> err(K);
    if (threads <= 0) threads = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    threads = std::min(threads, K);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (;;) {
            int s = next.fetch_add(1);
            if (s >= K) break;
            err[s] = build_sub(X, s, S.subs[s]);
        }
    };
    std::vector<std::thread> pool;
    try {
        for (int t = 1; t < threads; t++) pool.emplace_back(worker);
    } catch (const std::exception&) {
        // no more threads to be had: the ones that started and this one share the subdomains
    }
    worker();
    for (auto& t : pool) t.join();
    for (int s = 0; s < K; s++)
        if (!err[s].empty()) return err[s];
    for (auto& sb : S.subs) {
        S.max_n = std::max(S.max_n, sb.n);
        S.max_lev = std::max(S.max_lev, sb.nlev);
        S.total_rows += sb.n;
        S.total_slots += sb.nslot;
    }
    return "";
}

void local_map(const SysSym& S, int s, std::vector<int>& map) {
    const SubSym& o = S.subs[s];
    const int N = S.g.n_cells();
    map.assign(N, -1);
    const int nN = o.nf + o.nn;
    for (int p = nN; p < o.n; p++) {
        const int J = -1 - o.cells_of_row[o.cells_of_row_ptr[nN] + (p - nN)];
        for (int i = S.bptr[J]; i < S.bptr[J + 1]; i++) map[S.bcell[i]] = p;
    }
    for (int p = 0; p < nN; p++)
        for (int t = o.cells_of_row_ptr[p]; t < o.cells_of_row_ptr[p + 1]; t++) map[o.cells_of_row[t]] = p;
}

}  // namespace asm2
