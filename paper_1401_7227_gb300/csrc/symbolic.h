// Host symbolic analysis of the two-level additive Schwarz preconditioner: subdomain geometry,
// local patterns, assembly lists, wavefront levels, the factorisation program and the layout of
// the factor streams.  It depends on the grid, the partition and the block pattern of A only, so
// new values of A reuse it (Section 4: the coarsened matrices are rebuilt every non-linear
// iteration, the structure is not).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "asm2_internal.h"

namespace asm2 {

struct Geom {
    int nx = 0, ny = 0, nz = 0;
    int px = 1, py = 1, pz = 1;
    int ov = 0, nw = 0;
    int cn[3] = {1, 1, 1};
    int far_mode = 1;
    int cf[3] = {1, 1, 1};
    int n_cells() const { return nx * ny * nz; }
    int n_sub() const { return px * py * pz; }
};

// Pattern of A (host) and its ELL placement
struct Pattern {
    int n = 0;
    std::vector<int> rp, ci;  // BSR pattern
    int ell_w = 0, rows_pad = 0;
    std::vector<int> ell_loc;  // [nnzb] w * rows_pad + r
    std::vector<int> ell_col;  // [ell_w * rows_pad]
    int find(int r, int c) const;  // block index of (r, c) or -1
};

struct SubSym {
    int n = 0, nf = 0, nn = 0, nfar = 0, nlev = 0, nslot = 0;
    int chunk_cap = 0;    // capacity of this subdomain's stream chunks (kStreamChunkMin .. Max)
    // local pattern by local row, slot = CSR position
    std::vector<int> prp, pci, pdiag;
    // assembly: slot value = C[acs] (if >= 0) + sum of signed ELL blocks aloc[aptr[s] .. aptr[s+1])
    std::vector<int> aptr, aloc, acs;
    // rows <-> positions (level order), levels as position ranges
    std::vector<int> row_of_pos, pos_of_row, lv_pos0;
    // factorisation program
    std::vector<int> tgt_lv, tgt, pp, ls_lv, diag_of_pos;
    std::vector<int> pair;  // (L slot, U slot) interleaved
    std::vector<int> ls;    // (L slot, diag slot) interleaved
    // fine index / lump index of every local row (-1 in the other space)
    std::vector<int> fidx_of_row, cidx_of_row;
    // restriction: fcell by fine index; lump rows by lump index (rptr/rsrc/rbox), clong = lump
    // rows with long lists; owned-cell scatter (own_pos = fine index)
    std::vector<int> fcell, rptr, rsrc, rbox, clong, own_pos, own_cell;
    // Sum lists (rsrc, corr_cells, and SysSym::bsum) hold cells (>= 0) and cell groups (~g < 0):
    // an aligned 2 x 2 x 2 group whose cells inside the grid all belong to the list stands for
    // them; its sum is formed once per apply (cell_group()).
    // far lumps: rcorr = index of the lump's correction list (or -1); corr_ptr/corr_cells = the
    // near-region cells of each far box, summed by a gather pass and subtracted from the box sum
    std::vector<int> rcorr, corr_ptr, corr_cells;
    // factor stream: chunks (byte offset, size) in consumption order; the first n_fwd_chunks
    // belong to the forward sweep
    std::vector<LevelInfo> lv;
    std::vector<long long> chunk_off;
    std::vector<int> chunk_bytes;
    int n_fwd_chunks = 0;
    std::vector<unsigned char> stream;  // indices filled in, values zero
    std::vector<long long> pk_off_f, pk_off_c;
    std::vector<int> pk_src_f, pk_src_c;
    // cell -> local row over the whole grid is not stored; map_region gives it for parity hooks
    std::vector<int> cells_of_row_ptr, cells_of_row;  // fine cell or lump cells, by local row
    long long apply_index_bytes = 0;
};

struct SysSym {
    Geom g;
    int prec = 0;  // element size class of the fine-row values: 0 f64, 1 f32, 2 f16
    int lump32 = 0;  // lump-row values stored in FP32 (else FP64)
    int colsum = 1;
    int chunk_force = 0;  // stream-chunk capacity asked for (bytes; 0: each subdomain's own rule)
    // far boxes
    int nboxes = 0;
    std::vector<int> farbox;     // [N]
    std::vector<int> bptr, bcell;
    std::vector<int> bsum_ptr, bsum;  // each far box's cells as a sum list (cells and cell groups)
    // coarse (far-box) coupling matrix C: blocks summed over box pairs
    int nC = 0;
    std::vector<int> cptr, cloc;
    std::vector<SubSym> subs;
    int max_n = 0, max_lev = 0;
    long long total_rows = 0, total_slots = 0;
};

// Builds the whole symbolic structure; returns "" or an error message.  prec: 0 f64, 1 f32,
// 2 f16 element storage of fine-row factors; lump32: lump-row factors stored in FP32 (else FP64);
// colsum: compensation on/off.  threads <= 0: auto.  chunk_force: 0, or the stream-chunk capacity
// in bytes (a multiple of 4096 in [kStreamChunkMin, kStreamChunkMax]) for every subdomain, raised
// where one row needs more.
std::string build_symbolic(const Geom& g, const Pattern& A, int prec, int lump32, int colsum, SysSym& out,
                           int threads, int chunk_force = 0);

// Aligned 2 x 2 x 2 cell groups: group of a cell, group count, and a group's cells in the grid
// (x, y, z each in {2 g, 2 g + 1} within the grid; z fastest, as cells are numbered)
inline int group_dims(int n) { return (n + 1) / 2; }
inline int cell_group(const Geom& g, int c) {
    const int z = c % g.nz, t = c / g.nz, x = t % g.nx, y = t / g.nx;
    return (z >> 1) + group_dims(g.nz) * ((x >> 1) + group_dims(g.nx) * (y >> 1));
}
inline int n_groups(const Geom& g) { return group_dims(g.nx) * group_dims(g.ny) * group_dims(g.nz); }

// local row of every cell for subdomain s (-1 = outside), from the stored lists
void local_map(const SysSym& S, int s, std::vector<int>& map);

std::string build_pattern(int n, const int* rp, const int* ci, int nnzb, Pattern& P);

}  // namespace asm2
