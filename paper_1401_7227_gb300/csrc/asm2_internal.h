// Internal declarations shared by the host runtime and the CUDA kernels of libasm2.
//
// Everything on the device is described by small tables of absolute pointers, so one kernel
// launch can work on any mix of systems: a single solve is a batch of one system.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace asm2 {

// ---------------------------------------------------------------------------------------------
// Krylov workspace layout.  Each system owns one device block of vectors of n3p doubles
// (n3 = 3 * n_cells rounded up to VEC_CHUNK), addressed by slot number.
// ---------------------------------------------------------------------------------------------
constexpr int VEC_CHUNK = 4096;   // elements per vector work item (256 threads x 16)
// bytes of one factor-stream chunk (= one shared-memory ring slot of the apply): chosen per subdomain
// so that its largest fine level fits one chunk, within [kStreamChunkMin, kStreamChunkMax]
constexpr int kStreamChunkMin = 8192, kStreamChunkMax = 24576;
constexpr int kLongLumpRow = 16;     // lump rows with more stored blocks are swept by a whole warp
// The apply runs one 256-thread CTA per subdomain.  With all its local vectors in shared memory
// one or two CTAs fit on an SM; with the fine-row vector in device memory (L1/L2) four fit, which
// wins once a launch has more subdomains than the shared-memory variant runs at once.  The lump
// vector (and, for FP64 lump rows, its FP32 mirror) then stays in shared memory when four CTAs'
// worth fit, else it goes to device memory too.
constexpr int kApplyThreadsDev = 256;
enum ApplyY { Y_SMEM = 0, Y_LUMPS = 1, Y_DEVICE = 2 };  // where the apply's local vectors live
struct ApplyConfig {
    int ymode;  // ApplyY
    int smem;   // dynamic shared memory of the vectors (bytes)
    int slots;  // factor-stream ring slots (2..4; the tiling tuner measured deeper rings slower)
    int chunk;  // bytes of one ring slot: the largest chunk capacity of the launch's subdomains
};
// Chunk header word 6: bit 0 = last chunk of its wavefront level; bits 8..11 = log2 of the entry
// slots S of the short lump rows (each such row takes 3 S lanes: 3 output components x S slots);
// kChunkLongLumps = the chunk holds a lump row of more than kLongLumpRow blocks.
constexpr int kChunkLongLumps = 1 << 12;
constexpr int VEC_THREADS = 256;
constexpr int kCgsMax = 64;  // classical Gram-Schmidt: at most kCgsMax - 2 basis vectors (restart)
enum VecSlot { VX = 0, VB = 1, VR = 2, VW = 3, VZ = 4, VU = 5, VV0 = 6 };  // V_k = VV0 + k; Z_k after V

// GMRES phases of one system
enum Phase { PH_DONE = 0, PH_ARNOLDI = 1, PH_RESTART = 2, PH_INIT = 3, PH_OM = 4, PH_OM_FINAL = 5 };
// PH_OM: one ORTHOMIN direction (apply, mat-vec, projections, update); PH_OM_FINAL: true residual.

// Per-system control words (device, int32), written by the state kernels.
enum Ctl {
    C_PHASE = 0,
    C_J,          // Arnoldi index j of the step in progress
    C_JEND,       // columns of H used by the pending update
    C_ITERS,      // preconditioned mat-vecs so far
    C_RESTARTS,
    C_STATUS,     // asm_status of the system
    C_CONVERGED,
    C_APPLY_IN,   // vector slot fed to the preconditioner (-1: skip the apply)
    C_APPLY_OUT,
    C_SPMV_IN,    // vector slot of the SpMV input (-1: skip)
    C_SPMV_OUT,
    C_SPMV_B,     // slot of b for y = b - A x, or -1 for y = A x
    C_MAXIT,
    C_CNT_RED,    // arrival counter of the chunk reduction in flight
    C_CNT_FIN,    // arrival counter of the finishing kernel
    C_BREAKDOWN,
    C_OM_STORED,  // ORTHOMIN: directions held (at most k)
    C_OM_SLOT,    // ORTHOMIN: ring slot of the direction in progress (0 .. k)
    C_NCTL = 20
};

// Per-system scalars (device, double) at fixed offsets; H is (m+1) x m row-major.
struct ScalLayout {
    int bnorm, beta, tol, w0, hn, red0, red1, H, cs, sn, g, y, om_qq, om_beta, om_alpha, n;
    __host__ __device__ static ScalLayout make(int m) {
        ScalLayout L;
        int o = 0;
        L.bnorm = o++;
        L.beta = o++;
        L.tol = o++;
        L.w0 = o++;
        L.hn = o++;
        L.red0 = o++;
        L.red1 = o++;
        L.H = o;
        o += (m + 1) * m;
        L.cs = o;
        o += m;
        L.sn = o;
        o += m;
        L.g = o;
        o += m + 1;
        L.y = o;
        o += m;
        L.om_qq = o;  // ORTHOMIN: (q_s, q_s) of every ring slot
        o += m + 1;
        L.om_beta = o;  // ORTHOMIN: projection coefficients of the step in progress
        o += m;
        L.om_alpha = o++;
        L.n = o;
        return L;
    }
};

// Per-system table (device copy).  Pointers are absolute.
struct SysTab {
    double* ws;          // vector workspace base (slots of n3p doubles)
    long long n3p;       // padded vector length
    int n3;              // 3 * n_cells
    int n_cells;
    int m;               // GMRES restart length, or ORTHOMIN direction count k
    int flexible;        // keep Z_k = B^{-1} V_k (slots after V)
    int krylov;          // asm_krylov: 0 GMRES (slots V_k, Z_k), 1 ORTHOMIN (slots P_s, then Q_s)
    int ortho;           // asm_ortho: 0 modified, 1 classical Gram-Schmidt (single-system GMRES)
    int nchunk;          // vector work items of this system
    double* scal;        // scalars (ScalLayout)
    int* ctl;            // control words (Ctl)
    double* partial;     // [2 * nchunk] chunk partial sums
    // A in ELL form: slot w, element t of row r at ell_val[(w*9 + t) * rows_pad + r]
    const double* ell_val;
    const int* ell_col;  // [w * rows_pad + r]; padding slots point at r with zero values
    int ell_w;
    int rows_pad;
    // preconditioner
    double* boxsum;      // [n_boxes * 3] far-box sums of the apply input
    double* corr;        // [n_corr * 3] near-region sums subtracted from far-lump box sums
    double* gsum;        // [n_groups * 3] sums of the apply input over aligned 2x2x2 cell groups
    float4* r32;         // [n_cells] the apply input rounded to FP32 (written with gsum), or null
    int gnx, gny, gnz;   // grid size (for the cells of a group)
    int* dev_err;        // device status word: nonzero after a bounded wait expired
    long long wait_limit;  // polls of the first wait on each factor-stream copy of the apply kernels
    // classical coarse-grid correction (0 none, 1 two-level, 2 two-stage; Eqs. 3.5-3.8)
    int cmode;
    int cnb;             // coarse boxes
    const int* cbox;     // [n_cells] coarse box of each cell
    const double* caug;  // [3 cnb][6 cnb]: the right half holds A_C^{-1}
    double* crc;         // [3 cnb] R_C x
    double* cyc;         // [3 cnb] A_C^{-1} R_C x
    double* cw;          // [3 n_cells] two-stage residual r - A z
};

// Work items
struct VecItem {   // VEC_CHUNK elements [e0, e0 + VEC_CHUNK) of system sys; chunk index within system
    int sys, chunk;
};
struct RowItem {   // rows [r0, r0 + 256) of system sys
    int sys, r0;
};
// kind 0 / 1: sum over the sum list cells[b0 .. b1) (cells >= 0 and cell groups ~g) of the apply
// input into boxsum[out] / corr[out]; kind 2: the group sums gsum of groups b0 .. b1 - 1 (these
// items come first and run in their own launch, before the lists that read them)
struct BoxItem {
    int sys, out, b0, b1;
    int kind, pad_;
    const int* cells;
};

// One wavefront level of a local factor: its nf fine rows have fine indices f0 .. f0+nf-1 and
// its nc lump rows lump indices c0 .. c0+nc-1.  Forward/backward segments are byte offsets into
// the subdomain's factor stream; every array inside a segment starts on a 16-byte boundary.
// A stored column is a fine index (>= 0) or ~lump index (< 0).
struct LevelInfo {
    int f0, nf, c0, nc;
    int eLf, eLc, eUf, eUc;
    long long fwd_off, bwd_off;
};

// One subdomain work item of the preconditioner apply.
struct SubDesc {
    int sys;
    int nf;           // fine rows
    int nc;           // lump rows
    int n_chunks;     // factor-stream chunks (forward then backward)
    int n_fwd;        // forward chunks
    int n_own;
    int n_long;       // lump rows restricted by a whole warp
    int corr0;        // first correction sum of this subdomain in SysTab::corr
    int chunk_cap;    // bytes of this subdomain's ring slots (its largest chunk fits one)
    const double* dinv;          // exact local solves: [A_i | A_i^{-1}] (3n x 6n), fine then lump order
    const int2* chunks;          // (byte offset, bytes) of every chunk, consumption order
    const unsigned char* stream; // 16-byte aligned
    double* y;        // the local vectors in device memory (written by k_restrict, 16-byte aligned)
    int y_fine;       // byte offsets within y: fine rows, and the FP32 mirror of FP64 lumps; lumps at 0
    int y_mirror;
    int y_bytes;      // bytes of all local vectors (the shared-memory copy of Y_SMEM)
    const int* fcell; // [nf] cell of each fine row
    const int* rptr;  // [nc + 1] cells summed into each near lump (far lumps: empty)
    const int* rsrc;
    const int* rbox;  // [nc] far box whose sum is the far lump's base, or -1
    const int* rcorr; // [nc] correction sum subtracted from it (index from corr0), or -1
    const int* clong; // [n_long] lump rows with long source lists
    const int* own_pos;  // fine index of each owned cell
    const int* own_cell;
};

// One subdomain work item of the numeric factorisation (slot values in FP64).
struct FactDesc {
    int sys;
    int nlev;
    int n;
    int pad_;
    double* slot;           // [nslot * 9] assembled values, factored in place
    double* dpiv;           // [n * 9] final pivot blocks, by local row
    const int* lv_pos0;     // [nlev + 1] position ranges of the levels
    const int* diag_of_pos; // [n] slot of the diagonal block of each position
    const int* row_of_pos;  // [n]
    const int* tgt_lv;      // [nlev + 1] ranges into tgt
    const int* tgt;         // target slots finalised at each level
    const int* pp;          // [ntgt + 1] pair ranges
    const int2* pair;       // (L slot, U slot) to subtract, in the right-looking update order
    const int* ls_lv;       // [nlev + 1] ranges into ls
    const int2* ls;         // (L slot, diagonal slot of its column): L = A * D^{-1}
};

// Device error record of the factorisation (first singular pivot)
struct FactErr {
    int flag, sub, row, pad_;
};

// One subdomain of the nested-factorisation local solver (Appendix A): a local problem without
// lumps, i.e. the box of bx * by * bz fine cells, local cell p = z + bz (x + bx y).
struct NFDesc {
    int sys;
    int sub;          // subdomain index (error location)
    int bx, by, bz, n;
    int colsum;       // Eq. A.7 (1) or Eq. A.6 alone (0)
    int n_own;
    int c0, gnz, gnx;    // grid cell of local (0, 0, 0); cell of (x, y, z) = c0 + z + gnz (x + gnx y)
    int own_lo[3], own_hi[3];  // the owned box in local (x, y, z)
    int line_bytes;      // one line packet of the apply (nf_line_bytes)
    const double* slot;  // the subdomain's assembled blocks of A_i (9 doubles each)
    const int* bands;    // [7 n]: slot of D, L1, U1, L2, U2, L3, U3 in cell p's row, or -1
    double* g;           // [9 n] the diagonal blocks G
    double* gi;          // [9 n] their inverses
    double* work;        // nf_work_doubles(bx, by, bz) doubles of scratch (factorisation)
    void* fband;         // [7 n] the band blocks of each cell, compute type (factorisation)
    void* pack;          // [by * bx] line packets (16-byte aligned), compute type
    void* yv;            // [by] planes of the apply's forward result, nf_plane_bytes(bx bz) apart
};

// ---------------------------------------------------------------------------------------------
// Kernel launchers (kernels.cu)
// ---------------------------------------------------------------------------------------------
// slot values of the local matrices from the array-of-blocks copy of A (lists of BSR block indices,
// ~index for a subtracted block); slots whose lists hold kLongAssembly or more blocks are
// summed by a warp each (long_slots, nlong; null: every slot by the per-element kernel)
constexpr int kLongAssembly = 32;
void launch_assemble(const int* aptr, const int* aloc, const int* acs, const double* bsr_val, const double* cval,
                     double* slot, long long nslot, cudaStream_t st, const int* long_slots = nullptr, int nlong = 0);
void launch_coarse(const int* cptr, const int* cloc, const double* bsr_val, double* cval, int nc, cudaStream_t st);
void launch_factor(const FactDesc* fd, int nsub, FactErr* err, const int* sub_ids, cudaStream_t st);
void launch_pack(const long long* off, const int* src, long long n, int prec, unsigned char* stream_base,
                 const double* slot_base, cudaStream_t st);
void launch_ell_fill(const double* bsr_vals, const int* row_ptr, int n, int ell_w, double* ell_val, int rows_pad,
                     cudaStream_t st);

// items[0 .. ngroup): group-sum items (kind 2), then the box and correction sums
void launch_boxsum(const SysTab* st_tab, const BoxItem* items, int nitems, int ngroup, cudaStream_t st);
// ysmem: shared memory for the local vectors (0 = they stay in the global scratch SubDesc.y);
// the ring of factor-stream slots is added on top
void launch_apply(const SysTab* st_tab, const SubDesc* subs, int nsub, int prec, bool lump32, ApplyConfig cfg,
                  cudaStream_t st);
// CTAs of that apply launch resident per SM (0 when it cannot launch)
int apply_ctas_per_sm(int prec, bool lump32, ApplyConfig cfg);
// R_i r of every subdomain into its device-memory local vectors (items: subdomain, first local row
// of 256; fine rows first, then lump rows)
void launch_restrict(const SysTab* tab, const SubDesc* subs, const int2* items, int nitems, int prec, bool lump32,
                     cudaStream_t st);
// shared memory the local vectors of a subdomain need (nf fine rows, nc lump rows), and the ring
// Layout of one subdomain's apply local vectors (the same in device and in shared memory): lumps at
// byte 0 (FP64, or FP32 with lump32), fine rows at `fine` (FP64 with FP64 factors, else FP32), and
// the FP32 mirror of FP64 lumps under FP32/FP16 fine rows at `mirror`; every part 16-byte aligned.
// With FP32 lumps every row (fine or lump) is four floats, 16 bytes.
// The lumps-in-shared-memory placement keeps lumps and mirror as [lumps | mirror] (mirror at `fine`).
struct YLayout {
    size_t fine, mirror, total, lump_part;
};
inline YLayout y_layout(int nf, int nc, int prec, bool lump32) {
    const auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    if (prec != 0 && lump32) return YLayout{16 * (size_t)nc, 16 * (size_t)(nc + nf), 16 * (size_t)(nc + nf), 16 * (size_t)nc};
    const size_t tl = 8, tc = prec == 0 ? 8 : 4;
    const size_t yc = a16(3 * tl * (size_t)nc), yf = a16(3 * tc * (size_t)nf);
    const size_t ycf = prec != 0 && !lump32 ? a16(12 * (size_t)nc) : 0;
    return YLayout{yc, yc + yf, yc + yf + ycf, yc + ycf};
}
size_t apply_smem_bytes(int nf, int nc, int prec, bool lump32);  // all local vectors of one subdomain
size_t apply_lump_bytes(int nc, int prec, bool lump32);  // its lump vector (and FP32 mirror of FP64 lumps)
// Placement of one apply launch's local vectors.  all_bytes / lump_bytes: the largest subdomain's
// needs (0: not available); smem_slots: ring slots of the all-shared-memory variant; chunk: bytes of
// one ring slot (the largest chunk capacity of the launch's subdomains); force: 0
// automatic (all in shared memory while the launch's nsub CTAs run at once at that occupancy, else
// lumps in shared memory when four CTAs fit, else device memory), Y_SMEM + 1 / Y_LUMPS + 1 /
// Y_DEVICE + 1 to ask for one placement (taken when it fits).  smem_slots: ring slots with all
// local vectors in shared memory; other_slots: with the other placements.
ApplyConfig apply_local_vectors(int nsub, int all_bytes, int lump_bytes, int smem_slots, int chunk, int sm_smem,
                                int sms, int force, int other_slots = 2);
size_t apply_ring_bytes(int slots, int chunk);
void launch_spmv(const SysTab* st_tab, const RowItem* items, int nitems, cudaStream_t st);

void launch_init(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st);
void launch_prep(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st);
void launch_post(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st);
void launch_mgs(const SysTab* tab, const VecItem* items, int nitems, int k, cudaStream_t st);
void launch_finish(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st);
// ORTHOMIN(k): projection pass l of the direction in progress (l = 0 also reduces ||r|| of
// initial systems and ||b - A x|| of finishing ones), then x += alpha p, r -= alpha q.
// Dense matrices inverted in place by Gauss-Jordan elimination with partial pivoting: aug = [A | I]
// (n x 2n, row-major), prow / fcol scratch of 2n / n doubles.
struct GJMat {
    double* aug;
    int n;
    double* prow;
    double* fcol;
};
void launch_gj_init(const GJMat* mats, const int2* rows, int nrows, cudaStream_t st);
// one cooperative launch; err[m] = 1 + pivot column of a singular matrix m (else untouched)
cudaError_t launch_gj_run(const GJMat* mats, int nmat, int nmax, double* part, int part_cap, int* err, int device,
                          cudaStream_t st);
void launch_dense_scatter(const double* slot, const long long* off, const int* mat_of_slot, const GJMat* mats,
                          long long nslot, cudaStream_t st);
// exact local solves: R_i r (one CTA per subdomain), then the owned rows of A_i^{-1} R_i r
// (items: (subdomain work item, first of 8 owned rows)) written to the apply output
void launch_dense_restrict(const SysTab* tab, const SubDesc* subs, int nsub, cudaStream_t st);
void launch_dense_apply(const SysTab* tab, const SubDesc* subs, const int2* items, int nitems, cudaStream_t st);
// Nested factorisation: G and G^{-1} of every subdomain (one warp each; *err gets the first
// singular G) and the line packets of the apply (nmax: largest n; prec 0 FP64, else FP32); the
// apply z[owned] = (B_i^{-1} R_i r)[owned], one CTA of one warp per subdomain, smem = the largest
// nf_apply_smem of the descriptors at that ring depth
size_t nf_work_doubles(int bx, int by, int bz);
size_t nf_line_bytes(int bz, int prec);
size_t nf_plane_bytes(int S, int prec);  // one plane of the apply's y (stride of NFDesc::yv)
size_t nf_apply_smem(int bx, int bz, int prec, int slots);
// ring slots of the apply (2..4) for ndesc subdomains of at most bx_max x bz_max planes
int nf_apply_slots(int ndesc, int bx_max, int bz_max, int prec, int sm_smem, int sms, int dev_smem);
void launch_nf_factor(const NFDesc* descs, int ndesc, int nmax, int prec, FactErr* err, cudaStream_t st);
void launch_nf_apply(const SysTab* tab, const NFDesc* descs, int ndesc, int prec, int slots, size_t smem,
                     cudaStream_t st);
void launch_om(const SysTab* tab, const VecItem* items, int nitems, int l, cudaStream_t st);
void launch_om_update(const SysTab* tab, const VecItem* items, int nitems, cudaStream_t st);
// Coarse-grid correction: [A_C | I] from the box-pair blocks, then in-place Gauss-Jordan (one
// cooperative launch; *err = 1 + column of a zero pivot); and the per-apply kernels
// (two-stage residual, R_C, A_C^{-1} product, R_C^T added to the apply output).
struct GJMat;
cudaError_t launch_coarse_invert(const long long* keys, const double* blocks, int nkeys, int nb, double* aug,
                                 const GJMat* mat, double* part, int part_cap, int* err, int device, cudaStream_t st);
void launch_coarse_apply(const SysTab* tab, const RowItem* rows, int nrows, const BoxItem* boxes, int nboxes,
                         const RowItem* grows, int ngrows, const VecItem* vecs, int nvecs, bool two_stage,
                         cudaStream_t st);
// Whole Gram-Schmidt + state step of a single system in one cooperative launch (grid <= the
// co-resident limit from ortho_coop_grid); part2 holds 4 * nchunk doubles.
int ortho_coop_grid(int device);
cudaError_t launch_ortho_coop(const SysTab* tab, double* part2, int grid, cudaStream_t st);

// Read-only view of the device matrix of a handle (used by the no-allocation residual)
struct MatrixView {
    const double* ell_val;
    const int* ell_col;
    int ell_w, rows_pad, n_cells, device;
    cudaStream_t stream;
};
// Loads the no-allocation residual's scratch array and kernel onto `device` (current) and keeps
// the array's device address; called by asm_create, while the caller can still allocate.
int noalloc_prepare(int device);

}  // namespace asm2

struct asm_ctx;
// ASM_OK and *out filled when h holds a matrix, else ASM_ERR_STATE
int handle_matrix_view(asm_ctx* h, asm2::MatrixView* out);
