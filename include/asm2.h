/*
 * asm2 -- two-level ("boundary conditioning") additive Schwarz preconditioned Krylov solver for
 * fully implicit reservoir Jacobians with 3x3 blocks per cell, on one NVIDIA GB300 (sm_103a).
 *
 * Method: H. Jackson, M. Taroni, D. K. Ponting, "A Two-Level Variant of Additive Schwarz
 * Preconditioning for Use in Reservoir Simulation", arXiv:1401.7227.
 *   - Linear problem r = b - A x = 0, A = -J (Section 2).
 *   - Each subdomain i solves with A_i = R_i A R_i^T (Eq. 3.4), where R_i is the identity on the
 *     subdomain's fine cells and coarsens the rest of the grid into near-field and far-field lumps
 *     by plain summation (Eq. 4.1, Section 4, Appendix B).
 *   - A_i is approximately inverted by a block ILU(0) whose dropped fill is moved to the diagonal
 *     block of its column, so that E = B - A has zero column sums (Section 2; cf. Eq. A.7).
 *   - B^{-1} r = sum_i P_i R_i^T A_i^{-1} R_i r: each cell takes the local solution of the
 *     subdomain that owns it; the coarse parts are discarded (Eqs. 4.2-4.5).
 *   - The Krylov accelerator is GMRES(m) or ORTHOMIN(k), right-preconditioned (Section 2).
 *
 * Conventions for every call:
 *   - Cells are numbered z fastest: cell = k + nz * (i + nx * j) for grid position (i, j, k).
 *   - Vectors hold 3 doubles per cell (cell-major); a matrix block is 9 doubles, row-major.
 *   - Every call returns an asm_status; nothing throws across this boundary.
 *   - A handle is used from one host thread at a time.  Device work is issued in order on the
 *     CUDA stream given to asm_create (NULL = the legacy default stream); calls that take caller
 *     buffers return after that work has completed.
 *   - "on_device" says whether caller vector/matrix pointers are device memory (1) or host
 *     memory (0).  Caller buffers stay owned by the caller.  The library copies everything given
 *     to asm_set_* / asm_update_values into device memory it owns, freed by asm_destroy.
 *   - Partition geometry (Section 4): the grid is split into px*py*pz boxes, part t of n cells
 *     in a dimension being [n*t/p, n*(t+1)/p); subdomain s = tz + pz*(tx + px*ty).  Its fine
 *     set is its box grown by `overlap` cells (clipped); near lumps are the c_near-sized boxes
 *     aligned at 0 that meet the ring of width `near_width` around the fine set, minus the fine
 *     set; far lumps are the far boxes (the partition boxes, or c_far-sized aligned boxes) minus
 *     the fine set and the near lumps.  Empty lumps are dropped.  Local order: fine cells by cell
 *     index, then near lumps, then far lumps, each by box index bz + nbz*(bx + nbx*by).
 */
#ifndef ASM2_H
#define ASM2_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ASM_OK = 0,
    ASM_ERR_INVALID_ARG = 1,   /* bad size, index, pointer or option; checked on the host */
    ASM_ERR_PATTERN = 2,       /* block pattern not structurally symmetric / missing a diagonal */
    ASM_ERR_ZERO_PIVOT = 3,    /* singular 3x3 pivot in a local factorisation */
    ASM_ERR_NOT_CONVERGED = 4, /* max_iter reached; x holds the last iterate */
    ASM_ERR_OOM = 5,           /* device (or host) allocation failed */
    ASM_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    ASM_ERR_TIMEOUT = 7,       /* a bounded device wait expired */
    ASM_ERR_STATE = 8          /* call out of order (e.g. solve before factor) */
} asm_status;

typedef enum {
    ASM_PREC_FP64 = 0,  /* local factors stored and applied in FP64 */
    ASM_PREC_FP32 = 1,  /* fine-cell factor rows stored and applied in FP32; lump rows as
                           asm_options.lump_precision says */
    ASM_PREC_FP16S = 2  /* fine-cell factor rows stored in FP16 (with a power-of-two exponent per
                           block), applied in FP32; lump rows as asm_options.lump_precision says */
} asm_precision;

/* Lump rows (the near- and far-field unknowns of the coarsened outer region, Section 4) of the
 * local ILU factors under FP32 or FP16S fine rows.  The factorisation itself always runs in FP64;
 * Gram-Schmidt, the true residual and the classical coarse-grid solve stay FP64 either way. */
typedef enum {
    ASM_LUMP_FP64 = 0,  /* lump rows stored and applied in FP64 */
    ASM_LUMP_FP32 = 1   /* (default) lump rows stored and applied in FP32 like the fine rows: every
                           ILU factor row of the mixed-precision path is FP32 (FP64 factors ignore
                           it) */
} asm_lump_precision;

typedef enum { ASM_KRYLOV_GMRES = 0, ASM_KRYLOV_ORTHOMIN = 1 } asm_krylov;

typedef enum {
    ASM_LOCAL_BILU0_COLSUM = 0, /* block ILU(0) with column-sum compensation (default) */
    ASM_LOCAL_BILU0 = 1,        /* plain block ILU(0): dropped fill is discarded */
    ASM_LOCAL_EXACT = 2         /* exact local solves A_i^{-1} (Section 5: the paper's own setting,
                                   Gaussian elimination): every A_i is inverted at asm_factor by
                                   Gauss-Jordan elimination with partial pivoting (FP64 only; at most
                                   4096 local block rows; (3 n_i)^2 * 16 bytes of device memory each) */
    ,
    ASM_LOCAL_NF_COLSUM = 3,    /* nested factorisation with column-sum compensation (Appendix A,
                                   Eqs. A.2-A.4 and A.7): for local problems without lumps only
                                   (near_width 0 and ASM_FAR_NONE), whose A_i is hepta-banded on the
                                   box of the fine set, ordered z fastest, then x, then y.  G is always
                                   computed in FP64; the apply runs in FP64 (ASM_PREC_FP64) or in FP32
                                   (ASM_PREC_FP32; ASM_PREC_FP16S is refused at asm_create).  asm_factor
                                   returns ASM_ERR_INVALID_ARG when a local problem has lumps or a line of
                                   a fine box (its z extent) is too long for the apply's shared memory
                                   (about 180 cells in FP64, 280 in FP32), and ASM_ERR_PATTERN when an
                                   A_i has a block off the seven bands */
    ASM_LOCAL_NF = 4            /* nested factorisation without compensation: G = D - L1 G^{-1} U1
                                   (Eq. A.6); same conditions */
} asm_local_solver;

/* Orthogonalisation of the GMRES Arnoldi step (Section 2 uses modified Gram-Schmidt).  The
 * paper has no classical option; it is offered because on this GPU every projection of MGS is a
 * global reduction (a grid-wide barrier per projection), while classical Gram-Schmidt takes the
 * same FP64 work with two global reductions per step.  It rounds differently and keeps the basis
 * less orthogonal (loss ~ cond^2 eps instead of cond eps), so iteration counts may differ from
 * MGS and from the oracle; tests hold it to the solution tolerance.  It applies to single-system
 * GMRES solves with the cooperative Gram-Schmidt (ASM_TUNE_COOP_ORTHO = 1) and restart <= 62;
 * batched solves use MGS. */
typedef enum {
    ASM_ORTHO_MGS = 0, /* modified Gram-Schmidt (default; the oracle's arithmetic order) */
    ASM_ORTHO_CGS = 1  /* classical Gram-Schmidt: all projections, then the norm, from two reductions */
} asm_ortho;

typedef enum {
    ASM_FAR_NONE = 0,      /* no far field: cells outside fine set + near lumps are left out */
    ASM_FAR_PARTITION = 1, /* far lumps = the partition boxes */
    ASM_FAR_BOXES = 2      /* far lumps = aligned boxes of size c_far */
} asm_far_mode;

typedef struct {
    int precision;    /* asm_precision */
    int krylov;       /* asm_krylov */
    int restart;      /* GMRES restart length m, or ORTHOMIN direction count k; 1..512 */
    int local_solver; /* asm_local_solver */
    int flexible;     /* GMRES update: 1 keeps Z_j = B^{-1} v_j and sets x += Z y; 0 sets
                         x += B^{-1}(V y); -1 = automatic (0 for FP64, 1 otherwise) */
    int device;       /* CUDA device ordinal */
    int lump_precision; /* asm_lump_precision (default ASM_LUMP_FP32) */
    int ortho;          /* asm_ortho (default ASM_ORTHO_MGS) */
} asm_options;

typedef struct {
    int iterations;      /* preconditioned matrix-vector products */
    int restarts;        /* completed GMRES cycles (true-residual evaluations) */
    int converged;       /* 1 when ||b - A x||_2 <= rtol * ||b||_2, FP64 true residual */
    int status;          /* asm_status of this system */
    double rel_residual; /* final FP64 true relative residual */
} asm_solve_info;

typedef struct {
    int n_cells;                 /* N */
    int n_sub;                   /* subdomains K */
    long long local_rows;        /* sum over subdomains of n_i (fine cells + lumps) */
    int max_local_rows;          /* max n_i */
    int max_levels;              /* max wavefront levels of a local factor */
    long long local_blocks;      /* sum over subdomains of the local pattern size (blocks) */
    long long factor_bytes;      /* factor-stream bytes read by one preconditioner apply */
    long long apply_index_bytes; /* restriction/scatter list bytes read by one apply */
    long long matrix_bytes;      /* values + column indices of A read by one SpMV */
    long long alg_apply_bytes;   /* minimum bytes one apply must move: every off-diagonal factor
                                    block (9 values + a 4-byte index) and every D^{-1} block at its
                                    storage precision, plus r read and z written (48 N) */
    double setup_ms;             /* host symbolic analysis time of the last asm_factor */
    double factor_ms;            /* device assembly + factorisation time of the last asm_factor */
    /* the ILU apply's tiling (0 for other local solvers): */
    int chunk_max_kb;            /* largest stream-chunk capacity of the subdomains (a ring slot) */
    long long stream_chunks;     /* stream chunks of all subdomains, both sweeps */
    int apply_placement;         /* placement a single-system apply runs with now: 3 all in shared
                                    memory, 2 lumps, 0 device (the online tuner's choice once made) */
    int apply_slots;             /* its ring slots */
    int last_solve_placement;    /* placement the last asm_solve / asm_solve_batch with this handle
                                    ran its applies in (a batch shares one; -1: no solve yet) */
    int last_solve_slots;        /* its ring slots */
    int last_solve_chunk_kb;     /* its ring slot size: the largest chunk capacity of the batch */
} asm_stats;

/* Device time of each part of the solver, accumulated while profiling is on (CUDA events on the
 * handle's stream around each launch group), and the number of kernels launched. */
typedef struct {
    double apply_ms;        /* far-box sums + fused local solves (preconditioner apply) */
    double spmv_ms;         /* SpMV (A z, and b - A x at restarts) */
    double ortho_ms;        /* Gram-Schmidt / norms / Givens / vector updates */
    double factor_ms;       /* assembly + factorisation + factor packing */
    long long apply_launches;   /* preconditioner applies timed in apply_ms */
    long long kernel_launches;  /* every kernel launched by the library (counted always) */
} asm_profile_info;

typedef struct asm_ctx* asm_handle;

/* Defaults: FP64, GMRES, m = 30, column-sum ILU(0), automatic flexibility, device 0. */
void asm_default_options(asm_options* opt);

/* Text of a status code (static storage, never NULL). */
const char* asm_error_string(int status);

/* Create a handle.  opt NULL = defaults.  cuda_stream: a cudaStream_t of opt->device, or NULL.
 * Errors: INVALID_ARG (bad option / device), CUDA. */
int asm_create(asm_handle* h, const asm_options* opt, void* cuda_stream);

/* Free every device and host resource of h (NULL is a no-op). */
int asm_destroy(asm_handle h);

/* Grid of the problem (Section 1: one cell = one 3x3 block row).  Must precede the matrix. */
int asm_set_grid(asm_handle h, int nx, int ny, int nz);

/* The matrix A (Section 2: A = -J) as BSR with 3x3 blocks: row_ptr[n_cells+1], col_idx[nnzb]
 * (ascending within a row, diagonal present, pattern structurally symmetric), vals[nnzb*9]
 * row-major blocks.  n_cells must equal nx*ny*nz.  The pattern is validated on the host
 * (INVALID_ARG for bad indices, PATTERN for asymmetry or a missing diagonal); on_device applies
 * to vals only (row_ptr/col_idx are always host arrays).  Invalidates any factorisation. */
int asm_set_matrix_bsr(asm_handle h, int n_cells, int nnzb, const int* row_ptr, const int* col_idx,
                       const double* vals, int on_device);

/* New values for the same pattern (vals[nnzb*9]); keeps the symbolic analysis, so the next
 * asm_factor only re-assembles and re-factors on the device (a new Newton iteration, Section 4:
 * the coarsened matrices are rebuilt once per non-linear iteration). */
int asm_update_values(asm_handle h, const double* vals, int on_device);

/* Subdomain partition and coarsening (Section 4, Eq. 4.1, Figs. 2-3; geometry in the file
 * header).  c_near[3]: near-box size (x, y, z), required when near_width > 0.  far_mode:
 * asm_far_mode; c_far[3] is the far-box size for ASM_FAR_BOXES (else ignored, may be NULL).
 * Errors: INVALID_ARG (p > n, negative widths, box sizes < 1). */
int asm_set_partition_boxes(asm_handle h, int px, int py, int pz, int overlap, int near_width,
                            const int* c_near, int far_mode, const int* c_far);

/* Classical coarse-grid corrections, the methods the paper compares its boundary conditioning
 * with (Section 3, Fig. 6), added to the preconditioner set by asm_set_partition_boxes (B_AS):
 *   ASM_COARSE_TWO_LEVEL  B^{-1} = B_AS^{-1} + R_C^T A_C^{-1} R_C                      (Eq. 3.5)
 *   ASM_COARSE_TWO_STAGE  B^{-1} = B_AS^{-1} + R_C^T A_C^{-1} R_C (I - A B_AS^{-1})    (Eqs. 3.7-3.8)
 * R_C sums the 3-vectors of the cells of each coarse box, R_C^T copies a box's value to each of
 * its cells, and A_C = R_C A R_C^T (Eq. 3.6) is inverted exactly at asm_factor (Gauss-Jordan
 * elimination with partial pivoting, FP64, on the device).  c_box: the coarse box size (x, y, z)
 * in cells, boxes aligned at 0 and numbered bz + nbz*(bx + nbx*by); NULL or {0,0,0} takes the
 * partition boxes (box = subdomain).  At most 1024 coarse boxes.  ASM_COARSE_NONE removes the
 * correction.  Invalidates the factorisation.  Errors: INVALID_ARG (mode, box size, too many
 * boxes), STATE (no grid or partition yet); a singular A_C makes asm_factor return ZERO_PIVOT
 * with error location (-1, coarse block row).  The serving loop does not take these options. */
typedef enum { ASM_COARSE_NONE = 0, ASM_COARSE_TWO_LEVEL = 1, ASM_COARSE_TWO_STAGE = 2 } asm_coarse_mode;
int asm_set_coarse_correction(asm_handle h, int mode, const int* c_box);

/* Build B: host symbolic analysis (cached across asm_update_values), then on the device the
 * local matrices A_i = R_i A R_i^T (Eq. 3.4, B.3) and their block ILU(0) (+ colsum, Section 2).
 * Errors: STATE (no matrix/partition), ZERO_PIVOT (see asm_get_error_location), OOM, CUDA. */
int asm_factor(asm_handle h);

/* z = B^{-1} r = sum_i P_i R_i^T A_i^{-1} R_i r (Eqs. 4.2-4.5); r, z: 3N doubles. */
int asm_apply_precond(asm_handle h, const double* r, double* z, int on_device);

/* y = A x; x, y: 3N doubles. */
int asm_spmv(asm_handle h, const double* x, double* y, int on_device);

/* Solve A x = b to ||b - A x||_2 <= rtol ||b||_2 (FP64 true residual) with the Krylov method of
 * the options, x0 = 0 (Section 2).  x receives the solution (or the last iterate with
 * NOT_CONVERGED).  info may be NULL.
 *   GMRES(m): restarted, modified Gram-Schmidt, Givens rotations; stops when the Arnoldi residual
 *   estimate reaches rtol, then confirms on the true residual (a restart otherwise).
 *   ORTHOMIN(k): p = B^{-1} r, q = A p, A-orthogonalised (newest first) against the k most
 *   recent directions, x += alpha p, r -= alpha q with alpha = (r, q) / (q, q); stops when the
 *   updated residual reaches rtol or max_iter steps have run, or on (q, q) = 0; the reported
 *   status and rel_residual are those of the true residual at that point (no restart). */
int asm_solve(asm_handle h, const double* b, double* x, double rtol, int max_iter, int on_device,
              asm_solve_info* info);

/* Solve n independent factored systems together: every Krylov step of all unfinished systems
 * runs in the same kernel launches.  Handles must share device, stream, factor precision and
 * Krylov method.
 * b[k], x[k] belong to hs[k]; infos[k] (may be NULL) receives its result.  Each system's
 * arithmetic does not depend on the others in the batch.  Returns the worst status. */
int asm_solve_batch(asm_handle* hs, int n, const double* const* b, double* const* x, double rtol,
                    int max_iter, int on_device, asm_solve_info* infos);

/* Sizes and timings of the current factorisation. */
int asm_get_stats(asm_handle h, asm_stats* st);

/* Tuning switches of the kernels (none changes the arithmetic of a fine row; results are bitwise
 * the same, except where ASM_TUNE_CHUNK_KB says otherwise):
 *   ASM_TUNE_APPLY_SMEM  where the apply keeps each subdomain's local vectors.  1 (default):
 *                        all in shared memory (256-thread CTAs) when every subdomain CTA of the
 *                        launch then runs at once; else the lump vector in shared memory and the
 *                        fine-row vector in device memory when that fits; else all in device memory
 *                        (256-thread CTAs).  0: all in device memory; 2: lumps in shared memory;
 *                        3: all in shared memory (2 and 3 fall back to device memory when they do
 *                        not fit);
 *   ASM_TUNE_COOP_ORTHO  1 (default) runs the Gram-Schmidt step of a single-system solve in one
 *                        cooperative launch, 0 in one launch per projection.
 * Errors: INVALID_ARG for an unknown key or value. */
typedef enum {
    ASM_TUNE_APPLY_SMEM = 0,
    ASM_TUNE_COOP_ORTHO = 1,
    ASM_TUNE_AUTOTUNE = 2, /* 1 (default): a solve's first apply steps try every placement of the
                              local vectors that fits (a warm-up round, then a timed round) and
                              keep the fastest; remembered per handle for single-system solves.
                              Placements give bitwise equal results.  0: the placement rule only. */
    ASM_TUNE_GRAPHS = 3,   /* 1 (default): batched solves replay each Krylov step as a captured
                              CUDA graph (one per projection count); 0: plain launches */
    ASM_TUNE_WAIT_LIMIT = 4, /* failure-detection hook (0..30, default 22): the apply kernels (ILU
                              sweeps and nested factorisation) give up waiting for a factor-stream
                              copy after 2^value polls, 0 polls for value 0, and the call returns
                              ASM_ERR_TIMEOUT without a result.  Before it leaves, each CTA waits
                              with the full bound for its own copies in flight, so the device stays
                              usable.  Value 0 makes every wait expire at once, which tests the
                              timeout path without a fault; restore 22 afterwards */
    ASM_TUNE_CHUNK_KB = 5,   /* stream-chunk capacity of the ILU factor stream (the wavefront
                              levels' rows are cut into chunks of at most this size; one ring slot
                              of the apply holds one chunk).  0 (default): each subdomain's own
                              rule (its largest fine level, 8..24 KB); 8, 12, 16, 20 or 24: that
                              capacity in KB for every subdomain, raised where one row needs more.
                              Takes effect at the next asm_factor, which then rebuilds the
                              symbolic structure.  Fine rows compute the same bits under every
                              capacity; FP64 lump rows may round differently (their entry slots
                              are chosen per chunk) */
    ASM_TUNE_APPLY_SLOTS = 6 /* ring slots of the apply: 0 (default) with all local vectors in
                              shared memory as many as keep two CTAs per SM, else 4, and 2 with the
                              other placements; 2, 3 or 4 for every placement */
} asm_tune_key;
int asm_set_tuning(asm_handle h, int key, int value);

/* The tiling tuner (no counterpart in the paper, which leaves the blocking of the local solves to
 * the implementation).  For a factored handle with ILU(0) local solves it measures the
 * preconditioner apply under every stream-chunk capacity (ASM_TUNE_CHUNK_KB: the rule, 8, 12, 16,
 * 20, 24 KB; capacities that give every subdomain the same chunks as an earlier one are skipped)
 * crossed with every placement of the local vectors that fits (all in shared memory, lumps in
 * shared memory, all in device memory) and 2, 3 or 4 ring slots, each as the median of `reps` timed
 * applies after two untimed ones.  It then leaves the fastest in place (ASM_TUNE_CHUNK_KB,
 * ASM_TUNE_APPLY_SLOTS and ASM_TUNE_APPLY_SMEM set, the online placement tuner off) with the
 * handle factored again, and reports every measurement.  Each capacity costs one symbolic rebuild
 * and factorisation, so this is a set-up step to run once per structure.  The handle's values are
 * factored again as they are.
 * Errors: STATE if not factored; INVALID_ARG for another local solver, reps < 1 or out == NULL. */
#define ASM_TILING_MAX 64
typedef struct {
    int chunk_kb;      /* ASM_TUNE_CHUNK_KB value (0: the per-subdomain rule) */
    int chunk_max_kb;  /* the largest capacity the subdomains got (a ring slot's size) */
    long long chunks;  /* stream chunks of all subdomains, both sweeps */
    int placement;     /* ASM_TUNE_APPLY_SMEM value: 3 all in shared memory, 2 lumps, 0 device */
    int slots;         /* ring slots */
    int ctas_per_sm;   /* apply CTAs resident per SM */
    double apply_ms;   /* median time of one preconditioner apply (all its kernels) */
} asm_tiling_entry;
typedef struct {
    int n;               /* entries measured */
    int best;            /* index of the entry left in place */
    double rule_ms;      /* the default (rule capacity, automatic placement), measured first */
    asm_tiling_entry e[ASM_TILING_MAX];
} asm_tiling_report;
int asm_tune_tiling(asm_handle h, int reps, asm_tiling_report* out);

/* The same search for a batch (asm_solve_batch's arguments): every handle gets each stream-chunk
 * capacity in turn (one symbolic rebuild and factorisation each), and the batch is solved twice
 * per capacity, the first solve untimed (its first steps run the online placement tuner), the
 * second timed.  Each entry's apply_ms holds that timed batched solve's time, and its placement
 * and slots are what the online tuner chose for the batch; rule_ms is the rule's entry.  The
 * fastest capacity is left in place (handles factored again); placements stay with the online
 * tuner.  x receives the last solve's iterates.  Errors as asm_solve_batch, plus STATE if a
 * handle is not factored and INVALID_ARG for another local solver or out == NULL. */
int asm_tune_tiling_batch(asm_handle* hs, int n, const double* const* b, double* const* x, double rtol, int max_iter,
                          int on_device, asm_tiling_report* out);

/* Profiling switch (0/1): when on, launch groups are bracketed by CUDA events. */
int asm_set_profiling(asm_handle h, int enable);
/* Accumulated profile since the last reset (counters keep running when profiling is off). */
int asm_get_profile(asm_handle h, asm_profile_info* p);
/* Zero the accumulated profile and launch counters. */
int asm_reset_profile(asm_handle h);

/* After ZERO_PIVOT: the subdomain and local block row of the first singular pivot found. */
int asm_get_error_location(asm_handle h, int* sub, int* row);

/* Parity hooks (copies to caller HOST memory, in the local order of the file header):
 * counts[3] = {fine cells, near lumps, far lumps}; map[N] = local row of each cell or -1;
 * the local matrix A_s as BSR (row_ptr[n+1], col_idx[nnzb], vals[nnzb*9]); its factors in the
 * same pattern (lu[nnzb*9]: L below, U above, D^{-1} on the diagonal; dpiv[n*9]: pivot blocks),
 * as FP64 before any down-cast of the stored factors.  Any output pointer may be NULL.  With
 * nested factorisation dpiv receives the diagonal blocks G of Eqs. A.6-A.7 by local row and lu
 * must be NULL; with exact local solves asm_get_local_factors returns ASM_ERR_INVALID_ARG. */
int asm_get_local_info(asm_handle h, int s, int* n, int* nnzb, int* counts, int* n_levels);
int asm_get_local_map(asm_handle h, int s, int* map);
int asm_get_local_matrix(asm_handle h, int s, int* row_ptr, int* col_idx, double* vals);
int asm_get_local_factors(asm_handle h, int s, double* lu, double* dpiv);

/* ------------------------------------------------------------------------------------------
 * Serving loop (continuous batching).  Requests of any grid size are submitted as they arrive;
 * asm_server_progress admits them while the active-system limit and the device-memory budget
 * allow (a request whose matrix key is already resident reuses its factors; a new structure --
 * grid, partition, precision and a 64-bit FNV-1a hash of the block pattern; the pattern itself is
 * not compared -- is analysed once on a host worker thread and cached), and advances every active
 * system by Krylov steps in the same kernel launches; finished systems leave the batch between
 * steps.  Each system's arithmetic does not depend on the others in the batch.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int precision;        /* asm_precision of every served system (default FP32) */
    int restart;          /* GMRES m (default 30) */
    int device;           /* CUDA device */
    int max_active;       /* systems advanced together, 0 = no limit (default 64) */
    int max_cached;       /* idle factored systems kept for matrix reuse, LRU (default 16) */
    long long hbm_budget; /* device bytes for resident systems; 0 = 85% of free memory */
    int lump_precision;   /* asm_lump_precision of every served system (default ASM_LUMP_FP32) */
} asm_server_options;

typedef struct {
    int nx, ny, nz, n_cells, nnzb;
    const int* row_ptr;    /* host, borrowed until the result is collected */
    const int* col_idx;    /* host, borrowed until the result is collected */
    const double* vals;    /* host, borrowed until the result is collected */
    int px, py, pz, overlap, near_width, c_near[3], far_mode, c_far[3]; /* asm_set_partition_boxes */
    const double* b;       /* host, copied at submission */
    double rtol;
    int max_iter;
    long long matrix_key;  /* >= 0: requests with the same key carry the same matrix */
} asm_request;

typedef struct {
    long long submitted, admitted, completed, steps, reuse_hits, structure_builds, evictions;
    long long resident_bytes, budget_bytes;
    int active, pending;
    /* where the host time goes (wall clock, ms, cumulative): structure analysis on the worker
     * thread; admission (every call of it), of which building new systems (allocation, structure
     * upload, values, factorisation) and re-keying idle systems of the same structure (values and
     * factorisation only); Krylov steps (control-word reads, batch tables, launches; admission and
     * retiring excluded); retiring (result download) */
    double analysis_ms, admit_ms, build_ms, rekey_ms, step_ms, retire_ms;
    long long progress_calls, structure_reuses;
    double build_factor_ms; /* of build_ms: the numeric factorisation (the rest: allocation, uploads) */
} asm_server_stats;

/* Defaults: FP32 factors, GMRES(30), device 0, 64 active systems, 16 cached, budget 0 (85% of the
 * free device memory at creation). */
void asm_server_default_options(asm_server_options* opt);
typedef struct asm_server* asm_server_handle;
/* cuda_stream: the stream all served work is issued on (NULL = legacy default stream).
 * Errors: INVALID_ARG (bad option / device index), CUDA (no usable device), OOM. */
int asm_server_create(asm_server_handle* s, const asm_server_options* opt, void* cuda_stream);
/* Queue a request; *ticket identifies it.  Errors: INVALID_ARG (inconsistent sizes, or grid and
 * partition arguments that asm_set_grid / asm_set_partition_boxes refuse). */
int asm_server_submit(asm_server_handle s, const asm_request* req, long long* ticket);
/* Admit what fits, then run up to max_steps Krylov steps of the active systems. */
int asm_server_progress(asm_server_handle s, int max_steps, int* n_active, int* n_pending);
/* STATE while the request is unfinished; else copies x (3N doubles, host) and its info, forgets
 * the ticket and returns OK (also when not converged: see info.status) or the request's error. */
int asm_server_result(asm_server_handle s, long long ticket, double* x, asm_solve_info* info);
/* Counters since creation, and the current resident bytes, budget, active and pending counts. */
int asm_server_get_stats(asm_server_handle s, asm_server_stats* stats);
/* Stops the analysis thread and frees every system, cached factor and uncollected request. */
int asm_server_destroy(asm_server_handle s);

/* No-allocation true residual: r = b - A x and *norm = ||r||_2 for the matrix held by h.
 * The paper has no counterpart: this entry point is for callers that cannot allocate device
 * memory when they need it -- code running under a memory pool that forbids further device
 * allocations, or code that must keep its allocations fixed after start-up (certified or
 * real-time simulators).  b, x (3N doubles, read), r (3N doubles, written) and norm (one
 * double, written) are caller-owned DEVICE pointers; the call allocates nothing and calls no
 * allocating routine.  The partial sums of the norm go to a scratch array compiled into the
 * library (16384 doubles + a counter, 128 KB, held by every GPU that loads the library until the
 * process exits), so N is limited to 256 * 16384 = 4,194,304 cells (INVALID_ARG beyond).  CUDA
 * loads a library's kernels and device arrays lazily, and loading allocates device memory, so
 * asm_create loads this entry point's kernel and array onto the handle's device: later calls,
 * the first one included, allocate nothing.  All calls share the array and each leaves its
 * counter at zero: calls that overlap on the GPU race.  r must not overlap x (INVALID_ARG); r may
 * be b.  Work is issued on the handle's stream, and the call waits for that stream before it
 * returns.
 * Errors: INVALID_ARG (NULL pointer, N too large, r overlapping x), STATE (no matrix), CUDA. */
int asm_residual_noalloc(asm_handle h, const double* b, const double* x, double* r, double* norm);

#ifdef __cplusplus
}
#endif

#endif
