/*
 * sc.h -- C ABI of the GB300 supernodal sparse Cholesky library (libsc).
 *
 * Right-looking supernodal Cholesky A = L L^T of a sparse symmetric positive
 * definite matrix, in the two variants of Karsavuran, Ng, Peyton and Peyton,
 * "Some new techniques to use in serial sparse Cholesky factorization
 * algorithms" (arXiv 2409.13090):
 *   RL  -- Algorithm 4 (Sec. 2.2.1): one update matrix U_J per supernode,
 *          assembled into the ancestors through relative indices;
 *   RLB -- Algorithm 5 (Sec. 2.2.2): SYRK/GEMM updates applied block by block
 *          straight into the ancestors' factor storage, with no floating-point
 *          working storage and no assembly.
 * The solution pipeline is the four steps of Sec. 1: ordering, symbolic
 * factorization (host), numeric factorization (GPU), solution (GPU).
 *
 * Conventions shared by every entry point
 *  - Indices are 0-based. A is given by its lower triangle including the
 *    diagonal, compressed sparse column (CSC): colptr[n+1] (int64), rowind
 *    (int32), row indices strictly ascending within a column, the diagonal
 *    entry present and first in its column. values are FP64, aligned with
 *    rowind (Sec. 2.1.1: on entry the factor storage holds the entries of the
 *    lower triangle of A).
 *  - Return value: SC_OK (0) on success; -i when argument i (1-based) is
 *    invalid; a positive k when the matrix is not positive definite, k being
 *    the 1-based index (in the caller's ordering) of the column whose pivot
 *    was not positive; otherwise one of the named SC_ERR_* codes below.
 *  - Ownership: the library copies what it needs from caller arrays during
 *    the call; the caller keeps ownership of every pointer it passes. Handles
 *    are released with their _free function. An sc_numeric keeps a reference
 *    to its sc_symbolic; sc_symbolic_free on a symbolic handle that still has
 *    live numeric handles fails with SC_ERR_IN_USE.
 *  - Streams: cuda_stream is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream). Device work is enqueued on it; entry points that
 *    return device results to the host synchronise that stream.
 *  - Threading: a handle must not be used from two threads at once.
 */
#ifndef SC_H
#define SC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
#define SC_OK 0
#define SC_ERR_CUDA (-101)          /* a CUDA runtime call failed            */
#define SC_ERR_TIMEOUT (-102)       /* a bounded device-side wait gave up    */
#define SC_ERR_NOT_CONVERGED (-103) /* refinement hit its cap; X = best iterate */
#define SC_ERR_OOM (-104)           /* host or device allocation failed      */
#define SC_ERR_IN_USE (-105)        /* symbolic handle still referenced      */
#define SC_ERR_INTERNAL (-106)      /* an internal consistency check failed  */
#define SC_ERR_UNSUPPORTED (-107)   /* option not available in this library  */
#define SC_ERR_IO (-108)            /* a file could not be written or read, or is
                                       not a valid symbolic file of this library */

/* --------------------------------------------------------------- options */
/* SC_ORDER_GRID_ND: geometric nested dissection of an nx x ny x nz grid
 * (grid[] and nd_leaf); SC_ORDER_GRAPH_ND: nested dissection of the matrix
 * graph by breadth-first level structures (nd_leaf), for inputs without a
 * grid; SC_ORDER_GRAPH_ML: as SC_ORDER_GRAPH_ND, but each separator is the
 * smaller of the level separator and that of a multilevel bisection (heavy-edge
 * coarsening, FM refinement), which finds the plane separators of stencils with
 * diagonal coupling. All stand in for the paper's METIS ordering (Sec. 3.1). */
enum sc_ordering {
    SC_ORDER_NATURAL = 0,
    SC_ORDER_GRID_ND = 1,
    SC_ORDER_USER = 2,
    SC_ORDER_GRAPH_ND = 3,
    SC_ORDER_GRAPH_ML = 4
};
enum sc_variant { SC_RLB = 0, SC_RL = 1 };
/* Arithmetic of the numeric factorization:
 *   SC_FP64  every operation in FP64 (the paper's precision, Sec. 3.1);
 *   SC_FP32  factor stored and computed in FP32 (SIMT FMA);
 *   SC_TF32  factor stored in FP32, large update products on the TF32 tensor
 *            cores with FP32 accumulation.
 *   SC_TF32X3  as SC_TF32, but each large product is formed from split
 *            operands x = hi + lo (hi = TF32 rounding of x, lo = TF32 rounding
 *            of x - hi) as hi*hi' + hi*lo' + lo*hi' on the tensor cores: close
 *            to FP32 accuracy at tensor-core rate, so fewer refinement steps.
 *            Holds two extra FP32 copies of the factor storage.
 * With SC_FP32 / SC_TF32 / SC_TF32X3 the solve refines in FP64 (residual
 * r = b - A x and the update x += d in FP64) until the backward error reaches
 * ir_tol. */
enum sc_precision { SC_FP64 = 0, SC_FP32 = 1, SC_TF32 = 2, SC_TF32X3 = 3 };

/* Launch-plan settings (host-side choices only: every setting runs the same
 * kernels on the same data, so the factor agrees with the default plan up to
 * the rounding order of the update sums). A zero field means the library
 * default, given in brackets. sc_tune picks them by timing; a caller may also
 * pass a table through sc_options.tune.
 *   tile_min_entries  an Alg. 5 product (B, B') becomes a tiled task when it
 *                     has >= this many outputs and K >= tile_min_k, or >= 8x
 *                     this many outputs; smaller ones run in the device loops [1024]
 *   tile_min_k        see tile_min_entries [16]
 *   loop_budget       work bound of one device-loop item, in outputs x (K + 4) [32768]
 *   lookahead         1 = products into the next level's chunks run first and
 *                     the rest overlap the next level (RLB with graph replay
 *                     only), -1 = off [1]
 *   tc_min_k          tensor-core tiles only for K >= tc_min_k (>= 32) [32]
 *   tc_wide_n         128-column tensor-core tiles for products at least this
 *                     wide, 64-column tiles below (>= 16) [96]
 *   thin_dim          products with min(m, n) <= thin_dim (1..8) go to the
 *                     warp-block kernel, -1 = none [8]
 *   defer_width       trailing updates inside a supernode are deferred in
 *                     levels: a chunk updates the rest of its 256-column macro
 *                     panel (K = chunk width), a macro panel's last chunk the
 *                     rest of its defer_width-column block (K = 256), and that
 *                     block's last chunk every later column (K = defer_width).
 *                     256..2^20, rounded down to a multiple of the macro panel;
 *                     256 = two levels only [512]. Wider outer blocks mean fewer
 *                     read-modify-write passes over each target with longer K.
 *   fused             1 = every level of an FP64 / FP32 RLB factorization runs as
 *                     one persistent launch (POTRF, TRSM, products, device loops
 *                     and the previous level's lookahead products, ordered by
 *                     device-side counters), -1 = one launch per kernel class
 *                     (each class at its own occupancy) [-1]
 *   tc_wide256        products at least this wide (that would take 128-column
 *                     tiles) take 256-column tensor-core tiles, which read
 *                     each A row from shared memory once per 256 outputs
 *                     (16..2^20; above every product's width = off) [256]
 *   solve_group       the solve sweeps' units: a wide chunk's row tiles after
 *                     its first, taken by one CTA in runs of up to this many
 *                     (1..1024): fewer CTAs wait for one chunk's solution, at
 *                     the price of later arrivals from a run's last tiles
 *                     [2 for FP64 factors, 4 for FP32 / TF32 / TF32x3]
 *   tc_multicast      1 = the 256-column tensor-core tiles run in clusters of
 *                     two CTAs that take vertically adjacent tiles and share
 *                     the B tiles by TMA multicast (each loads half), -1 = one
 *                     CTA per tile [1]
 *   factor_ms         out (sc_tune): median factor time of this setting */
typedef struct sc_tune_table {
    int32_t tile_min_entries;
    int32_t tile_min_k;
    int32_t loop_budget;
    int32_t lookahead;
    int32_t tc_min_k;
    int32_t tc_wide_n;
    int32_t thin_dim;
    int32_t defer_width;
    int32_t fused;
    int32_t tc_wide256;
    int32_t solve_group;
    int32_t tc_multicast;
    int32_t reserved[2];
    double factor_ms;
} sc_tune_table;

typedef struct sc_options {
    int32_t ordering;          /* enum sc_ordering                                  */
    int32_t grid[3];           /* nx, ny, nz for SC_ORDER_GRID_ND (id = x+nx*(y+ny*z)) */
    int32_t nd_leaf;           /* ND: a box or vertex set of at most this many
                                  points is a leaf (grid and graph orderings)      */
    const int32_t *user_perm;  /* SC_ORDER_USER: perm[new] = old, length n          */
    int32_t pr;                /* 1 = partition-refinement reordering within supernodes */
    int32_t variant;           /* enum sc_variant                                   */
    int32_t precision;         /* enum sc_precision (default for sc_factor)         */
    int32_t chunk;             /* panel width for the dense work inside a supernode (8..64) */
    double ir_tol;             /* refinement stops at backward error <= ir_tol      */
    int32_t ir_maxit;          /* refinement iteration cap                          */
    double pivot_tau;          /* low-precision pivot d_jj <= tau * |A_jj| redone in FP64 */
    int64_t spin_limit;        /* iteration limit of every bounded device wait      */
    int32_t use_graph;         /* 1 = replay the factor schedule as a CUDA graph    */
    double merge_frac;         /* supernode merging budget (Sec. 3.1): merge child-parent
                                  pairs by least new fill while the added storage stays
                                  <= merge_frac x the fundamental storage; 0 = off */
    const sc_tune_table *tune; /* launch-plan settings (copied), NULL = defaults     */
    int32_t deterministic;     /* 1 = bit-reproducible factor: every entry of L gets its
                                  updates in one fixed order, so two factorizations of
                                  the same values give the same bits. Needs variant
                                  SC_RL: the U_J products are stored, never accumulated
                                  (no inner-dimension splitting), and each level's
                                  assembly is owned by the targets (a CTA per row slab
                                  of Lnz(P) adds P's update matrices in source order).
                                  The solve's reductions stay unordered. 0 = off. */
    int32_t threads;           /* host threads of sc_analyze: the graph orderings
                                  (SC_ORDER_GRAPH_ND, SC_ORDER_GRAPH_ML) order the two
                                  halves of each of the top nested-dissection splits
                                  concurrently, and the partition refinement, the
                                  per-supernode glbind sort and the map of A's entries
                                  into Lnz run in blocks on these threads. The analysis is the same for every
                                  value. 0 = the host's hardware threads (at most 64);
                                  1 = serial; < 0 or > 1024 is an argument error (-4). */
    int32_t reserved[2];
} sc_options;

/* Fills o with the defaults: SC_ORDER_NATURAL, nd_leaf 8, pr 1, SC_RLB, SC_FP64,
 * chunk 64, ir_tol 1e-14, ir_maxit 30, pivot_tau 2^-10, spin_limit 1<<22,
 * use_graph 1, merge_frac 0 (fundamental supernodes), tune NULL, deterministic 0, threads 0. Returns
 * SC_OK, or -1 if o is NULL. */
int sc_options_default(sc_options *o);

/* ------------------------------------------------------------- symbolic */
typedef struct sc_symbolic sc_symbolic;

/* Symbolic analysis (Sec. 1 steps 1-2; Sec. 2.1.2; Sec. 3.1): ordering, then
 * elimination tree, postorder, column counts, fundamental supernodes, optional
 * supernode merging, supernodal elimination tree, partition refinement within supernodes,
 * relind(J, p(J)), blocks and relindB(J, P) (Alg. 5), levels, and the
 * device schedule. Host only; no device memory is touched.
 *   n        order of A (>= 1)
 *   colptr   n+1 column pointers into rowind (host)
 *   rowind   row indices of the lower triangle (host)
 *   o        options (host); NULL = defaults
 *   out      receives the new handle
 * Errors: -1..-5 for invalid arguments (unsorted or duplicate indices,
 * entries above the diagonal or a missing diagonal give -3; an option out of
 * range, or deterministic with a variant other than SC_RL, gives -4), SC_ERR_OOM. */
int sc_analyze(int64_t n, const int64_t *colptr, const int32_t *rowind, const sc_options *o,
               sc_symbolic **out);

/* Read-only view of the symbolic structures, for verification. Pointers stay
 * valid until the handle is freed. All arrays are host memory. */
typedef struct sc_symbolic_view {
    int64_t n, nsuper, nnzL, nblocks, npairs;  /* nnzL: entries stored (incl. merged zeros) */
    double flops;               /* sum over columns j of |L_{*,j}|^2, true (fundamental) structure */
    const int32_t *perm;        /* [n]  final ordering, perm[new] = old      */
    const int32_t *sup_ptr;     /* [nsuper+1] first column of each supernode */
    const int32_t *sup_parent;  /* [nsuper]   p(J), -1 for a root            */
    const int64_t *gl_ptr;      /* [nsuper+1] offsets into glbind            */
    const int32_t *glbind;      /* rows of each supernode, ascending         */
    const int64_t *ri_ptr;      /* [nsuper+1] offsets into relind            */
    const int32_t *relind;      /* relind(J, p(J)): |S_J| entries per J       */
    const int64_t *blk_ptr;     /* [nsuper+1] offsets into the block arrays   */
    const int32_t *blk_first;   /* first (global) row of each block           */
    const int32_t *blk_size;    /* rows in each block                         */
    const int32_t *blk_owner;   /* supernode whose columns hold the block     */
    const int64_t *rb_pair_ptr; /* [nsuper+1] offsets into the (J,P) pairs    */
    const int32_t *rb_pair_P;   /* ancestor P of each pair, from p(J) upward  */
    const int64_t *rb_val_ptr;  /* [npairs+1] offsets into rb_val             */
    const int32_t *rb_val;      /* relindB(J,P): one entry per block of J at or above P */
    const int32_t *level;       /* [nsuper] height in the supernodal etree    */
    const int32_t *cparent;     /* [n] column elimination tree of the final ordering */
} sc_symbolic_view;

/* Fills v with the view of s. Errors: -1, -2 for NULL arguments. */
int sc_symbolic_export(const sc_symbolic *s, sc_symbolic_view *v);

/* relind composition of Alg. 4 (a host utility): out[k] =
 * rCP[lenCP - 1 - rJC[k]], i.e. each distance in relind(J,C) picks the entry
 * of relind(C,P) at that distance from its bottom. Errors: -1..-5 when a
 * pointer is NULL or a distance is outside relind(C,P). */
int sc_relind_compose(const int32_t *rJC, int64_t lenJC, const int32_t *rCP, int64_t lenCP, int32_t *out);

/* Writes s to the file at path (created or truncated): the options, the
 * launch-plan settings and every host structure of the analysis, with a
 * checksum, so that a later process can factor without analysing again.
 * Errors: -1, -2 for NULL arguments, SC_ERR_IO, SC_ERR_OOM, SC_ERR_INTERNAL
 * for a handle altered by a test hook. */
int sc_symbolic_save(const sc_symbolic *s, const char *path);

/* Reads a file written by sc_symbolic_save into a new handle (equal to the
 * saved one in every array sc_symbolic_export shows; the device schedule is
 * rebuilt and passes sc_check_schedule before the handle is returned). The
 * file is portable between little-endian 64-bit hosts. Errors: -1, -2 for
 * NULL arguments, SC_ERR_IO (unreadable, truncated, checksum or version
 * mismatch, inconsistent sizes), SC_ERR_OOM. */
int sc_symbolic_load(const char *path, sc_symbolic **out);

/* Frees s. Returns SC_ERR_IN_USE (and frees nothing) while numeric handles
 * made from s are alive; SC_OK otherwise (also for NULL). */
int sc_symbolic_free(sc_symbolic *s);

/* -------------------------------------------------------------- numeric */
typedef struct sc_numeric sc_numeric;

typedef struct sc_factor_info {
    int64_t failed_col;     /* 0, or 1-based caller-order column of the first bad pivot */
    int32_t precision;      /* precision actually used                          */
    int32_t pivot_fallbacks;/* diagonal blocks redone in FP64 (low precision only) */
    double flops;           /* sum_j |L_{*,j}|^2                                */
    double factor_ms;       /* device time of the factorization (CUDA events)   */
    int64_t device_bytes;   /* device memory held by the numeric handle         */
    int32_t kernel_launches;/* kernels launched by one factorization            */
    int32_t reserved[5];
} sc_factor_info;

/* Numeric factorization (Sec. 1 step 3): Alg. 5 (RLB) or Alg. 4 (RL) as set
 * in the symbolic handle's options, on the GPU.
 *   s                symbolic handle (from sc_analyze)
 *   values           FP64 values aligned with the rowind given to sc_analyze;
 *                    host memory if values_on_device == 0, device memory otherwise
 *   precision        enum sc_precision, or -1 for the handle's option
 *   cuda_stream      stream for the device work
 *   out              receives a new numeric handle (device memory is allocated)
 *   info             optional (may be NULL)
 * Returns SC_OK, a positive column index when A is not positive definite
 * (the handle is still returned so it can be freed or refactored), or an
 * error code. Synchronises cuda_stream. */
int sc_factor(sc_symbolic *s, const double *values, int values_on_device, int precision,
              void *cuda_stream, sc_numeric **out, sc_factor_info *info);

/* Refactors an existing numeric handle with new values of the same pattern,
 * reusing its device memory and its captured launch schedule. Same argument
 * meaning and return codes as sc_factor. Synchronises cuda_stream. */
int sc_refactor(sc_numeric *h, const double *values, int values_on_device, void *cuda_stream,
                sc_factor_info *info);

typedef struct sc_solve_info {
    int32_t iterations;    /* refinement iterations (0 for a plain FP64 solve)   */
    int32_t converged;     /* 1 if max backward error <= ir_tol                  */
    double eta_max;        /* max over right-hand sides of the backward error    */
    double solve_ms;       /* device time of the whole solve incl. refinement    */
    double *eta;           /* optional [nrhs] output, caller-owned host memory   */
    int32_t refine;        /* in: -1 = by precision (refine low-precision factors),
                              1 = refine, 0 = no refinement. Without info (NULL)
                              the solve refines by precision.                */
    int32_t kernel_launches; /* out: kernels launched by this solve                */
    int32_t method;        /* in: 0 = classical refinement x += solve(b - A x);
                              1 = conjugate gradients on A x = b preconditioned by
                              the factor (FP64 vectors), for matrices whose
                              condition number times the factor's unit roundoff
                              is too large for classical refinement to converge */
    int32_t max_iterations; /* in: iteration cap of this solve (0 = ir_maxit)    */
    float copy_in_ms;      /* out: device time of copying B in (host -> device
                              when on_device = 0), part of solve_ms           */
    float copy_out_ms;     /* out: device time of copying X out, part of solve_ms */
} sc_solve_info;

/* Solves A X = B (Sec. 1 step 4): permute, forward solve with L, backward
 * solve with L^T, un-permute; with a low-precision factor (or refine = 1),
 * iterative refinement in FP64 until the backward error
 *   eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
 * is at most ir_tol for every column, or ir_maxit iterations.
 *   h        numeric handle
 *   nrhs     number of right-hand sides (>= 1)
 *   B, ldb   n x nrhs column-major FP64 right-hand sides
 *   X, ldx   n x nrhs column-major FP64 solution (may not alias B)
 *   on_device  1 if B and X are device pointers, 0 if host pointers
 *   info     optional; its eta field, when set, receives nrhs values
 * Returns SC_OK, SC_ERR_NOT_CONVERGED (X holds the best iterate), or an
 * error code. Synchronises cuda_stream. */
int sc_solve(sc_numeric *h, int64_t nrhs, const double *B, int64_t ldb, double *X, int64_t ldx,
             int on_device, void *cuda_stream, sc_solve_info *info);

/* Batched symbolic analysis for many independent matrices (the batch is
 * factored as one block-diagonal problem whose levels are aligned by height,
 * so every level of every matrix is in one launch sequence).
 *   count    number of matrices (>= 1)
 *   syms     count symbolic handles (each from sc_analyze); not consumed
 *   out      receives the combined handle; its unknowns are the matrices'
 *            unknowns concatenated in order, and its values array is the
 *            matrices' values arrays concatenated in order.
 * Errors: -1..-3 (-2 also when the handles differ in variant or
 * deterministic), SC_ERR_OOM. */
int sc_analyze_batch(int count, sc_symbolic *const *syms, sc_symbolic **out);

/* Batched numeric factorization of many independent matrices in one launch
 * sequence (a convenience over sc_analyze_batch + sc_factor): the values of
 * matrix i (FP64, aligned with the rowind of syms[i]) are gathered into the
 * batch handle's concatenated values array, and the block-diagonal problem is
 * factored at once.
 *   count      number of matrices (>= 1)
 *   syms       count symbolic handles (each from sc_analyze); not consumed
 *   values     count pointers; values[i] holds nnz(A_i) doubles
 *   values_on_device  1 if every values[i] is a device pointer, 0 if host
 *   precision  enum sc_precision
 *   batch_sym  receives the combined symbolic handle (free it with
 *              sc_symbolic_free after the numeric handle)
 *   out        receives the numeric handle of the batch; solve with sc_solve
 *              on right-hand sides whose rows are the matrices' unknowns
 *              concatenated in order
 *   info       optional, as for sc_factor
 * Returns as sc_factor (a positive value: the failing column of the batch's
 * concatenated ordering), -i for an invalid argument i (count, syms or a NULL
 * syms[i] / values[i], values, values_on_device, precision, batch_sym, out),
 * SC_ERR_OOM or SC_ERR_CUDA. */
int sc_factor_batch(int count, sc_symbolic *const *syms, const double *const *values, int values_on_device,
                    int precision, void *cuda_stream, sc_symbolic **batch_sym, sc_numeric **out,
                    sc_factor_info *info);

/* Copies L to host memory in the canonical supernodal layout: for each
 * supernode J, an m_J x |J| row-major block (row r = glbind(J)[r], column
 * c = column f_J + c of the final ordering, entries above the diagonal 0),
 * blocks concatenated in supernode order, as FP64. out must hold
 * sum_J m_J |J| doubles. Synchronises the handle's last stream. */
int sc_numeric_export_L(const sc_numeric *h, double *out);

/* Read-only view of the factor where it lives, in device memory: for callers
 * that check or use L on the GPU without copying it to the host (at the
 * largest sizes the host copy of sc_numeric_export_L is tens of GB). Storage
 * layout (Sec. 2.1.1's Lnz, one panel per supernode): supernode J is a
 * row-major m_J x panel_ld[J] panel at element offset panel_off[J] of lnz;
 * row r is global row glbind(J)[r] (sc_symbolic_view), column c < |J| is
 * column f_J + c of the final ordering. Entries with c > r (above the
 * diagonal of the panel's top block) and columns c >= |J| (row padding) are
 * not part of L. Entries are FP64 (elt 8) or FP32 (elt 4, every low-precision
 * factor).
 *   lnz        device pointer, valid until the handle is refactored or freed;
 *              the caller must not write through it
 *   panel_off, panel_ld  host arrays [nsuper], valid while the symbolic
 *              handle lives
 * Synchronises the handle's last stream (the factor is complete on return).
 * Errors: -1, -2 for NULL arguments, SC_ERR_CUDA. */
typedef struct sc_factor_view {
    const void *lnz;
    int32_t elt;
    int32_t precision;
    int64_t size;       /* entries of the storage (panels and their padding) */
    int64_t nsuper;
    const int64_t *panel_off;
    const int32_t *panel_ld;
} sc_factor_view;
int sc_numeric_view(const sc_numeric *h, sc_factor_view *v);

/* Per-kernel-class profile of one factorization, for roofline reporting: the
 * factorization runs once outside the CUDA graph with CUDA events around every
 * launch on cuda_stream. Each output array has SC_PROF_CLASSES entries, in the
 * class order: value load (K0), POTRF, TRSM, SIMT tiled products,
 * tensor-core tiled products, warp products, RL update matrices, RL assembly,
 * device-side RLB loops.
 *   ms        summed device time per class (milliseconds, host array)
 *   flops     algorithmic flops per class (2 per multiply-add; POTRF w^3/3,
 *             TRSM rows * w^2; RL assembly counts one per added entry)
 *   launches  launches per class
 * Same values/stream conventions and return codes as sc_refactor. */
#define SC_PROF_CLASSES 9
int sc_factor_profile(sc_numeric *h, const double *values, int values_on_device, void *cuda_stream, double *ms,
                      double *flops, int32_t *launches);

/* Measured FMA throughput of the current GPU (the roofline denominator of the
 * SIMT kernels): a kernel of independent FMA chains timed with CUDA events,
 * best of three. kind 0 = FP64, 1 = FP32. Writes FLOP/s (2 per FMA) to
 * *flops_per_s. Errors: -1 bad kind, -3 NULL output, SC_ERR_CUDA, SC_ERR_OOM. */
int sc_probe_fma_peak(int kind, void *cuda_stream, double *flops_per_s);

/* Size of the launch plan a factorization in `precision` would use (host only,
 * no device memory): out[0..nout) receives, in order, the chunk levels, chunks,
 * product tasks, warp-sized tasks, tiled tasks, SIMT tiles, tensor-core tiles,
 * TRSM tiles, RL assembly pairs, device-loop items, warp-block units, SIMT
 * tiles split along the inner dimension (added atomically), target-owned RL
 * assembly slabs (deterministic plans) and the tensor-core tiles that are 256
 * columns wide. Errors: -1, -2, -3. */
int sc_plan_stats(const sc_symbolic *s, int precision, int64_t *out, int nout);

/* Host-side check of the device schedule of s (no device work): recomputes,
 * from the symbolic structures alone, every address range the factor kernels
 * derive from a product task, a device-loop item (Alg. 5's SYRK on B and GEMMs
 * of the runs B' through relindB) or an RL assembly pair (Alg. 4, relind), and
 * checks that each lies inside its source panel / target panel, in the lower
 * trapezoid of the target, that the target is the source's own panel (in-panel
 * updates, the only plain non-atomic writes) or an ancestor's, that a run B'
 * maps to consecutive rows of P, that the columns read are factored at the
 * product's level or before and the columns written after it, and that the
 * critical-product flag matches the target's chunk level. Where each entry
 * lands is checked against its definition: the target row and column are the
 * positions in glbind(P) of the source rows (the relind maps are not used).
 *   out[0..nout): products checked, loop products checked, RL assembly entries
 *   checked, level of the first violation (-1 if none), its kind (0 if none:
 *   1 source range, 2 target range, 3 trapezoid, 4 not an ancestor, 5 level
 *   order, 6 critical flag, 7 run mapping, 8 RL pool, 9 RL relind, 10 plain
 *   write outside the own panel, 11 an entry not landing at its row's and
 *   column's positions in glbind(P), 12 a product that the tensor-core
 *   precisions route to tcgen05 tiles would multiply panel columns past its
 *   inner dimension: its K is not a whole number of 8-column MMA steps and
 *   real columns of the source panel follow it; 13 in a deterministic
 *   schedule, a launch plan (FP64 or tensor-core) with a product tile split
 *   along the inner dimension, or a target row of an RL assembly pair that no
 *   slab of its target owns, or a slab whose pairs are not one target's in
 *   source order).
 * Returns SC_OK, SC_ERR_INTERNAL when a violation is found, -1 / -2 for NULL
 * arguments. */
int sc_check_schedule(const sc_symbolic *s, int64_t *out, int nout);

/* Test hook: plants one mistake of the given kind (1 a GEMM target one row
 * too high, 2 a critical product marked as other, 3 an in-panel update reading
 * one column too many, 4 a loop item reaching past its blocks, 5 tensor-core
 * routing that ignores the K-tail rule, 6 a deterministic plan whose first
 * level of assembly slabs misses a target row) in s's schedule
 * so that a test can see sc_check_schedule find it. s can no longer be factored
 * (sc_factor returns SC_ERR_INTERNAL). Returns SC_OK, -1, -2 for a bad kind,
 * or SC_ERR_UNSUPPORTED when the schedule has no entry of that kind. */
int sc_test_perturb_schedule(sc_symbolic *s, int kind);

/* Launch-plan autotuner for one matrix (the level schedule and the product
 * routing of Alg. 4/5 are fixed by the structure; the thresholds that cut
 * products into tiled tasks, device-loop items, tensor-core or warp-block
 * work, and the lookahead split, are chosen here). Starting from s's current
 * table, it visits the fields of sc_tune_table one at a time (coordinate
 * descent, one pass), factors the matrix under each candidate value (one
 * untimed factorization, then `reps` timed ones; CUDA events) and keeps a
 * value when its median time is below 0.98x the best so far. The winner is
 * stored in s (every later sc_factor of s uses it) and written to *best with
 * its time.
 *   s            symbolic handle with no live numeric handles
 *   values       FP64 values as for sc_factor (host or device)
 *   precision    enum sc_precision, or -1 for the handle's option
 *   reps         timed factorizations per candidate (1..15)
 *   cuda_stream  stream for the device work (synchronised)
 *   best         out: the chosen table, factor_ms set
 *   tried        optional out: settings timed (incl. the starting one)
 * Errors: -1..-8 for invalid arguments, SC_ERR_IN_USE when numeric handles of
 * s are alive, a positive column when A is not positive definite, and the
 * codes of sc_factor. On error s keeps its previous table. */
int sc_tune(sc_symbolic *s, const double *values, int values_on_device, int precision, int reps, void *cuda_stream,
            sc_tune_table *best, int32_t *tried);

/* Allocation-free residual and backward error. The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory during a call -- applications that give all device memory to
 * their own pool up front, or latency-critical loops where a cudaMalloc (which
 * can synchronise the whole device) is not acceptable. It computes, for each
 * column c of X,
 *   R_c = B_c - A X_c  and  eta_c = ||R_c||_inf / (||A||_inf ||X_c||_inf + ||B_c||_inf),
 * the same check sc_solve reports, and calls no allocation routine.
 *   n                 order of A (>= 1)
 *   row_ptr, col, val A as a full symmetric CSR (both triangles): row_ptr[n+1]
 *                     int64, col int32, val FP64 -- device memory
 *   nrhs              columns of B, X, R: 1..SC_NOALLOC_MAX_RHS
 *   B, ldb / X, ldx   column-major FP64 inputs (device memory), ld >= n
 *   R, ldr            column-major FP64 output (device memory), ld >= n. R may
 *                     be B itself (R == B with ldr == ldb: each row reads its
 *                     B entry before writing R) but must not overlap X, which
 *                     other rows are still reading.
 *   eta               nrhs FP64 outputs (device memory); NaN for a column whose
 *                     residual, X, B or ||A|| holds a NaN or an infinity, so a
 *                     test eta <= tol never passes on such a column
 *   cuda_stream       stream for the work; the call returns without waiting
 * Working memory is one fixed array of 3 * SC_NOALLOC_MAX_RHS + 1 doubles
 * (about 24 KB) built into the library; every GPU that loads the library
 * holds it until the process exits. Each call looks up that array's device
 * address on the current device (so it is current again after a device reset),
 * except while cuda_stream is being captured, when the address found by the
 * last call on that device is reused: the first call on a device therefore
 * has to come before any stream capture (a first call during a capture returns
 * SC_ERR_CUDA). All calls share the array and each call clears it
 * first, so calls whose work overlaps on the GPU (other streams, other
 * threads) race and must be serialised by the caller.
 * Errors: -1..-12 for the arguments in order (-5: nrhs outside 1..max),
 * SC_ERR_CUDA. */
#define SC_NOALLOC_MAX_RHS 1024
int sc_residual_eta_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val, int64_t nrhs,
                            const double *B, int64_t ldb, const double *X, int64_t ldx, double *R, int64_t ldr,
                            double *eta, void *cuda_stream);

/* Test hook for the failure path of the solve's bounded waits (no counterpart
 * in the paper). The next sc_solve on h runs with the forward sweep expecting
 * one arrival more at chunk `chunk` (0-based, in the order of the level
 * schedule; nchunks - 1 is the root's last chunk) than the sweep delivers, so
 * the waits at that chunk give up after spin_limit polls and sc_solve returns
 * SC_ERR_TIMEOUT; every other wait sees the error and stops. The expected
 * count is restored afterwards, so later solves on h run normally. Nothing
 * faults: the wait ends by its iteration limit.
 * Errors: -1 (h NULL), -2 (chunk < 0; a chunk beyond the last makes the next
 * sc_solve return -1). */
int sc_test_stall_solve(sc_numeric *h, int64_t chunk);

/* Test hook for the failure path of the per-level persistent kernel's bounded
 * waits (fused plans; no counterpart in the paper). The next sc_refactor on h
 * runs with the units that read chunk `chunk` (0-based, in the order of the
 * level schedule) waiting for one more POTRF / TRSM completion than the chunk
 * delivers: their waits give up after spin_limit polls, every other wait sees
 * the error and stops, and sc_refactor returns SC_ERR_TIMEOUT. The target is
 * restored afterwards, so later factorizations run normally. Nothing faults.
 * Errors: -1 (h NULL), -2 (chunk < 0); the next factorization returns
 * SC_ERR_UNSUPPORTED if h has no per-level kernel or chunk is out of range. */
int sc_test_stall_factor(sc_numeric *h, int64_t chunk);

/* Frees h and its device memory. NULL is accepted. */
void sc_numeric_free(sc_numeric *h);

/* Human-readable text for a return code. Never NULL. */
const char *sc_strerror(int code);

/* Build identification: the CUDA architecture the kernels were compiled for. */
const char *sc_build_info(void);

#ifdef __cplusplus
}
#endif
#endif /* SC_H */
