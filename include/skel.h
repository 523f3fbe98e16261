/*
 * skel.h — C-ABI of the GB300 skeletonized fast multipole apply.
 *
 * The library evaluates u_i = sum_{j != i} G(x_i, x_j) q_j (Section 1,
 * Eq. (1)) for the Laplace kernels of Eq. (2) and the 3D low-frequency
 * Helmholtz kernel of Eq. (5) (normalised as e^{i kappa r} / (4 pi r)) with
 * the strong recursive skeletonization FMM of the paper:
 *   - skel_build: adaptive 2:1-balanced tree and neighbor lists (Section 3.1)
 *     and the proxy-surface interpolative decompositions of Algorithm 1
 *     (Section 2.1), computed on the host in FP64 / complex128 and uploaded
 *     to the GPU once;
 *   - skel_apply: Algorithm 2 (upward pass, ifo / ifs / tfo translations,
 *     level-1 sum, downward pass) in hand-written sm_103a CUDA kernels.
 *
 * Conventions shared by every entry point:
 *   - Every function returns SKEL_OK (0) or a negative SKEL_ERR_* code; no
 *     C++ exception crosses this boundary. skel_last_error() gives a
 *     message for the last failure on the calling thread.
 *   - Points are host FP64, row-major n x dim, and are copied.
 *   - Charges q and potentials u are n x nrhs with each right-hand side
 *     contiguous (column-major, user point order). FP64 precision uses
 *     double (complex128 as interleaved (re, im) for Helmholtz); FP32 and
 *     FP32_TC use float (complex64).
 *   - A handle owns all host and device memory of its plan. One handle may be
 *     used by one apply at a time (it owns the apply's workspace).
 */
#ifndef SKEL_H
#define SKEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define SKEL_OK            0
#define SKEL_ERR_ARG      (-1)  /* invalid argument (null, size, range, layout) */
#define SKEL_ERR_OOM      (-2)  /* host or device allocation failed            */
#define SKEL_ERR_CUDA     (-3)  /* a CUDA runtime call failed                  */
#define SKEL_ERR_TIMEOUT  (-4)  /* a bounded device wait gave up               */
#define SKEL_ERR_NUMERIC  (-5)  /* non-finite input                            */
#define SKEL_ERR_STATE    (-6)  /* handle not in the right state (e.g. host-only plan) */

/* ---- kernels (Eq. (2), Eq. (5)) ----------------------------------------- */
#define SKEL_LAPLACE_2D    0    /* G = -log|x-y| / (2 pi)          */
#define SKEL_LAPLACE_3D    1    /* G = 1 / (4 pi |x-y|)            */
#define SKEL_HELMHOLTZ_3D  2    /* G = e^{i kappa r} / (4 pi r)    */
#define SKEL_HELMHOLTZ_2D  3    /* G = (i/4) H_0^(1)(kappa r), kappa > 0 (the 2D Helmholtz
                                   experiments of Section 5); complex like HELMHOLTZ_3D */

/* ---- apply precisions ------------------------------------------------- */
#define SKEL_FP64     0   /* FP64 arithmetic, double charges/potentials            */
#define SKEL_FP32     1   /* FP32 arithmetic on the CUDA cores, float in/out       */
#define SKEL_FP32_TC  2   /* FP32 kernel evaluation, tensor-core contractions over
                             right-hand sides (3-pass TF32 split, FP32 accumulate)
                             in passes of 32 columns (3D Helmholtz: 16 complex
                             columns, [u_r | u_i] = G_r [q_r | q_i] + G_i [-q_i | q_r]);
                             2D / 3D Laplace and 3D Helmholtz with nrhs >= 4 —
                             otherwise the FP32 CUDA-core path runs */

typedef struct skel_plan* skel_handle;

typedef struct {
    int    kind;    /* SKEL_LAPLACE_2D | SKEL_LAPLACE_3D | SKEL_HELMHOLTZ_3D | SKEL_HELMHOLTZ_2D */
    double kappa;   /* wavenumber, Helmholtz only                             */
} skel_kernel;

typedef struct {
    int proxy_p;      /* proxy Chebyshev nodes per box edge; 0 = default (2D: 32, 3D: 12) */
    int nrhs_max;     /* largest nrhs any later apply will use, <= 256; 0 = 32           */
    int host_only;    /* 1 = build the plan on the host only; apply returns SKEL_ERR_STATE */
    int num_threads;  /* host threads used by the build; 0 = all                          */
    int device_build; /* 1 = Algorithm 1 (proxy matrices, pivoted QR, T) on the current
                         CUDA device in FP64, one CTA per box; 0 = on the host. Same
                         ranks and operators up to rounding (ties in the pivot order
                         may resolve differently). Needs host_only = 0.               */
    int store_tiles;  /* stored-operator mode: evaluate the kernel values of the
                         tensor-core translations once at build and keep them on the
                         device (skel_stats.stored_tile_bytes); FP32_TC applies then
                         read them instead of evaluating the kernel.
                         1 = per-tile store: every tile's rows x 32 values; results
                             equal the on-the-fly apply bit for bit.
                         2 = symmetric store: the real kernels are symmetric, so a
                             block two tiles share is stored once (about half the
                             bytes) and read transposed by one of them; results equal
                             the on-the-fly apply up to FP32 rounding of those values.
                         0 = none. Real kernels only (ignored otherwise).
                         SKEL_ERR_OOM if the values do not fit.                         */
    int store_stages; /* per-tile store: the form of its apply kernel: 4 bulk-copy
                         stages per CTA (two CTAs per SM), 8 (one CTA per SM), or 5 =
                         split rings (5 slots of kernel values released when read,
                         3 of B operand released by the MMAs); 0 = 4. Same result
                         every way; skel_autotune may change it.                        */
    int updown_tc;    /* 1 = FP32_TC applies of a real kernel also run the upward and
                         downward skeleton GEMMs on the tensor cores (three-part TF32
                         split, 6 products); the plan keeps T in tile order (about the
                         size of T twice). The tensor core's accumulation is less
                         accurate than FP32 FMAs on these cancelling sums (relative error
                         1.3e-6 instead of 7.8e-7 at N = 2^20, tol 1e-6), so the default
                         0 keeps them on the CUDA cores.                               */
} skel_options;

typedef struct {
    int64_t n_points;
    int     dim;
    int     n_levels;        /* L: deepest level (root = level 0)                     */
    int64_t n_boxes;         /* including the root                                     */
    int64_t n_leaves;
    int     k_max;           /* largest skeleton rank on levels >= 2                   */
    int64_t n_index;         /* sum over boxes of |I_B|                                */
    int64_t n_T;             /* sum over boxes of k_B (|I_B| - k_B) (T entries)        */
    int64_t n_colleague, n_coarse, n_fine;   /* neighbor-list entries                  */
    int64_t pairs_direct;    /* kernel evaluations per apply between touching leaves   */
    int64_t pairs_far;       /* kernel evaluations per apply on all other translations */
    int64_t n_work_items;    /* near-field work items of the device plan               */
    double  t_tree;          /* seconds: tree + balance + neighbor lists               */
    double  t_skel;          /* seconds: Algorithm 1 (all IDs)                         */
    double  t_upload;        /* seconds: device plan construction and upload           */
    int64_t device_bytes;    /* device memory held by the plan (all precisions)       */
    int64_t n_tc_items;      /* FP32_TC: tensor-core work items (128 target rows each) */
    int64_t n_tc_tiles;      /* FP32_TC: source tiles streamed by them (32 sources)    */
    int64_t n_mix_items;     /* FP32_TC: CUDA-core items for the remaining small boxes */
    int64_t pairs_tc;        /* FP32_TC: kernel evaluations (of pairs_direct + pairs_far)
                                done by the tensor-core items, per 32 right-hand sides */
    int     skel_on_device;  /* 1 if Algorithm 1 ran on the GPU (device_build)          */
    double  t_id_kernels;    /* device build: seconds inside the ID kernels (CUDA events) */
    double  id_gflop;        /* device build: GFLOP of the QR reflector updates (FP64)   */
    int64_t stored_tile_bytes; /* store_tiles: device bytes of the stored kernel tiles   */
    int     n_proxy;         /* proxy points per box (2D: 4p, 3D: 6p^2; Section 2.1)     */
    int64_t pairs_stored;    /* FP32_TC: kept kernel values the symmetric store holds
                                once (of pairs_tc; the others are the same values read
                                transposed)                                              */
    int     store_mode;      /* stored-operator mode the plan holds: 0 none, 1 per-tile,
                                2 symmetric                                              */
} skel_stats;

/*
 * skel_build — tree, neighbor lists (Section 3.1) and Algorithm 1 (on the
 * host, or on the GPU with opts.device_build), then the device plan.
 *   points     host, n x dim row-major FP64, copied; must be finite
 *   n, dim     n >= 1; dim = 2 for SKEL_LAPLACE_2D, 3 otherwise
 *   k          kernel (kappa >= 0 for Helmholtz)
 *   tol        ID tolerance, 0 < tol < 1 (rank rule |R_kk| > tol |R_00|)
 *   leaf_size  b >= 1: boxes with more than b points are split (Section 3.1)
 *   opts       may be NULL (defaults)
 *   out        receives the handle; untouched on error
 * The upload goes to the CUDA device that is current on the calling thread.
 * Errors: SKEL_ERR_ARG, SKEL_ERR_NUMERIC (non-finite point), SKEL_ERR_OOM,
 * SKEL_ERR_CUDA.
 */
int skel_build(const double* points, int64_t n, int dim, skel_kernel k,
               double tol, int leaf_size, const skel_options* opts,
               skel_handle* out);

/*
 * skel_build_batch — skel_build for nsets independent point sets with the
 * same kernel, tolerance, leaf size and options (the batched workload of many
 * small sets; pair it with skel_apply_batch).
 *   points     nsets host pointers, set i: n[i] x dim row-major FP64, copied
 *   n          nsets sizes, each >= 1
 *   out        nsets handles; all written on success, none on error
 * Every argument of every set is checked before any work. The host phases of
 * many sets run in parallel, one set per host thread (when nsets is at least
 * the thread count and Algorithm 1 runs on the host); the device plans are
 * created one after the other. On any error every plan built so far is
 * freed; the message names the failing set. Errors as skel_build.
 */
int skel_build_batch(int nsets, const double* const* points, const int64_t* n, int dim,
                     skel_kernel k, double tol, int leaf_size,
                     const skel_options* opts, skel_handle* out);

/*
 * skel_apply — u = A~ q by Algorithm 2 on the GPU.
 *   q, u       n x nrhs (see conventions); device pointers (the common case:
 *              asynchronous on `stream`, no allocation, CUDA-graph
 *              capturable) or host pointers: page-locked host memory
 *              (cudaHostAlloc, cudaHostRegister) is read and written in place
 *              by the apply's permutation kernels, other host memory is
 *              staged through device buffers that the handle allocates on
 *              first use; either way the call synchronises `stream` before
 *              returning. q and u must not overlap; u is overwritten.
 *   nrhs       1 <= nrhs <= opts.nrhs_max
 *   precision  SKEL_FP64 | SKEL_FP32 | SKEL_FP32_TC
 *   stream     a cudaStream_t, or NULL for the legacy default stream
 * Errors: SKEL_ERR_ARG, SKEL_ERR_STATE (host-only plan), SKEL_ERR_CUDA,
 * SKEL_ERR_OOM (host staging only).
 */
int skel_apply(skel_handle h, const void* q, void* u, int nrhs, int precision,
               void* stream);

/*
 * skel_apply_transpose — qbar = A~^T ubar (plain transpose, no conjugation).
 * Source: the factorisation of Section 2.2, where a well-separated block is
 * A_{Bi,Bj} ~ E_{Bi} A_{Si,Sj} F_{Bj} with F_B = [T_B  I] and E_B = F_B^*
 * (E_B = [T_B^*; I]), applied level by level by Algorithm 2. Transposing
 * every factor gives F_{Bj}^T A_{Sj,Si} E_{Bi}^T: for the complex-symmetric
 * Helmholtz kernels that is the same algorithm with every T replaced by
 * conj(T) in both passes (the kernel blocks are complex-symmetric and the
 * neighbor relations symmetric); for the real Laplace kernels A~ is
 * symmetric and this equals skel_apply.
 * Same arguments, layout, ownership and errors as skel_apply.
 */
int skel_apply_transpose(skel_handle h, const void* ubar, void* qbar, int nrhs,
                         int precision, void* stream);

/*
 * skel_apply_batch — skel_apply (transpose = 0) or skel_apply_transpose
 * (transpose = 1) on nsets independent plans, queued back to back on one
 * stream with no host synchronisation, so that a whole batch of point sets
 * (and its adjoint) can be captured into one CUDA graph.
 *   hs         nsets handles, all with device plans on the current device
 *   q, u       nsets device pointers each (plan i: n_i x nrhs column-major);
 *              host pointers are rejected (no staging inside a batch)
 *   nrhs       1 <= nrhs <= every plan's nrhs_max
 * Every argument is checked before anything is queued (SKEL_ERR_ARG,
 * SKEL_ERR_STATE); each plan works in its own buffers, so the sets share no
 * memory. The paper applies one point set at a time; batching independent
 * sets is this library's addition.
 */
int skel_apply_batch(const skel_handle* hs, int nsets, const void* const* q, void* const* u, int nrhs,
                     int precision, int transpose, void* stream);

/*
 * skel_merge — one plan that applies many independent plans in a single
 * pass: each phase of Algorithm 2 (permutation, upward pass per level,
 * translations, downward pass per level, permutation) runs as one launch
 * over the boxes, items and points of all sets, instead of one apply per
 * set. This is the paper's batching of same-shaped work across boxes (its
 * GPU implementation, Section 5.2) carried across point sets; the merge
 * itself is this library's addition. The merged plan's points are the sets'
 * points one after the other: set i holds points [o_i, o_i + n_i) with
 * o_i = n_0 + ... + n_{i-1}, so q and u are N x nrhs column-major with
 * N = n_0 + ... + n_{nsets-1} (in each right-hand side, set 0's n_0 values,
 * then set 1's, ...). skel_apply, skel_apply_transpose, skel_autotune,
 * skel_set_profiling, skel_device_status and skel_info work on it as on any
 * plan (skel_info sums the sets' statistics; k_max and n_levels are the
 * largest); the plan-exchange calls return SKEL_ERR_STATE. No translation
 * crosses a set, and every set's values equal its own apply bit for bit.
 *   hs      nsets >= 1 handles of one kernel (kind, kappa) and dim, built by
 *           skel_build / skel_build_batch / skel_plan_import (not merged);
 *           they stay valid and independent (the merged plan has its own
 *           device copy of every operator)
 *   opts    nrhs_max, store_tiles and host_only are read (NULL: 32, no
 *           stored tiles, a device plan; host_only = 1 forms the merged
 *           layout and its statistics only, and applies return SKEL_ERR_STATE)
 *   out     receives the merged handle; untouched on error
 * The upload goes to the current CUDA device.
 * Errors: SKEL_ERR_ARG, SKEL_ERR_OOM, SKEL_ERR_CUDA.
 */
int skel_merge(const skel_handle* hs, int nsets, const skel_options* opts, skel_handle* out);

/*
 * skel_free — release the handle and all the host and device memory that
 * skel_build (or skel_plan_import) allocated for it: the tree, the index sets
 * and every interpolation matrix T_B (the paper's M_proj, the memory of all
 * T_B in the results notation of Section 5.2), the device operators and the
 * apply's workspace. NULL is a no-op. No apply on the handle may still be
 * running (the call does not wait for the caller's streams).
 */
void skel_free(skel_handle h);

/*
 * skel_info — the quantities the paper reports for a run (results notation of
 * Section 5.2): N (n_points), k_max (largest skeleton rank on levels
 * >= 2), T_tree (t_tree: tree, 2:1
 * balance and neighbor lists of Section 3.1), T_skel (t_skel: Algorithm 1)
 * and the size of all T_B (n_T entries; M_proj = n_T x 8 or 16 bytes), plus
 * the work counts of the apply (Section 4's cost terms: kernel evaluations
 * of the translations, boxes, neighbor-list entries) and device figures.
 *   h   a handle from skel_build / skel_plan_import
 *   s   caller-owned, filled completely (fields that do not apply are 0)
 * Errors: SKEL_ERR_ARG (NULL argument).
 */
int skel_info(skel_handle h, skel_stats* s);

/*
 * skel_last_error — message of the last failed call on this thread (or an
 * empty string). The pointer stays valid until the next call on the thread.
 * The paper has no counterpart (it is this C-ABI's error reporting).
 */
const char* skel_last_error(void);

/*
 * ---- plan exchange ----------------------------------------------------
 * A plan is the tree plus one ID per box, in this flat format (boxes in
 * (level, Morton key) order, children by child index sum_d bit_d 2^d):
 *   level[b], coord[b*dim + d]   box level and integer cell coordinates
 *   parent[b]                    parent box, -1 for the root
 *   is_leaf[b]                   1 for leaves
 *   idx[idx_ptr[b] ..]           I_B as user point indices in slot order
 *                                (leaf: ascending; tree box: the children's
 *                                skeletons concatenated in child order)
 *   piv[idx_ptr[b] ..]           positions within I_B: the first k[b] are the
 *                                skeleton S_B in pivot order, then R_B
 *   T[T_ptr[b] ..]               k_b x (|I_B| - k_b), column-major; complex
 *                                plans store interleaved (re, im) pairs and
 *                                T_ptr counts complex entries
 * The root (level 0) has an empty index set unless it is the only box.
 */
typedef struct {
    int64_t n_boxes;
    int64_t n_index;
    int64_t n_T;          /* entries (complex entries count once)      */
    int     dim;
    int     is_complex;
    double  center[3];    /* root box centre (dim entries used)        */
    double  side;         /* root box side                             */
} skel_plan_dims;

/* skel_plan_get_dims — sizes needed to export a plan. */
int skel_plan_get_dims(skel_handle h, skel_plan_dims* d);

/*
 * skel_plan_export — copy the plan into caller-owned host arrays sized by
 * skel_plan_get_dims (level, parent, is_leaf, k: n_boxes; coord:
 * n_boxes*dim; idx_ptr, T_ptr: n_boxes+1; idx, piv: n_index; T: n_T, doubled
 * for complex). Any pointer may be NULL to skip that array.
 */
int skel_plan_export(skel_handle h, int32_t* level, int32_t* coord,
                     int64_t* parent, int8_t* is_leaf, int64_t* idx_ptr,
                     int64_t* idx, int64_t* piv, int32_t* k, int64_t* T_ptr,
                     double* T);

/*
 * skel_plan_import — build a handle from an externally computed plan in the
 * format above (for example the IDs of another implementation of Algorithm
 * 1) instead of running the library's own tree and ID. The library checks
 * the plan's consistency (box order, parents, slot structure of every index
 * set, permutations), derives the neighbor lists itself and uploads.
 *   points, n, dim, k   as for skel_build
 *   center, side        root box (dim entries of center)
 * Errors: SKEL_ERR_ARG for any inconsistency, plus those of skel_build.
 */
int skel_plan_import(const double* points, int64_t n, int dim, skel_kernel k,
                     const double* center, double side, int64_t n_boxes,
                     const int32_t* level, const int32_t* coord,
                     const int64_t* parent, const int8_t* is_leaf,
                     const int64_t* idx_ptr, const int64_t* idx,
                     const int64_t* piv, const int32_t* kk,
                     const int64_t* T_ptr, const double* T,
                     const skel_options* opts, skel_handle* out);

/*
 * skel_neighbors_export — one neighbor relation in CSR form.
 *   which   0 = colleagues (same level, touching, self included),
 *           1 = coarse neighbors (leaves one level up touching the box),
 *           2 = fine neighbors (boxes one level down touching a leaf)
 *   ptr     n_boxes + 1 entries (always filled)
 *   list    ptr[n_boxes] entries, or NULL to query the size only
 */
int skel_neighbors_export(skel_handle h, int which, int64_t* ptr, int64_t* list);

/*
 * ---- phase timing -------------------------------------------------------
 * skel_set_profiling(h, m) makes each of the next m applies record CUDA
 * events on its stream at the boundaries of its six phases: permutation in,
 * upward pass, translations (the near-field kernel), reduction of partial
 * sums, downward pass, permutation out, plus one where the main translation
 * kernel starts (eight event records per apply and nothing else; the events
 * are created here, not in the apply). m = 0 turns it off. skel_last_timings
 * waits for the captured applies and returns each phase's duration summed
 * over them, in milliseconds, with the number of kernels they launched and
 * the number of applies captured.
 */
typedef struct {
    double ms[6];          /* permute_in, upward, translations, reduce, downward, permute_out */
    int    launches;       /* kernels launched by the captured applies                        */
    int    n_applies;      /* applies captured                                                */
    double ms_main;        /* the part of ms[2] spent in the main translation kernel: the
                              tensor-core launches of FP32_TC, else the whole phase          */
    int    main_launches;  /* launches of that kernel                                         */
} skel_timings;

/* skel_set_profiling — capture the next max_applies applies (0 = off, <= 100000). */
int skel_set_profiling(skel_handle h, int max_applies);

/* skel_last_timings — summed phase durations of the captured applies;
 * SKEL_ERR_STATE if profiling is off. */
int skel_last_timings(skel_handle h, skel_timings* t);

/*
 * skel_device_status — the tensor-core apply waits on its own tensor-core
 * completions with bounded spins. If one ever gives up, the kernel raises a
 * device status word (and that apply's result is invalid) instead of hanging.
 * This call waits for the device, returns SKEL_ERR_TIMEOUT if the word was
 * raised since the last call (else SKEL_OK) and clears it.
 */
int skel_device_status(skel_handle h);

/*
 * ---- failure-detection test hooks (the paper has no counterpart) ---------
 * skel_test_withhold_tile — the next FP32_TC apply on h (tensor-core path)
 * holds back the bulk copies of the first source tile of its first
 * tensor-core item until the compute warps' bounded wait for them has run
 * out, with every bounded wait of that apply limited to wait_limit_ms
 * (0 < wait_limit_ms <= 2000). The copies are then issued and waited for,
 * so every barrier phase still completes once per tile and nothing faults
 * or hangs; that apply's result is invalid and the next skel_device_status
 * returns SKEL_ERR_TIMEOUT. Later applies are unaffected.
 * Errors: SKEL_ERR_ARG, SKEL_ERR_STATE (host-only plan, 2D Helmholtz, or
 * no tensor-core items).
 */
int skel_test_withhold_tile(skel_handle h, double wait_limit_ms);

/*
 * skel_test_fail_alloc — the countdown-th device allocation (plan arrays,
 * stored tiles, host-pointer staging) the library makes after this call
 * fails as if memory were exhausted; countdown = 0 turns the hook off.
 * Process-wide. The failing call returns SKEL_ERR_OOM after freeing what it
 * had allocated, and leaves its output handle untouched.
 * Errors: SKEL_ERR_ARG (countdown < 0).
 */
int skel_test_fail_alloc(int countdown);

/*
 * skel_test_set_updown — force the launch shape of every level's FP32
 * upward and downward pass on h (what skel_autotune otherwise picks per
 * level): code 0 = the default rule, 1 / 2 / 4 / 8 = the plain kernel with
 * that many warps per CTA, 17 / 18 / 20 / 24 = the asynchronous-copy kernel
 * with 1 / 2 / 4 / 8 warps. Every shape gives the same result bit for bit,
 * which tests check with it.
 * Errors: SKEL_ERR_ARG (NULL handle, other codes), SKEL_ERR_STATE (host-only
 * plan).
 */
int skel_test_set_updown(skel_handle h, int code);

/*
 * skel_autotune — pick, by measurement on this plan and device, the variants
 * the FP32 applies of nrhs right-hand sides will use: per tree level and
 * direction the launch shape of the up/down kernel (1, 2, 4 or 8 warps per
 * CTA sharing a 32-row block, with the blocks staged through registers or by
 * asynchronous copies; every shape adds the same partial sums in the same
 * order), the pipeline depth of the on-the-fly tensor-core kernel (4, 6
 * or 8 bulk-copy stages; same arithmetic), and for the tensor-core
 * translations (real kernels, nrhs >= 4) whether the
 * kernel values are evaluated on the fly or read from a store (the choice
 * between operators stored and evaluated on the fly: the per-tile and the
 * symmetric store are each tried if allow_store and they fit the free device
 * memory with 2 GB to spare; the fastest of the three is kept, stores that
 * lose are freed). Every launch shape computes the same result; the
 * symmetric store differs from the others by FP32 rounding only, so tuning
 * changes speed and memory, not accuracy. Synchronous on `stream`, uses the
 * plan's own buffers (no concurrent apply on the handle; not capturable).
 *   h            plan with a device part; real kernels only
 *   nrhs         1 .. nrhs_max
 *   out          may be NULL; receives the measurements
 * Errors: SKEL_ERR_ARG, SKEL_ERR_STATE (host-only plan), SKEL_ERR_OOM,
 * SKEL_ERR_CUDA, SKEL_ERR_TIMEOUT (a bounded wait of the fill pass gave up).
 */
typedef struct {
    double ms_onfly;          /* one tensor-core pass, kernel evaluated on the fly (-1: not timed) */
    double ms_stored;         /* the same reading the per-tile store (-1: not timed)            */
    int    stored;            /* store mode the plan keeps after tuning: 0 none, 1 per-tile,
                                 2 symmetric                                                     */
    int    n_updown;          /* up/down level launches tuned (levels x 2 directions)           */
    int    n_changed;         /* of those, choices unlike the default rule                      */
    double ms_updown_default; /* their summed time with the default rule                        */
    double ms_updown_tuned;   /* and with the chosen variants                                   */
    int    tc_stages;         /* pipeline depth (bulk-copy stages) chosen for the on-the-fly
                                 tensor-core kernel: 4, 6 or 8 (0: not tuned)                  */
    double ms_sym;            /* one tensor-core pass reading the symmetric store (-1: not timed) */
    int    tcs_stages;        /* form chosen for the per-tile stored kernel (store_stages: 4, 5
                                 or 8); 0: not tuned                                             */
} skel_tuning;
int skel_autotune(skel_handle h, int nrhs, int allow_store, void* stream, skel_tuning* out);

/*
 * skel_direct_noalloc — u = A q by direct summation (FP64; complex128 for
 * Helmholtz), for callers that cannot allocate device memory: code running
 * inside a framework that owns (and has reserved) the device memory pool, or
 * a loop that must not take the device-wide synchronisation a cudaMalloc or
 * cudaFree can cause. The paper has no counterpart: it is the plan-free form
 * of the translation kernel's partial-sum scheme, and it allocates nothing.
 *   points     device, n x dim row-major FP64
 *   q, u       device, n x nrhs (each right-hand side contiguous); u is
 *              overwritten; asynchronous on `stream`
 *   n, dim, k  as for skel_build, kappa rules included (coincident points
 *              contribute nothing)
 * Its partial sums live in one 32 MiB __device__ array inside the library:
 * every GPU that loads the library holds it until the process exits, and all
 * calls share it, so calls that overlap on the GPU race. Each call overwrites
 * every scratch value it reads; nothing has to start at zero. The first call
 * on a device looks up the array's device address there; make that first
 * call before any stream capture.
 * Errors: SKEL_ERR_ARG for NULL or host pointers, pointers to another
 * device's memory, a bad kernel, kappa or size, or a problem whose partial
 * sums exceed the array (n up to 131,072 for real kernels, 91,168 for the
 * Helmholtz kernels); SKEL_ERR_CUDA for an error the caller's earlier work
 * left pending (reported and cleared before anything is launched) or for a
 * failed launch of this call's kernels.
 */
int skel_direct_noalloc(const double* points, int64_t n, int dim, skel_kernel k,
                        const double* q, double* u, int nrhs, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SKEL_H */
