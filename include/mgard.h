/*
 * mgard.h -- C ABI of the GB300 (sm_103a) multilevel decomposition library.
 *
 * The library computes the multigrid-based hierarchical decomposition of a
 * structured 1D-3D grid and its inverse (Chen et al., "Accelerating
 * Multigrid-based Hierarchical Scientific Data Refactoring on GPUs",
 * Section II-A, Eq. 1 and Eq. 2):
 *
 *   decomposition, level l = L .. 1:
 *     coefficients  c = u - Pi_{l-1} u          on N_l \ N_{l-1}
 *     load vector   f = R_l M_l vec(C_l)        C_l = c, zero on N_{l-1}
 *     correction    M_{l-1} z = f               (tensor-product mass matrix)
 *     update        u(N_{l-1}) += z
 *   recomposition runs the same stages in reverse, level 1 .. L.
 *
 * Layout (Fig. 3): the field is a dense row-major array, dims[0] slowest.
 * The transform is in place: after decomposition every node of
 * N_l \ N_{l-1} holds its level-l coefficient and the nodes of N_0 hold the
 * coarsest values.  N_l is the set of nodes whose indices are multiples of
 * 2^(L-l) in every dimension.
 *
 * Shapes: 1 <= ndim <= 3; every dims[k] >= 2 with (dims[k]-1) divisible by
 * 2^L.  Dimensions of size 1 are squeezed away.  nlevels = -1 selects the
 * largest L allowed by the shape.
 *
 * Memory: every pointer named d_* is device memory owned by the caller; every
 * pointer named h_* is host memory owned by the caller (pinned for
 * asynchronous copies).  The plan owns its small device tables (interpolation
 * weights, stencil and tridiagonal factors); nothing on the call path
 * allocates.  Calls are asynchronous on the given stream (a cudaStream_t
 * passed as void*, NULL = legacy default stream); the data and workspace must
 * stay untouched until the stream reaches the call.  Functions never abort:
 * they return a status, and mgard_last_error() gives a readable reason for
 * the most recent failure on the calling thread.
 */
#ifndef MGARD_GB300_H
#define MGARD_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MGARD_API __attribute__((visibility("default")))
#else
#define MGARD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MGARD_OK = 0,
    MGARD_ERR_INVALID_ARG = 1,       /* NULL pointer, bad enum, bad level count   */
    MGARD_ERR_UNSUPPORTED_SHAPE = 2, /* dims not of the form k*2^L+1, > 3 dims    */
    MGARD_ERR_WORKSPACE = 3,         /* workspace missing, misaligned or too small */
    MGARD_ERR_CUDA = 4,              /* a CUDA runtime call or launch failed       */
    MGARD_ERR_TIMEOUT = 5,           /* a bounded device-side wait ran out         */
    MGARD_ERR_INTERNAL = 6
} mgard_status;

typedef enum {
    MGARD_F32 = 0,       /* float storage, float arithmetic                        */
    MGARD_F64 = 1,       /* double storage, double arithmetic                      */
    MGARD_F32_MIXED = 2  /* float field; finest-level stencils in float; tridiagonal
                            solves, the coarse-level arrays and the correction
                            accumulation across levels in double                 */
} mgard_dtype;

typedef struct mgard_plan mgard_plan;

/* Create a plan for one grid shape and precision.
 *   ndim     number of dimensions, 1..3
 *   dims     ndim node counts, slowest first
 *   nlevels  number of levels L to process, or -1 for the largest allowed
 *   coords   NULL for a uniform grid (x_i = i/(n-1)), else ndim host arrays,
 *            coords[k] of length dims[k], strictly increasing (Section II-A:
 *            non-uniformly spaced structured grids)
 *   dtype    element type and precision scheme
 *   out      receives the plan; NULL on failure
 * The plan copies what it needs; coords may be freed afterwards.  Creating a
 * plan allocates and fills its device tables synchronously on the current
 * device; the plan is bound to that device. */
MGARD_API mgard_status mgard_plan_create(int ndim, const int64_t *dims, int nlevels,
                               const double *const *coords, mgard_dtype dtype,
                               mgard_plan **out);

/* A plan with a level count per dimension: dimension k coarsens in the
 * first levels[k] steps from the finest level and keeps all its nodes after
 * that (P = I along it: no interpolation, and its stencil factor M and the
 * solve with M cancel), so short sides stop early while the others go on;
 * L = max_k levels[k].  levels: ndim entries (entries of size-1 dims are
 * ignored), -1 = that dimension's maximum; NULL = every dimension its
 * maximum.  Not part of the paper's runs (equal sides only, Section IV);
 * Eq. 1-2 hold unchanged on the nested tensor-product spaces.  With equal
 * counts the plan is the plain one (mgard_plan_create with nlevels = L).
 * Otherwise mgard_decompose / mgard_recompose (and their _host forms) run
 * the levels on the persistent kernel of the batch calls, as a batch of one
 * field: the shape must fit it (fine rows of at most 1025 nodes, coarse
 * planes within a block's shared memory), else
 * MGARD_ERR_UNSUPPORTED_SHAPE; calls of one direction must be ordered (one
 * stream).  The adjoints, mgard_recompose_classes, the quantization calls
 * and mgard_plan_tune return MGARD_ERR_UNSUPPORTED_SHAPE for such a plan. */
MGARD_API mgard_status mgard_plan_create_per_dim(int ndim, const int64_t *dims, const int *levels,
                                                 const double *const *coords, mgard_dtype dtype,
                                                 mgard_plan **out);

/* Release a plan and its device tables (NULL is accepted). */
MGARD_API mgard_status mgard_plan_destroy(mgard_plan *plan);

/* Number of levels L the plan processes. */
MGARD_API int mgard_plan_levels(const mgard_plan *plan);

/* Bytes of device workspace one decompose/recompose call needs (256-byte
 * aligned base required). */
MGARD_API size_t mgard_workspace_bytes(const mgard_plan *plan);

/* Kernel launches one mgard_decompose / mgard_recompose call issues. */
MGARD_API int mgard_plan_launches(const mgard_plan *plan, int recompose);

/* Multilevel decomposition in place (Section II-A, Eq. 1-2; Fig. 3 layout).
 *   d_data   device array of prod(dims) elements of the plan's dtype
 *            (float for MGARD_F32 and MGARD_F32_MIXED, double for MGARD_F64)
 *   d_ws     device workspace of at least mgard_workspace_bytes(plan) bytes,
 *            256-byte aligned; its contents on entry do not matter
 *   stream   cudaStream_t as void* */
MGARD_API mgard_status mgard_decompose(const mgard_plan *plan, void *d_data, void *d_ws,
                             size_t ws_bytes, void *stream);

/* Inverse of mgard_decompose, in place (Section II-A, recomposition runs the
 * decomposition stages in reverse order).  Same arguments. */
MGARD_API mgard_status mgard_recompose(const mgard_plan *plan, void *d_data, void *d_ws,
                             size_t ws_bytes, void *stream);

/* Recomposition from the first `nclasses` coefficient classes, in place
 * (Section I, Fig. 1: a field is rebuilt to a chosen fidelity from a number
 * of coefficient classes; Section II-A, overall process: the omitted
 * coefficients are left out of the recomposition).  Class 0 is the coarsest
 * values on N_0, class l the level-l coefficients on N_l \ N_{l-1}; the
 * classes l >= nclasses are treated as zero (what their nodes of d_data
 * hold does not affect the result).  On return every node of d_data holds the rebuilt field, which is
 * the L2 projection Q_k u of the decomposed field onto V_k, k = nclasses-1,
 * evaluated on the finest grid; nclasses = L + 1 is mgard_recompose.
 *   nclasses  1 .. L + 1 (MGARD_ERR_INVALID_ARG otherwise)
 *   d_data, d_ws, ws_bytes, stream as for mgard_decompose. */
MGARD_API mgard_status mgard_recompose_classes(const mgard_plan *plan, int nclasses, void *d_data,
                                               void *d_ws, size_t ws_bytes, void *stream);

/* Launch-shape tuning of one level (step j = 0 is the finest level L).
 * Params 0-2 change only tile shapes and kernel variants, not the result.
 *   param 0  restriction tile: 0 = 8 x 64, 1 = 4 x 64, 2 = 16 x 64 coarse nodes per
 *            block, 3 = 8 x 30 (FP64: 4 x 30) per warp (levels with at least
 *            30 coarse columns and one strip of rows; the default where it
 *            applies)
 *   param 1  correction solves: 0 = automatic (a warp per chunk of 9, 17
 *            or 33 (FP32 only) nodes of every line, 32 lines across the
 *            lanes, where a line splits evenly into at most 16 chunks; with FP64 working
 *            arrays one thread per line instead along the slowest dimension
 *            when it has at least 128 lines per SM and along strided
 *            dimensions too long for those chunks; else chunks of about 16
 *            nodes per warp), -1 = one thread per line, 1..32 = that many
 *            warps (chunks) per line in the shared-memory panel kernel
 *   param 2  coarse planes per restriction work item (0 = automatic)
 *   param 3  plan-wide (any valid level): 0 = run the coarse end of the
 *            hierarchy in a single launch per direction (default); 1 = run
 *            every level with the tiled per-level kernels.
 *   param 4  plan-wide: 0 = the single launch is the cooperative kernel when
 *            the plan has one (every level from the first whose sides are
 *            <= 129 nodes, the grid running each level and one block the
 *            last few in shared memory), else the single-block kernel (the
 *            levels whose array fits one block's shared memory, at most
 *            227 KB, sides <= 257); 1 = always the single-block kernel.
 *   The forms of params 3 and 4 differ only in floating-point rounding order.
 *   param 6  plan-wide: polls of a grid-barrier wait in the cooperative
 *            kernel before the wait gives up and records it (0 = default,
 *            2^22 polls of tens of nanoseconds each).  A wait runs out only
 *            when the limit is far too small for the work between barriers;
 *            the result is then wrong, and mgard_plan_check reports it.
 *   param 7  plan-wide: the row-chunk kernels (one warp per row segment
 *            of 256 or 512 columns, moved in coalesced 16-byte words through
 *            a per-warp shared-memory ring of asynchronous copies; the
 *            restriction also solving along the contiguous dimension when a
 *            row is one segment) on the levels they take: 2D/3D, rows of
 *            2^k 256 + 1 nodes, n1 = 1 mod 8, a 16-byte aligned array.  The
 *            value is a mask of the ones kept out: bit 0 the coefficient and
 *            interpolation sweeps, bit 1 the restriction (default 2: the
 *            row-chunk sweeps with the strip restriction); 3 = the tile and
 *            strip kernels on every level.  All forms differ only in
 *            floating-point rounding order.  The
 *            row-chunk kernels read whole 16-byte words: up to 12 bytes
 *            beyond an array's last element, inside the word that holds it.
 *   param 9  plan-wide: coarse intervals (sweeps) or planes (restriction)
 *            per work item of the row-chunk kernels (0 = automatic).
 *   param 10 plan-wide: 0 = the slab load-vector kernel on the levels it
 *            takes (default): 3D levels whose array holds 4-byte elements
 *            (FP32, and level 0 of the mixed scheme) in rows of 64 k + 1
 *            nodes, k <= 16.  A block takes a band of coarse rows over whole
 *            rows and a chunk of coarse planes; each fine plane's rows that
 *            feed the band, one contiguous range, are staged in shared memory
 *            by a single bulk asynchronous copy.  It reads whole 16-byte
 *            words: up to 12 bytes before and after a range, inside the
 *            words that hold its ends.  1 = the strip / tile / row-chunk
 *            kernels instead.  The forms differ only in floating-point
 *            rounding order.
 *   param 11 coarse planes per slab work item of the level (0 = automatic:
 *            the largest count that still gives every resident block two
 *            items).
 *   param 12 plan-wide: coarse rows per slab band, 4, 6 or 8 (0 = automatic:
 *            6, or fewer on levels with fewer coarse rows).
 *   param 13 plan-wide: ring slots (planes staged at once) of the slab
 *            kernel, 2 .. 16 (0 = automatic: 2); a count whose shared memory
 *            does not fit leaves the affected levels to the other kernels.
 *   param 15 plan-wide: the slab kernel's register budget, for 2 or 3
 *            blocks per SM (0 = automatic: 3 where they fit, 2 for the FP64
 *            coarse rows of the mixed scheme).
 *   param 16 plan-wide: 1 = the slab kernel also solves M_{l-1} along the
 *            contiguous dimension, one warp per finished row, and the
 *            separate solve of that dimension is skipped; 0 = the solve
 *            kernels do it (default: measured faster on this GPU).  The
 *            forms differ only in rounding order.
 *   param 14 plan-wide test hook: v > 0 announces each slab block's first
 *            copy with 16 bytes more than it moves, so its wait runs out
 *            after v microseconds (the block records it and returns; the
 *            results are not valid and mgard_plan_check reports
 *            MGARD_ERR_TIMEOUT); 0 = off, with the normal limit of 2 s per
 *            wait.
 *   mgard_plan_get_tune also reports param 5: the first level the
 *   cooperative kernel runs (-1: none), param 8: the row-chunk
 *   restriction's segment width of the level (512 or 256 columns; 0: not a
 *   row-chunk level), and for params 11 .. 13, 15 and 16 the level's values
 *   (0: not a slab level).
 * Returns MGARD_ERR_INVALID_ARG for an unknown parameter or value. */
MGARD_API mgard_status mgard_plan_tune(mgard_plan *plan, int level, int param, int value);

/* Current value of a tuning parameter of level j (-1 on error). */
MGARD_API int mgard_plan_get_tune(const mgard_plan *plan, int level, int param);

/* Status of the bounded waits of the plan's last calls: synchronizes
 * `stream`, then returns MGARD_ERR_TIMEOUT if a wait for a bulk copy of the
 * slab load-vector kernel ran out since the last check (the plan's sticky
 * status word, cleared by this call), or if a grid-barrier wait of the last
 * cooperative launch that used workspace d_ws (the plan's layout) ran out;
 * the results of such a call are not valid.  Else MGARD_OK (also when the
 * plan runs neither kernel).  No paper counterpart: a safeguard of this
 * implementation's bounded waits. */
MGARD_API mgard_status mgard_plan_check(const mgard_plan *plan, const void *d_ws, void *stream);

/* End-to-end forms with host buffers: copy h_in (host, prod(dims) elements,
 * pinned for overlap) into d_data, transform it in place, copy the result
 * into h_out (host, may equal h_in).  All three steps are queued on `stream`;
 * the caller synchronizes the stream before reading h_out.  d_data and d_ws
 * as for mgard_decompose. */
MGARD_API mgard_status mgard_decompose_host(const mgard_plan *plan, const void *h_in, void *h_out,
                                  void *d_data, void *d_ws, size_t ws_bytes, void *stream);
MGARD_API mgard_status mgard_recompose_host(const mgard_plan *plan, const void *h_in, void *h_out,
                                  void *d_data, void *d_ws, size_t ws_bytes, void *stream);

/* Kernel timing (measurement support, not part of the method).  When
 * enabled, the next calls on the plan record a CUDA event pair on the call's
 * stream around every launch of the `levels` finest levels (0 = off).
 * mgard_profile_read synchronizes on the recorded events and returns the
 * accumulated time per kernel kind and level since the last read:
 *   kinds[i]   0 coefficient+load-vector (decompose), 1 load-vector
 *              (recompose), 2 solve sweep, 3 fused last solve sweep with
 *              the correction update, 4 coarse placement, 5 interpolation
 *   levels_out[i]  step index j (0 = finest level L)
 *   launches[i], ms[i]  launch count and summed event time
 * At most `cap` entries are written; the return value is the number of
 * entries (or -1 on error).  Calls made while profiling must not overlap on
 * different streams. */
MGARD_API mgard_status mgard_profile_enable(mgard_plan *plan, int levels);
MGARD_API int mgard_profile_read(mgard_plan *plan, int cap, int *kinds, int *levels_out,
                                 int *launches, double *ms);

/* Transposes of the two linear maps, in place, same arguments as
 * mgard_decompose: d_data holds a cotangent of the map's output and receives
 * the cotangent of its input (back-propagation through the map).  Per level,
 * with K = R M_l the restriction stencil and M_l P = K^T (M symmetric):
 *   decomposition^T  w = c_bar + [K^T M_{l-1}^{-1} e_bar]_odd,
 *                    e_bar <- e_bar - Pi^T w        (coarsest level first)
 *   recomposition^T  e_tot = e_bar + Pi^T o_bar,
 *                    o_bar <- o_bar - [K^T M_{l-1}^{-1} e_tot]_odd
 *                                                   (finest level first)
 * (transposes of Section II-A, Eq. 1-2). */
MGARD_API mgard_status mgard_decompose_adjoint(const mgard_plan *plan, void *d_data, void *d_ws,
                                     size_t ws_bytes, void *stream);
MGARD_API mgard_status mgard_recompose_adjoint(const mgard_plan *plan, void *d_data, void *d_ws,
                                     size_t ws_bytes, void *stream);

/* Batches of independent fields (each with its own plan: shapes, levels and
 * tile settings may differ).  Not part of the paper (its fields are
 * processed one at a time); the level steps are those of Section II-A.
 * A batch call is one CUDA-graph launch in one of two forms:
 *  - persistent (the default when every field fits it): one launch of a
 *    persistent kernel whose blocks pull work items -- planes, line panels,
 *    the small tail and the final placement of every level of every field --
 *    from a device queue.  The host orders the items by a list-scheduling
 *    model of the launch (largest fields first, a few in flight at a time);
 *    an item waits (bounded) until the tasks it depends on are done.  A
 *    field fits when its fine rows (its last dimension; for 2D fields the
 *    columns) have at most 1025 nodes, every level fits one block's shared
 *    memory (3D: coarse planes of up to 129 x 129 nodes in FP32), and all
 *    fields share one element type.
 *  - a graph of every field's per-level kernels spread over `streams`
 *    internal streams, captured on the first call for a set of data
 *    pointers / workspace and re-captured when they change.
 *   mgard_batch_create     plans: nfields plan pointers, kept (not copied)
 *                          and not freed by the batch; streams: 1..32
 *   mgard_batch_workspace_bytes   one workspace that serves both forms
 *   mgard_batch_decompose / mgard_batch_recompose
 *                          d_data: nfields device pointers (host array);
 *                          the launch goes to `stream`.  Calls of one
 *                          direction must be ordered (one stream): they
 *                          share the batch's counters.
 *   mgard_batch_tune       param 0: 1 = persistent, 0 = graph of per-field
 *                          launches (MGARD_ERR_INVALID_ARG for 1 when a
 *                          field does not fit); 1: polls of a dependency
 *                          wait before it gives up (>= 1); 2: test hook,
 *                          1 = the first item also waits for a count that
 *                          nothing reaches (its wait runs out); 3: blocks
 *                          per SM of the persistent grid (0 = as many as
 *                          fit; rebuilds the work lists); 4: measurement,
 *                          1 = every block records its busy and waiting
 *                          time per item kind; 5: queue order, 0 = fields
 *                          by decreasing modelled time (a few in flight),
 *                          1 = the longest modelled path to the end of a
 *                          field first (rebuilds the work lists)
 *   mgard_batch_profile_read   dir 0 / 1: per item kind (A, B, C, D, small
 *                          tail, placement) the block-milliseconds busy and
 *                          waiting for dependencies, and the items, summed
 *                          over the calls since the last read (6 entries
 *                          each, host arrays); synchronizes the device and
 *                          clears the record
 *   mgard_batch_get        0 persistent on, 1 poll limit, 2 test hook,
 *                          3 blocks per SM requested, 4 every field fits,
 *                          5 grid blocks, 6 blocks per SM that fit,
 *                          7 / 8 work items of a decomposition /
 *                          recomposition, 9 / 10 their modelled time (us),
 *                          11 dynamic shared memory bytes, 12 queue
 *                          order; -1 otherwise
 *   mgard_batch_check      synchronizes `stream`, then MGARD_ERR_TIMEOUT if
 *                          a dependency wait of the persistent kernel ran
 *                          out since the last check (the results of that
 *                          call are then not valid), else MGARD_OK; clears
 *                          the record.
 * The first call of a direction captures its graph: it must not itself be
 * inside a stream capture. */
typedef struct mgard_batch mgard_batch;
MGARD_API mgard_status mgard_batch_create(int nfields, mgard_plan *const *plans, int streams,
                                          mgard_batch **out);
MGARD_API mgard_status mgard_batch_destroy(mgard_batch *batch);
MGARD_API size_t mgard_batch_workspace_bytes(const mgard_batch *batch);
MGARD_API mgard_status mgard_batch_decompose(mgard_batch *batch, void *const *d_data, void *d_ws,
                                             size_t ws_bytes, void *stream);
MGARD_API mgard_status mgard_batch_recompose(mgard_batch *batch, void *const *d_data, void *d_ws,
                                             size_t ws_bytes, void *stream);
MGARD_API mgard_status mgard_batch_tune(mgard_batch *batch, int param, int value);
MGARD_API long long mgard_batch_get(const mgard_batch *batch, int param);
MGARD_API mgard_status mgard_batch_check(mgard_batch *batch, void *stream);
MGARD_API mgard_status mgard_batch_profile_read(mgard_batch *batch, int dir, double *busy_ms, double *wait_ms,
                                                long long *items);

/* ---- Decomposition without any device allocation --------------------------
 * The paper has no counterpart: it is a deployment variant of
 * mgard_decompose for callers that cannot allocate device memory where they
 * need the transform -- e.g. a process whose device memory is held by its own
 * pool allocator, or a loop that must not call cudaMalloc/cudaFree because
 * they synchronize the whole device.  It computes what mgard_plan_create on a
 * uniform grid (coords = NULL) followed by mgard_decompose computes.
 *
 *   ndim, dims, nlevels, dtype   as for mgard_plan_create (uniform grid)
 *   d_data                       the field, device memory, in place
 *   stream                       cudaStream_t as void*, NULL = legacy default
 *
 * The tables and the workspace live in one static device array of
 * MGARD_NOALLOC_SCRATCH_BYTES bytes (one per device, created when the
 * library's module is loaded on it).  A shape whose tables plus workspace do
 * not fit fails with MGARD_ERR_WORKSPACE before anything is launched.  The
 * workspace takes about 8/7 bytes per node in 3D and 8/3 in 2D for FP32
 * (twice that for FP64 and mixed): 257^3 and 2049^2 fit in FP32,
 * 257x257x129 in FP64.
 * Nothing in the array has to start at zero: each call writes, on `stream`,
 * the tables and workspace regions it then reads.  All calls on a device
 * share the array, so calls must not overlap: two calls on different streams,
 * or from different host threads, without an order between them, race on
 * it.  Calls in sequence on one stream are safe.  Every call looks up the
 * current device's array (cudaGetSymbolAddress).  The tables are uploaded
 * from pageable host memory on every call, so the call may block the host
 * until the work queued before it on `stream` has run; for the same reason
 * it cannot be captured into a CUDA graph: on a stream under capture it
 * returns MGARD_ERR_INVALID_ARG and queues nothing.  It runs no kernel that
 * waits on other blocks (the coarse levels take the single-block or
 * per-level kernels, never the cooperative one), so no wait can run out. */
#define MGARD_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
MGARD_API mgard_status mgard_decompose_noalloc(int ndim, const int64_t *dims, int nlevels, mgard_dtype dtype,
                                               void *d_data, void *stream);

/* ---- Quantization of the coefficient classes ------------------------------
 * Section V-B (lossy compression): the quantization and de-quantization of
 * the decomposed field run on the GPU between the decomposition and an
 * entropy coder.  The paper does not state the quantizer; these calls use a
 * uniform quantizer with one bin width per coefficient class:
 *   class of a node: the class it holds in the in-place layout (Fig. 3):
 *     class 0 = the coarsest values N_0, class l = the level-l coefficients
 *     N_l \ N_{l-1}, l = 1 .. L;
 *   code = sign(c) floor(|c| / bin_k + 1/2), computed in the field's
 *     precision (FP32 for MGARD_F32 and MGARD_F32_MIXED, FP64 for MGARD_F64)
 *     as one rounded product with 1 / bin_k (itself rounded to that
 *     precision) and one rounded addition, saturating at +-(2^31 - 1);
 *   de-quantized value = code x bin_k (rounded to the field's precision).
 * |c - code x bin_k| <= bin_k / 2 up to rounding of the product (unless
 * saturated).
 *   bins      host array of L + 1 positive finite bin widths, index = class
 *             (MGARD_ERR_INVALID_ARG otherwise, nothing launched)
 *   d_data    the decomposed field (device, the plan's shape and type)
 *   d_codes   int32 device array of the field's node count, same layout
 * Asynchronous on `stream`; no workspace.  mgard_decompose_quantize is
 * mgard_decompose then mgard_quantize on `stream` (d_data ends up holding
 * the decomposed field); mgard_dequantize_recompose is mgard_dequantize into
 * d_data then mgard_recompose. */
MGARD_API mgard_status mgard_quantize(const mgard_plan *plan, const double *bins, const void *d_data,
                                      int32_t *d_codes, void *stream);
MGARD_API mgard_status mgard_dequantize(const mgard_plan *plan, const double *bins, const int32_t *d_codes,
                                        void *d_data, void *stream);
MGARD_API mgard_status mgard_decompose_quantize(const mgard_plan *plan, const double *bins, void *d_data,
                                                int32_t *d_codes, void *d_ws, size_t ws_bytes, void *stream);
MGARD_API mgard_status mgard_dequantize_recompose(const mgard_plan *plan, const double *bins,
                                                  const int32_t *d_codes, void *d_data, void *d_ws,
                                                  size_t ws_bytes, void *stream);

/* ---- Measurement support --------------------------------------------------
 * FP64 fused multiply-add rate of the current device in TFLOP/s (2 flops per
 * FMA), measured with CUDA events on `stream` over one launch of
 * independent FMA chains on every SM (about a million FMAs per thread);
 * synchronizes `stream`.  The paper has no counterpart: it is the
 * denominator of the FP64 compute roofline of the benchmark.
 *   tflops   out, host pointer (MGARD_ERR_INVALID_ARG when NULL) */
MGARD_API mgard_status mgard_probe_fp64_peak(double *tflops, void *stream);

/* Human-readable name of a status code (static string). */
MGARD_API const char *mgard_status_string(mgard_status status);

/* Reason for the most recent failure on the calling thread ("" if none). */
MGARD_API const char *mgard_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MGARD_GB300_H */
