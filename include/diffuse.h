/*
 * diffuse.h -- C-ABI of the GB300 task-and-kernel-fusion runtime.
 *
 * The interface follows the paper's statement of the problem (Section 3,
 * Fig. 2a; Section 4 opening; Section 5.1):
 *   - applications (array libraries) create STORES -- rectangular arrays -- and
 *     aliasing VIEWS of them (Section 3.1, Fig. 1a);
 *   - they describe how each index task sees a store through a PARTITION:
 *     None (replicated) or an affine Tiling(shape, offset, projection)
 *     (Section 3.1, Fig. 3);
 *   - they SUBMIT index tasks: IndexTask(launch domain, [(store, partition,
 *     privilege)]) with privileges R, W, RW and Rd (Section 3.2);
 *   - tasks are buffered in a WINDOW; FLUSH (flush_window, Section 5.1) runs
 *     the fusion pass -- greedy longest fusible prefixes under the
 *     launch-domain, true-dependence, anti-dependence and reduction
 *     constraints (Section 4.2, Fig. 5), temporary-store elimination
 *     (Def. 4) and memoization of isomorphic windows (Section 5.2) -- and
 *     launches one generated sm_103a kernel per launch group;
 *   - RELEASE drops the application's reference; stores stay alive while
 *     pending tasks use them (the split reference count of Section 5.1).
 *
 * Conventions
 *   - Every entry point returns 0 (DFS_OK) on success or a negative dfs_status.
 *     dfs_last_error() then describes the failure in text.
 *   - Handles (dfs_store, dfs_partition) are positive integers owned by the
 *     context; they are never reused within a context.
 *   - Submission validates shapes, dtypes, partitions and privileges
 *     synchronously.  Device-side failures (a grid-barrier timeout) are
 *     deferred and reported by dfs_sync() or dfs_store_read().
 *   - All device work of a context is ordered on one CUDA stream.
 *   - A context is not thread-safe: one host thread at a time.
 *   - Arrays are row-major; shapes and offsets are in elements.
 */
#ifndef DIFFUSE_H
#define DIFFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DFS_MAX_DIM 3

typedef struct dfs_ctx dfs_ctx;
typedef int64_t dfs_store;     /* > 0 */
typedef int64_t dfs_partition; /* > 0 */

typedef enum {
  DFS_OK = 0,
  DFS_ERR_INVALID = -1,         /* bad argument or illegal task */
  DFS_ERR_NO_DEVICE = -2,       /* operation needs a device; context is analysis-only */
  DFS_ERR_CUDA = -3,            /* a CUDA runtime/driver call failed */
  DFS_ERR_COMPILE = -4,         /* NVRTC failed to compile a generated kernel */
  DFS_ERR_OOM = -5,             /* device allocation failed */
  DFS_ERR_BARRIER_TIMEOUT = -6, /* a grid barrier gave up waiting (deferred) */
  DFS_ERR_STATE = -7,           /* handle released / unknown, or wrong call order */
  DFS_ERR_BUFFER = -8,          /* caller's buffer too small (see *needed) */
  DFS_ERR_TOO_LARGE = -9        /* input exceeds a fixed capacity (dfs_dot_noalloc) */
} dfs_status;

typedef enum { DFS_F32 = 0, DFS_F64 = 1, DFS_I32 = 2, DFS_I64 = 3 } dfs_dtype;

/* Privileges of Section 3.2; DFS_PRIV_IMM marks an immediate scalar operand. */
typedef enum {
  DFS_PRIV_R = 1,
  DFS_PRIV_W = 2,
  DFS_PRIV_RW = 3,
  DFS_PRIV_RD = 4,
  DFS_PRIV_IMM = 8
} dfs_privilege;

typedef enum { DFS_REDOP_NONE = 0, DFS_REDOP_SUM = 1 } dfs_redop;

/*
 * Task bodies (the array libraries' operators; Section 2, Fig. 1e; Section 6,
 * Fig. 8a).  Operand order of dfs_submit's args:
 *   unary element-wise   [in0, out]          out[e] = f(in0[e])
 *   binary element-wise  [in0, in1, out]     out[e] = in0[e] (op) in1[e]
 *     in* are store args (R) or immediates (DFS_PRIV_IMM); a 0-d store read
 *     through the None partition broadcasts.  out is W (or RW).  Every store
 *     operand of one element-wise task has the same floating dtype, and every
 *     non-0-d operand's sub-store has the same shape at each point.
 *     Rounding: every operation rounds once to the store dtype (no
 *     contraction across operations), so a fused window equals the unfused
 *     stream bit for bit.
 *     ERF(x) = copysign(erf(|x|), x): the odd extension of an erf on
 *     [0, inf], so ERF(-x) = -ERF(x) bit for bit.  FP64 uses the CUDA math
 *     library's erf; FP32 uses this library's own approximation, within
 *     2 ulp of erf (the bound CUDA documents for erff).
 *     LOG(x): FP64 uses the CUDA math library's log; FP32 uses this
 *     library's own approximation, within 1 ulp of log (the bound CUDA
 *     documents for logf), with the IEEE results at 0, below 0, inf and NaN.
 *     NCDF(x) = 0.5 * (1 + ERF(x * (1/sqrt 2))), evaluated in that order.
 *   DFS_OP_DOT  [x R, y R, out RD(SUM)]   out (+)= sum_e x[e]*y[e]
 *   DFS_OP_SUM  [x R, out RD(SUM)]        out (+)= sum_e x[e]
 *     out is a 0-d store through None.  A reduction into a store that holds
 *     no value yet starts from zero; otherwise it folds into the value.
 *     The order of summation is fixed (per point, then over points in
 *     order), so results are reproducible run to run.
 *   DFS_OP_SPMV [rowptr R, col R, val R, x R, y W (, win R)]   y = A x, CSR
 *     rowptr/col are int32, val/x/y one float dtype; rowptr, col, val and x
 *     are read through None (any row may touch any column); y through a
 *     1-D Tiling whose sub-store at each point is the block of rows it owns.
 *     win (optional) is an access hint that does not change y: an int32 1-D
 *     store read through a Tiling of 6 elements per point (tile 6, offset 0
 *     relative to the store, one record per point of y's tiling), holding up
 *     to three windows (lo0, len0, lo1, len1, lo2, len2) of x, in elements of
 *     x, that the point's rows read (dfs_spmv_windows computes them).  A
 *     kernel that gives each point its own block of rows copies the windows
 *     into shared memory (bulk copies) before the rows run and reads x there;
 *     a record whose windows are out of x's bounds, not 16-byte aligned
 *     (start and size) or larger than DFS_SPMV_STAGE_BYTES in all is ignored
 *     for that point.  Results are bit-identical with and without win.
 */
#define DFS_SPMV_STAGE_BYTES 53248 /* shared memory for staged x windows per CTA */
typedef enum {
  DFS_OP_COPY = 1,
  DFS_OP_NEG = 2,
  DFS_OP_ABS = 3,
  DFS_OP_EXP = 4,
  DFS_OP_LOG = 5,
  DFS_OP_SQRT = 6,
  DFS_OP_ERF = 7,
  DFS_OP_NCDF = 8,
  DFS_OP_ADD = 32,
  DFS_OP_SUB = 33,
  DFS_OP_MUL = 34,
  DFS_OP_DIV = 35,
  DFS_OP_POW = 36,
  DFS_OP_MAX = 37,
  DFS_OP_MIN = 38,
  DFS_OP_DOT = 64,
  DFS_OP_SUM = 65,
  DFS_OP_SPMV = 96
} dfs_op;

/* One (store, partition, privilege) triple of IndexTask (Fig. 2a), or an
 * immediate scalar when privilege == DFS_PRIV_IMM (store/partition ignored). */
typedef struct {
  dfs_store store;
  dfs_partition partition;
  int32_t privilege; /* dfs_privilege */
  int32_t redop;     /* dfs_redop; DFS_REDOP_SUM with DFS_PRIV_RD */
  double imm;        /* value of an immediate */
} dfs_arg;

typedef enum {
  /* one kernel per fused task (the paper's execution: one task per prefix) */
  DFS_LAUNCH_PER_TASK = 0,
  /* all fused tasks of a flush in one cooperative kernel, grid barriers at
   * the points where the fusion constraints cut (GB300 execution) */
  DFS_LAUNCH_PERSISTENT = 1
} dfs_launch_mode;

typedef struct {
  int32_t device;            /* CUDA ordinal; -1 = analysis-only (no device) */
  int32_t fusion;            /* 1: the paper's fusion pass; 0: every task alone, no temporaries */
  int32_t launch_mode;       /* dfs_launch_mode */
  int32_t window_size;       /* tasks buffered before the window is analysed (>= 1) */
  void *stream;              /* cudaStream_t to use; NULL = the context creates one */
  int32_t block_threads;     /* threads per CTA: 128, 256, 512 or 1024 (0 = 256) */
  int32_t ctas_per_sm;       /* CTAs per SM (0 = as many as fit): sizes the grid and, when
                              * > 0, is the kernels' minimum resident CTAs per SM, which
                              * caps their registers per thread */
  int32_t unroll;            /* vectors per thread per loop trip, 1..8 (0 = 2) */
  double barrier_timeout_s;  /* grid-barrier spin limit in seconds (0 = 2.0) */
  const char *cache_dir;     /* on-disk cubin cache directory, or NULL */
  /* Test hook (0 = off): in generated kernels CTA 0 does not arrive at grid
   * barrier number k, so every CTA's wait runs out after barrier_timeout_s
   * and the launch ends with DFS_ERR_BARRIER_TIMEOUT at the next dfs_sync. */
  int32_t debug_skip_arrival;
  /* 1: record CUDA events immediately around every kernel launch; the
   * per-kernel device times appear in dfs_stats_json after dfs_sync. */
  int32_t time_launches;
  /* 1: automatic window growth (Section 7.2): when a window that filled up
   * (window_size tasks) fused completely into one task, the window size
   * doubles, up to window_max.  The current size is in dfs_stats_json. */
  int32_t window_growth;
  int32_t window_max;        /* cap of the growth (0 = 4096) */
} dfs_config;

/* Fills *cfg with the defaults above (device 0, fusion on, persistent). */
void dfs_config_default(dfs_config *cfg);

/* Creates a context.  With device >= 0 the CUDA device is made current and
 * the NVRTC compiler is loaded.  On failure *out is NULL. */
int dfs_init(dfs_ctx **out, const dfs_config *cfg);

/* Flushes, synchronizes and frees every resource of the context (library-
 * owned device memory included; wrapped memory is not freed).  NULL is ok. */
int dfs_shutdown(dfs_ctx *ctx);

/* Creates a store of `ndim` (0..3) dimensions.  Device memory is owned by the
 * library and allocated lazily, at the first flush that must materialise the
 * store; a store that the fusion pass proves temporary is never allocated.
 * Stores of 2 or 3 dimensions are pitched in device memory: each row (run of
 * the last dimension) starts on a 16-byte boundary, so row-wise kernels use
 * 16-byte accesses whatever the row length.  Host copies (dfs_store_write,
 * dfs_store_read) take and give densely packed rows. */
int dfs_store_create(dfs_ctx *ctx, int32_t dtype, int32_t ndim, const int64_t *shape,
                     dfs_store *out);

/* Creates a store over caller-owned device memory (dense, row-major,
 * 16-byte alignment recommended).  The memory must outlive every task that
 * uses the store; such a store is never treated as temporary. */
int dfs_store_wrap(dfs_ctx *ctx, int32_t dtype, int32_t ndim, const int64_t *shape,
                   void *dev_ptr, dfs_store *out);

/*
 * dfs_store_wrap_host -- a store over caller-owned, page-locked host memory
 * that is mapped into the device's address space (cudaHostAlloc, or memory
 * registered with cudaHostRegister and its mapping flag; on GB300 the GPU
 * reaches it over NVLink-C2C).  Kernels then read and write the host memory
 * directly: a one-pass program over host arrays needs no separate copies in
 * or out.  Layout: dense, row-major.  The memory must stay allocated while any
 * task uses the store; the store is never temporary.
 * The range [host_ptr, host_ptr + bytes) is checked before anything uses it:
 * CUDA must report both its first and its last byte as page-locked host
 * memory (pageable memory is refused even where the device could reach it,
 * since its pages can be unmapped under a running kernel), with device
 * mappings at the same distance apart.  The caller keeps the memory
 * allocated until every task that uses the store has completed (a
 * dfs_sync after its flush).  Returns DFS_OK; DFS_ERR_INVALID (nothing is created) for a
 * null pointer or memory that is not mapped pinned host memory;
 * DFS_ERR_NO_DEVICE in an analysis-only context.
 */
int dfs_store_wrap_host(dfs_ctx *ctx, int32_t dtype, int32_t ndim, const int64_t *shape, void *host_ptr,
                        dfs_store *out);

/*
 * dfs_host_alloc / dfs_host_free -- page-locked host memory mapped into the
 * address space of every device (cudaHostAlloc, mapped and portable), for
 * dfs_store_wrap_host and for fast copies.  *out receives the host address
 * (NULL for bytes == 0).  Returns DFS_OK, DFS_ERR_INVALID for a null `out`,
 * DFS_ERR_OOM when the allocation fails.  dfs_host_free(NULL) is a no-op.
 */
int dfs_host_alloc(size_t bytes, void **out);
int dfs_host_free(void *p);

/* Creates an aliasing view: the box [offset, offset+shape) of `parent`
 * (itself possibly a view), as array slicing does (Fig. 1a). */
int dfs_store_view(dfs_ctx *ctx, dfs_store parent, const int64_t *offset, const int64_t *shape,
                   dfs_store *out);

/* Drops the application's reference to a store or view.  Memory is freed
 * once no application reference and no pending task remain. */
int dfs_store_release(dfs_ctx *ctx, dfs_store s);

/* Copies `bytes` from host memory into a root store (after flushing pending
 * work; asynchronous with respect to the host for pinned memory). */
int dfs_store_write(dfs_ctx *ctx, dfs_store s, const void *host_src, size_t bytes);

/* Flushes, then copies the store (root or 1-/2-D view) to host memory and
 * synchronizes.  Returns any deferred device error. */
int dfs_store_read(dfs_ctx *ctx, dfs_store s, void *host_dst, size_t bytes);

/* Flushes, materialises the store's root and returns the device address of
 * the store's first element (for interoperation with other CUDA code).  Rows
 * of a created 2-D or 3-D store are pitched (see dfs_store_create): the row
 * pitch is the row length rounded up to 16 bytes. */
int dfs_store_device_ptr(dfs_ctx *ctx, dfs_store s, void **out);

/* The None partition: every point of the launch domain sees the whole store. */
int dfs_partition_none(dfs_ctx *ctx, dfs_partition *out);

/* Tiling(tile, offset, proj) (Section 3.1, Fig. 3e): point p of the launch
 * domain sees [proj(p)*tile, (proj(p)+1)*tile) + offset, clipped to the
 * store (or view) it is applied to.  proj[d] names the launch-domain
 * coordinate that drives store dimension d; NULL means the identity. */
int dfs_partition_tiling(dfs_ctx *ctx, int32_t ndim, const int64_t *tile, const int64_t *offset,
                         const int32_t *proj, dfs_partition *out);

/* Appends IndexTask(launch_domain, args) to the window (Section 3.2).  When
 * the window holds `window_size` tasks it is analysed and its complete fused
 * groups are launched. */
int dfs_submit(dfs_ctx *ctx, int32_t op, int32_t ndim, const int64_t *launch_domain,
               int32_t nargs, const dfs_arg *args);

/* flush_window(): analyses and launches every buffered task; asynchronous. */
int dfs_flush(dfs_ctx *ctx);

/* Waits for the context's stream; returns deferred device errors. */
int dfs_sync(dfs_ctx *ctx);

/* Text of the last error on this context (empty if none). */
const char *dfs_last_error(dfs_ctx *ctx);

/* JSON description of how the buffered window would be fused, without
 * launching it: {"groups": [[task indices]...], "temporaries": [store ids],
 * "launches": [[group indices]...], "barriers": n, "key": "..."}.
 * Writes at most len bytes (NUL-terminated) and the full size to *needed. */
int dfs_plan_json(dfs_ctx *ctx, char *buf, size_t len, size_t *needed);

/* JSON counters: tasks submitted, fused groups, launches, barriers, plan and
 * kernel cache hits/misses, NVRTC compile seconds, bytes allocated. */
int dfs_stats_json(dfs_ctx *ctx, char *buf, size_t len, size_t *needed);

/*
 * CUDA-graph capture of flushed windows.  The paper memoises the analysis and
 * code generation of isomorphic windows (Section 5.2); capture goes one step
 * further and records the launches themselves, so a steady-state loop body
 * (e.g. one iteration of an iterative solver whose state lives in stores the
 * application holds and updates in place) can be replayed with no host-side
 * issue cost.
 *
 * dfs_capture_begin flushes, then records instead of executing: every launch
 * of the following flushes, and the stream-ordered allocations and frees of
 * stores created and released inside the captured region, go into a graph.
 * Bookkeeping (which stores hold values) advances as if the work ran once.
 * dfs_capture_end flushes, ends the capture and instantiates the graph into
 * *out.  The captured work has NOT run; dfs_graph_launch runs it (any number
 * of times) on the context stream, on the same device addresses and with the
 * same immediate values.
 * Restrictions (DFS_ERR_STATE otherwise): no dfs_store_read / dfs_sync while
 * capturing; a store created inside the captured region must be released
 * before dfs_capture_end; stores the graph uses stay allocated until
 * dfs_graph_destroy even if released (replays may read them).
 */
typedef int64_t dfs_graph;
int dfs_capture_begin(dfs_ctx *ctx);
int dfs_capture_end(dfs_ctx *ctx, dfs_graph *out);
int dfs_graph_launch(dfs_ctx *ctx, dfs_graph g);
int dfs_graph_destroy(dfs_ctx *ctx, dfs_graph g);

/*
 * Batched execution of isomorphic windows (GB300 extension of the
 * memoisation of Section 5.2 to many problems at once).
 *
 * Between dfs_batch_begin and dfs_batch_end the application submits K
 * instances of one task sequence -- e.g. one iteration of each of K
 * independent solves of different sizes -- calling dfs_batch_next after each
 * instance.  The instances must be isomorphic: the same operations and
 * privileges, the same pattern of store, partition and launch-domain
 * identities, and the same liveness of their stores; sizes, tiles, store
 * addresses and immediate values may differ.  dfs_batch_end runs the fusion
 * pass once, generates one size-generic kernel whose sizes, pointers and
 * immediates come from per-instance descriptors in device memory, and
 * launches it once: each phase processes the points of all K instances
 * through a work list, so the uneven problems share one persistent launch
 * and its grid barriers.  Reductions keep one partial per point and each
 * instance's scalars are finished in a fixed order, so every instance's
 * results are bit-identical to running it alone with the same tiles.
 *
 * Batches whose instances are not isomorphic, or that use stores of rank
 * other than 0 and 1, are executed as an ordinary flush of all their tasks
 * (same results, no batching); dfs_stats_json counts both cases.
 * Descriptor tables are cached by content, so a batch that repeats the same
 * stores (in-place iterations) uploads nothing and can be captured in a
 * CUDA graph after it has run once.
 * Returns DFS_ERR_STATE for calls out of order.
 */
int dfs_batch_begin(dfs_ctx *ctx);
int dfs_batch_next(dfs_ctx *ctx);
int dfs_batch_end(dfs_ctx *ctx);

/*
 * dfs_batch_repeat -- issue the most recent batch n more times, as if the
 * application had submitted the same K instance windows again n times
 * (memoisation of Section 5.2 carried to the launch itself: no analysis, no
 * descriptor upload, one kernel launch per repetition).
 *
 * Allowed only while the batch is still "steady": every store it uses held a
 * value before it ran or was eliminated as a temporary (so each instance
 * only updates stores it already owns, as an in-place solver iteration
 * does), and since then no other window was launched, no graph was captured
 * or launched, and no store with device memory was freed.  dfs_batch_repeat
 * first flushes the pending window; if that launches anything the batch is
 * no longer steady.  n == 0 does nothing.
 * Returns DFS_OK; DFS_ERR_INVALID for n < 0; DFS_ERR_STATE when there is no
 * steady batch to repeat (nothing is launched); DFS_ERR_CUDA when a launch
 * fails.  Device errors are deferred as for any launch.
 */
int dfs_batch_repeat(dfs_ctx *ctx, int32_t n);

/*
 * dfs_read_scalars -- flushes, then copies the values of n 0-d stores to
 * host_out[0..n) as doubles (FP32 and integer values converted exactly where
 * representable) with one gather kernel and one device-to-host copy, and
 * synchronizes.  A serving loop uses it to read every active solve's
 * residual norm at once instead of n separate dfs_store_read calls.
 * stores: n handles of 0-d stores (roots or views) that hold values;
 * host_out: n doubles owned by the caller.  The context keeps a small device
 * buffer for the gather (grown as needed, freed at dfs_shutdown).
 * Returns DFS_OK; DFS_ERR_INVALID for null pointers, n < 0 or a store that
 * is not 0-d; DFS_ERR_STATE for an unknown or released store, one that holds
 * no value, or a call while capturing; DFS_ERR_NO_DEVICE in an
 * analysis-only context; any deferred device error, as dfs_store_read.
 */
int dfs_read_scalars(dfs_ctx *ctx, int32_t n, const dfs_store *stores, double *host_out);

/*
 * dfs_read_scalars_async -- the same gather as dfs_read_scalars, enqueued on
 * the context's stream without waiting: it flushes, checks the stores, and
 * returns once the descriptor upload, the gather kernel and the copy of the
 * n values to host_vals[0..n) are issued.  A serving loop reads one group of
 * solves' residuals this way while the GPU still has another group's
 * iterations queued behind the copy, so the GPU does not wait for the host.
 * host_work (2 n int64: the gather's descriptors) and host_vals (n doubles)
 * must be page-locked host memory (dfs_host_alloc) that the caller neither
 * reads nor writes until a ticket recorded after this call (dfs_record) has
 * completed.  Errors as dfs_read_scalars, plus DFS_ERR_INVALID when a host
 * buffer is not page-locked.  n == 0 issues nothing.
 */
int dfs_read_scalars_async(dfs_ctx *ctx, int32_t n, const dfs_store *stores, int64_t *host_work,
                           double *host_vals);

/*
 * Completion tickets.  dfs_record flushes the pending window and records a
 * CUDA event after all work issued on the context so far; *ticket names it.
 * dfs_wait blocks until that work has finished and then returns any deferred
 * device error (as dfs_sync does, but without waiting for work issued after
 * the ticket).  dfs_poll sets *done to 1 when the work has finished (then
 * returning deferred device errors) and to 0 otherwise, without blocking.
 * dfs_ticket_elapsed_ms gives the device time between two completed tickets
 * of the context (milliseconds, CUDA event resolution).  dfs_ticket_release
 * forgets a ticket; its event is reused.  Tickets not released are freed at
 * dfs_shutdown.
 * Returns DFS_OK; DFS_ERR_INVALID for null pointers; DFS_ERR_STATE for an
 * unknown ticket, a ticket not complete (elapsed time) or dfs_record while
 * capturing; DFS_ERR_NO_DEVICE in an analysis-only context; DFS_ERR_CUDA.
 */
int dfs_record(dfs_ctx *ctx, uint64_t *ticket);
int dfs_wait(dfs_ctx *ctx, uint64_t ticket);
int dfs_poll(dfs_ctx *ctx, uint64_t ticket, int32_t *done);
int dfs_ticket_elapsed_ms(dfs_ctx *ctx, uint64_t from, uint64_t to, float *ms);
int dfs_ticket_release(dfs_ctx *ctx, uint64_t ticket);

/*
 * Instance templates: the memoisation of Section 5.2 carried to task issue.
 * A serving loop issues the same iteration window for every solve of a size,
 * differing only in the stores; recording it once and replaying it with the
 * stores substituted costs one call per instance instead of one per task.
 *
 * dfs_template_begin starts recording.  Until dfs_template_end, every store
 * creation, view, task submission and store release is recorded as well as
 * performed.  Calls that a replay cannot repeat (dfs_store_write, _wrap,
 * _wrap_host, _read, the dfs_batch_* and capture/graph calls, the scalar
 * reads, dfs_record) fail with DFS_ERR_STATE while recording, and so does
 * releasing a store the recording did not create; either makes
 * dfs_template_end fail.  dfs_template_end also fails unless every store the
 * recording created (temporaries and views) was released by its end.  On
 * success *id names the template.
 *
 * The template's inputs are the stores it used but did not create, in first
 * use order; dfs_template_inputs copies up to cap of them to out and sets *n
 * to their number.  dfs_template_replay issues the recorded sequence again
 * with from[i] replaced by to[i] (n pairs): fresh stores for the recorded
 * creations and views, the same partitions, privileges and immediates.  Every
 * input must be mapped to a live store of the dtype and shape it had when it
 * was recorded (DFS_ERR_INVALID otherwise, checked before anything is
 * issued).  If a later step fails (say, a flush the window size triggers
 * cannot allocate), the call returns that step's error: tasks issued before
 * it stay issued, and the stores this replay created are released, so none
 * outlives what still uses it.  A replay may run inside a batch instance (between dfs_batch_begin
 * / dfs_batch_next).  A partition handle keeps the tiling it was created
 * with, so a template replays the tiling it recorded.
 * dfs_template_free forgets a template.  Templates are freed at dfs_shutdown.
 * Returns DFS_OK; DFS_ERR_INVALID for null pointers or bad counts;
 * DFS_ERR_STATE for nesting, an unknown template, or a failed recording.
 */
int dfs_template_begin(dfs_ctx *ctx);
int dfs_template_end(dfs_ctx *ctx, uint64_t *id);
int dfs_template_inputs(dfs_ctx *ctx, uint64_t id, int32_t cap, dfs_store *out, int32_t *n);
int dfs_template_replay(dfs_ctx *ctx, uint64_t id, int32_t n, const dfs_store *from, const dfs_store *to);
int dfs_template_free(dfs_ctx *ctx, uint64_t id);

/*
 * dfs_set_launch_config -- changes the launch parameters of a live context
 * (block_threads: 128, 256, 512 or 1024; unroll: 1..8; ctas_per_sm: 0 =
 * as many as fit, else that many, with registers capped to fit them; see
 * dfs_config), as an autotuner does between
 * timed trials.  Flushes the pending window first.  Kernels already
 * generated for other parameters stay cached.  Block size changes the
 * per-thread order of reductions inside a point, so reduction results may
 * differ in the last bits between settings; unroll and ctas_per_sm do not
 * change any result.
 * Returns DFS_OK; DFS_ERR_INVALID for values outside those ranges (nothing
 * changes); DFS_ERR_STATE inside a batch or a capture.
 */
int dfs_set_launch_config(dfs_ctx *ctx, int32_t block_threads, int32_t unroll, int32_t ctas_per_sm);

/*
 * Row-block partition over ranks (one process per GPU).  Section 3.2 splits
 * an index task's launch domain into point tasks, one per processor; across
 * GPUs the vectors of an iterative solver are tiled by row blocks and each
 * rank runs the point tasks of its own block (the weak-scaling setting of the
 * paper's evaluation, Section 7).  Rank r of P owns the rows
 * [floor(r n / P), floor((r + 1) n / P)).  Element-wise tasks and reductions
 * then need nothing from other ranks but the reductions' partial sums; a CSR
 * SpMV, which reads x through the None partition, also needs the entries of
 * x that its rows reference outside the block -- its HALO, received from
 * their owners before the SpMV.  These calls compute that plan on the host;
 * they need no device and allocate nothing the caller must free.
 *
 * dfs_rowblock_bounds: *lo, *hi = the rows rank `rank` of `nranks` owns out
 * of n.  Returns DFS_ERR_INVALID for n < 0, nranks < 1 or rank outside
 * [0, nranks), or null outputs.
 *
 * dfs_rowblock_sizes: sizes of rank `rank`'s plan for the square CSR matrix
 * (rowptr: n + 1 int32, rowptr[0] == 0, non-decreasing; col: rowptr[n]
 * int32 columns in [0, n)): owned rows, their stored entries, the distinct
 * halo columns, and the owned entries other ranks read (counted once per
 * reading rank).  Returns DFS_ERR_INVALID for a malformed matrix or bad rank.
 *
 * dfs_rowblock_plan: fills caller-owned arrays sized by dfs_rowblock_sizes:
 *   local_rowptr  (n_own + 1 int32)  the owned rows' row pointers, from 0;
 *   local_col     (nnz int32)        their columns renumbered: an owned
 *                 column g becomes g - row_lo, a halo column becomes
 *                 n_own + its halo slot (the values array is the caller's
 *                 val[rowptr[row_lo] .. rowptr[row_hi]) unchanged);
 *   halo_cols     (n_halo int64)     global column of each halo slot,
 *                 ascending, hence grouped by owning rank;
 *   recv_counts   (nranks int64)     halo slots owned by each rank;
 *   send_idx      (n_send int32)     owned local indices to send, grouped by
 *                 destination rank ascending, ascending within a group (the
 *                 order of the receiver's halo slots);
 *   send_counts   (nranks int64)     entries sent to each rank.
 * The halo exchange is then one all-to-all of send_idx's entries of x with
 * these counts, received into x[n_own ..].  Returns DFS_ERR_INVALID as
 * dfs_rowblock_sizes or for a null array that must hold entries,
 * DFS_ERR_TOO_LARGE when n_own + n_halo exceeds the int32 range.
 */
/*
 * dfs_spmv_windows -- the windows of x that each point of an SpMV reads, for
 * the optional `win` argument of DFS_OP_SPMV.  The matrix is CSR (rowptr:
 * nrows + 1 int32, rowptr[0] == 0, non-decreasing; col: rowptr[nrows] int32
 * in [0, ncols)); point p owns rows [p tile, min((p + 1) tile, nrows)).  For
 * each point, the distinct columns of its rows are merged into intervals
 * (gaps of up to 64 columns are absorbed), the closest intervals are merged
 * until at most three remain, and each interval is widened to 16-byte
 * boundaries of an x of `elem_bytes`-byte elements whose first element is
 * 16-byte aligned, then clipped to the 16-byte-aligned part of [0, ncols)
 * (columns left outside are read from global memory).  A point whose
 * windows exceed budget_bytes in all gets an empty record (all zeros).
 * out: 6 int32 per point, ceil(nrows / tile) points, owned by the caller.
 * Host only; needs no device.  Returns DFS_ERR_INVALID for a malformed
 * matrix, tile < 1, elem_bytes not 4 or 8, or a null pointer.
 */
int dfs_spmv_windows(const int32_t *rowptr, const int32_t *col, int64_t nrows, int64_t ncols, int64_t tile,
                     int32_t elem_bytes, int64_t budget_bytes, int32_t *out);

typedef struct {
  int64_t row_lo, row_hi; /* owned global rows */
  int64_t nnz;            /* stored entries of the owned rows */
  int64_t n_halo;         /* distinct columns outside [row_lo, row_hi) they read */
  int64_t n_send;         /* owned entries other ranks read, summed over ranks */
} dfs_rowblock_sizes_t;
int dfs_rowblock_bounds(int64_t n, int32_t nranks, int32_t rank, int64_t *lo, int64_t *hi);
int dfs_rowblock_sizes(const int32_t *rowptr, const int32_t *col, int64_t n, int32_t nranks, int32_t rank,
                       dfs_rowblock_sizes_t *out);
int dfs_rowblock_plan(const int32_t *rowptr, const int32_t *col, int64_t n, int32_t nranks, int32_t rank,
                      int32_t *local_rowptr, int32_t *local_col, int64_t *halo_cols, int64_t *recv_counts,
                      int32_t *send_idx, int64_t *send_counts);

/* Source of the generated CUDA for the most recent launch (debugging). */
int dfs_last_kernel_source(dfs_ctx *ctx, char *buf, size_t len, size_t *needed);

/* ABI version (major*100 + minor). */
int dfs_version(void);

/*
 * dfs_dot_noalloc -- *out = sum_i x[i]*y[i] over n FP64 elements, computed on
 * `stream` (a cudaStream_t; NULL = the legacy default stream) of the current
 * device WITHOUT allocating any device memory.
 *
 * The paper has no counterpart: this entry point serves callers that cannot
 * allocate when they need a reduction -- serving or real-time loops that
 * reserve all their device memory at start-up (an allocation later could
 * block, synchronise the device or fail under the memory budget), and
 * plug-ins whose host framework owns every device allocation and hands them
 * none.
 *
 * x, y: device pointers to n doubles (8-byte aligned); out: device pointer to
 * one double.  All three are owned by the caller.  The result is written
 * asynchronously on `stream`.  Summation order is fixed (one partial per
 * DFS_NOALLOC_TILE elements, a fixed tree inside each block, partials summed
 * in order), so repeated calls give identical bits.
 *
 * Scratch: a file-scope __device__ array of DFS_NOALLOC_MAX_N /
 * DFS_NOALLOC_TILE doubles (128 KB) plus the runtime's 160-byte control block
 * (exit counter; cleared by every call), held by every GPU that loads the
 * library until the process exits.  Every call on a device shares
 * it, so calls whose kernels overlap on the GPU (different streams, no
 * ordering between them) race and give wrong results; order them.
 * The first call on each device resolves the scratch's device address with
 * that device current (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Host threads may call concurrently.
 *
 * Returns DFS_OK; DFS_ERR_INVALID for null pointers or n < 0;
 * DFS_ERR_TOO_LARGE when n > DFS_NOALLOC_MAX_N (nothing is launched);
 * DFS_ERR_CUDA when a CUDA call fails.  n == 0 writes 0.0.
 */
#define DFS_NOALLOC_TILE 4096
#define DFS_NOALLOC_MAX_N (16384LL * DFS_NOALLOC_TILE) /* 2^26 elements; 128 KB of scratch */
int dfs_dot_noalloc(const double *x, const double *y, int64_t n, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DIFFUSE_H */
