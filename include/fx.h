/*
 * fx.h - C ABI of the fused expression library (libfx.so).
 *
 * The library evaluates a whole linear-algebra expression tree - element-wise
 * operators, transposes, broadcasts and a terminal reduction - in one fused
 * CUDA kernel on one GB300 (sm_103a). This is the method of Curtin, Edel and
 * Sanderson, "Fast GPU Linear Algebra via Compile Time Expression Fusion":
 * the tree is a compile-time C++ type (Sec. 3, the AST-as-type paragraph),
 * instantiated at build time into kernels, so that the expression is computed
 * in one pass over its input matrices (Sec. 5). Expressions are therefore
 * chosen by name from the set compiled into the library (fx_list_count and
 * fx_list_get).
 *
 * Conventions that hold for every call:
 *  - Matrices are column-major: element (r, c) is ptr[r + c*ld] (Sec. 3, the
 *    element-access rule of the base matrix type), with ld >= rows.
 *  - Every pointer handed to fx_expr_bind / fx_eval_batch is a DEVICE pointer
 *    owned by the caller, except the host pointers of fx_eval_host. The
 *    library never frees caller memory.
 *  - Calls are asynchronous and stream-ordered (Sec. 2: all operations are
 *    dispatched asynchronously; the caller synchronises). A stream argument
 *    is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *  - No call throws or aborts. Every call returns an fx_status; on failure,
 *    fx_last_error_string() describes it (thread-local, valid until the next
 *    failing call on the same thread).
 *  - One fx_expr is evaluated on one stream at a time: its reduction
 *    workspace is shared by its launches, so two overlapping evaluations of
 *    the same fx_expr on different streams race. Distinct fx_expr objects
 *    are independent.
 */
#ifndef FX_H
#define FX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FX_MAX_SLOTS 24   /* inputs + outputs of one expression */
#define FX_MAX_SCALARS 8

typedef struct fx_expr fx_expr; /* opaque; created and destroyed by the library */

typedef enum {
  FX_OK = 0,
  FX_E_ARG = -1,         /* null pointer, bad slot or scalar index, bad enum */
  FX_E_SHAPE = -2,       /* bound shapes disagree with the expression */
  FX_E_DTYPE = -3,       /* no instantiation for this storage type */
  FX_E_ALIGN = -4,       /* pointer not aligned to its element size */
  FX_E_UNBOUND = -5,     /* a slot needed by the call has no buffer */
  FX_E_UNSUPPORTED = -6, /* the expression has no such entry point */
  FX_E_CUDA = -7,        /* a CUDA runtime error (message has the details) */
  FX_E_NOMEM = -8,       /* workspace allocation failed */
  FX_E_NOTFOUND = -9     /* no expression of that name */
} fx_status;

typedef enum { FX_F32 = 0, FX_F64 = 1, FX_BF16 = 2, FX_F16 = 3 } fx_dtype;

/* What the expression's root produces. */
typedef enum {
  FX_KIND_ELEMENTWISE = 0, /* one output matrix, same shape as the tree */
  FX_KIND_FULL_REDUCE = 1, /* accu / norm: one scalar */
  FX_KIND_DIM_REDUCE = 2,  /* sum / max along a dimension: a row or column vector */
  FX_KIND_MULTI = 3        /* output matrix Z plus one scalar s: accu(Z), or the
                              accu of a second tree over the same leaves (the
                              formula then lists both trees, "Z-tree ; s-tree") */
} fx_kind;

/* Autotuner modes (fx_tune). */
typedef enum { FX_TUNE_OFF = 0, FX_TUNE_CACHE = 1, FX_TUNE_SEARCH = 2 } fx_tune_mode;

/* One matrix of a batch: a device pointer and leading dimension for every
 * slot (inputs, then outputs), and the shape (rows x cols) of the tree for
 * this matrix. ld[k] == 0 means "contiguous" (the slot's own row count); a
 * leading dimension per slot lets a batch address submatrices of larger
 * arrays, as fx_expr_bind does for one matrix. A
 * transposed leaf of a rows x cols tree is cols x rows. A scalar output
 * (accu) points to one element. */
typedef struct {
  void* ptr[FX_MAX_SLOTS];
  int64_t ld[FX_MAX_SLOTS];
  int64_t rows;
  int64_t cols;
} fx_batch_item;

/* ---- discovery -------------------------------------------------------- */

/* Number of compiled (name, storage) instantiations. */
int fx_list_count(void);

/* Instantiation i (0 <= i < fx_list_count()): its name, storage type and
 * the tree it computes (an S-expression, e.g. "(- (+ (% A B) (* s0 (exp C)))
 * (t D))"; s0, s1 ... are its scalars). Strings are static. FX_E_ARG if i is
 * out of range; null out-pointers are skipped. */
fx_status fx_list_get(int i, const char** name, fx_dtype* storage, const char** formula);

/* ---- expression objects ----------------------------------------------- */

/* Creates an expression object for the compiled tree `name` with `storage`
 * element type (FX_E_NOTFOUND: unknown name; FX_E_DTYPE: name known but not
 * compiled for that storage type). Scalars start at their compiled
 * defaults; no slot is bound. Allocates host memory only. */
fx_status fx_expr_create(const char* name, fx_dtype storage, fx_expr** out);

/* Frees the object, its device workspace and any cached CUDA graph. Waits
 * for nothing: the caller must make sure no launch of this object is still
 * running (synchronise its stream first). NULL is accepted. */
fx_status fx_expr_destroy(fx_expr* x);

/* Counts of input slots, output slots and scalars, and the root's kind (the
 * kind tells a caller which outputs to bind: a matrix, a scalar, a vector,
 * or a matrix and its sum). */
fx_status fx_expr_info(const fx_expr* x, int* n_inputs, int* n_outputs, int* n_scalars,
                       fx_kind* kind);

/* Name of slot `slot` (inputs first, then outputs), e.g. "A" or "Z". */
fx_status fx_expr_slot_name(const fx_expr* x, int slot, const char** name);

/* Storage type of a slot's buffer. Every slot of a tree has the tree's
 * storage type (the fx_expr_create argument) except inputs a definition
 * fixes otherwise (expr3's Y is FP64 in an FP32 tree, read as its FP32
 * rounding); reduction outputs are FP32 (FP64 for FP64 trees). */
fx_status fx_expr_slot_dtype(const fx_expr* x, int slot, fx_dtype* dtype);

/* Binds a device buffer to a slot: `rows` x `cols`, column-major with
 * leading dimension `ld` (>= rows; ld may be anything >= 1 for rows <= 1).
 * The element type is the expression's storage type for inputs and
 * element-wise outputs; reduction outputs hold float for f32/bf16/f16
 * storage and double for f64. Checks: slot range, non-null pointer when the
 * shape is non-empty, alignment to the element size, ld. Shapes are checked
 * against each other at evaluation. The buffer stays owned by the caller and
 * must stay valid until the last evaluation that uses it has completed. */
fx_status fx_expr_bind(fx_expr* x, int slot, void* dev_ptr, int64_t rows, int64_t cols,
                       int64_t ld);

/* Sets scalar `idx` (s0, s1 ... in the formula) to `v`; it is applied in the
 * compute type (float, or double for f64 storage). */
fx_status fx_expr_set_scalar(fx_expr* x, int idx, double v);
fx_status fx_expr_get_scalar(const fx_expr* x, int idx, double* v);

/* ---- evaluation --------------------------------------------------------- */

/* Fused evaluation: every input element is read once and every output
 * element written once (Sec. 5: one pass over the input matrices).
 * Reductions finish on the device: a deterministic two-stage combine (per
 * block partials, then one block sums them in a fixed order in FP64), so
 * results are bitwise repeatable for fixed shapes and tuning. Asynchronous.
 * Empty shapes are valid: nothing is read; accu/norm of an empty tree write
 * 0, sum along a dimension writes zeros, max of an empty slice writes -inf. */
fx_status fx_eval(fx_expr* x, void* stream);

/* The same tree evaluated one operator at a time (one kernel per node,
 * every intermediate materialised in the storage type in library
 * workspace): the unfused baseline the fused path is measured against.
 * Its kernels always run at the library's default launch shapes; a shape
 * set by fx_tune or fx_expr_set_launch_shape applies to the fused path
 * only. */
fx_status fx_eval_unfused(fx_expr* x, void* stream);

/* End-to-end evaluation from and to HOST memory. The slots must be bound
 * to device buffers as for fx_eval; host_in[k] (k < n_inputs) is copied to
 * input slot k, the tree is evaluated, and output slot j is copied to
 * host_out[j]. Host buffers are dense column-major (ld = rows) and should be
 * pinned (cudaHostAlloc) for asynchronous copies. Element-wise trees with
 * at least 32 columns whose inputs are each read in one mode run as a
 * pipeline of up to 8 column chunks: chunk i's inputs are copied up on an
 * internal stream while chunk i-1 is evaluated on `stream` and chunk i-2's
 * output is copied down on a second internal stream (the object owns both
 * streams; `stream` waits for them before the call's work is complete).
 * Other trees copy, evaluate and copy back in order on `stream`. Returns
 * after enqueueing; the caller synchronises `stream` before reading
 * host_out. */
fx_status fx_eval_host(fx_expr* x, const void* const* host_in, void* const* host_out,
                       void* stream);

/* Batched evaluation of one tree over `n` independent matrices of uneven
 * shapes in one persistent launch over a host-built work-list of tiles,
 * plus one launch that combines per-tile partial sums for accu outputs.
 * With use_graph != 0 the two launches are captured in a CUDA graph the
 * first time a given items array (same contents) is seen and replayed
 * afterwards. The item array is read on the host during the call only.
 * Every matrix operand of an item (inputs and Z) must span fewer than 2^31
 * elements (ld * (cols - 1) + rows), since the batched kernel addresses a
 * matrix with 32-bit offsets: FX_E_SHAPE otherwise, before any launch.
 * FX_E_UNSUPPORTED for trees without a batched entry. */
fx_status fx_eval_batch(fx_expr* x, int64_t n, const fx_batch_item* items, void* stream,
                        int use_graph);

/* Fused backward of an accu(...) root: for every input slot k with
 * grad_ptrs[k] != NULL, writes dL/d(input k) scaled by *grad_out into
 * grad_ptrs[k] (device, same shape as input k, dense column-major, storage
 * type). grad_out is a DEVICE pointer to one reduction-type scalar (float,
 * or double for f64), or NULL for 1: a device pointer rather than a host
 * value, so that a backward pass queued behind the forward pass and the
 * caller's own loss arithmetic needs no host synchronisation. The tree is recomputed element by
 * element (no stored intermediates); gradients of broadcast leaves are
 * reduced along the broadcast dimension with the same deterministic
 * combine as fx_eval. FX_E_UNSUPPORTED for other roots. */
fx_status fx_eval_backward(fx_expr* x, const void* grad_out, void* const* grad_ptrs,
                           void* stream);

/* Autotuner (it takes the caller's stream, so that its timed trials run in
 * stream order with the caller's other work). FX_TUNE_OFF: built-in launch
 * shapes. FX_TUNE_CACHE: use the
 * cached choice for this (expression, storage, shape class, device) if the
 * cache file has one. FX_TUNE_SEARCH: time every candidate launch shape
 * on the currently bound buffers (writes the outputs; synchronises the
 * stream), keep the fastest (the built-in shape unless a candidate is at
 * least 1% faster than it), and record it in the cache file
 * ($FX_TUNE_CACHE, default ./fx_tune.json). */
fx_status fx_tune(fx_expr* x, fx_tune_mode mode, void* stream);

/* Autotuner of the batched entry (fx_eval_batch): times the batched
 * kernel's launch shapes - threads per block 256 or 512 (512 not for BF16 /
 * FP16), 2, 3 or 4 pipeline stages (reported as unroll 2, 4, 8), blocks per
 * SM 0 (as many as fit), 1 or 2, and the vector width each thread
 * evaluates per step (reported as pipeline 0: 16 bytes of elements, 1: 8
 * bytes) - on the given items without graph capture,
 * keeps the fastest and caches it under (expression, storage, device, n).
 * FX_TUNE_CACHE reads the cache; FX_TUNE_OFF restores the defaults. The
 * next fx_eval_batch uses the chosen shape (and re-captures its graph). */
fx_status fx_tune_batch(fx_expr* x, int64_t n, const fx_batch_item* items, fx_tune_mode mode,
                        void* stream);

/* Launch shape currently chosen (for reports): threads per block, vectors
 * per thread per step, blocks per SM (0: as many as fit), and the kernel
 * variant (see fx_expr_set_launch_shape). Null pointers are skipped. */
fx_status fx_expr_launch_shape(const fx_expr* x, int* block, int* unroll, int* blocks_per_sm,
                               int* pipeline);

/* Fixes the launch shape (what FX_TUNE_SEARCH would choose) until the next
 * fx_tune call. block: threads per block of the streaming kernels, a
 * multiple of 32 in [64, 512]; unroll: 2, 4 or 8 vectors per thread per
 * step; blocks_per_sm: 0 (as many as fit) to 32 (the shared-memory
 * pipelines take 1 or 2); pipeline: the kernel variant.
 *   0: the library's choice per tree: tensor-map (TMA) tiles for trees
 *      with transposed leaves, bulk-copy chunks for dense trees of five or
 *      more leaves, register loads otherwise;
 *   1: copy pipelines wherever a tree has one: cp.async tiles for
 *      transposed leaves, bulk-copy chunks for dense trees, bulk-copy row
 *      segments for sum/max along dim 1;
 *   2: register loads everywhere.
 * A variant whose alignment rules the operands miss (TMA and bulk copies:
 * 16-byte aligned bases; TMA also leading dimensions of a multiple of 16
 * bytes) falls back to register loads. Results agree within each kernel's
 * rounding rules; the choice changes speed only.
 * FX_E_ARG for a value out of range (the shape is then unchanged). */
fx_status fx_expr_set_launch_shape(fx_expr* x, int block, int unroll, int blocks_per_sm,
                                   int pipeline);

/* Number of kernel launches the last evaluation call on this object
 * enqueued (for launch accounting). */
int fx_expr_last_launches(const fx_expr* x);

/* Synchronises `stream`, then reports FX_E_CUDA if an asynchronous CUDA
 * error is pending or if a kernel of this object gave up one of its bounded
 * waits (the bulk-copy pipelines poll their shared-memory barriers a fixed
 * number of times, then record the failure and finish without combining);
 * the record is cleared. FX_OK otherwise. */
fx_status fx_expr_sync_status(fx_expr* x, void* stream);

/* ---- device probes (these allocate and free a small device buffer) ----- */

/* Measured FP64 FMA throughput of the current device in flop/s (two flops
 * per FMA): a short launch of independent FMA chains on every SM, timed
 * with CUDA events on `stream` (synchronises it). The denominator of the
 * ALU roofline of FP64 trees, whose exp, sqrt and division sequences run
 * on the FP64 pipe. */
fx_status fx_fp64_fma_rate(void* stream, double* flops_per_s);

/* Self-test of the bounded waits: one warp waits on a shared-memory
 * mbarrier that nothing arrives on, gives up after 1000 polls and records
 * the timeout; *word receives the error word (1 = a wait gave up). The
 * kernel always finishes; synchronises `stream`. */
fx_status fx_selftest_wait_timeout(void* stream, unsigned int* word);

/* ---- evaluation without device allocation ------------------------------ */

/* Bytes of the fixed device array behind fx_sqdiff_accu_f32_noalloc: room
 * for 4096 per-block partial sums (16 bytes each) and a completion ticket. */
#define FX_NOALLOC_SCRATCH (4096 * 16 + 256)

/* s = accu(square(A - B)) for FP32 matrices A and B (rows x cols,
 * column-major, leading dimension ld, device pointers), written to the
 * device float *s. Same kernel, launch plan and result as fx_eval on
 * "sqdiff_accu" with f32 storage, but this call allocates no device memory
 * and needs no fx_expr object. The paper has no counterpart: it is for
 * callers that cannot call cudaMalloc while they compute - code working
 * inside a device-memory budget fixed in advance, code that must not add
 * the device synchronisation cudaMalloc/cudaFree can cause, or a host whose
 * allocator belongs to another framework.
 *  - Scratch: a file-scope device array of FX_NOALLOC_SCRATCH bytes, held
 *    by every GPU that loads the library until the process exits.
 *  - The first call on each device looks up that array's device address
 *    (cudaGetSymbolAddress) with the device current and keeps it; make that
 *    first call before any stream capture on the device. The kept address
 *    belongs to the device's context: do not call this entry point again
 *    after cudaDeviceReset in the same process.
 *  - Every call on a device shares the one array, which keeps what the last
 *    call left; the call clears the part that must start at zero. Calls
 *    whose kernels overlap on the GPU (different streams, no ordering) race
 *    on it: order them on one stream or with events.
 *  - An empty matrix (rows or cols 0) writes 0.
 *  - FX_E_UNSUPPORTED if the launch would need more than 4096 partial sums
 *    (a 152-SM GB300 at the default launch shape needs at most 1216);
 *    FX_E_ARG / FX_E_SHAPE / FX_E_ALIGN as for fx_expr_bind (4-byte
 *    alignment), FX_E_SHAPE also for extents whose element indices would
 *    overflow 64 bits; FX_E_CUDA if a CUDA call fails. Asynchronous on
 *    `stream`. */
fx_status fx_sqdiff_accu_f32_noalloc(const float* A, const float* B, int64_t rows, int64_t cols,
                                     int64_t ld, float* s, void* stream);

/* ---- errors ------------------------------------------------------------- */

const char* fx_last_error_string(void);
const char* fx_status_string(fx_status s);

#ifdef __cplusplus
}
#endif
#endif /* FX_H */
