/*
 * qsd.h -- C ABI of the GB300 sparse COO tensor transposition library.
 *
 * The library transposes a COO tensor whose entries are sorted
 * lexicographically under one complete mode ordering (the input order tau)
 * into lexicographic order under a requested complete ordering sigma
 * (the problem of Section 2.2, "Transposition": transposition is a change of
 * the storage order; the result is the entries re-sorted under sigma, with
 * the relative order of equal coordinates kept, since every partial sort of
 * Sections 3.1-3.2 is stable).
 *
 * It follows the method of Section 3: a host planner (qsd_plan) computes the
 * minimal sequence of PartialSort calls of Algorithm 3 (QuesadillaSort) and
 * merges the calls that share a prefix into one stable sort of each bucket of
 * equal prefix by a bit-packed key; qsd_transpose runs that plan with CUDA
 * kernels on one GPU. No call synchronises with the device unless stated.
 *
 * Conventions for every entry point:
 *   - mode labels and positions are 0-based;
 *   - "device" pointers are CUDA device memory of the current device, "host"
 *     pointers are ordinary (ideally page-locked) host memory;
 *   - a `stream` argument is a cudaStream_t passed as void* (NULL = legacy
 *     default stream); device work is stream-ordered on it;
 *   - argument errors are reported synchronously as a qsd_status and nothing
 *     is enqueued; errors found on the device (invalid input under the
 *     `validate` option, a bounded wait that expired) are recorded in a
 *     device status word that qsd_get_async_status / qsd_workspace_status
 *     read. No kernel traps or asserts.
 */
#ifndef QSD_H_
#define QSD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QSD_MAX_ORDER 8

typedef enum {
  QSD_OK = 0,
  QSD_ERR_INVALID_ARGUMENT = 1,   /* bad permutation, dims < 1, null pointer, ... */
  QSD_ERR_UNSUPPORTED = 2,        /* order > QSD_MAX_ORDER, nnz >= 2^30, ... */
  QSD_ERR_OUT_OF_MEMORY = 3,      /* a device allocation failed */
  QSD_ERR_CUDA = 4,               /* a CUDA runtime call failed */
  QSD_ERR_UNSORTED_INPUT = 5,     /* device: input not sorted under tau (validate) */
  QSD_ERR_COORD_OUT_OF_RANGE = 6, /* device: a coordinate outside [0, dim) (validate) */
  QSD_ERR_TIMEOUT = 7,            /* device: a bounded wait expired */
  QSD_ERR_BUDGET = 8,             /* a request does not fit a memory budget */
  QSD_ERR_WORKSPACE_TOO_SMALL = 9 /* workspace_bytes below qsd_workspace_bytes() */
} qsd_status;

/* Immutable host-side plan. Thread-safe to share across host threads and
 * streams once created. */
typedef struct qsd_plan_s* qsd_plan_t;

/* Coordinates: a double buffer of structure-of-arrays int32 mode rows.
 * Mode m of entry j is buf[s][m * stride + j] (device memory). The data to
 * transpose is in buf[selector]; on return qsd_transpose sets selector to
 * the buffer that holds the result (it may be either buffer). The other
 * buffer's contents are scratch during the call. */
typedef struct {
  int32_t* buf[2];
  int64_t stride; /* elements between mode rows, >= nnz */
  int selector;   /* 0 or 1 */
} qsd_coords;

/* Values: a double buffer of opaque elem_bytes-sized payloads (device
 * memory), moved bit for bit with their coordinates. elem_bytes is 4 or 8,
 * or 0 when the tensor carries no values (buf may then be NULL). The
 * selector is updated together with the coordinates' selector. */
typedef struct {
  void* buf[2];
  int elem_bytes;
  int selector;
} qsd_values;

/* Planner options (qsd_plan_ex). Zero-initialise for defaults. */
typedef struct {
  int validate;          /* nonzero: check on the device that coordinates lie
                            in [0, dim) and that the input is sorted under the
                            input order; failures set the async status */
  int digit_bits;        /* radix digit width of the global passes, 1..8;
                            0 = automatic */
  int local_capacity;    /* largest bucket (entries) sorted in shared memory
                            by one thread block, a power of two in
                            [1024, 8192]; 0 = automatic (4096). The library
                            lowers it when the staged rows of the tensor's
                            order and value width would leave room for fewer
                            than two blocks per SM */
  int no_skip;           /* nonzero: ignore the input ordering and run a full
                            radix sort over every mode (the baseline of
                            Section 3 that the method improves on) */
  int tile;              /* entries a global pass stages in shared memory at
                            once: 1024, 2048, 3584 or 4096 (smaller when the
                            rows do not fit); 0 = automatic */
  int chunk_tiles;       /* tiles per chunk, the unit of the per-chunk digit
                            counts, 1..256; 0 = automatic (2) */
  int global_groups;     /* nonzero: run every group that has a prefix as one
                            global sort by (prefix, key) instead of sorting
                            each bucket of equal prefix by the key (the same
                            result: the group's input is sorted by its
                            prefix); more digit passes, no bucket work */
  int top_k;             /* K > 0: Top-K-sadilla (Section 3.6): Algorithm 3
                            sorts to the order of the first K target modes
                            (the other modes keep their input order), then
                            every bucket of equal first-K coordinates is
                            sorted completely by the remaining target modes;
                            the same result. 0, or K >= order - 1: plain
                            Quesadilla; ignored under no_skip.
                            0 <= K <= QSD_MAX_ORDER */
  int key_index;         /* nonzero: every group without a prefix whose key
                            fits 64 bits and takes two or more digit passes
                            sorts (packed key, entry index) pairs instead of
                            whole entries, and moves the coordinates and the
                            values once at the end, gathered through the
                            final index (Algorithm 2's perm array); the same
                            result, fewer bytes per pass, one random read of
                            every entry. Needs 8 (key <= 32 bits) or 12 bytes
                            per entry more workspace */
  int first_digit_bits;  /* 0 < b < the digit width: the least significant
                            digit of every group takes b bits and the rest
                            of the key is split evenly, where that needs no
                            more passes than the even split (fewer runs per
                            tile where the key's low bits are near uniform);
                            0 = even split. 0 <= b <= 8 */
} qsd_plan_options;

/* Description of a plan (qsd_plan_get_info). */
typedef struct {
  int order;
  int input_mode_order[QSD_MAX_ORDER];
  int target_perm[QSD_MAX_ORDER];
  /* The PartialSort calls of Algorithm 3, in execution order: call i is
   * PartialSort(A, (target_perm[0..call_prefix_len[i])), call_mode[i]);
   * it is bucketed (Algorithm 2) when call_prefix_len[i] > 0, else
   * non-bucketed (Algorithm 1). num_calls equals b(tau, sigma). */
  int num_calls;
  int num_bucketed_calls;
  int call_prefix_len[QSD_MAX_ORDER];
  int call_mode[QSD_MAX_ORDER];
  /* Execution groups: group g stably sorts every bucket of equal
   * target_perm[0..group_prefix_len[g]) coordinates by the key made of the
   * modes target_perm[group_prefix_len[g] .. + group_num_keys[g]) (most
   * significant first), bit-packed to group_key_bits[g] bits and sorted in
   * group_digit_passes[g] radix digits. */
  int num_groups;
  int group_prefix_len[QSD_MAX_ORDER];
  int group_num_keys[QSD_MAX_ORDER];
  int group_key_bits[QSD_MAX_ORDER];
  int group_digit_passes[QSD_MAX_ORDER];
  int local_capacity;
  /* 1 where group g runs in (key, index) form (qsd_plan_options.key_index) */
  int group_key_index[QSD_MAX_ORDER];
} qsd_plan_info;

/* Builds the plan for transposing an order-`order` tensor with the given
 * dimensions, sorted under `input_mode_order` (tau), into `target_perm`
 * (sigma) order. Follows Algorithm 3 (Section 3.5), relabelled for a
 * non-simple tau as Section 2.2 allows. Host only; never touches the GPU.
 *   order:            1..QSD_MAX_ORDER
 *   dims:             host array[order], each 1 <= dims[m] <= 2^31 - 1
 *   input_mode_order: host array[order], a permutation of 0..order-1
 *   target_perm:      host array[order], a permutation of 0..order-1
 *   out:              receives the plan; release with qsd_plan_destroy
 * Returns QSD_ERR_INVALID_ARGUMENT / QSD_ERR_UNSUPPORTED on bad input. */
qsd_status qsd_plan(int order, const int64_t* dims, const int* input_mode_order,
                    const int* target_perm, qsd_plan_t* out);

/* qsd_plan with options (opts may be NULL = defaults). Also returns
 * QSD_ERR_UNSUPPORTED when a group's packed key would need more than 32
 * digit passes at the chosen digit width (possible only below 8 bits). */
qsd_status qsd_plan_ex(int order, const int64_t* dims,
                       const int* input_mode_order, const int* target_perm,
                       const qsd_plan_options* opts, qsd_plan_t* out);

/* Copies the plan's description into *info (host memory). */
qsd_status qsd_plan_get_info(qsd_plan_t plan, qsd_plan_info* info);

/* Releases a plan. NULL is ignored. */
void qsd_plan_destroy(qsd_plan_t plan);

/* Device scratch (bytes) that qsd_transpose_ws needs for `nnz` entries.
 * Independent of the data; 0 <= nnz < 2^30. */
qsd_status qsd_workspace_bytes(qsd_plan_t plan, int64_t nnz, size_t* bytes);

/* Transposes in place of the double buffers: on return (stream-ordered) the
 * result is in coords->buf[coords->selector] and vals->buf[vals->selector].
 * Scratch is taken with cudaMallocAsync on `stream` and released on it.
 * coords, vals: host structs describing device buffers (vals may be NULL
 * when the tensor has no values). 0 <= nnz < 2^30; nnz = 0 does nothing.
 * Asynchronous device errors: see qsd_get_async_status. */
qsd_status qsd_transpose(qsd_coords* coords, qsd_values* vals, int64_t nnz,
                         qsd_plan_t plan, void* stream);

/* As qsd_transpose, with caller-provided device scratch `workspace` of
 * `workspace_bytes` >= qsd_workspace_bytes(plan, nnz), 256-byte aligned.
 * Makes no allocation. The workspace must not be used by another call that
 * may overlap on the device; its first 4 bytes hold this call's device
 * status word (see qsd_workspace_status). */
qsd_status qsd_transpose_ws(qsd_coords* coords, qsd_values* vals, int64_t nnz,
                            qsd_plan_t plan, void* workspace,
                            size_t workspace_bytes, void* stream);

/* Out-of-place transpose: reads the input from `in_coords` (device; mode m
 * of entry j at in_coords[m * in_stride + j]) and `in_vals` (device,
 * out_vals->elem_bytes per entry; NULL when there are no values) and leaves
 * them unchanged; the result is written to out_coords->buf[selector] /
 * out_vals->buf[selector], the selectors being set on return. Both output
 * buffers serve as scratch and must not alias the input. Same workspace
 * rules as qsd_transpose_ws; makes no allocation. A plan with no pass copies
 * the input. This is the call for tensors kept resident and transposed
 * repeatedly (the input stays sorted under tau). */
qsd_status qsd_transpose_from_ws(const int32_t* in_coords, int64_t in_stride,
                                 const void* in_vals, qsd_coords* out_coords,
                                 qsd_values* out_vals, int64_t nnz,
                                 qsd_plan_t plan, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* Transposes exactly like qsd_transpose_ws, but allocates nothing and takes
 * no workspace: for callers that cannot allocate device memory, such as code
 * that runs inside a host framework or serving engine which owns all device
 * memory through its own allocator and budget, or a latency-critical path
 * where a device allocation (which can synchronise the device) is not
 * acceptable. (The paper has no counterpart; this is a library service.)
 *
 * Scratch comes from one file-scope device array of 64 MiB that every GPU
 * loading this library reserves until the process exits. Requests whose
 * qsd_workspace_bytes(plan, nnz) exceeds 64 MiB are rejected with
 * QSD_ERR_WORKSPACE_TOO_SMALL before anything is enqueued (for plans with a
 * bucketed group that is roughly 12 million entries; use qsd_transpose_ws
 * beyond that). All calls on a device share the array and each call resets
 * the parts that must start at zero, so calls that may overlap on the GPU
 * (different streams, or streams not ordered with each other) race and must
 * not be issued; calls ordered on one stream are fine. The first call on each
 * device resolves the array's device address (cudaGetSymbolAddress) and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not call this entry point after a reset of the
 * device's primary context (cudaDeviceReset), which reloads the module and
 * leaves the kept address stale. While the launch profiler
 * (qsd_profile_enable) is on, the call returns QSD_ERR_UNSUPPORTED before
 * anything is enqueued, because the profiler allocates buffers of its own.
 * The array lies outside any memory budget of the serving loop below.
 * Arguments, result buffers and errors are as for qsd_transpose_ws. */
qsd_status qsd_transpose_noalloc(qsd_coords* coords, qsd_values* vals,
                                 int64_t nnz, qsd_plan_t plan, void* stream);

/* End-to-end transpose of HOST arrays: copies the input (host_coords rows of
 * length nnz at host_stride, host_vals) into the caller's device double
 * buffers, transposes with `workspace`, copies the result into host_out_*,
 * and waits for `stream`. Host arrays should be page-locked for full copy
 * bandwidth. host_vals / host_out_vals may be NULL when dev_vals is NULL or
 * has elem_bytes 0. Returns the call's device status as well. */
qsd_status qsd_transpose_host(const int32_t* host_coords, int64_t host_stride,
                              const void* host_vals, int32_t* host_out_coords,
                              int64_t host_out_stride, void* host_out_vals,
                              int64_t nnz, qsd_plan_t plan,
                              qsd_coords* dev_coords, qsd_values* dev_vals,
                              void* workspace, size_t workspace_bytes,
                              void* stream);

/* qsd_transpose_host without the wait: enqueues the copy in, the
 * transposition and the copy out on `stream` and returns. The host arrays,
 * device buffers and workspace must stay untouched until the stream has
 * passed the call; the device status is read afterwards with
 * qsd_workspace_status(workspace, stream). With page-locked host arrays,
 * calls on two streams (each with its own device buffers and workspace)
 * overlap one call's copy out with the next call's copy in and kernels.
 * Argument errors are returned at once, as for qsd_transpose_host. */
qsd_status qsd_transpose_host_async(const int32_t* host_coords, int64_t host_stride,
                                    const void* host_vals, int32_t* host_out_coords,
                                    int64_t host_out_stride, void* host_out_vals,
                                    int64_t nnz, qsd_plan_t plan,
                                    qsd_coords* dev_coords, qsd_values* dev_vals,
                                    void* workspace, size_t workspace_bytes,
                                    void* stream);

/* Waits for `stream`, then reads the status word of a workspace used by
 * qsd_transpose_ws (QSD_OK if no device error was recorded). */
qsd_status qsd_workspace_status(const void* workspace, void* stream,
                                qsd_status* out);

/* Waits for `stream`, then returns and clears the current device's sticky
 * status word, which every transpose on that device ORs its errors into. */
qsd_status qsd_get_async_status(void* stream, qsd_status* out);

/* ---- Graph-captured calls ----
 * One out-of-place transposition (the arguments of qsd_transpose_from_ws)
 * captured once into a CUDA graph and replayed by a single graph launch per
 * call: for repeated transpositions of resident tensors, especially small
 * ones, whose time otherwise goes to launching a dozen or so kernels and
 * memsets one by one. The pointers, nnz and plan are bound at creation and
 * must stay valid (and unmodified in meaning) until qsd_exec_destroy; the
 * input must be re-filled in place if it changes. Each launch computes the
 * whole transposition anew, writes the same output buffer every time (its
 * selector is returned), and uses the workspace like qsd_transpose_from_ws
 * (its status word reports device errors; launches that may overlap on the
 * device must not share a workspace). (No counterpart in the paper.)
 *
 * qsd_exec_create captures without running anything on the device; it
 * returns the argument errors of qsd_transpose_from_ws, and
 * QSD_ERR_UNSUPPORTED while the launch profiler is on.
 * qsd_exec_launch launches on `stream` and stores the result's selectors
 * (coordinates and values; either pointer may be NULL).
 * qsd_exec_destroy releases the graph. NULL is ignored. */
typedef struct qsd_exec_s* qsd_exec_t;
qsd_status qsd_exec_create(const int32_t* in_coords, int64_t in_stride, const void* in_vals,
                           const qsd_coords* out_coords, const qsd_values* out_vals,
                           int64_t nnz, qsd_plan_t plan, void* workspace,
                           size_t workspace_bytes, qsd_exec_t* out);
qsd_status qsd_exec_launch(qsd_exec_t exec, void* stream, int* selector, int* vals_selector);
void qsd_exec_destroy(qsd_exec_t exec);

/* ---- Bounded waits: test-only controls ----
 * Every wait of a kernel on another part of itself (a staging buffer that a
 * bulk copy fills, a hand-off between its warps) gives up after a limit,
 * records QSD_ERR_TIMEOUT in the device status word and returns; no kernel
 * traps, and the context stays usable. These two calls exist so that a test
 * can make such a wait expire on purpose and watch the status. They are
 * process-wide, apply to the current device, synchronise with it, and must
 * not be called while library work is in flight. (No counterpart in the
 * paper.)
 *
 * qsd_debug_set_spin_limit_ns: the limit of every bounded wait, in ns;
 * 0 restores the default (2 s). At most 60 s (else
 * QSD_ERR_INVALID_ARGUMENT).
 * qsd_debug_set_stall: 1 = from the next launch on, block 0 of the digit-pass
 * move kernel arms its first staging slot for the slot's bulk copies but
 * issues none of them, so every wait on that slot expires and the block's
 * warps leave through their abort path (the pass's output is then
 * undefined and the status word reads QSD_ERR_TIMEOUT); 0 = off (default).
 * Other values: QSD_ERR_INVALID_ARGUMENT. */
qsd_status qsd_debug_set_spin_limit_ns(uint64_t limit_ns);
qsd_status qsd_debug_set_stall(int stall);

/* ---- Plan tuner ----
 * The paper ranks plans by their number of partial sorts and leaves choosing
 * by measured cost to future work. qsd_plan_tune does that for one tensor:
 * starting from the plan's options it times out-of-place transpositions of
 * the caller's data (qsd_transpose_from_ws, `reps` timed runs per candidate,
 * CUDA events on `stream`) under one changed option at a time -- groups with
 * a prefix as bucket sorts or as global sorts (global_groups), digit width,
 * tile size, bucket capacity, chunk length -- keeps the fastest, and writes
 * its options to *best (and its time per transposition to *best_ms, may be
 * NULL). Every candidate gives the same result (the plan's calls are
 * fixed). Candidates needing more than workspace_bytes are skipped;
 * qsd_plan_tune_workspace_bytes gives an amount that fits all of them. The
 * output buffers are overwritten. Synchronises `stream`. */
qsd_status qsd_plan_tune_workspace_bytes(qsd_plan_t plan, int64_t nnz, size_t* bytes);
qsd_status qsd_plan_tune(qsd_plan_t plan, const int32_t* in_coords, int64_t in_stride,
                         const void* in_vals, qsd_coords* out_coords, qsd_values* out_vals,
                         int64_t nnz, void* workspace, size_t workspace_bytes, void* stream,
                         int reps, qsd_plan_options* best, float* best_ms);

/* ---- Compressed sparse fiber levels ----
 * The CSF tree of Section 2.1 for a tensor sorted under sigma (for example a
 * result of qsd_transpose with target_perm sigma): level l (1..order) has one
 * node per maximal run of entries with equal coordinates in modes
 * sigma[0..l-1], in order. Level l's node ids are the coordinates of mode
 * sigma[l-1]; node k of level l < order has children ptr[l][k] ..
 * ptr[l][k+1]-1 on level l+1 (level 0 is the root); leaf k covers entries
 * ptr[order][k] .. ptr[order][k+1]-1 (more than one only for duplicate
 * coordinates), which index the values array. All arrays are device int32. */
typedef struct {
  int32_t* ids[QSD_MAX_ORDER];      /* ids[l]: level l+1's node ids, capacity >= nnz */
  int32_t* ptr[QSD_MAX_ORDER + 1];  /* ptr[0]: capacity 2; ptr[l], l >= 1: capacity >= nnz + 1 */
} qsd_csf;

/* Device scratch (bytes) qsd_csf_build needs. */
qsd_status qsd_csf_workspace_bytes(int order, int64_t nnz, size_t* bytes);

/* Builds the CSF levels of the device rows `coords` (mode m at
 * coords + m * stride, sorted under sigma) on `stream`: fills out->ids[0..order-1],
 * out->ptr[0..order] and nodes[0..order] (device int32; nodes[l] = nodes on
 * level l, nodes[0] = 1). One count, scan and write pass over the entries.
 * Unsorted input gives a tree of the runs it does have (no error, every
 * write in bounds). Errors: QSD_ERR_INVALID_ARGUMENT, QSD_ERR_UNSUPPORTED,
 * QSD_ERR_WORKSPACE_TOO_SMALL, QSD_ERR_CUDA. */
qsd_status qsd_csf_build(const int32_t* coords, int64_t stride, int64_t nnz, int order,
                         const int* sigma, const qsd_csf* out, int32_t* nodes,
                         void* workspace, size_t workspace_bytes, void* stream);

/* Transposition and the CSF levels of its result in one call: as
 * qsd_transpose_from_ws followed by qsd_csf_build on the result (sigma =
 * the plan's target order), but the comparisons of neighbouring output
 * entries the levels are made of are done by the transposition's last
 * movement, which has both entries in shared memory (the paper's closing
 * section proposes fusing format conversion into the sort): it leaves one
 * byte per entry, the first level at which the entry differs from the one
 * before it (0 where that entry was written by another tile or bucket
 * batch), and the CSF pass reads those bytes instead of every coordinate
 * row, working out the unknown ones from the rows. Arguments as for
 * qsd_transpose_from_ws and qsd_csf_build; `workspace` must hold
 * qsd_transpose_csf_workspace_bytes(plan, nnz), 256-byte aligned. The
 * tree is the same as qsd_csf_build gives. */
qsd_status qsd_transpose_csf_workspace_bytes(qsd_plan_t plan, int64_t nnz, size_t* bytes);
qsd_status qsd_transpose_csf_from_ws(const int32_t* in_coords, int64_t in_stride,
                                     const void* in_vals, qsd_coords* out_coords,
                                     qsd_values* out_vals, int64_t nnz, qsd_plan_t plan,
                                     const qsd_csf* csf, int32_t* nodes, void* workspace,
                                     size_t workspace_bytes, void* stream);

/* ---- Batches ----
 * Many independent tensors transposed together. The paper transposes one
 * tensor at a time; a batch runs the same method (each tensor gets its own
 * plan and result, bit for bit the result qsd_transpose gives) but shares
 * the launches among the tensors: each stage (bucket discovery, bucket
 * sort, and every radix pass's count, offset and move kernels) is one
 * launch of persistent thread blocks that take work items of every tensor
 * at that stage. Tensors whose plans have several groups run them in
 * rounds; a tensor with fewer passes drops out of the later passes. The
 * whole launch sequence is captured once in a CUDA graph and replayed by
 * each qsd_batch_run (one graph launch per run).
 *
 * A batch binds its buffers at creation: each tensor's input is read-only
 * and its result goes to its own double buffer, so a batch can be run any
 * number of times (each run recomputes the same results). */
typedef struct qsd_batch_s* qsd_batch_t;

/* One tensor of a batch. All pointers are device memory. */
typedef struct {
  qsd_plan_t plan;       /* its plan (copied by qsd_batch_create) */
  int64_t nnz;           /* entries, >= 0 */
  const int32_t* in;     /* input rows, mode m at in + m * in_stride, sorted
                            under the plan's input order; read only */
  int64_t in_stride;     /* >= nnz */
  const void* in_vals;   /* input values (val_bytes each); NULL when the
                            batch carries no values */
  int32_t* out[2];       /* result double buffer, mode m at
                            out[s] + m * out_stride; must not overlap `in` */
  int64_t out_stride;    /* >= nnz */
  void* out_vals[2];     /* value double buffer (NULL without values) */
} qsd_batch_item;

/* Execution options of a batch (zero-initialise for defaults). digit_bits
 * and local_capacity replace every plan's own when nonzero; tile and
 * chunk_tiles are as in qsd_plan_options. */
typedef struct {
  int digit_bits;      /* 0 = each plan's own */
  int local_capacity;  /* 0 = 4096 */
  int tile;            /* 0 = automatic */
  int chunk_tiles;     /* 0 = 2 */
  int no_graph;        /* nonzero: launch directly instead of replaying a graph */
  int use_tuned;       /* nonzero: take the options the tuning cache holds for
                          a batch of this shape, if any (qsd_batch_tune) */
} qsd_batch_options;

/* Creates a batch of n >= 1 tensors. val_bytes is 0 (no values), 4 or 8 for
 * every tensor. opts may be NULL. Checks every item (plans, strides,
 * pointers, total entries below 2^30) and uploads the batch's work tables
 * to the device (synchronously). Errors: QSD_ERR_INVALID_ARGUMENT,
 * QSD_ERR_UNSUPPORTED, QSD_ERR_OUT_OF_MEMORY, QSD_ERR_CUDA. */
qsd_status qsd_batch_create(const qsd_batch_item* items, int n, int val_bytes,
                            const qsd_batch_options* opts, qsd_batch_t* out);

/* Device scratch (bytes) qsd_batch_run needs. */
qsd_status qsd_batch_workspace_bytes(qsd_batch_t batch, size_t* bytes);

/* Transposes every tensor of the batch on `stream`. workspace: device
 * memory of at least qsd_batch_workspace_bytes bytes, 256-byte aligned; its
 * first word is the status word qsd_workspace_status reads. The first run
 * with a given workspace captures the graph (not on `stream` itself); later
 * runs replay it. A batch is not safe to run from two host threads at once.
 * Errors: QSD_ERR_WORKSPACE_TOO_SMALL, QSD_ERR_INVALID_ARGUMENT,
 * QSD_ERR_CUDA (nothing enqueued on an argument error). */
qsd_status qsd_batch_run(qsd_batch_t batch, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Which buffer of item i's double buffer holds its result after a run. */
qsd_status qsd_batch_result(qsd_batch_t batch, int i, int* selector);

/* The options the batch runs with. */
qsd_status qsd_batch_get_options(qsd_batch_t batch, qsd_batch_options* out);

/* Autotuner. Times qsd_batch_run under candidate options (tile size, digit
 * width, shared-memory bucket capacity, chunk length; coordinate search from
 * the current options, `reps` timed runs each, CUDA events on `stream`),
 * keeps the fastest, stores it in the process's tuning cache under the
 * batch's shape and writes it to *best (may be NULL). Candidates whose
 * workspace exceeds workspace_bytes are skipped. Synchronises `stream`. */
qsd_status qsd_batch_tune(qsd_batch_t batch, void* workspace, size_t workspace_bytes,
                          void* stream, int reps, qsd_batch_options* best);

/* Writes / reads the tuning cache as text (one shape and its options per
 * line); loading adds to the cache. */
qsd_status qsd_tune_cache_save(const char* path);
qsd_status qsd_tune_cache_load(const char* path);

/* Releases a batch (its device tables and graph). NULL is ignored. */
void qsd_batch_destroy(qsd_batch_t batch);

/* ---- Serving ----
 * A request loop over resident tensors (no counterpart in the paper, which
 * transposes one tensor per call). Callers register tensors that stay in
 * device memory, then submit requests (tensor, target order) from any host
 * thread. An engine thread admits queued requests in arrival order while the
 * in-flight limit and the device memory budget (results and scratch of the
 * admitted requests) allow, and launches each step's admitted requests as
 * one batch (qsd_batch_*) on one of several streams: steps overlap on the
 * device, and requests that arrive while others run join the next step
 * (continuous batching). Each result is bit for bit the one a single
 * qsd_transpose call gives. Results stay in the server's memory until
 * released. Times are seconds of qsd_server_clock(); completion times come
 * from CUDA events on the device. The budget covers the server's own
 * reservation only: the 64 MiB scratch array of qsd_transpose_noalloc, which
 * every GPU loading this library holds, is not counted in it. */
typedef struct qsd_server_s* qsd_server_t;

typedef struct {
  size_t memory_budget;    /* device bytes for results and scratch of admitted
                              requests; reserved when the server is created */
  int max_inflight;        /* admitted, not yet completed requests (0 = 1024) */
  int streams;             /* engine streams = steps in flight at once (0 = 2) */
  int max_batch;           /* requests per step (0 = 256) */
  int val_bytes;           /* value width of every tensor: 0, 4 or 8 */
  qsd_batch_options batch; /* execution options of every step (launched
                              directly; no_graph and use_tuned are ignored) */
} qsd_server_options;

typedef struct {
  int64_t request;        /* id from qsd_server_submit */
  int tensor;             /* the request's tensor */
  int status;             /* qsd_status: QSD_OK, QSD_ERR_BUDGET (the request
                             alone exceeds the budget; no result), or a device
                             error recorded during its step */
  const int32_t* coords;  /* device: result rows, mode m at coords + m * stride
                             (valid until qsd_server_release) */
  int64_t stride;
  const void* vals;       /* device: result values (NULL without values) */
  int64_t nnz;
  double arrival_s;       /* the request's arrival time */
  double admit_s;         /* when its step was launched */
  double done_s;          /* when its step completed on the device */
} qsd_server_result;

typedef struct {
  int64_t submitted, admitted, completed, rejected, released, steps;
  int64_t entries_completed; /* entries transposed by completed requests */
  int queue_depth, max_queue_depth;
  int inflight, max_inflight_seen;
  size_t bytes_in_use, peak_bytes; /* of the budget */
} qsd_server_stats;

/* Creates a server on the current device and starts its engine thread.
 * Errors: QSD_ERR_INVALID_ARGUMENT, QSD_ERR_OUT_OF_MEMORY (the budget could
 * not be reserved), QSD_ERR_CUDA. */
qsd_status qsd_server_create(const qsd_server_options* opts, qsd_server_t* out);

/* Registers a resident tensor: device rows (mode m at coords + m * stride,
 * sorted under input_mode_order; NULL = identity) and values, owned by the
 * caller and kept unchanged while the server lives. *tensor_id receives its
 * id (0, 1, ...). */
qsd_status qsd_server_add_tensor(qsd_server_t server, int order, const int64_t* dims,
                                 const int* input_mode_order, const int32_t* coords,
                                 int64_t stride, const void* vals, int64_t nnz,
                                 int* tensor_id);

/* Queues a request to transpose tensor_id into target_perm. arrival_s: its
 * arrival time (<= 0: now). Never blocks on the device. */
qsd_status qsd_server_submit(qsd_server_t server, int tensor_id, const int* target_perm,
                             double arrival_s, int64_t* request_id);

/* Moves up to max_results completed requests (in completion order) into
 * out, waiting up to wait_ms milliseconds for the first one; *n receives the
 * count. */
qsd_status qsd_server_poll(qsd_server_t server, qsd_server_result* out, int max_results,
                           int wait_ms, int* n);

/* Copies a completed request's result into caller device buffers (rows with
 * stride dst_stride, values) on `stream`. */
qsd_status qsd_server_copy_result(qsd_server_t server, int64_t request_id, int32_t* dst_coords,
                                  int64_t dst_stride, void* dst_vals, void* stream);

/* Returns a completed request's result memory to the budget. A copy made
 * by qsd_server_copy_result must have completed on its stream first: the
 * memory can be reused by the next step at once. */
qsd_status qsd_server_release(qsd_server_t server, int64_t request_id);

qsd_status qsd_server_get_stats(qsd_server_t server, qsd_server_stats* out);

/* Seconds of the monotonic clock the server stamps times with. */
double qsd_server_clock(void);

/* Stops the engine: queued requests are dropped, steps in flight are waited
 * for, and all server memory is freed. NULL is ignored. */
void qsd_server_destroy(qsd_server_t server);

/* ---- Launch profiler (off by default) ----
 * When enabled, every kernel launch of the library on this process is
 * bracketed by CUDA events on its stream and tagged with the entries it
 * processed and the algorithmic bytes that implies (one read and one write
 * of every moved entry's coordinates and value; key or prefix rows read for
 * the histogram and bucket-discovery kernels). Used to compute per-kernel
 * throughput against the HBM roofline. */
typedef struct {
  char kernel[32];    /* "onesweep", "local_sort", "digit_hist", ... */
  int group;          /* plan group index (-1: not group-specific) */
  int pass;           /* radix pass within the group (-1: n/a) */
  int64_t entries;    /* entries the launch processed (-1: unknown) */
  int64_t algo_bytes; /* algorithmic bytes of the launch (-1: unknown) */
  float ms;           /* CUDA-event duration on the launching stream */
} qsd_profile_record;

/* Turns recording on (nonzero) or off for subsequent launches. */
qsd_status qsd_profile_enable(int enable);
/* Waits for the recorded launches and copies up to max_records of them, in
 * launch order, into out (host memory); *n_records receives the number
 * recorded since the last reset. */
qsd_status qsd_profile_read(qsd_profile_record* out, int max_records,
                            int* n_records);
/* Drops all records. */
qsd_status qsd_profile_reset(void);

/* Human-readable name of a status code (static storage). */
const char* qsd_status_string(qsd_status status);

/* Library version string (static storage). */
const char* qsd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QSD_H_ */
