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
                            [1024, 8192]; 0 = automatic */
  int no_skip;           /* nonzero: ignore the input ordering and run a full
                            radix sort over every mode (the baseline of
                            Section 3 that the method improves on) */
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

/* qsd_plan with options (opts may be NULL = defaults). */
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
 * device resolves the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture. The launch profiler
 * (qsd_profile_enable) must be off, as it allocates its own buffers.
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

/* Waits for `stream`, then reads the status word of a workspace used by
 * qsd_transpose_ws (QSD_OK if no device error was recorded). */
qsd_status qsd_workspace_status(const void* workspace, void* stream,
                                qsd_status* out);

/* Waits for `stream`, then returns and clears the current device's sticky
 * status word, which every transpose on that device ORs its errors into. */
qsd_status qsd_get_async_status(void* stream, qsd_status* out);

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
