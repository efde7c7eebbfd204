// Kernel argument structures and launcher declarations (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsd_internal.h"

namespace qsd {

// Workspace counter slots (int32), zeroed before every group.
enum Counter {
  kCntSegTile = 0,       // dynamic tile id of the bucket discovery kernel
  kCntNumSeg = 1,        // number of buckets found
  kCntNumLarge = 2,      // buckets too large for one thread block
  kCntNumChunks = 3,     // chunks over all large buckets
  kCntNumGroups = 4,     // chunk groups over all large buckets
  kCntLargeEntries = 5,  // entries inside large buckets
  kCntClaim = 6,         // per pass: chunk claims of the histogram and move kernels
  kCntPassChunks = 6 + 2 * kMaxPasses,  // per pass (batches): active chunks
  kCntPassGroups = 6 + 3 * kMaxPasses,  // per pass (batches): active chunk groups
  kNumCounters = 6 + 4 * kMaxPasses
};

// Chunks per chunk group (the unit of the offset scan).
constexpr int kGroupChunks = 64;

// Structure-of-arrays tensor buffers as the kernels see them.
struct Cols {
  const int32_t* in;   // mode m at in + m * in_stride
  int32_t* out;
  const void* vin;     // values (may be null when vbytes == 0)
  void* vout;
  int64_t in_stride;   // elements between input mode rows
  int64_t out_stride;  // elements between output mode rows
  int order;
  int vbytes;          // 0, 4 or 8
};

// The buckets sorted by the global digit passes, cut into chunks (contiguous
// entry ranges of at most `chunk` entries inside one bucket) and chunk
// groups (kGroupChunks consecutive chunks of one bucket). When `single` is
// set there is one bucket [0, nnz) and the tables are implicit.
struct LargeSegs {
  int single;
  int nnz;
  int tile;                 // entries per tile (the unit staged in shared memory)
  int chunk;                // entries per chunk, a multiple of tile
  const int* counters;      // kCntNumLarge / kCntNumChunks / kCntNumGroups
  const int2* seg;          // [start, end) of each large bucket
  const int* chunk_base;    // first chunk of each large bucket
  const int* group_base;    // first group of each large bucket
  const int* chunk_owner;   // large bucket of each chunk
  const int* group_owner;   // large bucket of each group
};

struct PassList {
  int npasses;
  PassDesc pass[kMaxPasses];
};

// ---------------------------------------------------------------------------
// Batches. One round of a batch runs the same group index of many tensors
// together: they lie end to end in one index space, tensor k holding entries
// [jbase[k], jbase[k+1]), and its buckets, chunks and output slots are
// numbered in that space. A tensor's rows are reached through pointers
// shifted back by jbase[k] elements, so entry J of the space is element J of
// them and the kernels' index arithmetic is the single-tensor one.

// Bucket discovery of a round: tensor k covers discovery tiles
// [tile_base[k], tile_base[k+1]); its buckets are the runs of equal prefix
// coordinates (a tensor with no prefix is one bucket).
struct SegTensor {
  const int32_t* col[kMaxOrder];  // shifted prefix rows
  int n;                          // prefix length
};
struct SegBatch {
  int n;                  // tensors; 0 = one tensor (the launch's own arguments)
  const int* jbase;       // [n + 1]
  const int* tile_base;   // [n + 1]
  const SegTensor* t;     // [n]
};

// A tensor of a round as the shared-memory bucket sort sees it.
struct LsTensor {
  Cols c;                // shifted; input rows -> the rows its group ends in
  int npasses;           // key passes of its group
  const PassDesc* pass;  // [npasses], device memory
};
struct LsBatch {
  int n;                 // 0 = one tensor
  const int* jbase;      // [n + 1]
  const LsTensor* t;     // [n]
};

// A tensor at one pass of a round: its buffers and the pass's digit.
struct PassTensor {
  Cols c;  // shifted
  PassDesc pd;
};

// The work of one pass of a round: the chunks (and chunk groups) of the
// tensors that have this pass, listed by the classification.
struct PassBatch {
  const PassTensor* t;      // [tensors]; null = one tensor
  const int* large_tensor;  // tensor of each large bucket
  const int* chunks;        // active chunk ids
  const int* groups;        // active chunk-group ids
  const int* counters;      // kCntPassChunks + pass / kCntPassGroups + pass
  int pass;
};

// Where the classification records a round's per-pass work.
struct ClassifyBatch {
  int n;                  // 0 = one tensor
  const int* jbase;       // [n + 1]
  const LsTensor* t;      // [n] (for npasses)
  int* large_tensor;      // [max_large]
  int* pass_chunks;       // [max_passes][max_chunks]
  int* pass_groups;       // [max_passes][max_groups]
  int max_chunks;
};

// Launch helpers (return a CUDA error code; 0 on success).
cudaError_t launch_seg_discover(const int32_t* const* prefix_cols, int nprefix,
                                int nnz, int* seg_start, uint32_t* seg_lb,
                                int* counters, unsigned* status,
                                cudaStream_t stream);
// The same over a batch round of `ntiles` discovery tiles and `nnz` entries.
cudaError_t launch_seg_discover_batch(const SegBatch& sb, int ntiles, int nnz, int* seg_start,
                                      uint32_t* seg_lb, int* counters, cudaStream_t stream);
int seg_tile_entries();  // entries per discovery tile
// Buckets larger than small_max are numbered and cut into chunks of `chunk`
// entries and groups of kGroupChunks chunks; their group sums for every pass
// (group_sum[pass][group][kRadix]) are zeroed.
cudaError_t launch_seg_classify(const int* seg_start, int* counters, int nnz, int small_max,
                                int chunk, int2* large, int* chunk_base, int* group_base,
                                int* chunk_owner, int* group_owner, uint32_t* group_sum,
                                int npasses, int max_groups, const ClassifyBatch& cb,
                                cudaStream_t stream);
cudaError_t launch_validate(const int32_t* coords, int64_t stride, int order,
                            const int64_t* dims, const int* tau, int nnz,
                            unsigned* status, cudaStream_t stream);

// Global digit passes (reduce, scan, move):
// Entries per tile and per chunk; `tile` and `chunk_tiles` are requests
// (0 = automatic), honoured when the tile fits shared memory.
int digit_tile(int order, int vbytes, int tile = 0);
int digit_chunk(int order, int vbytes, int tile = 0, int chunk_tiles = 0);
// Per chunk: histogram of the pass's digit into chunk_hist[chunk][kRadix];
// adds each chunk's counts into group_sum[group][kRadix] (zeroed before).
// With a batch (pb.t set) `c` only gives the layout (largest order, value
// width) and `pd` is unused: each chunk takes its tensor's buffers and digit.
cudaError_t launch_chunk_hist(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                              uint32_t* chunk_hist, uint32_t* group_sum, int* claim,
                              int max_chunks, const PassBatch& pb, cudaStream_t stream);
// Per chunk group: turns chunk_hist into each chunk's first output slot per
// digit (bucket start + digits below + the same digit in earlier chunks).
// Over one whole tensor (ls.single, no batch) of more than 16 chunk groups,
// group_sum is first turned, in place, into each group's first slot per digit.
cudaError_t launch_chunk_scan(const LargeSegs& ls, uint32_t* chunk_hist,
                              uint32_t* group_sum, int max_groups, const PassBatch& pb,
                              cudaStream_t stream);
// CSF levels from the last movement of a transposition: for every output
// position g it writes lev[g] = the first level (1-based, in sigma order)
// whose coordinate differs from the entry at g - 1 (order + 1: equal
// coordinates), or 0 where the entry before g is not at hand (another tile
// or batch); lev == nullptr: nothing written.
struct LevOut {
  uint8_t* lev;
  int order;
  int sigma[kMaxOrder];
};

// Moves every row of every chunk to its digit's slots, tile by tile.
cudaError_t launch_digit_move(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                              const uint32_t* chunk_off, int* claim, int max_chunks,
                              unsigned* status, const PassBatch& pb, cudaStream_t stream,
                              const LevOut* lv = nullptr);

// The bucket capacity the shared-memory sort runs with: the largest power of
// two in [1024, want] whose staged rows fit shared memory.
int local_sort_capacity(int want, int order, int vbytes);
// With a batch (lb.n > 0) `c` gives the staging layout (largest order, value
// width) and `pl` is unused.
cudaError_t launch_local_sort(const Cols& c, const PassList& pl,
                              const int* seg_start, const int* counters,
                              int single, int nnz, int capacity,
                              unsigned* status, const LsBatch& lb, cudaStream_t stream,
                              const LevOut* lv = nullptr);

// CSF levels of a tensor sorted under sigma (rows given in sigma order).
struct CsfOut {
  int32_t* ids[kMaxOrder];      // level l + 1 node ids
  int32_t* ptr[kMaxOrder + 1];  // level l: first child (l < order) / first entry (l == order)
};
// lev (nullable, nnz bytes, 16-byte aligned): the first differing level of
// every entry as a transposition's last movement left it (0 = unknown);
// the unknown ones are filled in from the rows first.
cudaError_t launch_csf(const int32_t* const* rows_in_sigma_order, int order, int nnz,
                       const CsfOut& out, int32_t* nodes, uint32_t* tile_count,
                       cudaStream_t stream, uint8_t* lev = nullptr);
size_t csf_workspace_bytes(int order, int nnz);

// Copies every coordinate row and the values from c.in to c.out (entries
// [0, nnz)): a zero-pass plan asked for a distinct output buffer.
cudaError_t launch_copy(const Cols& c, int nnz, cudaStream_t stream);

// (key, index) form of a group: key mode i (a coordinate row) at bit
// base[i] of the packed key; `words` key words (1 or 2).
struct KeyPack {
  int nkeys;
  int words;
  int mode[kMaxOrder];
  int base[kMaxOrder];
};
// Writes the rows c.out + k * c.out_stride (c.out_stride a multiple of 4,
// c.out 16-byte aligned): k < words the packed key's 32-bit words, k = words
// the entry index, for entries [0, nnz) of the rows c.in.
cudaError_t launch_pack(const Cols& c, const KeyPack& kp, int nnz, cudaStream_t stream);
// out rows / values [j] = in rows / values [idx[j]] for j in [0, nnz); idx
// is 16-byte aligned.
cudaError_t launch_gather(const Cols& c, const int32_t* idx, int nnz, cudaStream_t stream);

int seg_lookback_words(int nnz);

// Profiling (qsd_profile_*): when enabled, each launch is bracketed by CUDA
// events on its stream and tagged with the entries it processed. `entries`
// is the host-known count, or -1 to read it from *dev_entries after the
// launch (when `complement` is set the count is total - *dev_entries).
struct ProfTag {
  const char* kernel;
  int group;
  int pass;
  int64_t entries;
  const int* dev_entries;
  int complement;
  int64_t total;
  int64_t bytes_per_entry;
};
bool prof_enabled();
int prof_begin(const ProfTag& tag, cudaStream_t st);
void prof_end(int rec, cudaStream_t st);

cudaError_t launch_fold_status(const unsigned* ws_status, cudaStream_t stream);

// Test-only words of each translation unit with bounded waits: the spin
// limit (ns) and the move kernel's stall (qsd_debug_set_*).
cudaError_t debug_words_digit_pass(unsigned long long limit_ns, int stall);
cudaError_t debug_words_local_sort(unsigned long long limit_ns, int stall);
cudaError_t read_and_clear_sticky(unsigned* out, cudaStream_t stream);

}  // namespace qsd
