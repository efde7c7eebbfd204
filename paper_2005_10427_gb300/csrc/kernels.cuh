// Kernel argument structures and launcher declarations (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsd_internal.h"

namespace qsd {

// Workspace counter slots (int32), zeroed before every group.
enum Counter {
  kCntSegTile = 0,   // dynamic tile id of the bucket discovery kernel
  kCntNumSeg = 1,    // number of buckets found
  kCntNumLarge = 2,  // number of buckets too large for one thread block
  kCntNumTiles = 3,  // digit-pass tiles over all large buckets
  kCntLargeEntries = 4,  // entries inside large buckets
  kCntPassTile = 5,  // dynamic tile ids of the digit passes: 5 .. 5+kMaxPasses
  kNumCounters = 5 + kMaxPasses
};

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

// The buckets handled by the global digit passes. When `single` is set there
// is one bucket [0, nnz) and no device tables.
struct LargeSegs {
  int single;
  int nnz;
  int single_tiles;          // tiles of the single bucket
  const int* counters;       // kCntNumLarge / kCntNumTiles
  const int2* seg;           // [start, end) of each large bucket
  const int* tile_base;      // first tile of each large bucket
  const int* tile_owner;     // large bucket of each tile
};

struct PassList {
  int npasses;
  PassDesc pass[kMaxPasses];
};

// Launch helpers (return a CUDA error code; 0 on success).
cudaError_t launch_seg_discover(const int32_t* const* prefix_cols, int nprefix,
                                int nnz, int* seg_start, uint32_t* seg_lb,
                                int* counters, unsigned* status,
                                cudaStream_t stream);
cudaError_t launch_seg_classify(const int* seg_start, int* counters, int nnz,
                                int small_max, int tile, int2* large,
                                int* tile_base, int* tile_owner, uint32_t* hist,
                                int npasses, cudaStream_t stream);
cudaError_t launch_validate(const int32_t* coords, int64_t stride, int order,
                            const int64_t* dims, const int* tau, int nnz,
                            unsigned* status, cudaStream_t stream);

int onesweep_tile();  // entries per digit-pass tile
cudaError_t launch_digit_hist(const Cols& c, const LargeSegs& ls,
                              const PassList& pl, uint32_t* hist, uint32_t* lb0,
                              int max_tiles, unsigned* status,
                              cudaStream_t stream);
cudaError_t launch_digit_scan(const LargeSegs& ls, int npasses, uint32_t* hist,
                              int max_large, cudaStream_t stream);
cudaError_t launch_onesweep_pass(const Cols& c, const LargeSegs& ls,
                                 const PassDesc& pd, int pass_index, int npasses,
                                 const uint32_t* digit_base, uint32_t* lb,
                                 uint32_t* lb_next, int* tile_counter,
                                 int max_tiles, unsigned* status,
                                 cudaStream_t stream);

cudaError_t launch_local_sort(const Cols& c, const PassList& pl,
                              const int* seg_start, const int* counters,
                              int single, int nnz, int capacity,
                              unsigned* status, cudaStream_t stream);

// Copies every coordinate row and the values from c.in to c.out (entries
// [0, nnz)): a zero-pass plan asked for a distinct output buffer.
cudaError_t launch_copy(const Cols& c, int nnz, cudaStream_t stream);

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
cudaError_t read_and_clear_sticky(unsigned* out, cudaStream_t stream);

}  // namespace qsd
