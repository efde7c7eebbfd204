// Batch internals shared by the batch entry points and the serving engine.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace qsd {

constexpr size_t kWsAlign = 256;
constexpr int64_t kMaxBatchNnz = (int64_t(1) << 30) - 1;

inline size_t ws_align_up(size_t x) { return (x + kWsAlign - 1) & ~(kWsAlign - 1); }

// One tensor of a batch (host view).
struct BatchTensor {
  qsd_plan_s plan;  // its plan (re-planned when the batch overrides the digit width)
  qsd_plan_options base_opts;
  int64_t nnz;
  const int32_t* in;
  int64_t in_stride;
  const void* in_vals;
  int32_t* out[2];
  int64_t out_stride;
  void* out_vals[2];
  int result;  // selector of the result after a run
};

// One tensor in one round: its group, passes and buffers (-1 = the input).
struct BatchMember {
  int tensor, group, P, cur, F;
};

struct BatchRound {
  std::vector<BatchMember> m;  // by pass count, descending
  int n = 0, N = 0, ntiles = 0, maxP = 0;
  int max_large = 0, max_chunks = 0, max_groups = 0;
  // byte offsets of the round's tables in the table block
  size_t jbase = 0, tile_base = 0, seg = 0, ls = 0, pool = 0;
  size_t pass[kMaxPasses] = {0};
};

// Byte offsets of the workspace's parts.
struct BatchLayout {
  size_t status, counters, seg_start, seg_lb, large, chunk_base, group_base, chunk_owner,
      group_owner, large_tensor, chunk_hist, group_sum, pass_chunks, pass_groups, total;
  int max_chunks, max_groups, max_passes;
};

// A batch's schedule: tensors, rounds, workspace layout, and where its
// device tables are.
struct BatchCore {
  int n = 0, vbytes = 0;
  qsd_batch_options opts{};
  std::vector<BatchTensor> t;
  std::vector<BatchRound> rounds;
  std::vector<int> copies;  // tensors with entries and no pass: copied to out[0]
  int max_order = 1, T = 0, CH = 0, C = 0;
  BatchLayout L{};
  size_t table_bytes = 0;
  const void* dtab = nullptr;  // device tables (table_bytes)
};

// Plans the rounds and the workspace layout for the core's tensors and
// options (host only; sets table_bytes).
qsd_status batch_prepare(BatchCore& b);
// Writes the table image (table_bytes) for tables living at device address
// dev_base.
void batch_fill_tables(const BatchCore& b, const void* dev_base, uint8_t* image);
// Enqueues one run on `st` (tables at b.dtab, workspace ws of L.total bytes).
qsd_status batch_issue(const BatchCore& b, void* ws, cudaStream_t st);

}  // namespace qsd
