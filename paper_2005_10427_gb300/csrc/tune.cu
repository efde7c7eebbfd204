// Plan tuner (qsd_plan_tune): a measured choice among equivalent plans.
//
// The paper orders plans by the number of partial sorts (Theorems 2-3) and
// proposes, as future work, choosing by actual cost. Every candidate here
// computes the same result and differs in how: Quesadilla or Top-K-sadilla
// for a K (Section 3.6: fewer calls of Algorithm 3, then one complete sort of
// the buckets of the first K target modes), whether groups with a prefix
// sort bucket by bucket or as one global sort by (prefix, key), the radix
// digit width (how many passes), the tile and chunk sizes, the bucket
// capacity of the shared-memory sort, whether groups without a prefix sort
// (key, index) pairs and gather the entries once at the end, and the width
// of the least significant digit.
// Each candidate is timed with CUDA events over real out-of-place
// transpositions of the caller's data; a coordinate search keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace {

qsd_status plan_with(const qsd_plan_s* base, const qsd_plan_options& o, qsd_plan_t* out) {
  return qsd_plan_ex(base->order, base->dims, base->tau, base->sigma, &o, out);
}

bool has_prefix_group(const qsd_plan_s* p) {
  for (int g = 0; g < p->ngroups; ++g)
    if (p->groups[g].npasses > 0 && p->groups[g].prefix_len > 0) return true;
  return false;
}

// The values each option takes in the search (0 = the library's choice);
// top_k takes 0 .. order - 2.
constexpr int kDims = 8;
const int kKeyIndex[] = {0, 1};
const int kFirstDigit[] = {0, 6, 5, 7};
const int kStructure[] = {0, 1};
const int kDigits[] = {8, 7, 6, 5};
const int kTiles[] = {0, 4096, 3584, 2048};
const int kCaps[] = {4096, 2048, 8192, 1024};
const int kChunks[] = {2, 4, 1};

template <typename F>
void for_each_candidate_value(int dim, int order, F f) {
  switch (dim) {
    case 0: for (int v = 0; v <= std::max(0, order - 2); ++v) f(v); break;
    case 1: for (int v : kStructure) f(v); break;
    case 2: for (int v : kDigits) f(v); break;
    case 3: for (int v : kTiles) f(v); break;
    case 4: for (int v : kCaps) f(v); break;
    case 5: for (int v : kChunks) f(v); break;
    case 6: for (int v : kKeyIndex) f(v); break;
    case 7: for (int v : kFirstDigit) f(v); break;
  }
}

int& field(qsd_plan_options& o, int dim) {
  switch (dim) {
    case 0: return o.top_k;
    case 1: return o.global_groups;
    case 2: return o.digit_bits;
    case 3: return o.tile;
    case 4: return o.local_capacity;
    case 5: return o.chunk_tiles;
    case 6: return o.key_index;
    default: return o.first_digit_bits;
  }
}

// Whether the plan under options o has a group in (key, index) form.
bool has_key_index_group(const qsd_plan_s* base, const qsd_plan_options& o) {
  qsd_plan_t p = nullptr;
  if (plan_with(base, o, &p) != QSD_OK) return false;
  bool r = false;
  for (int g = 0; g < p->ngroups; ++g) r |= p->groups[g].key_index != 0;
  qsd_plan_destroy(p);
  return r;
}

// Whether the plan under options o has a group sorted bucket by bucket.
bool has_prefix_group(const qsd_plan_s* base, const qsd_plan_options& o) {
  qsd_plan_t p = nullptr;
  if (plan_with(base, o, &p) != QSD_OK) return false;
  const bool r = has_prefix_group(p);
  qsd_plan_destroy(p);
  return r;
}

}  // namespace

extern "C" {

qsd_status qsd_plan_tune_workspace_bytes(qsd_plan_t plan, int64_t nnz, size_t* bytes) {
  if (!plan || !bytes || nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  size_t best = 0;
  auto take = [&](const qsd_plan_options& c) {
    qsd_plan_t p = nullptr;
    if (plan_with(plan, c, &p) != QSD_OK) return;
    size_t b = 0;
    if (qsd_workspace_bytes(p, nnz, &b) == QSD_OK) best = std::max(best, b);
    qsd_plan_destroy(p);
  };
  // For every structure (top_k, global_groups): every single change of the
  // other options (the search only ever combines the current best with one
  // changed option, and the sizes are small enough to take the maximum over
  // all of them from any start), and the smallest capacity, digit, chunk
  // and tile together (the most chunk groups).
  for (int k = 0; k <= std::max(0, plan->order - 2); ++k)
    for (int gg = 0; gg < 2; ++gg) {
      qsd_plan_options o = plan->opts;
      o.top_k = k;
      o.global_groups = gg;
      take(o);
      for (int dim = 2; dim < kDims; ++dim)
        for_each_candidate_value(dim, plan->order, [&](int v) {
          qsd_plan_options c = o;
          field(c, dim) = v;
          take(c);
        });
      qsd_plan_options c = o;
      c.local_capacity = 1024;
      c.digit_bits = 5;
      c.chunk_tiles = 1;
      c.tile = 2048;
      take(c);
      c.key_index = 1;
      take(c);
    }
  *bytes = best;
  return QSD_OK;
}

qsd_status qsd_plan_tune(qsd_plan_t plan, const int32_t* in_coords, int64_t in_stride,
                         const void* in_vals, qsd_coords* out_coords, qsd_values* out_vals,
                         int64_t nnz, void* workspace, size_t workspace_bytes, void* stream,
                         int reps, qsd_plan_options* best_out, float* best_ms_out) {
  if (!plan || !out_coords || !best_out || !workspace) return QSD_ERR_INVALID_ARGUMENT;
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return QSD_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return QSD_ERR_CUDA;
  }
  // ms per transposition under options o (< 0: no such plan, or not runnable
  // in the workspace)
  auto measure = [&](const qsd_plan_options& o, float* ms) -> qsd_status {
    *ms = -1.f;
    qsd_plan_t p = nullptr;
    qsd_status s = plan_with(plan, o, &p);
    if (s == QSD_ERR_UNSUPPORTED) return QSD_OK;  // e.g. too many digits for the key
    if (s != QSD_OK) return s;
    size_t need = 0;
    s = qsd_workspace_bytes(p, nnz, &need);
    if (s == QSD_OK && need <= workspace_bytes) {
      s = qsd_transpose_from_ws(in_coords, in_stride, in_vals, out_coords, out_vals, nnz, p,
                                workspace, workspace_bytes, stream);  // warm-up
      if (s == QSD_OK && cudaEventRecord(e0, st) != cudaSuccess) s = QSD_ERR_CUDA;
      for (int r = 0; r < reps && s == QSD_OK; ++r)
        s = qsd_transpose_from_ws(in_coords, in_stride, in_vals, out_coords, out_vals, nnz, p,
                                  workspace, workspace_bytes, stream);
      if (s == QSD_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess))
        s = QSD_ERR_CUDA;
      float t = 0.f;
      if (s == QSD_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) s = QSD_ERR_CUDA;
      if (s == QSD_OK) *ms = t / reps;
    }
    qsd_plan_destroy(p);
    return s;
  };
  qsd_plan_options best = plan->opts;
  if (!best.digit_bits) best.digit_bits = qsd::kRadixBits;
  if (!best.local_capacity) best.local_capacity = 4096;
  if (!best.chunk_tiles) best.chunk_tiles = 2;
  float best_ms = -1.f;
  qsd_status s = measure(best, &best_ms);
  for (int dim = 0; dim < kDims && s == QSD_OK; ++dim) {
    const bool prefix = has_prefix_group(plan, best);
    if (dim == 1 && !prefix) continue;  // no bucketed group: one structure only
    // the bucket capacity only matters when a bucket sort runs: a group with
    // a prefix, or a whole tensor small enough for one block
    if (dim == 4 && (!prefix || best.global_groups) && nnz > 8192) continue;
    // the (key, index) form only changes groups without a prefix that take
    // two or more passes
    if (dim == 6) {
      qsd_plan_options k = best;
      k.key_index = 1;
      if (!has_key_index_group(plan, k)) continue;
    }
    qsd_plan_options base = best;
    for_each_candidate_value(dim, plan->order, [&](int v) {
      if (s != QSD_OK || field(base, dim) == v) return;
      qsd_plan_options c = base;
      field(c, dim) = v;
      if (dim == 4 && c.global_groups) return;  // no bucket sort to size
      float ms = -1.f;
      s = measure(c, &ms);
      if (s == QSD_OK && ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best = c;
      }
    });
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return s;
}

}  // extern "C"
