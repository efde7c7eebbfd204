// Bucket discovery (Algorithm 2's first loop, parallelised as Section 3.2
// suggests: each bucket is a maximal run of entries with equal prefix
// coordinates, found by comparing adjacent entries) and the split of buckets
// into those one thread block sorts in shared memory and those the global
// digit passes sort.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

constexpr int kSegThreads = 256;
constexpr int kSegItems = 16;
constexpr int kSegTile = kSegThreads * kSegItems;
constexpr int kSegWarps = kSegThreads / 32;

struct PrefixCols {
  const int32_t* col[kMaxOrder];
  int n;
};

// One tile of kSegTile entries per block (dynamic tile id, so look-back
// predecessors are always running). flag[j] = 1 when j starts a bucket
// (j == 0 or some prefix coordinate differs from entry j-1). The flagged
// positions are compacted, in order, into seg_start; the last tile appends
// seg_start[nseg] = nnz and stores nseg.
__global__ void __launch_bounds__(kSegThreads)
k_seg_discover(PrefixCols pc, int nnz, int ntiles, int* __restrict__ seg_start,
               uint32_t* __restrict__ lb, int* __restrict__ counters,
               unsigned* status) {
  __shared__ int s_tile;
  __shared__ uint32_t s_tmp[kSegWarps + 1];
  __shared__ uint32_t s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(&counters[kCntSegTile], 1);
  __syncthreads();
  const int t = s_tile;
  if (t >= ntiles) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int base = t * kSegTile + w * kSegItems * 32;
  uint32_t ballots[kSegItems];
  uint32_t wcount = 0;
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    const int j = base + i * 32 + lane;
    bool flag = false;
    if (j < nnz) {
      flag = (j == 0);
      for (int m = 0; m < pc.n; ++m) {
        const int32_t* c = pc.col[m];
        if (j > 0) flag |= __ldg(c + j) != __ldg(c + j - 1);
      }
    }
    ballots[i] = __ballot_sync(0xffffffffu, flag);
    wcount += __popc(ballots[i]);
  }
  // block scan of per-warp counts (lane 0 of each warp contributes)
  uint32_t total;
  uint32_t wexcl = block_exclusive_sum<kSegWarps>(lane == 0 ? wcount : 0u, s_tmp, &total);
  wexcl = __shfl_sync(0xffffffffu, wexcl, 0);
  // decoupled look-back on the tile totals
  if (threadIdx.x == 0) {
    uint32_t excl = 0;
    if (t == 0) {
      st_relaxed(lb + t, kLbInclusive | total);
    } else {
      st_relaxed(lb + t, kLbAggregate | total);
      for (int p = t - 1; p >= 0; --p) {
        uint32_t v = wait_flag(lb + p, status);
        excl += v & kLbCountMask;
        if ((v & kLbStateMask) == kLbInclusive) break;
      }
      st_relaxed(lb + t, kLbInclusive | (excl + total));
    }
    s_excl = excl;
    if (t == ntiles - 1) {
      counters[kCntNumSeg] = (int)(excl + total);
      seg_start[excl + total] = nnz;
    }
  }
  __syncthreads();
  uint32_t pos = s_excl + wexcl;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    if (ballots[i] >> lane & 1u)
      seg_start[pos + __popc(ballots[i] & lt)] = base + i * 32 + lane;
    pos += __popc(ballots[i]);
  }
}

// Buckets larger than small_max go to the digit passes: each gets an index,
// a contiguous range of chunk ids and of chunk-group ids (so a bucket's
// chunks are consecutive), and zeroed group sums for every pass.
__global__ void k_seg_classify(const int* __restrict__ seg_start, int* __restrict__ counters,
                               int small_max, int chunk, int2* __restrict__ large,
                               int* __restrict__ chunk_base, int* __restrict__ group_base,
                               int* __restrict__ chunk_owner, int* __restrict__ group_owner,
                               uint32_t* __restrict__ group_sum, int npasses, int max_groups) {
  const int nseg = counters[kCntNumSeg];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += gridDim.x * blockDim.x) {
    const int a = seg_start[i], b = seg_start[i + 1];
    if (b - a <= small_max) continue;
    const int idx = atomicAdd(&counters[kCntNumLarge], 1);
    const int nc = (b - a + chunk - 1) / chunk;
    const int ng = (nc + kGroupChunks - 1) / kGroupChunks;
    const int cb = atomicAdd(&counters[kCntNumChunks], nc);
    const int gb = atomicAdd(&counters[kCntNumGroups], ng);
    atomicAdd(&counters[kCntLargeEntries], b - a);
    large[idx] = make_int2(a, b);
    chunk_base[idx] = cb;
    group_base[idx] = gb;
    for (int j = 0; j < nc; ++j) chunk_owner[cb + j] = idx;
    for (int j = 0; j < ng; ++j) {
      group_owner[gb + j] = idx;
      for (int p = 0; p < npasses; ++p) {
        uint4* row = reinterpret_cast<uint4*>(group_sum + ((size_t)p * max_groups + gb + j) * kRadix);
        for (int k = 0; k < kRadix / 4; ++k) row[k] = make_uint4(0, 0, 0, 0);
      }
    }
  }
}

// Optional input check: coordinates within [0, dim) and entries sorted
// (non-decreasing) lexicographically under the input order tau.
struct ValidateArgs {
  const int32_t* coords;
  int64_t stride;
  int order;
  int nnz;
  int tau[kMaxOrder];
  int64_t dims[kMaxOrder];
};

__global__ void k_validate(ValidateArgs a, unsigned* status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.nnz;
       j += gridDim.x * blockDim.x) {
    int cmp = 0;  // -1: entry j-1 < entry j, 1: greater
    for (int p = 0; p < a.order; ++p) {
      const int m = a.tau[p];
      const int32_t c = a.coords[(int64_t)m * a.stride + j];
      if (c < 0 || (int64_t)c >= a.dims[m]) set_status(status, QSD_ERR_COORD_OUT_OF_RANGE);
      if (j > 0 && cmp == 0) {
        const int32_t cp = a.coords[(int64_t)m * a.stride + j - 1];
        cmp = cp < c ? -1 : (cp > c ? 1 : 0);
      }
    }
    if (cmp > 0) set_status(status, QSD_ERR_UNSORTED_INPUT);
  }
}

__device__ unsigned g_sticky_status;

__global__ void k_fold_status(const unsigned* ws_status) {
  const unsigned s = *ws_status;
  if (s) atomicCAS(&g_sticky_status, 0u, s);
}

}  // namespace

cudaError_t launch_seg_discover(const int32_t* const* prefix_cols, int nprefix,
                                int nnz, int* seg_start, uint32_t* seg_lb,
                                int* counters, unsigned* status,
                                cudaStream_t stream) {
  PrefixCols pc;
  pc.n = nprefix;
  for (int m = 0; m < kMaxOrder; ++m) pc.col[m] = m < nprefix ? prefix_cols[m] : nullptr;
  const int ntiles = (nnz + kSegTile - 1) / kSegTile;
  if (ntiles == 0) return cudaSuccess;
  k_seg_discover<<<ntiles, kSegThreads, 0, stream>>>(pc, nnz, ntiles, seg_start,
                                                      seg_lb, counters, status);
  return cudaGetLastError();
}

int seg_lookback_words(int nnz) { return (nnz + kSegTile - 1) / kSegTile + 1; }

cudaError_t launch_seg_classify(const int* seg_start, int* counters, int nnz, int small_max,
                                int chunk, int2* large, int* chunk_base, int* group_base,
                                int* chunk_owner, int* group_owner, uint32_t* group_sum,
                                int npasses, int max_groups, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (nnz + 255) / 256;
  if (blocks > sms * 8) blocks = sms * 8;
  if (blocks < 1) blocks = 1;
  k_seg_classify<<<blocks, 256, 0, stream>>>(seg_start, counters, small_max, chunk, large,
                                             chunk_base, group_base, chunk_owner, group_owner,
                                             group_sum, npasses, max_groups);
  return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t* coords, int64_t stride, int order,
                            const int64_t* dims, const int* tau, int nnz,
                            unsigned* status, cudaStream_t stream) {
  ValidateArgs a;
  a.coords = coords;
  a.stride = stride;
  a.order = order;
  a.nnz = nnz;
  for (int m = 0; m < kMaxOrder; ++m) {
    a.tau[m] = m < order ? tau[m] : 0;
    a.dims[m] = m < order ? dims[m] : 1;
  }
  int blocks = (nnz + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) return cudaSuccess;
  k_validate<<<blocks, 256, 0, stream>>>(a, status);
  return cudaGetLastError();
}

cudaError_t launch_fold_status(const unsigned* ws_status, cudaStream_t stream) {
  k_fold_status<<<1, 1, 0, stream>>>(ws_status);
  return cudaGetLastError();
}

cudaError_t read_and_clear_sticky(unsigned* out, cudaStream_t stream) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyFromSymbol(out, g_sticky_status, sizeof(unsigned));
  if (e != cudaSuccess) return e;
  const unsigned zero = 0;
  return cudaMemcpyToSymbol(g_sticky_status, &zero, sizeof(unsigned));
}

}  // namespace qsd
