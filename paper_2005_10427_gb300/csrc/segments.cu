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

// Bucket starts in three steps with no dependency between blocks:
//   k_seg_count  per tile of kSegTile entries: flag[j] = 1 when j starts a
//                bucket (j is the tensor's first entry, or a prefix
//                coordinate differs from entry j-1); the flags are kept as
//                one bit per entry (the warp ballots) and the tile's count is
//                stored;
//   k_seg_scan   one block: exclusive prefix of the tile counts, the bucket
//                count, and the sentinel seg_start[nseg] = nnz;
//   k_seg_write  per tile: the flagged positions, compacted in order into
//                seg_start.
// Each warp covers kSegItems consecutive 32-entry pieces, so the ballot of
// round i of warp w holds entries [j0 + 32 * (w * kSegItems + i), +32) of the
// tile starting at entry j0, stored at word tile * kSegTile / 32 +
// w * kSegItems + i. A batch round gives each tensor its own tiles.

// The entries [j0, j1) of discovery tile t and the tensor's first entry.
struct SegTileSpan {
  int j0, j1, first, k;
};

__device__ __forceinline__ int upper_bound_int(const int* a, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ SegTileSpan seg_tile_span(const SegBatch& sb, int nnz, int t) {
  SegTileSpan sp;
  if (sb.n == 0) {
    sp.k = 0;
    sp.first = 0;
    sp.j0 = t * kSegTile;
    sp.j1 = nnz;
  } else {
    sp.k = upper_bound_int(sb.tile_base, 0, sb.n + 1, t) - 1;
    sp.first = __ldg(sb.jbase + sp.k);
    sp.j0 = sp.first + (t - __ldg(sb.tile_base + sp.k)) * kSegTile;
    sp.j1 = __ldg(sb.jbase + sp.k + 1);
  }
  if (sp.j1 > sp.j0 + kSegTile) sp.j1 = sp.j0 + kSegTile;
  return sp;
}

__global__ void __launch_bounds__(kSegThreads)
k_seg_count(PrefixCols pc1, SegBatch sb, int nnz, uint32_t* __restrict__ bits,
            uint32_t* __restrict__ tile_count) {
  __shared__ uint32_t s_warp[kSegWarps];
  __shared__ const int32_t* s_col[kMaxOrder];
  __shared__ int s_n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x;
  const SegTileSpan sp = seg_tile_span(sb, nnz, t);
  if (threadIdx.x < kMaxOrder) {
    if (sb.n == 0) {
      s_col[threadIdx.x] = pc1.col[threadIdx.x];
      if (threadIdx.x == 0) s_n = pc1.n;
    } else {
      s_col[threadIdx.x] = sb.t[sp.k].col[threadIdx.x];
      if (threadIdx.x == 0) s_n = sb.t[sp.k].n;
    }
  }
  __syncthreads();
  const int np = s_n;
  const int base = sp.j0 + w * kSegItems * 32;
  const int wbase = t * (kSegTile / 32) + w * kSegItems;
  uint32_t cnt = 0;
  int32_t prev[kMaxOrder];
  // the entry before this warp's first one
  for (int m = 0; m < np; ++m) {
    const int jp = base + lane - 1;
    prev[m] = (lane == 0 && jp >= sp.first && jp < sp.j1) ? __ldg(s_col[m] + jp) : 0;
  }
#pragma unroll 4
  for (int i = 0; i < kSegItems; ++i) {
    const int j = base + i * 32 + lane;
    const bool in = j < sp.j1;
    bool flag = in && j == sp.first;
    for (int m = 0; m < np; ++m) {
      const int32_t v = in ? __ldg(s_col[m] + j) : 0;
      // entry j-1: lane-1's value, or for lane 0 the previous round's last lane
      int32_t p = __shfl_up_sync(0xffffffffu, v, 1);
      const int32_t last = __shfl_sync(0xffffffffu, v, 31);
      if (lane == 0) p = prev[m];
      prev[m] = last;
      flag |= in && j > sp.first && v != p;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, flag);
    if (lane == 0 && (base + i * 32) < sp.j1) bits[wbase + i] = bal;
    cnt += __popc(bal);
  }
  if (lane == 0) s_warp[w] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int k = 0; k < kSegWarps; ++k) tot += s_warp[k];
    tile_count[t] = tot;
  }
}

// k_seg_count for one tensor whose prefix rows are 16-byte aligned: each lane
// reads four consecutive entries per row with one 16-byte load, so a warp
// covers its 512 entries in four rounds of 128. The flags of a round are the
// lanes' 4-bit groups; lanes 8q .. 8q+7 together give word q of the round
// (entries 32q .. 32q+31), the same words k_seg_count stores.
__global__ void __launch_bounds__(kSegThreads)
k_seg_count_vec(PrefixCols pc, int nnz, uint32_t* __restrict__ bits,
                uint32_t* __restrict__ tile_count) {
  __shared__ uint32_t s_warp[kSegWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x;
  const int j0 = t * kSegTile;
  const int j1 = min(j0 + kSegTile, nnz);
  const int np = pc.n;
  const int base = j0 + w * kSegItems * 32;
  const int wbase = t * (kSegTile / 32) + w * kSegItems;
  int32_t prev[kMaxOrder];
  // the entry before this warp's first one (lane 0's predecessor in round 0)
#pragma unroll
  for (int m = 0; m < kMaxOrder; ++m)
    prev[m] = (m < np && base > 0 && base - 1 < j1) ? __ldg(pc.col[m] + base - 1) : 0;
  uint32_t cnt = 0;
#pragma unroll
  for (int r = 0; r < kSegItems / 4; ++r) {
    const int jv = base + r * 128 + 4 * lane;  // the lane's first entry
    uint32_t nib = 0;
#pragma unroll
    for (int m = 0; m < kMaxOrder; ++m) {
      if (m >= np) break;
      int4 v;
      if (jv + 4 <= j1) {
        v = __ldg(reinterpret_cast<const int4*>(pc.col[m] + jv));
      } else {
        v.x = jv < j1 ? __ldg(pc.col[m] + jv) : 0;
        v.y = jv + 1 < j1 ? __ldg(pc.col[m] + jv + 1) : 0;
        v.z = jv + 2 < j1 ? __ldg(pc.col[m] + jv + 2) : 0;
        v.w = jv + 3 < j1 ? __ldg(pc.col[m] + jv + 3) : 0;
      }
      // entry jv - 1: lane-1's last, or for lane 0 the previous round's lane 31
      int32_t p = __shfl_up_sync(0xffffffffu, v.w, 1);
      const int32_t last = __shfl_sync(0xffffffffu, v.w, 31);
      if (lane == 0) p = prev[m];
      prev[m] = last;
      nib |= (v.x != p ? 1u : 0u) | (v.y != v.x ? 2u : 0u) | (v.z != v.y ? 4u : 0u) |
             (v.w != v.z ? 8u : 0u);
    }
    if (jv == 0) nib |= 1u;  // the tensor's first entry starts a bucket
    const int nvalid = j1 - jv;
    nib &= nvalid >= 4 ? 15u : (nvalid > 0 ? (1u << nvalid) - 1u : 0u);
    uint32_t word = nib << (4 * (lane & 7));
    word |= __shfl_xor_sync(0xffffffffu, word, 1);
    word |= __shfl_xor_sync(0xffffffffu, word, 2);
    word |= __shfl_xor_sync(0xffffffffu, word, 4);
    const int q = lane >> 3;
    if ((lane & 7) == 0 && base + r * 128 + 32 * q < j1) bits[wbase + r * 4 + q] = word;
    cnt += __popc(nib);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) s_warp[w] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int k = 0; k < kSegWarps; ++k) tot += s_warp[k];
    tile_count[t] = tot;
  }
}

__global__ void __launch_bounds__(1024)
k_seg_scan(uint32_t* __restrict__ tile_count, int ntiles, int nnz, int* __restrict__ seg_start,
           int* __restrict__ counters) {
  __shared__ uint32_t s_tmp[33];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < ntiles; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < ntiles ? tile_count[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_sum<32>(v, s_tmp, &total);
    const uint32_t carry = s_carry;
    if (i < ntiles) tile_count[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    counters[kCntNumSeg] = (int)s_carry;
    seg_start[s_carry] = nnz;
  }
}

__global__ void __launch_bounds__(kSegThreads)
k_seg_write(SegBatch sb, int nnz, const uint32_t* __restrict__ bits,
            const uint32_t* __restrict__ tile_off, int* __restrict__ seg_start) {
  __shared__ uint32_t s_tmp[kSegWarps + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int t = blockIdx.x;
  const SegTileSpan sp = seg_tile_span(sb, nnz, t);
  const int base = sp.j0 + w * kSegItems * 32;
  const int wbase = t * (kSegTile / 32) + w * kSegItems;
  uint32_t bal[kSegItems], cnt = 0;
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    bal[i] = (base + i * 32) < sp.j1 ? bits[wbase + i] : 0u;
    cnt += __popc(bal[i]);
  }
  uint32_t total;
  uint32_t wexcl = block_exclusive_sum<kSegWarps>(lane == 0 ? cnt : 0u, s_tmp, &total);
  wexcl = __shfl_sync(0xffffffffu, wexcl, 0);
  uint32_t pos = tile_off[t] + wexcl;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    if (bal[i] >> lane & 1u) seg_start[pos + __popc(bal[i] & lt)] = base + i * 32 + lane;
    pos += __popc(bal[i]);
  }
}

// Buckets larger than small_max go to the digit passes: each gets an index,
// a contiguous range of chunk ids and of chunk-group ids (so a bucket's
// chunks are consecutive), and zeroed group sums for each of its passes. In
// a batch round the bucket's tensor is recorded, and its chunks and groups
// are listed for every pass that tensor has (tensors differ in passes).
__global__ void k_seg_classify(const int* __restrict__ seg_start, int* __restrict__ counters,
                               int small_max, int chunk, int2* __restrict__ large,
                               int* __restrict__ chunk_base, int* __restrict__ group_base,
                               int* __restrict__ chunk_owner, int* __restrict__ group_owner,
                               uint32_t* __restrict__ group_sum, int npasses, int max_groups,
                               ClassifyBatch cb) {
  const int nseg = counters[kCntNumSeg];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nseg; i += gridDim.x * blockDim.x) {
    const int a = seg_start[i], b = seg_start[i + 1];
    if (b - a <= small_max) continue;
    const int idx = atomicAdd(&counters[kCntNumLarge], 1);
    const int nc = (b - a + chunk - 1) / chunk;
    const int ng = (nc + kGroupChunks - 1) / kGroupChunks;
    const int cbase = atomicAdd(&counters[kCntNumChunks], nc);
    const int gbase = atomicAdd(&counters[kCntNumGroups], ng);
    atomicAdd(&counters[kCntLargeEntries], b - a);
    large[idx] = make_int2(a, b);
    chunk_base[idx] = cbase;
    group_base[idx] = gbase;
    int np = npasses;
    if (cb.n > 0) {
      const int k = upper_bound_int(cb.jbase, 0, cb.n + 1, a) - 1;
      cb.large_tensor[idx] = k;
      np = cb.t[k].npasses;
      for (int p = 0; p < np; ++p) {
        const int lc = atomicAdd(&counters[kCntPassChunks + p], nc);
        for (int j = 0; j < nc; ++j) cb.pass_chunks[(size_t)p * cb.max_chunks + lc + j] = cbase + j;
        const int lg = atomicAdd(&counters[kCntPassGroups + p], ng);
        for (int j = 0; j < ng; ++j) cb.pass_groups[(size_t)p * max_groups + lg + j] = gbase + j;
      }
    }
    for (int j = 0; j < nc; ++j) chunk_owner[cbase + j] = idx;
    for (int j = 0; j < ng; ++j) {
      group_owner[gbase + j] = idx;
      for (int p = 0; p < np; ++p) {
        uint4* row = reinterpret_cast<uint4*>(group_sum + ((size_t)p * max_groups + gbase + j) * kRadix);
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
  (void)status;
  PrefixCols pc;
  pc.n = nprefix;
  for (int m = 0; m < kMaxOrder; ++m) pc.col[m] = m < nprefix ? prefix_cols[m] : nullptr;
  const int ntiles = (nnz + kSegTile - 1) / kSegTile;
  if (ntiles == 0) return cudaSuccess;
  SegBatch sb;
  sb.n = 0;
  sb.jbase = nullptr;
  sb.tile_base = nullptr;
  sb.t = nullptr;
  // seg_lb holds the tile counts (ntiles words) followed by the flag bits
  uint32_t* tile_count = seg_lb;
  uint32_t* bits = seg_lb + ntiles + 1;
  bool aligned = true;  // every prefix row 16-byte aligned: 16-byte loads
  for (int m = 0; m < nprefix; ++m) aligned &= (reinterpret_cast<uintptr_t>(pc.col[m]) & 15) == 0;
  if (aligned)
    k_seg_count_vec<<<ntiles, kSegThreads, 0, stream>>>(pc, nnz, bits, tile_count);
  else
    k_seg_count<<<ntiles, kSegThreads, 0, stream>>>(pc, sb, nnz, bits, tile_count);
  k_seg_scan<<<1, 1024, 0, stream>>>(tile_count, ntiles, nnz, seg_start, counters);
  k_seg_write<<<ntiles, kSegThreads, 0, stream>>>(sb, nnz, bits, tile_count, seg_start);
  return cudaGetLastError();
}

cudaError_t launch_seg_discover_batch(const SegBatch& sb, int ntiles, int nnz, int* seg_start,
                                      uint32_t* seg_lb, int* counters, cudaStream_t stream) {
  if (ntiles == 0) return cudaSuccess;
  PrefixCols pc;
  pc.n = 0;
  for (int m = 0; m < kMaxOrder; ++m) pc.col[m] = nullptr;
  uint32_t* tile_count = seg_lb;
  uint32_t* bits = seg_lb + ntiles + 1;
  k_seg_count<<<ntiles, kSegThreads, 0, stream>>>(pc, sb, nnz, bits, tile_count);
  k_seg_scan<<<1, 1024, 0, stream>>>(tile_count, ntiles, nnz, seg_start, counters);
  k_seg_write<<<ntiles, kSegThreads, 0, stream>>>(sb, nnz, bits, tile_count, seg_start);
  return cudaGetLastError();
}

int seg_tile_entries() { return kSegTile; }

// Words of scratch for bucket discovery over nnz entries in one tensor:
// tile counts, then one bit per entry. (A batch round sizes it by its tile
// count: ntiles + 1 + ntiles * kSegTile / 32 + kSegItems.)
int seg_lookback_words(int nnz) {
  const int ntiles = (nnz + kSegTile - 1) / kSegTile;
  return ntiles + 1 + ntiles * (kSegTile / 32) + kSegItems;
}

cudaError_t launch_seg_classify(const int* seg_start, int* counters, int nnz, int small_max,
                                int chunk, int2* large, int* chunk_base, int* group_base,
                                int* chunk_owner, int* group_owner, uint32_t* group_sum,
                                int npasses, int max_groups, const ClassifyBatch& cb,
                                cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (nnz + 255) / 256;
  if (blocks > sms * 8) blocks = sms * 8;
  if (blocks < 1) blocks = 1;
  k_seg_classify<<<blocks, 256, 0, stream>>>(seg_start, counters, small_max, chunk, large,
                                             chunk_base, group_base, chunk_owner, group_owner,
                                             group_sum, npasses, max_groups, cb);
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
