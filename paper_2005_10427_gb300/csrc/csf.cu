// Compressed sparse fiber (CSF) levels of a tensor sorted under sigma.
//
// Section 2.1 describes CSF as a tree over the sorted coordinates: level l
// (1..r) holds one node per maximal run of entries with equal prefix
// (sigma_0..sigma_{l-1}), its id the coordinate of mode sigma_{l-1}, and each
// node points at its first child on the next level. For entry j let L(j) be
// the first level whose mode differs from entry j-1 (1 for j = 0, r + 1 for
// a duplicate coordinate): j starts a node on every level l >= L(j). Then the
// node index of j on level l is the number of entries before j with L <= l,
// so the levels come out of one count, scan, write sequence over the entries
// (the bucket-discovery pattern, once for all levels):
//   k_csf_count  per tile: entries with L <= l, for every level l;
//   k_csf_scan   one block: per level, the tiles' first node indices, the
//                node counts and the end markers of the pointer arrays;
//   k_csf_write  per tile: for every entry and every level l >= L(j), the
//                node id, the parent's first-child pointer (l > L(j)), and on
//                the last level the leaf's first entry.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

constexpr int kCsfThreads = 256;
constexpr int kCsfWarps = kCsfThreads / 32;
constexpr int kCsfItems = 16;
constexpr int kCsfTile = kCsfThreads * kCsfItems;

struct CsfIn {
  const int32_t* col[kMaxOrder];  // the rows in sigma order: col[l] = row sigma_l
  int order;
  int nnz;
};

// L(j) for the entries of a warp's rounds: lane l of round i holds entry
// base + 32 i + l. prev[] carries the previous round's last entry.
struct LevelScan {
  int32_t prev[kMaxOrder];
};

__device__ __forceinline__ int first_level(const CsfIn& in, int j, int lane, int32_t (&v)[kMaxOrder],
                                           LevelScan& ls, bool first_in_warp) {
  int L = in.order + 1;
  const bool ok = j < in.nnz;
#pragma unroll
  for (int l = 0; l < kMaxOrder; ++l) {  // unrolled to the largest order: registers only
    if (l < in.order) {
      v[l] = ok ? __ldg(in.col[l] + j) : 0;
      int32_t p = __shfl_up_sync(0xffffffffu, v[l], 1);
      const int32_t last = __shfl_sync(0xffffffffu, v[l], 31);
      if (lane == 0) p = ls.prev[l];
      ls.prev[l] = last;
      if (L > in.order && (j == 0 || v[l] != p)) L = l + 1;
    }
  }
  (void)first_in_warp;
  return ok ? L : in.order + 2;  // past the end: no node on any level
}

__device__ __forceinline__ void load_prev(const CsfIn& in, int base, int lane, LevelScan& ls) {
#pragma unroll
  for (int l = 0; l < kMaxOrder; ++l) {
    const int jp = base - 1;
    ls.prev[l] = (l < in.order && lane == 0 && jp >= 0 && jp < in.nnz) ? __ldg(in.col[l] + jp) : 0;
  }
}

__global__ void __launch_bounds__(kCsfThreads)
k_csf_count(CsfIn in, uint32_t* __restrict__ tile_count, int ntiles) {
  __shared__ uint32_t s_cnt[kCsfWarps][kMaxOrder];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, t = blockIdx.x;
  const int base = t * kCsfTile + w * kCsfItems * 32;
  LevelScan ls;
  load_prev(in, base, lane, ls);
  uint32_t cnt[kMaxOrder];
#pragma unroll
  for (int l = 0; l < kMaxOrder; ++l) cnt[l] = 0;
#pragma unroll 4
  for (int i = 0; i < kCsfItems; ++i) {
    int32_t v[kMaxOrder];
    const int L = first_level(in, base + i * 32 + lane, lane, v, ls, i == 0);
#pragma unroll
    for (int l = 0; l < kMaxOrder; ++l)
      if (l < in.order) cnt[l] += __popc(__ballot_sync(0xffffffffu, L <= l + 1));
  }
  if (lane == 0) {
#pragma unroll
    for (int l = 0; l < kMaxOrder; ++l)
      if (l < in.order) s_cnt[w][l] = cnt[l];
  }
  __syncthreads();
  if (threadIdx.x < in.order) {
    uint32_t tot = 0;
    for (int k = 0; k < kCsfWarps; ++k) tot += s_cnt[k][threadIdx.x];
    tile_count[(size_t)threadIdx.x * ntiles + t] = tot;
  }
}

// One block: per level, exclusive scan of the tile counts (in place), the
// node counts, and the pointer arrays' fixed entries: ptr[0] = {0, n_1},
// ptr[l][n_l] = n_{l+1}, ptr[r][n_r] = nnz.
__global__ void __launch_bounds__(1024)
k_csf_scan(uint32_t* __restrict__ tile_count, int ntiles, int order, int nnz, CsfOut out,
           int32_t* __restrict__ nodes) {
  __shared__ uint32_t s_tmp[33];
  __shared__ uint32_t s_carry;
  int parents = 1;  // nodes on the level above (the root); thread 0's copy is used
  for (int l = 0; l < order; ++l) {
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    uint32_t* tc = tile_count + (size_t)l * ntiles;
    for (int b0 = 0; b0 < ntiles; b0 += 1024) {
      const int i = b0 + threadIdx.x;
      const uint32_t v = i < ntiles ? tc[i] : 0u;
      uint32_t total;
      const uint32_t ex = block_exclusive_sum<32>(v, s_tmp, &total);
      const uint32_t carry = s_carry;
      if (i < ntiles) tc[i] = carry + ex;
      __syncthreads();
      if (threadIdx.x == 0) s_carry = carry + total;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int n = (int)s_carry;  // nodes on level l + 1
      nodes[l + 1] = n;
      out.ptr[l][parents] = n;
      parents = n;
      if (l == order - 1) out.ptr[order][n] = nnz;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    nodes[0] = 1;
    out.ptr[0][0] = 0;
  }
}

__global__ void __launch_bounds__(kCsfThreads)
k_csf_write(CsfIn in, const uint32_t* __restrict__ tile_off, int ntiles, CsfOut out) {
  __shared__ uint32_t s_cnt[kCsfWarps][kMaxOrder];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, t = blockIdx.x;
  const int base = t * kCsfTile + w * kCsfItems * 32;
  const uint32_t lt = (1u << lane) - 1u;
  // first sweep: L of every item (4 bits each), the warp's count per level
  LevelScan ls;
  load_prev(in, base, lane, ls);
  uint32_t Lp[kCsfItems / 8] = {0u, 0u};
  uint32_t cnt[kMaxOrder];
#pragma unroll
  for (int l = 0; l < kMaxOrder; ++l) cnt[l] = 0;
#pragma unroll
  for (int i = 0; i < kCsfItems; ++i) {
    int32_t v[kMaxOrder];
    const int L = first_level(in, base + i * 32 + lane, lane, v, ls, i == 0);
    Lp[i / 8] |= (uint32_t)L << ((i % 8) * 4);
#pragma unroll
    for (int l = 0; l < kMaxOrder; ++l)
      if (l < in.order) cnt[l] += __popc(__ballot_sync(0xffffffffu, L <= l + 1));
  }
  if (lane == 0) {
#pragma unroll
    for (int l = 0; l < kMaxOrder; ++l)
      if (l < in.order) s_cnt[w][l] = cnt[l];
  }
  __syncthreads();
  // the warp's first node index per level: the tile's, plus earlier warps'
  uint32_t run[kMaxOrder];
#pragma unroll
  for (int l = 0; l < kMaxOrder; ++l) {
    run[l] = 0;
    if (l < in.order) {
      run[l] = tile_off[(size_t)l * ntiles + t];
      for (int k = 0; k < w; ++k) run[l] += s_cnt[k][l];
    }
  }
  // second sweep: node indices and the writes
#pragma unroll
  for (int i = 0; i < kCsfItems; ++i) {
    const int j = base + i * 32 + lane;
    const int L = (int)((Lp[i / 8] >> ((i % 8) * 4)) & 15u);
    uint32_t pprev = 0;
#pragma unroll
    for (int l = 0; l < kMaxOrder; ++l) {
      if (l >= in.order) break;
      const bool starts = L <= l + 1;  // j starts a node on level l + 1
      const uint32_t bal = __ballot_sync(0xffffffffu, starts);
      const uint32_t p = run[l] + __popc(bal & lt);
      run[l] += __popc(bal);
      if (starts) {
        out.ids[l][p] = __ldg(in.col[l] + j);
        if (L <= l) out.ptr[l][pprev] = (int32_t)p;  // j also started the parent
        if (l == in.order - 1) out.ptr[in.order][p] = j;
      }
      pprev = p;
    }
  }
}

}  // namespace

cudaError_t launch_csf(const int32_t* const* rows_in_sigma_order, int order, int nnz,
                       const CsfOut& out, int32_t* nodes, uint32_t* tile_count,
                       cudaStream_t stream) {
  CsfIn in;
  in.order = order;
  in.nnz = nnz;
  for (int l = 0; l < kMaxOrder; ++l) in.col[l] = l < order ? rows_in_sigma_order[l] : nullptr;
  const int ntiles = (nnz + kCsfTile - 1) / kCsfTile;
  if (ntiles > 0) k_csf_count<<<ntiles, kCsfThreads, 0, stream>>>(in, tile_count, ntiles);
  k_csf_scan<<<1, 1024, 0, stream>>>(tile_count, ntiles, order, nnz, out, nodes);
  if (ntiles > 0) k_csf_write<<<ntiles, kCsfThreads, 0, stream>>>(in, tile_count, ntiles, out);
  return cudaGetLastError();
}

size_t csf_workspace_bytes(int order, int nnz) {
  const size_t ntiles = ((size_t)nnz + kCsfTile - 1) / kCsfTile;
  return sizeof(uint32_t) * ((size_t)order * ntiles + 1);
}

}  // namespace qsd

extern "C" {

qsd_status qsd_csf_workspace_bytes(int order, int64_t nnz, size_t* bytes) {
  if (!bytes || order < 1 || nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  if (order > QSD_MAX_ORDER) return QSD_ERR_UNSUPPORTED;
  if (nnz > (int64_t(1) << 30) - 1) return QSD_ERR_UNSUPPORTED;
  *bytes = (qsd::csf_workspace_bytes(order, (int)nnz) + 255) & ~size_t(255);
  return QSD_OK;
}

qsd_status qsd_csf_build(const int32_t* coords, int64_t stride, int64_t nnz, int order,
                         const int* sigma, const qsd_csf* out, int32_t* nodes, void* workspace,
                         size_t workspace_bytes, void* stream) {
  if (!out || !nodes || !sigma || order < 1 || nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  if (order > QSD_MAX_ORDER || nnz > (int64_t(1) << 30) - 1) return QSD_ERR_UNSUPPORTED;
  bool seen[QSD_MAX_ORDER] = {false};
  for (int i = 0; i < order; ++i) {
    if (sigma[i] < 0 || sigma[i] >= order || seen[sigma[i]]) return QSD_ERR_INVALID_ARGUMENT;
    seen[sigma[i]] = true;
  }
  for (int l = 0; l <= order; ++l) {
    if (!out->ptr[l]) return QSD_ERR_INVALID_ARGUMENT;
    if (l < order && nnz > 0 && !out->ids[l]) return QSD_ERR_INVALID_ARGUMENT;
  }
  if (nnz > 0 && (!coords || stride < nnz)) return QSD_ERR_INVALID_ARGUMENT;
  size_t need = 0;
  qsd_csf_workspace_bytes(order, nnz, &need);
  if (!workspace) return QSD_ERR_INVALID_ARGUMENT;
  if (workspace_bytes < need) return QSD_ERR_WORKSPACE_TOO_SMALL;
  const int32_t* rows[QSD_MAX_ORDER];
  for (int l = 0; l < order; ++l) rows[l] = nnz > 0 ? coords + (int64_t)sigma[l] * stride : nullptr;
  qsd::CsfOut o;
  for (int l = 0; l < qsd::kMaxOrder; ++l) o.ids[l] = l < order ? out->ids[l] : nullptr;
  for (int l = 0; l <= qsd::kMaxOrder; ++l) o.ptr[l] = l <= order ? out->ptr[l] : nullptr;
  if (qsd::launch_csf(rows, order, (int)nnz, o, nodes, static_cast<uint32_t*>(workspace),
                      (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return QSD_ERR_CUDA;
  }
  return QSD_OK;
}

}  // extern "C"

