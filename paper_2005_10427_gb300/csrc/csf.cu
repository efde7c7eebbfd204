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
constexpr int kCsfItems = 16;  // consecutive entries per thread
constexpr int kCsfTile = kCsfThreads * kCsfItems;

struct CsfIn {
  const int32_t* col[kMaxOrder];  // the rows in sigma order: col[l] = row sigma_l
  int order;
  int nnz;
  int vec;       // every row 16-byte aligned: 16-byte loads
  uint8_t* lev;  // L of every entry from the transposition (0 = unknown), or null
};

// The 16 values of row l at entries j0 .. j0 + 15 (j0 a multiple of 16), and
// the value of entry j0 - 1. Entries past the end read as 0.
__device__ __forceinline__ void load_run(const CsfIn& in, int l, int j0, uint32_t (&v)[kCsfItems],
                                         uint32_t& before) {
  const int32_t* row = in.col[l];
  before = j0 > 0 && j0 - 1 < in.nnz ? (uint32_t)__ldg(row + j0 - 1) : 0u;
  if (in.vec && j0 + kCsfItems <= in.nnz) {
    const uint4* r4 = reinterpret_cast<const uint4*>(row + j0);
#pragma unroll
    for (int q = 0; q < kCsfItems / 4; ++q) {
      const uint4 x = __ldg(r4 + q);
      v[4 * q] = x.x;
      v[4 * q + 1] = x.y;
      v[4 * q + 2] = x.z;
      v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kCsfItems; ++k)
      v[k] = j0 + k < in.nnz ? (uint32_t)__ldg(row + j0 + k) : 0u;
  }
}

// L(j) of one entry from the rows (j > 0).
__device__ __forceinline__ uint32_t level_at(const CsfIn& in, int j) {
  for (int l = 0; l < in.order; ++l)
    if (__ldg(in.col[l] + j) != __ldg(in.col[l] + j - 1)) return (uint32_t)l + 1;
  return (uint32_t)in.order + 1;
}

// L(j) of the thread's 16 entries (4 bits each): the first level (1-based)
// whose mode differs from the entry before (1 at entry 0, order + 1 for a
// duplicate, order + 2 past the end). Reads the rows level by level, or,
// when the transposition left the levels (in.lev), reads those and works
// out only the unknown ones from the rows (writing them back when
// `fix` is set).
__device__ __forceinline__ void first_levels(const CsfIn& in, int j0, uint32_t (&L)[2],
                                             bool fix = false) {
  uint32_t lv[kCsfItems];
  if (in.lev) {
    uint8_t b[kCsfItems];
    const bool full = j0 + kCsfItems <= in.nnz;
    if (full) {
      const uint4 x = *reinterpret_cast<const uint4*>(in.lev + j0);
      const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int k = 0; k < kCsfItems; ++k) b[k] = (uint8_t)(w[k / 4] >> (8 * (k % 4)));
    } else {
#pragma unroll
      for (int k = 0; k < kCsfItems; ++k) b[k] = j0 + k < in.nnz ? in.lev[j0 + k] : 0;
    }
    bool changed = false;
#pragma unroll
    for (int k = 0; k < kCsfItems; ++k) {
      const int j = j0 + k;
      if (j >= in.nnz) {
        lv[k] = in.order + 2;
      } else if (j == 0) {
        lv[k] = 1;
      } else if (b[k] == 0) {
        lv[k] = level_at(in, j);
        b[k] = (uint8_t)lv[k];
        changed = true;
      } else {
        lv[k] = b[k];
      }
    }
    if (fix && changed) {
#pragma unroll
      for (int k = 0; k < kCsfItems; ++k)
        if (j0 + k < in.nnz) in.lev[j0 + k] = b[k];
    }
    L[0] = L[1] = 0;
#pragma unroll
    for (int k = 0; k < kCsfItems; ++k) L[k / 8] |= lv[k] << ((k % 8) * 4);
    return;
  }
#pragma unroll
  for (int k = 0; k < kCsfItems; ++k)
    lv[k] = j0 + k >= in.nnz ? in.order + 2 : (j0 + k == 0 ? 1 : in.order + 1);
#pragma unroll 1
  for (int l = 0; l < in.order; ++l) {
    uint32_t v[kCsfItems], before;
    load_run(in, l, j0, v, before);
#pragma unroll
    for (int k = 0; k < kCsfItems; ++k) {
      const uint32_t prev = k ? v[k - 1] : before;
      if (lv[k] == (uint32_t)in.order + 1 && v[k] != prev) lv[k] = l + 1;
    }
  }
  L[0] = L[1] = 0;
#pragma unroll
  for (int k = 0; k < kCsfItems; ++k) L[k / 8] |= lv[k] << ((k % 8) * 4);
}

__device__ __forceinline__ uint32_t level_of(const uint32_t (&L)[2], int k) {
  return (L[k / 8] >> ((k % 8) * 4)) & 15u;
}

__global__ void __launch_bounds__(kCsfThreads)
k_csf_count(const __grid_constant__ CsfIn in, uint32_t* __restrict__ tile_count, int ntiles) {
  __shared__ uint32_t s_cnt[kCsfWarps][kMaxOrder];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, t = blockIdx.x;
  const int j0 = t * kCsfTile + threadIdx.x * kCsfItems;
  uint32_t L[2];
  first_levels(in, j0, L, true);
#pragma unroll
  for (int l = 0; l < kMaxOrder; ++l) {
    if (l >= in.order) break;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCsfItems; ++k) c += level_of(L, k) <= (uint32_t)l + 1 ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) s_cnt[w][l] = c;
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
k_csf_write(const __grid_constant__ CsfIn in, const uint32_t* __restrict__ tile_off, int ntiles,
            const __grid_constant__ CsfOut out) {
  __shared__ uint32_t s_tmp[kCsfWarps + 1];
  const int t = blockIdx.x;
  const int j0 = t * kCsfTile + threadIdx.x * kCsfItems;
  uint32_t L[2];
  first_levels(in, j0, L);
  // node index of each entry on the level above (valid where the entry starts
  // a node there)
  uint32_t above[kCsfItems];
#pragma unroll
  for (int k = 0; k < kCsfItems; ++k) above[k] = 0;
#pragma unroll 1
  for (int l = 0; l < in.order; ++l) {
    // the thread's first node index on level l + 1
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCsfItems; ++k) c += level_of(L, k) <= (uint32_t)l + 1 ? 1u : 0u;
    uint32_t total;
    uint32_t p = tile_off[(size_t)l * ntiles + t] + block_exclusive_sum<kCsfWarps>(c, s_tmp, &total);
    if (c != 0) {  // else none of the thread's entries starts a node here: no ids to read
      uint32_t v[kCsfItems], before;
      load_run(in, l, j0, v, before);
#pragma unroll
      for (int k = 0; k < kCsfItems; ++k) {
        const uint32_t lk = level_of(L, k);
        if (lk <= (uint32_t)l + 1) {  // entry j0 + k starts a node on level l + 1
          out.ids[l][p] = (int32_t)v[k];
          if (lk <= (uint32_t)l) out.ptr[l][above[k]] = (int32_t)p;  // and its parent
          if (l == in.order - 1) out.ptr[in.order][p] = j0 + k;
          above[k] = p;
          ++p;
        }
      }
    }
    __syncthreads();  // s_tmp is reused by the next level's scan (every thread)
  }
}

}  // namespace

cudaError_t launch_csf(const int32_t* const* rows_in_sigma_order, int order, int nnz,
                       const CsfOut& out, int32_t* nodes, uint32_t* tile_count,
                       cudaStream_t stream, uint8_t* lev) {
  CsfIn in;
  in.order = order;
  in.nnz = nnz;
  in.vec = 1;
  in.lev = lev;
  for (int l = 0; l < kMaxOrder; ++l) {
    in.col[l] = l < order ? rows_in_sigma_order[l] : nullptr;
    if (l < order && (reinterpret_cast<uintptr_t>(in.col[l]) & 15)) in.vec = 0;
  }
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

