// Global stable radix passes for buckets too large for one thread block
// (and for the whole tensor when a group has no prefix).
//
// A pass is the GPU form of one histogram partial sort (Algorithm 1: count,
// prefix-sum, stable move) over a radix digit of the packed key instead of a
// whole mode, so the count array has 2^8 bins rather than n_k (the cost the
// paper's discussion attributes to large modes). Three kernels:
//   k_digit_hist   one read of the key coordinates; per-bucket histograms of
//                  every pass's digit at once (counting for all passes up
//                  front, as the paper's conclusion suggests fusing the first
//                  loop of the next sort into the current one);
//   k_digit_scan   per (bucket, pass): exclusive prefix sum over digits plus
//                  the bucket's start = the first output slot of each digit;
//   k_onesweep     per tile: stable in-tile ranking by digit, decoupled
//                  look-back over the preceding tiles of the same bucket for
//                  each digit's running offset, then a move of every
//                  coordinate row and the values through shared memory so
//                  that each digit's run is written contiguously.
// Buckets never exchange entries (Section 3.2: coordinates do not leave
// their bucket), so each bucket's tiles chain only among themselves.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

constexpr int kOsThreads = 512;
constexpr int kOsWarps = kOsThreads / 32;
constexpr int kOsItems = 16;
constexpr int kOsTile = kOsThreads * kOsItems;

constexpr int kHistThreads = 512;

struct TileInfo {
  int seg;       // large-bucket index (0 when single)
  int start;     // first entry of the tile
  int end;       // one past the last entry
  int first;     // tile id of the bucket's first tile
};

__device__ __forceinline__ int num_tiles(const LargeSegs& ls) {
  return ls.single ? ls.single_tiles : ls.counters[kCntNumTiles];
}

__device__ __forceinline__ TileInfo tile_info(const LargeSegs& ls, int t) {
  TileInfo ti;
  if (ls.single) {
    ti.seg = 0;
    ti.start = t * kOsTile;
    ti.end = min(ti.start + kOsTile, ls.nnz);
    ti.first = 0;
  } else {
    const int s = ls.tile_owner[t];
    const int2 se = ls.seg[s];
    const int tb = ls.tile_base[s];
    ti.seg = s;
    ti.start = se.x + (t - tb) * kOsTile;
    ti.end = min(ti.start + kOsTile, se.y);
    ti.first = tb;
  }
  return ti;
}

__device__ __forceinline__ uint32_t entry_digit(const Cols& c, const PassDesc& pd, int j) {
  uint32_t d = 0;
  for (int k = 0; k < pd.nfields; ++k) {
    const DigitField f = pd.f[k];
    d |= field_bits((uint32_t)__ldg(c.in + (int64_t)f.mode * c.in_stride + j), f);
  }
  return d;
}

__global__ void __launch_bounds__(kHistThreads)
k_digit_hist(Cols c, LargeSegs ls, PassList pl, uint32_t* __restrict__ hist,
             uint32_t* __restrict__ lb0) {
  extern __shared__ uint32_t s_hist[];  // [npasses][kRadix]
  const int P = pl.npasses;
  const int ntiles = num_tiles(ls);
  const int per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * per;
  const int t1 = min(t0 + per, ntiles);
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < P * kRadix; i += kHistThreads) s_hist[i] = 0;
  __syncthreads();
  int cur = -1;
  auto flush = [&](int s) {
    __syncthreads();
    uint32_t* row = hist + (size_t)s * P * kRadix;
    for (int i = threadIdx.x; i < P * kRadix; i += kHistThreads) {
      const uint32_t v = s_hist[i];
      if (v) {
        atomicAdd(row + i, v);
        s_hist[i] = 0;
      }
    }
    __syncthreads();
  };
  for (int t = t0; t < t1; ++t) {
    const TileInfo ti = tile_info(ls, t);
    if (ti.seg != cur) {
      if (cur >= 0) flush(cur);
      cur = ti.seg;
    }
    for (int d = threadIdx.x; d < kRadix; d += kHistThreads)
      lb0[(size_t)t * kRadix + d] = 0;
    for (int base = ti.start; base < ti.end; base += kHistThreads) {
      const int j = base + threadIdx.x;
      const bool valid = j < ti.end;
      for (int p = 0; p < P; ++p) {
        const uint32_t d = valid ? entry_digit(c, pl.pass[p], j) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1)
          atomicAdd(&s_hist[p * kRadix + d], (uint32_t)__popc(peers));
      }
    }
  }
  if (cur >= 0) flush(cur);
}

// One warp per (bucket, pass) row: exclusive prefix over digits + start.
__global__ void k_digit_scan(LargeSegs ls, int P, uint32_t* __restrict__ hist) {
  const int nlarge = ls.single ? 1 : ls.counters[kCntNumLarge];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  constexpr int PER = kRadix / 32;
  for (int row = gw; row < nlarge * P; row += nw) {
    const int s = row / P;
    const uint32_t start = ls.single ? 0u : (uint32_t)ls.seg[s].x;
    uint32_t* h = hist + (size_t)row * kRadix;
    uint32_t v[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      v[j] = h[lane * PER + j];
      sum += v[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t run = start + incl - sum;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      h[lane * PER + j] = run;
      run += v[j];
    }
  }
}

template <int VB>
struct ValType {
  using T = uint32_t;
};
template <>
struct ValType<8> {
  using T = unsigned long long;
};

struct OsShared {
  uint32_t warp_hist[kOsWarps * kRadix];
  uint32_t bin_start[kRadix];
  uint32_t bin_count[kRadix];
  uint32_t gbase[kRadix];
  uint8_t dig[kOsTile];
  int tile;
};

template <int VB>
__global__ void __launch_bounds__(kOsThreads, 2)
k_onesweep(Cols c, LargeSegs ls, PassDesc pd, int pass_index, int npasses,
           const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ lb,
           uint32_t* __restrict__ lb_next, int* __restrict__ tile_counter,
           unsigned* status) {
  extern __shared__ __align__(16) uint8_t smem[];
  OsShared& S = *reinterpret_cast<OsShared*>(smem);
  uint8_t* stage = smem + ((sizeof(OsShared) + 15) & ~size_t(15));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ntiles = num_tiles(ls);
  while (true) {
    if (threadIdx.x == 0) S.tile = atomicAdd(tile_counter, 1);
    __syncthreads();
    const int t = S.tile;
    if (t >= ntiles) break;
    const TileInfo ti = tile_info(ls, t);
    const int n_valid = ti.end - ti.start;
    const int wbase = ti.start + w * kOsItems * 32 + lane;

    uint32_t dig[kOsItems], rank[kOsItems];
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) {
      const int j = wbase + i * 32;
      dig[i] = j < ti.end ? entry_digit(c, pd, j) : (uint32_t)(kRadix - 1);
    }
    block_rank<kOsWarps, kOsItems>(dig, rank, S.warp_hist, S.bin_start, S.bin_count);

    if (threadIdx.x < kRadix) {
      const int d = threadIdx.x;
      uint32_t cnt = S.bin_count[d];
      if (d == kRadix - 1) cnt -= (uint32_t)(kOsTile - n_valid);  // padding sorts last
      uint32_t* my = lb + (size_t)t * kRadix + d;
      uint32_t excl = 0;
      if (t == ti.first) {
        st_relaxed(my, kLbInclusive | cnt);
      } else {
        st_relaxed(my, kLbAggregate | cnt);
        for (int p = t - 1; p >= ti.first; --p) {
          const uint32_t v = wait_flag(lb + (size_t)p * kRadix + d, status);
          excl += v & kLbCountMask;
          if ((v & kLbStateMask) == kLbInclusive) break;
        }
        st_relaxed(my, kLbInclusive | (excl + cnt));
      }
      const uint32_t gpos =
          digit_base[((size_t)ti.seg * npasses + pass_index) * kRadix + d] + excl;
      S.gbase[d] = gpos - S.bin_start[d];
      if (lb_next) lb_next[(size_t)t * kRadix + d] = 0;
    }
#pragma unroll
    for (int i = 0; i < kOsItems; ++i) S.dig[rank[i]] = (uint8_t)dig[i];
    __syncthreads();

    // Move every coordinate row, then the values, through shared memory.
    uint32_t* st32 = reinterpret_cast<uint32_t*>(stage);
    for (int m = 0; m < c.order; ++m) {
      const int32_t* src = c.in + (int64_t)m * c.in_stride;
      int32_t* dst = c.out + (int64_t)m * c.out_stride;
      uint32_t v[kOsItems];
#pragma unroll
      for (int i = 0; i < kOsItems; ++i) {
        const int j = wbase + i * 32;
        v[i] = j < ti.end ? (uint32_t)__ldcs(src + j) : 0u;
      }
#pragma unroll
      for (int i = 0; i < kOsItems; ++i) st32[rank[i]] = v[i];
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kOsItems; ++k) {
        const int pos = k * kOsThreads + threadIdx.x;
        if (pos < n_valid) dst[S.gbase[S.dig[pos]] + pos] = (int32_t)st32[pos];
      }
      __syncthreads();
    }
    if constexpr (VB != 0) {
      using T = typename ValType<VB>::T;
      const T* src = reinterpret_cast<const T*>(c.vin);
      T* dst = reinterpret_cast<T*>(c.vout);
      T* stv = reinterpret_cast<T*>(stage);
      T v[kOsItems];
#pragma unroll
      for (int i = 0; i < kOsItems; ++i) {
        const int j = wbase + i * 32;
        v[i] = j < ti.end ? __ldcs(src + j) : T(0);
      }
#pragma unroll
      for (int i = 0; i < kOsItems; ++i) stv[rank[i]] = v[i];
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kOsItems; ++k) {
        const int pos = k * kOsThreads + threadIdx.x;
        if (pos < n_valid) dst[S.gbase[S.dig[pos]] + pos] = stv[pos];
      }
      __syncthreads();
    }
  }
}

template <int VB>
size_t onesweep_smem() {
  return ((sizeof(OsShared) + 15) & ~size_t(15)) + (size_t)kOsTile * (VB == 8 ? 8 : 4);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

template <int VB>
cudaError_t launch_onesweep_vb(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                               int pass_index, int npasses, const uint32_t* digit_base,
                               uint32_t* lb, uint32_t* lb_next, int* tile_counter,
                               int max_tiles, unsigned* status, cudaStream_t stream) {
  const size_t smem = onesweep_smem<VB>();
  cudaError_t e = cudaFuncSetAttribute(k_onesweep<VB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<VB>, kOsThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * sm_count();
  if (grid > max_tiles) grid = max_tiles;
  if (grid < 1) grid = 1;
  k_onesweep<VB><<<grid, kOsThreads, smem, stream>>>(c, ls, pd, pass_index, npasses,
                                                     digit_base, lb, lb_next,
                                                     tile_counter, status);
  return cudaGetLastError();
}

}  // namespace

int onesweep_tile() { return kOsTile; }

cudaError_t launch_digit_hist(const Cols& c, const LargeSegs& ls, const PassList& pl,
                              uint32_t* hist, uint32_t* lb0, int max_tiles,
                              unsigned* status, cudaStream_t stream) {
  (void)status;
  const size_t smem = (size_t)pl.npasses * kRadix * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(k_digit_hist,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int grid = sm_count() * 2;
  if (grid > max_tiles) grid = max_tiles;
  if (grid < 1) grid = 1;
  k_digit_hist<<<grid, kHistThreads, smem, stream>>>(c, ls, pl, hist, lb0);
  return cudaGetLastError();
}

cudaError_t launch_digit_scan(const LargeSegs& ls, int npasses, uint32_t* hist,
                              int max_large, cudaStream_t stream) {
  int rows = max_large * npasses;
  int blocks = (rows * 32 + 255) / 256;
  const int cap = sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_digit_scan<<<blocks, 256, 0, stream>>>(ls, npasses, hist);
  return cudaGetLastError();
}

cudaError_t launch_onesweep_pass(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                                 int pass_index, int npasses, const uint32_t* digit_base,
                                 uint32_t* lb, uint32_t* lb_next, int* tile_counter,
                                 int max_tiles, unsigned* status, cudaStream_t stream) {
  switch (c.vbytes) {
    case 0:
      return launch_onesweep_vb<0>(c, ls, pd, pass_index, npasses, digit_base, lb,
                                   lb_next, tile_counter, max_tiles, status, stream);
    case 4:
      return launch_onesweep_vb<4>(c, ls, pd, pass_index, npasses, digit_base, lb,
                                   lb_next, tile_counter, max_tiles, status, stream);
    case 8:
      return launch_onesweep_vb<8>(c, ls, pd, pass_index, npasses, digit_base, lb,
                                   lb_next, tile_counter, max_tiles, status, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qsd
