// Block-local bucket sort in shared memory.
//
// Section 3.2 parallelises the bucketed sort by bucket boundaries: entries
// never leave their bucket, so each processor sorts the buckets that begin
// in its region. Here each thread block owns a window of `CAP` entries and
// sorts the small buckets (at most CAP entries each) that begin in it, in
// batches of consecutive buckets that fit shared memory together. A batch is
// stably sorted by (bucket, key): least-significant-digit-first radix passes
// over the group's key digits, then over the bucket index -- the order
// Algorithm 2 uses (sort on the mode, then stably re-bucket) -- each pass a
// stable ranking in shared memory. Only a permutation of batch positions is
// sorted; each coordinate row and the values then move once: the row's batch
// range is staged in shared memory and written back permuted with coalesced
// stores, so the kernel may write its output over its input. In a batch
// round the buckets of several tensors share the index space; a batch of
// buckets never crosses from one tensor into the next, and each takes its
// tensor's rows and digits.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

constexpr int kLsThreads = 512;
constexpr int kLsWarps = kLsThreads / 32;

template <int VB>
struct LsVal {
  using T = uint32_t;
};
template <>
struct LsVal<8> {
  using T = unsigned long long;
};

template <int CAP>
struct LsShared {
  uint16_t warp_hist[kLsWarps * kRadix];
  uint32_t bin_start[kRadix];
  uint32_t bin_count[kRadix];
  uint32_t tmp[kLsWarps + 1];
  uint16_t perm[2][CAP];
  uint16_t segid[CAP];
  int first, last, batch_end;
  Cols c;                  // the current batch's tensor: rows
  const PassDesc* passes;  // and key passes
  int npasses;
};

// First index i in [lo, hi) with a[i] > x (or hi).
__device__ __forceinline__ int upper_bound_i(const int* a, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}
// First index i in [lo, hi) with a[i] >= x (or hi).
__device__ __forceinline__ int lower_bound_i(const int* a, int lo, int hi, int x) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int CAP, int VB>
__global__ void __launch_bounds__(kLsThreads)
k_local_sort(Cols c1, const __grid_constant__ PassList pl, const int* __restrict__ seg_start,
             const int* __restrict__ counters, int single, int nnz, LsBatch lb) {
  constexpr int ITEMS = CAP / kLsThreads;
  extern __shared__ __align__(16) uint8_t smem[];
  LsShared<CAP>& S = *reinterpret_cast<LsShared<CAP>*>(smem);
  uint8_t* stage = smem + ((sizeof(LsShared<CAP>) + 15) & ~size_t(15));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int win0 = blockIdx.x * CAP;
  if (win0 >= nnz) return;
  const int win1 = min(win0 + CAP, nnz);
  const int nseg = single ? 1 : counters[kCntNumSeg];

  if (threadIdx.x == 0) {
    S.c = c1;
    S.passes = pl.pass;
    S.npasses = pl.npasses;
    if (single) {
      S.first = 0;
      S.last = 1;
    } else {
      S.first = lower_bound_i(seg_start, 0, nseg, win0);
      S.last = lower_bound_i(seg_start, S.first, nseg, win1);
    }
  }
  __syncthreads();
  const int last = S.last;
  int s = S.first;
  while (s < last) {
    if (threadIdx.x == 0) {
      const int a = single ? 0 : seg_start[s];
      const int b = single ? nnz : seg_start[s + 1];
      int e;
      int lim = last;
      if (lb.n > 0) {  // the bucket's tensor; the batch ends where the next one starts
        const int k = upper_bound_i(lb.jbase, 0, lb.n + 1, a) - 1;
        S.c = lb.t[k].c;
        S.passes = lb.t[k].pass;
        S.npasses = lb.t[k].npasses;
        const int tb = lower_bound_i(seg_start, s + 1, nseg + 1, lb.jbase[k + 1]);
        if (tb < lim) lim = tb;
      }
      if (b - a > CAP) {
        e = -1;  // large bucket: sorted by the digit passes
      } else if (single) {
        e = 1;
      } else {
        e = upper_bound_i(seg_start, s + 1, nseg + 1, a + CAP) - 1;
        if (e > lim) e = lim;
      }
      S.batch_end = e;
    }
    __syncthreads();
    const int e = S.batch_end;
    __syncthreads();
    if (e < 0) {
      ++s;
      continue;
    }
    const Cols& c = S.c;
    const int key_passes = S.npasses;
    const PassDesc* const passes = S.passes;
    const int A = single ? 0 : seg_start[s];
    const int n = (single ? nnz : seg_start[e]) - A;
    const int nsb = e - s;

    // Bucket index of every batch position (marks at bucket starts, scanned).
    if (nsb > 1) {
      for (int i = threadIdx.x; i < CAP; i += kLsThreads) S.segid[i] = 0;
      __syncthreads();
      for (int k = s + 1 + threadIdx.x; k < e; k += kLsThreads) S.segid[seg_start[k] - A] = 1;
      __syncthreads();
      // blocked inclusive scan: thread owns ITEMS consecutive positions
      uint32_t loc[ITEMS], sum = 0;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        loc[i] = S.segid[threadIdx.x * ITEMS + i];
        sum += loc[i];
      }
      uint32_t total;
      uint32_t run = block_exclusive_sum<kLsWarps>(sum, S.tmp, &total);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        run += loc[i];
        S.segid[threadIdx.x * ITEMS + i] = (uint16_t)run;
      }
    }
    for (int i = threadIdx.x; i < CAP; i += kLsThreads) S.perm[0][i] = (uint16_t)i;
    __syncthreads();

    int cur = 0;
    int seg_bits = 0;
    while ((1 << seg_bits) < nsb) ++seg_bits;
    const int seg_passes = (seg_bits + kRadixBits - 1) / kRadixBits;
    for (int p = 0; p < key_passes + seg_passes; ++p) {
      uint32_t dig[ITEMS], rank[ITEMS], el[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int pos = w * ITEMS * 32 + i * 32 + lane;
        el[i] = S.perm[cur][pos];
        uint32_t d = kRadix - 1;
        if (pos < n) {
          if (p < key_passes) {
            const PassDesc& pd = passes[p];
            d = 0;
            for (int k = 0; k < pd.nfields; ++k) {
              const DigitField f = pd.f[k];
              d |= field_bits((uint32_t)__ldg(c.in + (int64_t)f.mode * c.in_stride + A + el[i]), f);
            }
          } else {
            d = ((uint32_t)S.segid[el[i]] >> ((p - key_passes) * kRadixBits)) & (kRadix - 1);
          }
        }
        dig[i] = d;
      }
      block_rank<kLsWarps, ITEMS>(dig, rank, S.warp_hist, S.bin_start, S.bin_count, S.tmp);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) S.perm[cur ^ 1][rank[i]] = (uint16_t)el[i];
      __syncthreads();
      cur ^= 1;
    }

    // Move the rows: stage the batch range, write it back permuted.
    uint32_t* st32 = reinterpret_cast<uint32_t*>(stage);
    for (int m = 0; m < c.order; ++m) {
      const int32_t* src = c.in + (int64_t)m * c.in_stride + A;
      int32_t* dst = c.out + (int64_t)m * c.out_stride + A;
      for (int i = threadIdx.x; i < n; i += kLsThreads) st32[i] = (uint32_t)src[i];
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += kLsThreads) dst[i] = (int32_t)st32[S.perm[cur][i]];
      __syncthreads();
    }
    if constexpr (VB != 0) {
      using T = typename LsVal<VB>::T;
      const T* src = reinterpret_cast<const T*>(c.vin) + A;
      T* dst = reinterpret_cast<T*>(c.vout) + A;
      T* stv = reinterpret_cast<T*>(stage);
      for (int i = threadIdx.x; i < n; i += kLsThreads) stv[i] = src[i];
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += kLsThreads) dst[i] = stv[S.perm[cur][i]];
      __syncthreads();
    }
    s = e;
  }
}

template <int CAP, int VB>
cudaError_t launch_ls(const Cols& c, const PassList& pl, const int* seg_start,
                      const int* counters, int single, int nnz, const LsBatch& lb,
                      cudaStream_t stream) {
  const size_t smem = ((sizeof(LsShared<CAP>) + 15) & ~size_t(15)) +
                      (size_t)CAP * (VB == 8 ? 8 : 4);
  cudaError_t e = cudaFuncSetAttribute(k_local_sort<CAP, VB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = single ? 1 : (nnz + CAP - 1) / CAP;
  if (grid < 1) return cudaSuccess;
  k_local_sort<CAP, VB><<<grid, kLsThreads, smem, stream>>>(c, pl, seg_start, counters,
                                                            single, nnz, lb);
  return cudaGetLastError();
}

template <int CAP>
cudaError_t launch_ls_cap(const Cols& c, const PassList& pl, const int* seg_start,
                          const int* counters, int single, int nnz, const LsBatch& lb,
                          cudaStream_t stream) {
  switch (c.vbytes) {
    case 0: return launch_ls<CAP, 0>(c, pl, seg_start, counters, single, nnz, lb, stream);
    case 4: return launch_ls<CAP, 4>(c, pl, seg_start, counters, single, nnz, lb, stream);
    case 8: return launch_ls<CAP, 8>(c, pl, seg_start, counters, single, nnz, lb, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_local_sort(const Cols& c, const PassList& pl, const int* seg_start,
                              const int* counters, int single, int nnz, int capacity,
                              unsigned* status, const LsBatch& lb, cudaStream_t stream) {
  (void)status;
  switch (capacity) {
    case 1024: return launch_ls_cap<1024>(c, pl, seg_start, counters, single, nnz, lb, stream);
    case 2048: return launch_ls_cap<2048>(c, pl, seg_start, counters, single, nnz, lb, stream);
    case 4096: return launch_ls_cap<4096>(c, pl, seg_start, counters, single, nnz, lb, stream);
    case 8192: return launch_ls_cap<8192>(c, pl, seg_start, counters, single, nnz, lb, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qsd
