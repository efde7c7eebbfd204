// Block-local bucket sort in shared memory.
//
// Section 3.2 parallelises the bucketed sort by bucket boundaries: entries
// never leave their bucket, so each processor sorts the buckets that begin
// in its region. Here each thread block owns a window of a few times `CAP`
// entries and sorts the small buckets (at most CAP entries each) that begin
// in it, in batches of consecutive buckets that fit shared memory together
// (a batch of tiny buckets is ranked by counting instead of the passes). A batch's
// rows are staged in shared memory by bulk asynchronous copies (unaligned
// edges by plain loads) while the block numbers the batch's buckets; the
// batch is then stably sorted by (bucket, key): least-significant-digit-first
// radix passes over the group's key digits, then over the bucket index -- the
// order Algorithm 2 uses (sort on the mode, then stably re-bucket) -- each
// pass a stable ranking in shared memory of a permutation of batch
// positions, reading the digits from the staged rows. Every row is then
// written back through the permutation with coalesced stores, so the kernel
// may write its output over its input. In a batch round the buckets of
// several tensors share the index space; a batch of buckets never crosses
// from one tensor into the next, and each takes its tensor's rows and digits.
#include <cuda_runtime.h>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

// Threads of a block: 512 for capacities of 4096 entries and more, 256
// below, where the smaller per-warp counter space lets three blocks share an
// SM (the sort is barrier-bound, and more blocks hide each other's waits).
template <int CAP>
constexpr int ls_threads() {
  return CAP >= 4096 ? 512 : 256;
}
constexpr int kTiny = 64;  // largest bucket of the rank-by-counting path
constexpr int kLsSpan = 4;  // windows of CAP entries per block

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
  static constexpr int kWarps = ls_threads<CAP>() / 32;
  uint32_t warp_hist[kWarps * kRadix];
  uint32_t bin_start[kRadix];
  uint32_t bin_count[kRadix];
  uint32_t tmp[kWarps + 1];
  uint16_t perm[2][CAP];
  uint16_t segid[CAP];
  int first, last, batch_end;
  Cols c;                  // the current batch's tensor: rows
  const PassDesc* passes;  // and key passes (pass[])
  int npasses;
  PassDesc pass[kMaxPasses];
  uint64_t ld;             // the batch's staged rows have landed
  int row_off[kMaxOrder + 1];   // byte offset of element 0 in each staged row
  int row_head[kMaxOrder + 1];  // elements [0, head) and [tail, n) come by plain loads
  int row_tail[kMaxOrder + 1];
};

template <int CAP>
size_t ls_smem(int order, int vbytes) {
  return ((sizeof(LsShared<CAP>) + 15) & ~size_t(15)) + (size_t)order * ((size_t)CAP * 4 + 16) +
         (vbytes ? (size_t)CAP * vbytes + 16 : 0);
}

// Search of a sorted array by a whole warp: the first index i in [lo, hi)
// with a[i] > x (UPPER) or a[i] >= x (else), or hi. Each round probes 32
// evenly spaced positions and keeps the gap between the last probe below x
// and the first above, so a range of n takes about log32(n) dependent loads
// (a binary search by one thread takes log2(n)). Every lane gets the result.
template <bool UPPER>
__device__ __forceinline__ int warp_search(const int* a, int lo, int hi, int x, int lane) {
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) >> 5;
    const int p = lo + lane * step;
    const bool past = p >= hi || (UPPER ? __ldg(a + p) > x : __ldg(a + p) >= x);
    const unsigned m = __ballot_sync(0xffffffffu, past);
    const int f = m ? __ffs(m) - 1 : 32;
    if (f == 0) return lo;
    const int nlo = lo + (f - 1) * step + 1;
    if (f < 32) hi = min(hi, lo + f * step);
    lo = nlo;
  }
  const int p = lo + lane;
  const bool past = p < hi && (UPPER ? __ldg(a + p) > x : __ldg(a + p) >= x);
  const unsigned m = __ballot_sync(0xffffffffu, past);
  return m ? lo + __ffs(m) - 1 : hi;
}

// Copies np pass descriptors word by word (the lanes of one warp).
__device__ __forceinline__ void copy_passes(PassDesc* dst, const PassDesc* src, int np, int lane) {
  static_assert(sizeof(PassDesc) % 4 == 0, "descriptors of whole words");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int x = lane; x < np * (int)(sizeof(PassDesc) / 4); x += 32) d[x] = s[x];
}

template <int CAP, int VB>
__global__ void __launch_bounds__(ls_threads<CAP>())
k_local_sort(Cols c1, const __grid_constant__ PassList pl, const int* __restrict__ seg_start,
             const int* __restrict__ counters, int single, int nnz, LsBatch lb, int lay_order,
             unsigned* status, const __grid_constant__ LevOut lv) {
  constexpr int kLsThreads = ls_threads<CAP>();
  constexpr int kLsWarps = kLsThreads / 32;
  constexpr int ITEMS = CAP / kLsThreads;
  constexpr size_t kRow4 = (size_t)CAP * 4 + 16;  // a staged coordinate row
  extern __shared__ __align__(16) uint8_t smem[];
  LsShared<CAP>& S = *reinterpret_cast<LsShared<CAP>*>(smem);
  uint8_t* stage = smem + ((sizeof(LsShared<CAP>) + 15) & ~size_t(15));
  uint8_t* const vstage = stage + (size_t)lay_order * kRow4;  // the value row
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * CAP * kLsSpan;
  if (w0 >= nnz) return;
  const int win0 = (int)w0;
  const int64_t w1 = w0 + (int64_t)CAP * kLsSpan;
  const int win1 = w1 < nnz ? (int)w1 : nnz;
  const int nseg = single ? 1 : counters[kCntNumSeg];

  // Warp 0 plans: the buckets that begin in the window are [first, last)
  // (bucket starts are distinct, so at most win1 - win0 of them).
  if (w == 0) {
    int first = 0, last = 1;
    if (!single) {
      first = warp_search<false>(seg_start, 0, nseg, win0, lane);
      last = warp_search<false>(seg_start, first, min(nseg, first + (win1 - win0) + 1), win1, lane);
    }
    // the key passes in shared memory: every digit read takes a field
    copy_passes(S.pass, pl.pass, pl.npasses, lane);
    if (lane == 0) {
      mbar_init(&S.ld, 1);
      S.c = c1;
      S.passes = S.pass;
      S.npasses = pl.npasses;
      S.first = first;
      S.last = last;
    }
  }
  __syncthreads();
  const int last = S.last;
  int s = S.first;
  unsigned phase = 0;
  // warp 0's view of the current tensor of a batch round: its index, where
  // the next tensor starts, and the first bucket of the next tensor
  int kt = -1, kt_end = 0, kt_seg = last;
  while (s < last) {
    if (w == 0) {
      const int a = single ? 0 : __ldg(seg_start + s);
      const int b = single ? nnz : __ldg(seg_start + s + 1);
      int lim = last;
      if (lb.n > 0) {  // the bucket's tensor; the batch ends where the next one starts
        if (kt < 0 || a >= kt_end) {
          kt = warp_search<true>(lb.jbase, 0, lb.n + 1, a, lane) - 1;
          kt_end = __ldg(lb.jbase + kt + 1);
          kt_seg = warp_search<false>(seg_start, s + 1, last + 1, kt_end, lane);
          const int np = lb.t[kt].npasses;
          copy_passes(S.pass, lb.t[kt].pass, np, lane);
          if (lane == 0) {
            S.c = lb.t[kt].c;
            S.npasses = np;
          }
        }
        lim = min(lim, kt_seg);
      }
      int e;
      if (b - a > CAP) {
        e = -1;  // large bucket: sorted by the digit passes
      } else if (single) {
        e = 1;
      } else {  // the most buckets from s whose entries fit CAP, within the tensor
        e = min(warp_search<true>(seg_start, s + 1, lim + 1, a + CAP, lane) - 1, lim);
      }
      if (lane == 0) S.batch_end = e;
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
    const int nrows = c.order + (VB ? 1 : 0);
    auto row_smem = [&](int r) -> uint8_t* { return r < c.order ? stage + (size_t)r * kRow4 : vstage; };
    auto row_gmem = [&](int r) -> uintptr_t {
      return r < c.order ? reinterpret_cast<uintptr_t>(c.in + (int64_t)r * c.in_stride + A)
                         : reinterpret_cast<uintptr_t>(c.vin) + (uintptr_t)A * VB;
    };

    // Stage the batch's rows: warp 0 starts one bulk copy per row for its
    // 16-byte-aligned body (lane r: row r).
    if (w == 0) {
      fence_proxy_async_smem();  // the previous batch's reads of the stage came first
      unsigned bytes = 0;
      int head = 0;
      if (lane < nrows) {
        const int es = lane < c.order ? 4 : VB;
        const uintptr_t g0 = row_gmem(lane), g1 = g0 + (uintptr_t)n * es;
        const uintptr_t a0 = (g0 + 15) & ~uintptr_t(15), a1 = g1 & ~uintptr_t(15);
        S.row_off[lane] = (int)(g0 & 15);
        if (a1 > a0) {
          head = (int)((a0 - g0) / es);
          S.row_head[lane] = head;
          S.row_tail[lane] = (int)((a1 - g0) / es);
          bytes = (unsigned)(a1 - a0);
        } else {
          S.row_head[lane] = n;
          S.row_tail[lane] = n;
        }
      }
      unsigned total = bytes;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
      if (lane == 0) mbar_arrive_expect_tx(&S.ld, total);
      __syncwarp();
      if (lane < nrows && bytes) {
        const int es = lane < c.order ? 4 : VB;
        bulk_g2s(row_smem(lane) + S.row_off[lane] + (size_t)head * es,
                 reinterpret_cast<const void*>(row_gmem(lane) + (uintptr_t)head * es), bytes, &S.ld);
      }
    }

    // Batches of tiny buckets (at most kTiny entries, typical where the prefix
    // is nearly unique) whose packed key fits the scratch are ranked by
    // counting inside each bucket (below); the others by radix passes.
    constexpr int kScratchWords = kLsWarps * kRadix;  // the ranking counters' space
    constexpr int kKeyBits = CAP * 2 <= kScratchWords ? 64 : CAP <= kScratchWords ? 32 : 0;
    int key_bits = 0;
    for (int p = 0; p < S.npasses; ++p) key_bits += S.passes[p].bits;
    bool small = kKeyBits > 0 && !single && key_bits <= kKeyBits;
    // One read of the batch's bucket starts, while the rows load: marks at
    // the starts (scanned below into every position's bucket index), the
    // starts themselves in the second permutation buffer (which the
    // counting path does not use otherwise) and whether every bucket is tiny.
    if (nsb > 1)
      for (int i = threadIdx.x; i < CAP; i += kLsThreads) S.segid[i] = 0;
    __syncthreads();
    if (!single)
      for (int k = s + threadIdx.x; k < e; k += kLsThreads) {
        const int a = seg_start[k] - A;
        small = small && seg_start[k + 1] - A - a <= kTiny;
        S.perm[1][k - s] = (uint16_t)a;
        if (k > s) S.segid[a] = 1;
      }
    const bool tiny = __syncthreads_and(small);

    if (nsb > 1) {
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
    __syncthreads();  // the row plans are visible
    // unaligned edges with plain loads
    for (int r = 0; r < nrows; ++r) {
      const int head = S.row_head[r], tail = S.row_tail[r], np = head + (n - tail);
      uint8_t* dst = row_smem(r) + S.row_off[r];
      const uintptr_t src = row_gmem(r);
      for (int x = threadIdx.x; x < np; x += kLsThreads) {
        const int i = x < head ? x : tail + (x - head);
        if (r < c.order || VB == 4)
          reinterpret_cast<uint32_t*>(dst)[i] = __ldg(reinterpret_cast<const uint32_t*>(src) + i);
        else
          reinterpret_cast<unsigned long long*>(dst)[i] =
              __ldg(reinterpret_cast<const unsigned long long*>(src) + i);
      }
    }
    __syncthreads();
    mbar_wait(&S.ld, phase, status);  // the bulk copies have landed
    phase ^= 1u;

    int cur = 0;
    int seg_bits = 0;
    while ((1 << seg_bits) < nsb) ++seg_bits;
    const int seg_passes = (seg_bits + kRadixBits - 1) / kRadixBits;
    if (kKeyBits > 0 && tiny) {
      // Rank by counting: an entry's place in its bucket is the number of the
      // bucket's entries with a smaller packed key, or an equal key earlier in
      // the bucket (stable). Packed keys (the key passes' digits, least
      // significant first) are built once into the counters' space. Each
      // thread handles its ITEMS entries side by side, so that their
      // shared-memory reads overlap.
      using KeyT = typename std::conditional<kKeyBits == 64, uint64_t, uint32_t>::type;
      KeyT* keys = reinterpret_cast<KeyT*>(S.warp_hist);
      KeyT key[ITEMS];
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) key[j] = 0;
      int off = 0;
      for (int p = 0; p < key_passes; ++p) {
        const int nf = passes[p].nfields;
        uint32_t d[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) d[j] = 0;
        for (int k = 0; k < nf; ++k) {
          const DigitField f = passes[p].f[k];
          const uint32_t* row =
              reinterpret_cast<const uint32_t*>(row_smem(f.mode) + S.row_off[f.mode]);
#pragma unroll
          for (int j = 0; j < ITEMS; ++j) {
            const int i = threadIdx.x + j * kLsThreads;
            if (i < n) d[j] |= field_bits(row[i], f);
          }
        }
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) key[j] |= (KeyT)d[j] << off;
        off += passes[p].bits;
      }
#pragma unroll
      for (int j = 0; j < ITEMS; ++j) {
        const int i = threadIdx.x + j * kLsThreads;
        if (i < n) keys[i] = key[j];
      }
      __syncthreads();
      // every entry walks its bucket (most buckets hold one or two entries)
      for (int i = threadIdx.x; i < n; i += kLsThreads) {
        const int b = nsb > 1 ? S.segid[i] : 0;
        const int lo = S.perm[1][b], hi = b + 1 < nsb ? S.perm[1][b + 1] : n;
        const KeyT ki = keys[i];
        int r = lo;
#pragma unroll 1
        for (int y = lo; y < hi; ++y) {
          const KeyT ky = keys[y];
          r += (ky < ki || (ky == ki && y < i)) ? 1 : 0;
        }
        S.perm[0][r] = (uint16_t)i;
      }
      __syncthreads();
    }
    for (int p = 0; p < (tiny ? 0 : key_passes + seg_passes); ++p) {
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
              const uint32_t* row =
                  reinterpret_cast<const uint32_t*>(row_smem(f.mode) + S.row_off[f.mode]);
              d |= field_bits(row[el[i]], f);
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

    // Every row back through the permutation (coalesced stores).
    for (int m = 0; m < c.order; ++m) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(row_smem(m) + S.row_off[m]);
      int32_t* dst = c.out + (int64_t)m * c.out_stride + A;
      for (int i = threadIdx.x; i < n; i += kLsThreads) dst[i] = (int32_t)src[S.perm[cur][i]];
    }
    if constexpr (VB != 0) {
      using T = typename LsVal<VB>::T;
      const T* src = reinterpret_cast<const T*>(vstage + S.row_off[c.order]);
      T* dst = reinterpret_cast<T*>(c.vout) + A;
      for (int i = threadIdx.x; i < n; i += kLsThreads) dst[i] = src[S.perm[cur][i]];
    }
    if (lv.lev) {
      // first differing level against the entry written just before (the
      // batch's first entry: unknown here)
      for (int i = threadIdx.x; i < n; i += kLsThreads) {
        uint32_t L = 0;
        if (i > 0) {
          const int a = S.perm[cur][i], b = S.perm[cur][i - 1];
          L = (uint32_t)lv.order + 1;
          for (int l = 0; l < lv.order; ++l) {
            const int m = lv.sigma[l];
            const uint32_t* row = reinterpret_cast<const uint32_t*>(row_smem(m) + S.row_off[m]);
            if (row[a] != row[b]) {
              L = (uint32_t)l + 1;
              break;
            }
          }
        }
        lv.lev[A + i] = (uint8_t)L;
      }
    }
    __syncthreads();  // the stage is free for the next batch
    s = e;
  }
}

template <int CAP, int VB>
cudaError_t launch_ls(const Cols& c, const PassList& pl, const int* seg_start,
                      const int* counters, int single, int nnz, const LsBatch& lb,
                      unsigned* status, cudaStream_t stream, const LevOut& lv) {
  // shared state, then the staged rows: c.order coordinate rows (the largest
  // order of a batch) and the value row
  const size_t smem = ls_smem<CAP>(c.order, VB);
  cudaError_t e = cudaFuncSetAttribute(k_local_sort<CAP, VB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = single ? 1 : (int)(((int64_t)nnz + (int64_t)CAP * kLsSpan - 1) / ((int64_t)CAP * kLsSpan));
  if (grid < 1) return cudaSuccess;
  k_local_sort<CAP, VB><<<grid, ls_threads<CAP>(), smem, stream>>>(c, pl, seg_start, counters,
                                                            single, nnz, lb, c.order, status,
                                                            lv);
  return cudaGetLastError();
}

template <int CAP>
cudaError_t launch_ls_cap(const Cols& c, const PassList& pl, const int* seg_start,
                          const int* counters, int single, int nnz, const LsBatch& lb,
                          unsigned* status, cudaStream_t stream, const LevOut& lv) {
  switch (c.vbytes) {
    case 0: return launch_ls<CAP, 0>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
    case 4: return launch_ls<CAP, 4>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
    case 8: return launch_ls<CAP, 8>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t debug_words_local_sort(unsigned long long limit_ns, int stall) {
  return set_debug_words(limit_ns, stall);
}

// The bucket capacity the sort runs with: the largest power of two in
// [1024, want] whose staged rows leave room for two blocks per SM (the
// loads of one block overlap the ranking of the other; below 4096 entries
// the smaller blocks leave room for three), else the largest that fits
// shared memory at all.
int local_sort_capacity(int want, int order, int vbytes) {
  constexpr size_t kMax = 227 * 1024, kTwo = 113 * 1024;
  const size_t sz[4] = {ls_smem<8192>(order, vbytes), ls_smem<4096>(order, vbytes),
                        ls_smem<2048>(order, vbytes), ls_smem<1024>(order, vbytes)};
  const int cap[4] = {8192, 4096, 2048, 1024};
  for (int k = 0; k < 4; ++k)
    if (cap[k] <= want && sz[k] <= kTwo) return cap[k];
  for (int k = 0; k < 4; ++k)
    if (cap[k] <= want && sz[k] <= kMax) return cap[k];
  return 1024;
}

cudaError_t launch_local_sort(const Cols& c, const PassList& pl, const int* seg_start,
                              const int* counters, int single, int nnz, int capacity,
                              unsigned* status, const LsBatch& lb, cudaStream_t stream,
                              const LevOut* lvp) {
  LevOut lv;
  if (lvp && lb.n == 0) {
    lv = *lvp;
  } else {
    lv.lev = nullptr;
    lv.order = 0;
  }
  switch (capacity) {
    case 1024: return launch_ls_cap<1024>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
    case 2048: return launch_ls_cap<2048>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
    case 4096: return launch_ls_cap<4096>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
    case 8192: return launch_ls_cap<8192>(c, pl, seg_start, counters, single, nnz, lb, status, stream, lv);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qsd
