// Global stable radix passes for buckets too large for one thread block
// (and for the whole tensor when a group has no prefix).
//
// A pass is the GPU form of one histogram partial sort (Algorithm 1: count,
// prefix-sum, stable move) over a radix digit of the packed key instead of a
// whole mode, so the count array has at most 2^8 bins rather than n_k (the
// cost the paper's discussion attributes to large modes). The count and the
// prefix sum are done per chunk (a run of consecutive entries inside one
// bucket), which makes the move free of any dependency between thread
// blocks:
//   k_chunk_hist   per chunk: histogram of the pass's digit (one read of the
//                  key coordinates the digit comes from); per chunk group:
//                  the sum of its chunks' histograms;
//   k_chunk_scan   per chunk group: every chunk's first output slot for each
//                  digit = bucket start + entries of smaller digits in the
//                  bucket + entries of the same digit in earlier chunks (over
//                  a whole tensor of many groups: k_group_prefix, then
//                  k_chunk_scan_parts);
//   k_digit_move   per chunk (claimed dynamically): tiles of the chunk are
//                  staged in shared memory by bulk asynchronous copies (the
//                  next tile's copies overlap the current tile), ranked
//                  stably by digit, and every row is written through the
//                  inverse permutation to the chunk's running slots.
// Buckets never exchange entries (Section 3.2: coordinates do not leave
// their bucket), so offsets are computed per bucket.
#include <cuda_runtime.h>

#include <type_traits>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

constexpr int kHistThreads = 256;
constexpr int kHistWarps = kHistThreads / 32;
constexpr int kMaxRows = kMaxOrder + 1;

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

__device__ __forceinline__ int n_chunks(const LargeSegs& ls) {
  return ls.single ? (ls.nnz + ls.chunk - 1) / ls.chunk : ls.counters[kCntNumChunks];
}
__device__ __forceinline__ int n_groups(const LargeSegs& ls) {
  return ls.single ? (n_chunks(ls) + kGroupChunks - 1) / kGroupChunks
                   : ls.counters[kCntNumGroups];
}

struct ChunkInfo {
  int seg;     // large-bucket index
  int start;   // first entry of the chunk
  int end;     // one past its last entry
  int group;   // its chunk group
  int lo, hi;  // the bucket's entry range
};

__device__ __forceinline__ ChunkInfo chunk_info(const LargeSegs& ls, int c) {
  ChunkInfo ci;
  int s, cb, gb, lo, hi;
  if (ls.single) {
    s = 0;
    cb = 0;
    gb = 0;
    lo = 0;
    hi = ls.nnz;
  } else {
    s = ls.chunk_owner[c];
    const int2 se = ls.seg[s];
    cb = ls.chunk_base[s];
    gb = ls.group_base[s];
    lo = se.x;
    hi = se.y;
  }
  const int lc = c - cb;
  ci.seg = s;
  ci.start = lo + lc * ls.chunk;
  ci.end = min(ci.start + ls.chunk, hi);
  ci.group = gb + lc / kGroupChunks;
  ci.lo = lo;
  ci.hi = hi;
  return ci;
}

// Copies a descriptor word by word (threads t, t + step, ... of a group).
template <typename D>
__device__ __forceinline__ void copy_words(D* dst, const D* src, int t, int step) {
  static_assert(sizeof(D) % 4 == 0, "descriptor of whole words");
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = t; i < (int)(sizeof(D) / 4); i += step) d[i] = s[i];
}

// ---------------------------------------------------------------------------
// Counts a lane's four consecutive digits into its warp's histogram h (valid
// lanes only; every lane of the warp calls it together). Lanes whose four
// digits are equal -- most of them where one bin takes most entries -- are
// combined across the warp: one match finds the lanes with the same digit
// and one of them adds 4 per lane, so a hot bin takes one shared atomic per
// warp instead of one per lane. Other lanes add one atomic per run of equal
// digits.
__device__ __forceinline__ void count4(uint32_t* h, const uint32_t (&e)[4], bool valid,
                                       int lane) {
  const bool same = valid && e[0] == e[1] && e[1] == e[2] && e[2] == e[3];
  const uint32_t m_same = __ballot_sync(0xffffffffu, same);
  if (same) {
    const uint32_t peers = __match_any_sync(m_same, e[0]);
    if (lane == __ffs(peers) - 1) atomicAdd(&h[e[0]], 4u * (uint32_t)__popc(peers));
  } else if (valid) {
    uint32_t run_d = e[0], run_n = 1;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      if (e[k] == run_d) {
        ++run_n;
      } else {
        atomicAdd(&h[run_d], run_n);
        run_d = e[k];
        run_n = 1;
      }
    }
    atomicAdd(&h[run_d], run_n);
  }
}

// ---------------------------------------------------------------------------
// Chunk histograms: 16-byte loads of the digit's rows (four in flight per
// thread), each vector of four consecutive entries counted into the warp's
// histogram (count4). The vector loops run with warp-uniform bounds so that
// every lane takes part in count4's warp operations. At most 40 registers, so
// six blocks share an SM: measured 8% faster than eight loads in flight per
// thread with four blocks per SM.
__global__ void __launch_bounds__(kHistThreads, 6)
k_chunk_hist(const __grid_constant__ PassTensor one, LargeSegs ls,
             uint32_t* __restrict__ chunk_hist, uint32_t* __restrict__ group_sum,
             int* __restrict__ claim, PassBatch pb) {
  __shared__ uint32_t s_hist[kHistWarps][kRadix];
  __shared__ int s_chunk;
  __shared__ PassTensor s_it;  // the chunk's tensor: buffers and digit
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = pb.t ? pb.counters[kCntPassChunks + pb.pass] : n_chunks(ls);
  const Cols& c = s_it.c;
  const PassDesc& pd = s_it.pd;
  if (!pb.t) copy_words(&s_it, &one, threadIdx.x, kHistThreads);
  // thread 0 claims one chunk ahead, so the claim's round trip overlaps the
  // current chunk's work
  auto claim_next = [&]() {
    const int idx = atomicAdd(claim, 1);
    return idx < nc ? (pb.t ? pb.chunks[idx] : idx) : -1;
  };
  int next = threadIdx.x == 0 ? claim_next() : -1;
  while (true) {
    for (int i = threadIdx.x; i < kHistWarps * kRadix; i += kHistThreads)
      (&s_hist[0][0])[i] = 0;
    if (threadIdx.x == 0) {
      s_chunk = next;
      if (next >= 0) next = claim_next();
    }
    __syncthreads();
    const int ch = s_chunk;
    if (ch < 0) break;
    const ChunkInfo ci = chunk_info(ls, ch);
    if (pb.t) {
      copy_words(&s_it, pb.t + pb.large_tensor[ci.seg], threadIdx.x, kHistThreads);
      __syncthreads();
    }
    const int nbins = 1 << pd.bits;
    // vectors line up across the digit's rows when there is one row, or when
    // the row stride is a multiple of 4 entries (every row then has the same
    // 16-byte phase)
    const bool vec = pd.nfields == 1 || (c.in_stride & 3) == 0;
    // Vector path: the digit's rows advance together in 16-byte steps when the
    // row stride is a multiple of 4 entries; entries before the first aligned
    // one and after the last full vector are counted one by one.
    int vbeg = ci.end, vend = ci.end;
    if (vec) {
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(c.in + (int64_t)pd.f[0].mode * c.in_stride +
                                                       ci.start);
      const int skip = (int)(((16 - (a0 & 15)) & 15) >> 2);
      vbeg = min(ci.start + skip, ci.end);
      vend = vbeg + ((ci.end - vbeg) & ~3);
    }
    const int nhead = vbeg - ci.start, ntail = ci.end - vend;
    for (int k = threadIdx.x; k < nhead + ntail; k += kHistThreads) {
      const int j = k < nhead ? ci.start + k : vend + (k - nhead);
      uint32_t d = 0;
      for (int f = 0; f < pd.nfields; ++f) {
        const DigitField fd = pd.f[f];
        d |= field_bits((uint32_t)__ldg(c.in + (int64_t)fd.mode * c.in_stride + j), fd);
      }
      atomicAdd(&s_hist[w][d], 1u);
    }
    const int nvec = (vend - vbeg) >> 2;
    // a digit from one row: 4 vectors (64 bytes) per thread in flight per round
    if (pd.nfields == 1) {
      const DigitField fd = pd.f[0];
      const uint4* col =
          reinterpret_cast<const uint4*>(c.in + (int64_t)fd.mode * c.in_stride + vbeg);
      // the warp's first lane decides the trip count (lanes differ by < 32)
      for (int q0 = threadIdx.x; q0 - lane < nvec; q0 += kHistThreads * 4) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * kHistThreads;
          v[u] = q < nvec ? __ldg(col + q) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t e[4] = {field_bits(v[u].x, fd), field_bits(v[u].y, fd),
                                 field_bits(v[u].z, fd), field_bits(v[u].w, fd)};
          count4(s_hist[w], e, q0 + u * kHistThreads < nvec, lane);
        }
      }
    }
    for (int q0 = threadIdx.x; q0 - lane < (pd.nfields == 1 ? 0 : nvec); q0 += kHistThreads * 4) {
      uint4 dv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) dv[u] = make_uint4(0, 0, 0, 0);
      for (int f = 0; f < pd.nfields; ++f) {
        const DigitField fd = pd.f[f];
        const uint4* col =
            reinterpret_cast<const uint4*>(c.in + (int64_t)fd.mode * c.in_stride + vbeg);
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u * kHistThreads;
          v[u] = q < nvec ? __ldg(col + q) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          dv[u].x |= field_bits(v[u].x, fd);
          dv[u].y |= field_bits(v[u].y, fd);
          dv[u].z |= field_bits(v[u].z, fd);
          dv[u].w |= field_bits(v[u].w, fd);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t e[4] = {dv[u].x, dv[u].y, dv[u].z, dv[u].w};
        count4(s_hist[w], e, q0 + u * kHistThreads < nvec, lane);
      }
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < nbins; dd += kHistThreads) {
      uint32_t v = 0;
#pragma unroll
      for (int ww = 0; ww < kHistWarps; ++ww) v += s_hist[ww][dd];
      chunk_hist[(size_t)ch * kRadix + dd] = v;
      if (v) atomicAdd(group_sum + (size_t)ci.group * kRadix + dd, v);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Group offsets of a pass over one whole tensor (ls.single): one block turns
// the chunk groups' digit counts into each group's first output slot per
// digit, in place: group_sum[g][d] <- (entries of smaller digits) + (entries
// of digit d in groups before g). Thread (part, d) takes digit d over a
// quarter of the groups; eight counts in flight per thread.
constexpr int kPrefixParts = 4;
__global__ void __launch_bounds__(kRadix * kPrefixParts)
k_group_prefix(LargeSegs ls, uint32_t* __restrict__ group_sum) {
  __shared__ uint32_t s_part[kPrefixParts][kRadix];
  __shared__ uint32_t s_below[kRadix];
  __shared__ uint32_t s_warp[kRadix / 32];
  const int d = threadIdx.x % kRadix, part = threadIdx.x / kRadix;
  const int ng = n_groups(ls);
  const int per = (ng + kPrefixParts - 1) / kPrefixParts;
  const int g0 = min(part * per, ng), g1 = min(g0 + per, ng);
  uint32_t sum = 0;
  for (int g = g0; g < g1; g += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = g + k < g1 ? group_sum[(size_t)(g + k) * kRadix + d] : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += v[k];
  }
  s_part[part][d] = sum;
  __syncthreads();
  if (part == 0) {  // the digit totals' exclusive scan (warps 0-7)
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < kPrefixParts; ++k) tot += s_part[k][d];
    const int lane = d & 31, w = d >> 5;
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    s_below[d] = incl - tot;  // within the warp for now
  }
  __syncthreads();
  uint32_t run = s_below[d];
  for (int k = 0; k < (d >> 5); ++k) run += s_warp[k];
  for (int k = 0; k < part; ++k) run += s_part[k][d];
  for (int g = g0; g < g1; g += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = g + k < g1 ? group_sum[(size_t)(g + k) * kRadix + d] : 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (g + k < g1) {
        group_sum[(size_t)(g + k) * kRadix + d] = run;
        run += v[k];
      }
  }
}

// ---------------------------------------------------------------------------
// Chunk offsets over one whole tensor, after k_group_prefix: one block per
// chunk group, four parts of 16 chunks each (kRadix threads per part, one per
// digit). Each part holds its 16 counts in registers (all loads in flight),
// the parts' sums give each part's first slot, then every chunk's first slot
// per digit replaces its counts.
constexpr int kScanParts = 4;
__global__ void __launch_bounds__(kRadix * kScanParts)
k_chunk_scan_parts(LargeSegs ls, uint32_t* __restrict__ chunk_hist,
                   const uint32_t* __restrict__ group_sum) {
  constexpr int kPer = kGroupChunks / kScanParts;
  static_assert(kPer * kScanParts == kGroupChunks, "parts cover a group");
  __shared__ uint32_t s_part[kScanParts][kRadix];
  const int d = threadIdx.x % kRadix, part = threadIdx.x / kRadix;
  const int ng = n_groups(ls), nc = n_chunks(ls);
  for (int G = blockIdx.x; G < ng; G += gridDim.x) {
    const int c0 = G * kGroupChunks + part * kPer;
    uint32_t h[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      h[k] = c0 + k < nc ? chunk_hist[(size_t)(c0 + k) * kRadix + d] : 0u;
      sum += h[k];
    }
    s_part[part][d] = sum;
    __syncthreads();
    uint32_t off = group_sum[(size_t)G * kRadix + d];  // k_group_prefix's first slot
    for (int q = 0; q < part; ++q) off += s_part[q][d];
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (c0 + k < nc) {
        chunk_hist[(size_t)(c0 + k) * kRadix + d] = off;
        off += h[k];
      }
    __syncthreads();  // s_part is reused by the next group
  }
}

// ---------------------------------------------------------------------------
// Chunk offsets. One block (kRadix threads, one per digit) per chunk group,
// each block adding up its bucket's groups (buckets, batches, and tensors of
// at most 16 groups; larger whole tensors take k_chunk_scan_parts).
__global__ void __launch_bounds__(kRadix)
k_chunk_scan(LargeSegs ls, uint32_t* __restrict__ chunk_hist,
             const uint32_t* __restrict__ group_sum, PassBatch pb) {
  __shared__ uint32_t s_tmp[kRadix / 32 + 1];
  const int d = threadIdx.x;
  const int ng_all = pb.t ? pb.counters[kCntPassGroups + pb.pass] : n_groups(ls);
  const int nc_all = n_chunks(ls);
  for (int gi = blockIdx.x; gi < ng_all; gi += gridDim.x) {
    const int G = pb.t ? pb.groups[gi] : gi;
    int s, gb, cb, ng, nc, lo;
    if (ls.single) {
      s = 0;
      gb = 0;
      cb = 0;
      ng = ng_all;
      nc = nc_all;
      lo = 0;
    } else {
      s = ls.group_owner[G];
      const int2 se = ls.seg[s];
      gb = ls.group_base[s];
      cb = ls.chunk_base[s];
      nc = (se.y - se.x + ls.chunk - 1) / ls.chunk;
      ng = (nc + kGroupChunks - 1) / kGroupChunks;
      lo = se.x;
    }
    (void)s;
    // bucket total and the sum over the bucket's earlier groups, per digit
    uint32_t total = 0, prior = 0;
    for (int g = gb; g < gb + ng; ++g) {
      const uint32_t v = group_sum[(size_t)g * kRadix + d];
      total += v;
      if (g < G) prior += v;
    }
    uint32_t tot_all;
    const uint32_t below = block_exclusive_sum<kRadix / 32>(total, s_tmp, &tot_all);
    uint32_t off = (uint32_t)lo + below + prior;
    const int c0 = cb + (G - gb) * kGroupChunks;
    const int c1 = min(c0 + kGroupChunks, cb + nc);
    for (int c = c0; c < c1; c += 8) {
      uint32_t h[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) h[k] = c + k < c1 ? chunk_hist[(size_t)(c + k) * kRadix + d] : 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (c + k < c1) {
          chunk_hist[(size_t)(c + k) * kRadix + d] = off;
          off += h[k];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The move, warp-specialised. One block per SM runs a three-role pipeline
// over the tiles of the chunks it claims:
//   producer (1 warp)  claims chunks, describes each tile in a ring slot,
//                      loads its rows' unaligned edges and starts bulk
//                      copies of the aligned bodies into the slot's staging
//                      buffer (NS slots);
//   rankers            compute the digits of tile k+1, rank them stably and
//                      turn the chunk's running output slots into each
//                      sorted position's destination;
//   writers            write tile k's rows through the inverse permutation.
// (16 ranking and 15 writing warps for tiles of 2048 entries and more, 8 and
// 8 for tiles of 1024.)
// Ranking and writing overlap, and the copies run NS-1 tiles ahead.
// A slot is released in two parts: the writers write a tile's key rows (the
// rows its digit is read from) first and then free them, so the next tile
// of that slot has its key rows loaded and ranked while the other rows of
// this tile are still being written; its other rows follow once the whole
// slot is free. (With one slot released as a whole, every slot waited for
// the load, the ranking and the writing of its tile in turn, and the two
// slots that fit 24-byte entries could not hide that chain.) In a batch the
// tiles' key rows differ from tensor to tensor, so there a slot is freed
// only as a whole. Hand-offs use mbarriers (every wait bounded); the rankers
// synchronise among themselves on named barrier 1.

// Role sizes: RW ranking warps, WW writing warps, one producer warp.
template <int RW, int WW>
struct Roles {
  static constexpr int kRank = RW * 32;
  static constexpr int kWrite = WW * 32;
  static constexpr int kThreads = kRank + kWrite + 32;
};

// Where one row of a tile lands in its shared-memory slot: entry i is at
// byte off + i * esz; entries [0, head) and [tail_from, n) arrive by plain
// loads, the 16-byte-aligned body between them by one bulk copy.
struct RowPlan {
  int off;
  int head;
  int tail_from;
};

// One unit of work: tile `k` of chunk `chunk` (chunk < 0: the end). Tile q
// is described in entry q % (2 NS) of a ring of these, so the producer can
// describe a tile once its slot's key rows are free, while the writers still
// read the description of the tile before it in that slot.
struct TileMeta {
  int chunk, k, ntile, start, end, lo, hi;
  unsigned kmask;  // the rows the pass's digit is read from
  RowPlan row[kMaxRows];
  PassTensor it;  // the chunk's tensor: buffers and digit
};

template <int T, int NS, int RW>
struct WsShared {
  uint64_t kfull[NS];    // producer -> rankers: the tile's key rows staged
  uint64_t full[NS];     // producer -> writers: the tile's other rows staged
  uint64_t kempty[NS];   // writers -> producer: the slot's key rows free
  uint64_t empty[NS];    // writers -> producer: the whole slot free
  uint64_t ranked[2];    // rankers -> writers: destinations ready
  uint64_t consumed[2];  // writers -> rankers: destinations used
  // a chunk's first tile: the chunk's first output slot per digit (loaded
  // with the key rows; only the rankers read it)
  alignas(16) uint32_t off0[NS][kRadix];
  TileMeta meta[2 * NS];
  uint32_t off[kRadix];  // rankers: running output slot per digit of the chunk
  uint32_t warp_hist[RW * kRadix];
  uint32_t rank_tmp[RW];  // block_rank's scan scratch
  uint32_t bin_start[kRadix];
  uint32_t bin_count[kRadix];
  uint32_t gbase[2][kRadix];  // destination of sorted position p = gbase[d] + p
  uint32_t invdig[2][T];      // sorted position -> (digit << 16) | tile position
  int rk_abort;  // the rankers gave up: the writers stop without writing
};

template <int T>
__host__ __device__ constexpr int row_slot(int esz) {
  return T * esz + 16;
}

template <int T, int NS, int RW>
__host__ __device__ constexpr size_t ws_header() {
  return (sizeof(WsShared<T, NS, RW>) + 15) & ~size_t(15);
}

template <int T, int VB>
__host__ __device__ constexpr size_t ws_buffer(int order) {
  return (size_t)order * row_slot<T>(4) + (VB ? row_slot<T>(VB) : 0);
}

__device__ __forceinline__ uintptr_t row_base(const Cols& c, int r) {
  return r < c.order ? reinterpret_cast<uintptr_t>(c.in + (int64_t)r * c.in_stride)
                     : reinterpret_cast<uintptr_t>(c.vin);
}

template <int T, int NS, int VB, int RW, int WW>
__global__ void __launch_bounds__(Roles<RW, WW>::kThreads, 1)
k_digit_move(const __grid_constant__ PassTensor one, int lay_order, LargeSegs ls,
             const uint32_t* __restrict__ chunk_off, int* __restrict__ claim, unsigned* status,
             PassBatch pb, const __grid_constant__ LevOut lv) {
  constexpr int kWsRankWarps = RW, kWsWriteWarps = WW;
  constexpr int kWsRankThreads = Roles<RW, WW>::kRank;
  constexpr int kWsWriteThreads = Roles<RW, WW>::kWrite;
  constexpr int ITEMS = T / kWsRankThreads;
  static_assert(ITEMS * kWsRankThreads == T, "rankers must cover the tile");
  constexpr int WITEMS = (T + kWsWriteThreads - 1) / kWsWriteThreads;
  extern __shared__ __align__(16) uint8_t smem[];
  WsShared<T, NS, RW>& S = *reinterpret_cast<WsShared<T, NS, RW>*>(smem);
  uint8_t* const stage = smem + ws_header<T, NS, RW>();
  const size_t bufsz = ws_buffer<T, VB>(lay_order);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nchunks = pb.t ? pb.counters[kCntPassChunks + pb.pass] : n_chunks(ls);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&S.kfull[s], 32);
      mbar_init(&S.full[s], 32);
      mbar_init(&S.kempty[s], kWsWriteThreads);
      mbar_init(&S.empty[s], kWsWriteThreads);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&S.ranked[j], kWsRankThreads);
      mbar_init(&S.consumed[j], kWsWriteThreads);
    }
    S.rk_abort = 0;
  }
  __syncthreads();

  if (warp == kWsRankWarps + kWsWriteWarps) {
    // ---------------- producer ----------------
    // One tensor: a tile's key rows load once its slot's key rows are free.
    // A batch: only once the whole slot is.
    const bool split = pb.t == nullptr;
    int ch = 0, k = 0, ntile = 0;
    // Tiles [0, issued_k) had their key rows' copies started, [0, issued_p)
    // the other rows'. Before the block exits it waits for the latest phase
    // of every slot's barriers that copies were started for; skip = the
    // tile whose phases an end marker in its slot has superseded.
    int issued_k = 0, issued_p = 0, skip = -1;
    // test-only stall (qsd_debug_set_stall): block 0 arms its first slot
    // for the copies of its first tile but issues none of them
    const bool stall = blockIdx.x == 0 && *(volatile int*)&g_debug_stall == 1;
    // the next chunk: an index into the pass's list, -1 when none is left
    auto claim_chunk = [&]() {
      int idx = 0;
      if (lane == 0) idx = atomicAdd(claim, 1);
      idx = __shfl_sync(0xffffffffu, idx, 0);
      return idx < nchunks ? (pb.t ? pb.chunks[idx] : idx) : -1;
    };
    // lane 0 waits (bounded) and the warp follows its outcome; then every
    // lane's own wait on the completed phase orders its stores after the
    // consumers' reads of the slot
    auto wait_warp = [&](uint64_t* bar, unsigned parity) {
      int ok = 1;
      if (lane == 0) ok = mbar_wait(bar, parity, status) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
      mbar_wait(bar, parity, status);
      return true;
    };
    ch = claim_chunk();
    for (int q = 0;; ++q) {
      const int s = q % NS;
      const unsigned prev = ((q / NS) - 1) & 1;  // phase parity of tile q - NS in slot s
      if (q >= NS) {
        if (!wait_warp(&S.kempty[s], prev)) break;
        if ((!split || ch < 0) && !wait_warp(&S.empty[s], prev)) break;
      }
      TileMeta& ts = S.meta[q % (2 * NS)];
      uint8_t* buf = stage + (size_t)s * bufsz;
      if (ch < 0) {
        if (lane == 0) ts.chunk = -1;
        __syncwarp();
        mbar_arrive(&S.kfull[s]);
        mbar_arrive(&S.full[s]);
        skip = q - NS;  // slot s now holds the end marker
        break;
      }
      const ChunkInfo ci = chunk_info(ls, ch);
      ntile = (ci.end - ci.start + T - 1) / T;
      const int start = ci.start + k * T, end = min(start + T, ci.end), n = end - start;
      copy_words(&ts.it, pb.t ? pb.t + pb.large_tensor[ci.seg] : &one, lane, 32);
      __syncwarp();
      const Cols& c = ts.it.c;
      const int nrows = c.order + (VB ? 1 : 0);
      // row plans: lane r handles row r
      unsigned bytes = 0;
      RowPlan rp;
      if (lane < nrows) {
        const int e = lane < c.order ? 4 : VB;
        const uintptr_t g0 = row_base(c, lane) + (uintptr_t)start * e, g1 = g0 + (uintptr_t)n * e;
        const uintptr_t a0 = (g0 + 15) & ~uintptr_t(15), a1 = g1 & ~uintptr_t(15);
        rp.off = (int)(g0 & 15);
        if (a1 > a0) {
          rp.head = (int)((a0 - g0) / e);
          rp.tail_from = (int)((a1 - g0) / e);
          bytes = (unsigned)(a1 - a0);
        } else {
          rp.head = n;
          rp.tail_from = n;
        }
        ts.row[lane] = rp;
      }
      // The rows the digit is read from (key rows) are staged first, under
      // their own barrier, so ranking starts while the other rows still load.
      unsigned kmask = 0;
      for (int f = 0; f < ts.it.pd.nfields; ++f) kmask |= 1u << ts.it.pd.f[f].mode;
      if (lane == 0) {
        ts.chunk = ch;
        ts.k = k;
        ts.ntile = ntile;
        ts.start = start;
        ts.end = end;
        ts.lo = ci.lo;
        ts.hi = ci.hi;
        ts.kmask = kmask;
      }
      __syncwarp();
      const bool is_key = lane < nrows && (kmask >> lane & 1u);
      auto issue = [&](int phase) {
        uint64_t* bar = phase == 0 ? &S.kfull[s] : &S.full[s];
        // unaligned edges of this phase's rows with plain loads (the whole warp)
        for (int r = 0; r < nrows; ++r) {
          if (((kmask >> r) & 1u) != (phase == 0 ? 1u : 0u)) continue;
          const RowPlan p = ts.row[r];
          const int nplain = p.head + (n - p.tail_from);
          uint8_t* dst = buf + (size_t)r * row_slot<T>(4) + p.off;
          for (int x = lane; x < nplain; x += 32) {
            const int i = x < p.head ? x : p.tail_from + (x - p.head);
            if (r < c.order)
              *reinterpret_cast<uint32_t*>(dst + (size_t)i * 4) =
                  (uint32_t)__ldg(c.in + (int64_t)r * c.in_stride + start + i);
            else if (VB == 8)
              *reinterpret_cast<unsigned long long*>(dst + (size_t)i * 8) =
                  __ldg(reinterpret_cast<const unsigned long long*>(c.vin) + start + i);
            else
              *reinterpret_cast<uint32_t*>(dst + (size_t)i * 4) =
                  __ldg(reinterpret_cast<const uint32_t*>(c.vin) + start + i);
          }
        }
        // bytes of this phase's bulk copies, then one transaction-counted arrival
        const bool mine = lane < nrows && is_key == (phase == 0);
        unsigned total = mine ? bytes : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
        // a chunk's first tile also brings the chunk's output offsets (1 KB)
        const bool offs = phase == 0 && k == 0;
        if (offs) total += kRadix * sizeof(uint32_t);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(bar, total);
        else mbar_arrive(bar);
        const bool no_copy = stall && q == 0;
        if (offs && lane == 31 && !no_copy)
          bulk_g2s(S.off0[s], chunk_off + (size_t)ch * kRadix, kRadix * sizeof(uint32_t), bar);
        if (mine && bytes && !no_copy) {
          const int e = lane < c.order ? 4 : VB;
          bulk_g2s(buf + (size_t)lane * row_slot<T>(4) + rp.off + (size_t)rp.head * e,
                   reinterpret_cast<const void*>(row_base(c, lane) + (uintptr_t)(start + rp.head) * e),
                   bytes, bar);
        }
      };
      issue(0);
      ++issued_k;
      // the other rows: once the writers are done with the whole slot
      if (split && q >= NS && !wait_warp(&S.empty[s], prev)) break;
      issue(1);
      ++issued_p;
      // next work item
      if (++k >= ntile) {
        k = 0;
        ch = claim_chunk();
      }
    }
    // The block exits only after the bulk copies it started have landed: on
    // a normal end these waits return at once; after a timeout elsewhere they
    // are bounded like every other wait.
    if (lane == 0) {
      for (int x = max(0, issued_k - NS); x < issued_k; ++x)
        if (x != skip) mbar_wait(&S.kfull[x % NS], (x / NS) & 1, status);
      for (int x = max(0, issued_p - NS); x < issued_p; ++x)
        if (x != skip) mbar_wait(&S.full[x % NS], (x / NS) & 1, status);
    }
  } else if (warp < kWsRankWarps) {
    // ---------------- rankers ----------------
    const int w = warp;
    for (int q = 0;; ++q) {
      const int s = q % NS, j = q & 1;
      const bool okf = mbar_wait(&S.kfull[s], (q / NS) & 1, status);
      const bool okc = q < 2 || mbar_wait(&S.consumed[j], ((q / 2) - 1) & 1, status);
      if (!(okf && okc)) S.rk_abort = 1;  // the writers stop without writing
      const TileMeta& ts = S.meta[q % (2 * NS)];
      // go: a tile to rank. The rankers share named barrier 1, so they agree
      // on it (at the ranking's first barrier) before any of them leaves.
      const bool go = okf && okc && ts.chunk >= 0;
      const uint8_t* buf = stage + (size_t)s * bufsz;
      const int n_valid = go ? ts.end - ts.start : 0;
      uint32_t dig[ITEMS], rank[ITEMS];
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) dig[i] = 0;
      const int nf = go ? ts.it.pd.nfields : 0;
      for (int f = 0; f < nf; ++f) {
        const DigitField fd = ts.it.pd.f[f];
        const uint32_t* row = reinterpret_cast<const uint32_t*>(
            buf + (size_t)fd.mode * row_slot<T>(4) + ts.row[fd.mode].off);
        // every position of the row's slot is inside it (positions past the
        // tile's end read stale words and are overwritten below)
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) dig[i] |= field_bits(row[w * ITEMS * 32 + i * 32 + lane], fd);
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        if (w * ITEMS * 32 + i * 32 + lane >= n_valid) dig[i] = kRadix - 1;  // padding sorts last
      if (!block_rank<RW, ITEMS, 1>(dig, rank, S.warp_hist, S.bin_start, S.bin_count, S.rank_tmp,
                                    go)) {
        mbar_arrive(&S.ranked[j]);  // the writers see the end marker (or the abort)
        break;
      }
      const PassDesc& pd = ts.it.pd;
      const int nbins = 1 << pd.bits;
      if (ts.k == 0)  // a new chunk: its first output slot per digit (staged with the tile)
        for (int d = threadIdx.x; d < nbins; d += kWsRankThreads) S.off[d] = S.off0[s][d];
      for (int d = threadIdx.x; d < nbins; d += kWsRankThreads) {
        uint32_t cnt = S.bin_count[d];
        if (d == kRadix - 1) cnt -= (uint32_t)(T - n_valid);
        const uint32_t o = S.off[d];
        S.gbase[j][d] = o - S.bin_start[d];
        S.off[d] = o + cnt;
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i)
        S.invdig[j][rank[i]] = (dig[i] << 16) | (uint32_t)(w * ITEMS * 32 + i * 32 + lane);
      mbar_arrive(&S.ranked[j]);
    }
  } else {
    // ---------------- writers ----------------
    const int t = threadIdx.x - kWsRankThreads;
    for (int q = 0;; ++q) {
      const int s = q % NS, j = q & 1;
      if (!mbar_wait(&S.ranked[j], (q / 2) & 1, status)) break;
      const TileMeta& ts = S.meta[q % (2 * NS)];
      if (ts.chunk < 0 || S.rk_abort) break;
      // the key rows have landed (the rankers waited for them); the level
      // bytes compare every row, so then all of them must have landed first
      if (!mbar_wait(&S.kfull[s], (q / NS) & 1, status)) break;
      if (lv.lev && !mbar_wait(&S.full[s], (q / NS) & 1, status)) break;
      const uint8_t* buf = stage + (size_t)s * bufsz;
      const Cols& c = ts.it.c;
      const int n_valid = ts.end - ts.start, lo = ts.lo, hi = ts.hi;
      const unsigned kmask = ts.kmask;
      int dst_pos[WITEMS], src_idx[WITEMS];
#pragma unroll
      for (int k = 0; k < WITEMS; ++k) {
        const int p = k * kWsWriteThreads + t;
        int g = -1, i = 0;
        if (p < n_valid) {
          const uint32_t x = S.invdig[j][p];
          g = (int)(S.gbase[j][x >> 16] + (uint32_t)p);
          i = (int)(x & 0xffffu);
          if (g < lo || g >= hi) g = -1;  // never write outside the bucket
        }
        dst_pos[k] = g;
        src_idx[k] = i;
      }
      if (lv.lev) {
        // the entry written just before position g is the one at sorted
        // position p - 1 when that has the same digit (the same run of
        // consecutive destinations); compare them level by level in sigma
        // order
#pragma unroll
        for (int k = 0; k < WITEMS; ++k) {
          const int p = k * kWsWriteThreads + t;
          if (dst_pos[k] < 0) continue;
          uint32_t L = 0;
          const uint32_t x = S.invdig[j][p];
          const uint32_t y = p > 0 ? S.invdig[j][p - 1] : 0xffffffffu;
          if (p > 0 && (y >> 16) == (x >> 16)) {
            const int a = src_idx[k], b = (int)(y & 0xffffu);
            L = (uint32_t)lv.order + 1;
            for (int l = 0; l < lv.order; ++l) {
              const int m = lv.sigma[l];
              const uint32_t* row = reinterpret_cast<const uint32_t*>(
                  buf + (size_t)m * row_slot<T>(4) + ts.row[m].off);
              if (row[a] != row[b]) {
                L = (uint32_t)l + 1;
                break;
              }
            }
          }
          lv.lev[dst_pos[k]] = (uint8_t)L;
        }
      }
      auto write_row = [&](int r) {
        const uint32_t* src =
            reinterpret_cast<const uint32_t*>(buf + (size_t)r * row_slot<T>(4) + ts.row[r].off);
        int32_t* dst = c.out + (int64_t)r * c.out_stride;
#pragma unroll
        for (int k = 0; k < WITEMS; ++k)
          if (dst_pos[k] >= 0) dst[dst_pos[k]] = (int32_t)src[src_idx[k]];
      };
      // key rows first: once they are written the producer may load the
      // key rows of the slot's next tile over them
      for (int r = 0; r < c.order; ++r)
        if (kmask >> r & 1u) write_row(r);
      mbar_arrive(&S.kempty[s]);
      if (!mbar_wait(&S.full[s], (q / NS) & 1, status)) break;
      for (int r = 0; r < c.order; ++r)
        if (!(kmask >> r & 1u)) write_row(r);
      if constexpr (VB != 0) {
        using V = typename std::conditional<VB == 8, unsigned long long, uint32_t>::type;
        const V* src = reinterpret_cast<const V*>(buf + (size_t)c.order * row_slot<T>(4) +
                                                  ts.row[c.order].off);
        V* dst = static_cast<V*>(c.vout);
#pragma unroll
        for (int k = 0; k < WITEMS; ++k)
          if (dst_pos[k] >= 0) dst[dst_pos[k]] = src[src_idx[k]];
      }
      mbar_arrive(&S.consumed[j]);
      mbar_arrive(&S.empty[s]);
    }
  }
}

template <int T, int NS, int VB, int RW>
size_t ws_smem(int order) {
  return ws_header<T, NS, RW>() + NS * ws_buffer<T, VB>(order);
}

template <int T, int NS, int VB, int RW, int WW>
cudaError_t launch_move_t(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                          const uint32_t* chunk_off, int* claim, int max_chunks,
                          unsigned* status, const PassBatch& pb, cudaStream_t stream,
                          const LevOut& lv) {
  const size_t smem = ws_smem<T, NS, VB, RW>(c.order);
  cudaError_t e = cudaFuncSetAttribute(k_digit_move<T, NS, VB, RW, WW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = sm_count();
  if (grid > max_chunks) grid = max_chunks;
  if (grid < 1) grid = 1;
  PassTensor one;
  one.c = c;
  one.pd = pd;
  k_digit_move<T, NS, VB, RW, WW><<<grid, Roles<RW, WW>::kThreads, smem, stream>>>(
      one, c.order, ls, chunk_off, claim, status, pb, lv);
  return cudaGetLastError();
}

// Ring depth for a tile size: three staging buffers when they fit 227 KB of
// shared memory, else two. Tiles of 4096 and 2048 entries use 16 ranking and
// 15 writing warps, tiles of 1024 entries 8 and 8.
template <int VB>
cudaError_t launch_move_vb(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                           const uint32_t* chunk_off, int* claim, int max_chunks,
                           unsigned* status, const PassBatch& pb, cudaStream_t stream,
                           const LevOut& lv) {
  constexpr size_t kMax = 227 * 1024;
#define QSD_MV(T_, NS_, RW_, WW_)                                                      \
  return launch_move_t<T_, NS_, VB, RW_, WW_>(c, ls, pd, chunk_off, claim, max_chunks, status, \
                                              pb, stream, lv)
  if (ls.tile == 4096) {
    if (ws_smem<4096, 3, VB, 16>(c.order) <= kMax) QSD_MV(4096, 3, 16, 15);
    QSD_MV(4096, 2, 16, 15);
  }
  if (ls.tile == 3584) {
    if (ws_smem<3584, 3, VB, 16>(c.order) <= kMax) QSD_MV(3584, 3, 16, 15);
    QSD_MV(3584, 2, 16, 15);
  }
  if (ls.tile == 2048) {
    if (ws_smem<2048, 3, VB, 16>(c.order) <= kMax) QSD_MV(2048, 3, 16, 15);
    QSD_MV(2048, 2, 16, 15);
  }
  if (ws_smem<1024, 3, VB, 8>(c.order) <= kMax) QSD_MV(1024, 3, 8, 8);
  QSD_MV(1024, 2, 8, 8);
#undef QSD_MV
}

}  // namespace

// Entries per tile. A requested size (4096, 3584, 2048 or 1024) is honoured
// if its two-slot ring fits 227 KB of shared memory, else the next smaller
// one that fits. Automatically: the largest of 4096 and 3584 entries whose
// three-slot ring fits (a third slot lets the loads run two tiles ahead;
// measured faster than two slots of a larger tile), else the largest tile
// whose two-slot ring fits.
int digit_tile(int order, int vbytes, int tile) {
  auto rows = [&](int T) {
    return (size_t)order * (T * 4 + 16) + (vbytes ? (size_t)T * vbytes + 16 : 0);
  };
  constexpr size_t kMax = 227 * 1024;
  const bool f4 = ws_header<4096, 2, 16>() + 2 * rows(4096) <= kMax;
  const bool f35 = ws_header<3584, 2, 16>() + 2 * rows(3584) <= kMax;
  const bool f2 = ws_header<2048, 2, 16>() + 2 * rows(2048) <= kMax;
  if (tile == 4096 && f4) return 4096;
  if ((tile == 3584 || tile == 4096) && f35) return 3584;
  if ((tile == 2048 || tile == 3584 || tile == 4096) && f2) return 2048;
  if (tile != 0) return 1024;
  if (ws_header<4096, 3, 16>() + 3 * rows(4096) <= kMax) return 4096;
  if (ws_header<3584, 3, 16>() + 3 * rows(3584) <= kMax) return 3584;
  if (f4) return 4096;
  if (f35) return 3584;
  if (f2) return 2048;
  return 1024;
}

// Entries per chunk: chunk_tiles tiles (default 2: of 1, 2, 4, 6 and 8 the
// fastest on the single-call and the batched workloads), at most 256.
int digit_chunk(int order, int vbytes, int tile, int chunk_tiles) {
  const int k = chunk_tiles >= 1 && chunk_tiles <= 256 ? chunk_tiles : 2;
  return k * digit_tile(order, vbytes, tile);
}

cudaError_t launch_chunk_hist(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                              uint32_t* chunk_hist, uint32_t* group_sum, int* claim,
                              int max_chunks, const PassBatch& pb, cudaStream_t stream) {
  int grid = sm_count() * 8;
  if (grid > max_chunks) grid = max_chunks;
  if (grid < 1) grid = 1;
  PassTensor one;
  one.c = c;
  one.pd = pd;
  k_chunk_hist<<<grid, kHistThreads, 0, stream>>>(one, ls, chunk_hist, group_sum, claim, pb);
  return cudaGetLastError();
}

cudaError_t launch_chunk_scan(const LargeSegs& ls, uint32_t* chunk_hist,
                              uint32_t* group_sum, int max_groups, const PassBatch& pb,
                              cudaStream_t stream) {
  int grid = sm_count() * 8;
  if (grid > max_groups) grid = max_groups;
  if (grid < 1) grid = 1;
  // with few groups each block's own sum over them is cheaper than a launch more
  const int prefixed = ls.single && !pb.t && max_groups > 16;
  if (prefixed) {
    k_group_prefix<<<1, kRadix * kPrefixParts, 0, stream>>>(ls, group_sum);
    int g4 = 2 * sm_count();
    if (g4 > max_groups) g4 = max_groups;
    k_chunk_scan_parts<<<g4, kRadix * kScanParts, 0, stream>>>(ls, chunk_hist, group_sum);
    return cudaGetLastError();
  }
  k_chunk_scan<<<grid, kRadix, 0, stream>>>(ls, chunk_hist, group_sum, pb);
  return cudaGetLastError();
}

cudaError_t debug_words_digit_pass(unsigned long long limit_ns, int stall) {
  return set_debug_words(limit_ns, stall);
}

cudaError_t launch_digit_move(const Cols& c, const LargeSegs& ls, const PassDesc& pd,
                              const uint32_t* chunk_off, int* claim, int max_chunks,
                              unsigned* status, const PassBatch& pb, cudaStream_t stream,
                              const LevOut* lvp) {
  LevOut lv;
  if (lvp && !pb.t) {
    lv = *lvp;
  } else {
    lv.lev = nullptr;
    lv.order = 0;
  }
  switch (c.vbytes) {
    case 0: return launch_move_vb<0>(c, ls, pd, chunk_off, claim, max_chunks, status, pb, stream, lv);
    case 4: return launch_move_vb<4>(c, ls, pd, chunk_off, claim, max_chunks, status, pb, stream, lv);
    case 8: return launch_move_vb<8>(c, ls, pd, chunk_off, claim, max_chunks, status, pb, stream, lv);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qsd
