// Device helpers shared by the kernels: status word, bounded waits, bulk
// copies, radix digit extraction and a stable block-wide ranking of radix
// digits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qsd_internal.h"

namespace qsd {

// ---------------------------------------------------------------------------
// Status word: the first error recorded wins; kernels never trap.
__device__ __forceinline__ void set_status(unsigned* status, unsigned code) {
  if (status) atomicCAS(status, 0u, code);
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Every spin in this library gives up after a limit (2 s by default; a
// legitimate wait lasts microseconds) and records QSD_ERR_TIMEOUT. Without
// relocatable device code each translation unit holds its own copy of these
// words; qsd_debug_set_spin_limit_ns and qsd_debug_set_stall set every copy
// through each unit's set_debug_words().
constexpr uint64_t kSpinLimitNs = 2000000000ull;  // 2 s
static __device__ unsigned long long g_spin_limit_ns = kSpinLimitNs;
// Test-only: 1 = the first tile the move kernel's block 0 stages is armed
// for its bulk copies but none is issued, so every wait on that staging slot
// expires (the abort path of the bounded waits runs).
static __device__ int g_debug_stall = 0;

// Host side: sets this translation unit's copies on the current device.
static inline cudaError_t set_debug_words(unsigned long long limit_ns, int stall) {
  cudaError_t e = cudaMemcpyToSymbol(g_spin_limit_ns, &limit_ns, sizeof(limit_ns));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_debug_stall, &stall, sizeof(stall));
  return e;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine, non-tensor form) into shared memory,
// completed on an mbarrier. Addresses and sizes must be multiples of 16 B.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One arrival that also announces `bytes` of incoming transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// A plain arrival (no transaction count).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
      "selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete. Returns false
// (and records QSD_ERR_TIMEOUT) if it did not within kSpinLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  const uint64_t limit = *(volatile unsigned long long*)&g_spin_limit_ns;
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit) {
      set_status(status, QSD_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Radix digit of one entry for one pass: OR of bit slices of its coordinates.
__device__ __forceinline__ uint32_t field_bits(uint32_t c, const DigitField& f) {
  return ((c >> f.shift) & ((1u << f.width) - 1u)) << f.dst;
}

// ---------------------------------------------------------------------------
// Stable block-wide ranking of kRadix-valued digits.
//
// Thread (warp w, lane l) holds ITEMS digits; item i is element
// w*ITEMS*32 + i*32 + l of the tile ("warp-striped"), so the warps cover
// consecutive ranges and each warp's rounds consecutive 32-element pieces.
// On return rank[i] is the element's position when the tile is stably sorted
// by digit; s_bin_start[d] / s_bin_count[d] give each digit's run.
// Inside a round, the lanes holding equal digits (a lane's peers) come from
// one ballot for lane 0's digit and a per-warp table of lane masks for the
// rest (a warp match instruction's cost grows with the number of distinct
// digits in the warp, eight ballots per round cost twice the table; both
// measured on this GPU). A per-warp running count per digit in shared memory
// orders the rounds.
// Barrier over the first NTHREADS threads: the whole block when BAR == 0,
// else named barrier BAR.
template <int BAR, int NTHREADS>
__device__ __forceinline__ void group_sync() {
  if constexpr (BAR == 0) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NTHREADS) : "memory");
  }
}

// True on every participant when `pred` holds on all of the first NTHREADS
// threads (named barrier BAR with an AND reduction): a group that must leave
// a loop together decides it here.
template <int BAR, int NTHREADS>
__device__ __forceinline__ bool group_all(bool pred) {
  unsigned r;
  asm volatile(
      "{ .reg .pred q, r; setp.ne.u32 q, %1, 0; bar.red.and.pred r, %2, %3, q; "
      "selp.u32 %0, 1, 0, r; }"
      : "=r"(r)
      : "r"((unsigned)pred), "n"(BAR), "n"(NTHREADS)
      : "memory");
  return r != 0;
}

// With BAR != 0 the ranking threads are the first NWARPS warps of the block
// and synchronise on named barrier BAR only (other warps of the block may be
// doing other work). Returns whether `ok` held on every ranking thread
// (reduced at the ranking's first barrier, so a group can agree to stop at
// no extra cost).
//
// After the per-warp counts, one block-wide exclusive scan over the counters
// taken digit-major (digit d's counters of warps 0..NWARPS-1, then digit d+1's)
// gives every (digit, warp) pair its first sorted position: thread t reads the
// counters of digit t / TPD for 8 consecutive warps (TPD = NWARPS / 8 threads
// per digit), so the scan is 8 independent loads per thread and one scan of
// one value per thread.
template <int NWARPS, int ITEMS, int BAR = 0>
__device__ __forceinline__ bool block_rank(const uint32_t (&dig)[ITEMS],
                                           uint32_t (&rank)[ITEMS],
                                           uint32_t* s_warp_hist,  // [NWARPS][kRadix]
                                           uint32_t* s_bin_start,  // [kRadix]
                                           uint32_t* s_bin_count,  // [kRadix]
                                           uint32_t* s_tmp,        // [NWARPS]
                                           bool ok = true)
{
  static_assert(NWARPS % 8 == 0, "8 warps per scanning thread: NWARPS * 32 == kRadix * TPD");
  constexpr int TPD = NWARPS / 8;  // scanning threads per digit
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  uint32_t* h = s_warp_hist + w * kRadix;  // the warp's counters, then its offsets
#pragma unroll
  for (int k = lane; k < kRadix; k += 32) h[k] = 0;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  // Peers of each round: the lanes that share lane 0's digit from one
  // ballot; every other lane ORs its bit into the warp's (zeroed) table slot
  // for its digit, reads the slot back and clears it again, so the table is
  // zero afterwards for the counts. Measured on this GPU against eight
  // ballots per round: fewer cycles on every digit distribution tried
  // (uniform to one value per round), since a round rarely holds many
  // distinct digits other than its most common one in large groups.
  uint32_t peers[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const bool e = dig[i] == __shfl_sync(0xffffffffu, dig[i], 0);
    const uint32_t z = __ballot_sync(0xffffffffu, e);
    if (!e) atomicOr(&h[dig[i]], 1u << lane);
    __syncwarp();
    peers[i] = e ? z : h[dig[i]];
    __syncwarp();
    if (!e) h[dig[i]] = 0;
    __syncwarp();
  }
  // one leader per digit and round adds the round's count to the warp's
  // counter; shared atomics of one warp to one address apply in issue order,
  // so each round sees the counts of the rounds before it
  uint32_t old[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    old[i] = 0;
    if (lane == __ffs(peers[i]) - 1) old[i] = atomicAdd(&h[dig[i]], (uint32_t)__popc(peers[i]));
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i)
    rank[i] = __shfl_sync(0xffffffffu, old[i], __ffs(peers[i]) - 1) + __popc(peers[i] & lt);
  bool all_ok;
  if constexpr (BAR == 0)
    all_ok = __syncthreads_and(ok) != 0;
  else
    all_ok = group_all<BAR, NWARPS * 32>(ok);
  // digit-major scan: thread t owns digit d = t / TPD, warps w0 .. w0 + 7
  const int d = threadIdx.x / TPD, w0 = (threadIdx.x % TPD) * 8;
  uint32_t c[8], local = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = s_warp_hist[(w0 + k) * kRadix + d];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t x = c[k];
    c[k] = local;  // exclusive within the thread's 8 warps
    local += x;
  }
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_tmp[w] = incl;
  // every counter has been read: from here the same words hold offsets
  group_sync<BAR, NWARPS * 32>();
  uint32_t wt = lane < NWARPS ? s_tmp[lane] : 0u;
#pragma unroll
  for (int o = 1; o < NWARPS; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, wt, o);
    if (lane >= o) wt += y;
  }
  const uint32_t woff = w ? __shfl_sync(0xffffffffu, wt, w - 1) : 0u;
  const uint32_t prefix = woff + incl - local;  // sorted positions before this thread's counters
  const uint32_t dstart = __shfl_up_sync(0xffffffffu, prefix, threadIdx.x % TPD);
  const int part = threadIdx.x % TPD;
  if (part == 0) s_bin_start[d] = prefix;
  if (part == TPD - 1) s_bin_count[d] = prefix + local - (TPD > 1 ? dstart : prefix);
#pragma unroll
  for (int k = 0; k < 8; ++k) s_warp_hist[(w0 + k) * kRadix + d] = prefix + c[k];
  group_sync<BAR, NWARPS * 32>();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) rank[i] += h[dig[i]];
  return all_ok;
}

// Block-wide exclusive sum of one value per thread; returns the thread's
// exclusive prefix and writes the block total to *total.
template <int NWARPS>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t* s_tmp,
                                                        uint32_t* total) {
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_tmp[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < NWARPS ? s_tmp[lane] : 0u;
    uint32_t xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += t;
    }
    if (lane < NWARPS) s_tmp[lane] = xi - x;
    if (lane == NWARPS - 1) s_tmp[NWARPS] = xi;
  }
  __syncthreads();
  uint32_t r = s_tmp[w] + incl - v;
  *total = s_tmp[NWARPS];
  __syncthreads();
  return r;
}

}  // namespace qsd
