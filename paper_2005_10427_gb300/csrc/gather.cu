// Row copy, key packing and gather kernels.
//
// k_copy    moves every coordinate row and the values unchanged (a plan with
//           no pass, asked for a distinct output);
// k_pack    writes, for a group sorted in (key, index) form, every entry's
//           packed key (one or two 32-bit words) and its index as rows;
// k_gather  moves every coordinate row and the values once through the
//           sorted index: out[j] = in[idx[j]] (Algorithm 2's perm array
//           applied to the records), with 128-bit stores of four
//           consecutive outputs where the rows are 16-byte aligned.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"

namespace qsd {

namespace {

constexpr int kCopyThreads = 256;

// One grid-stride pass per row; rows are copied with int4 when the base
// addresses of both rows are 16-byte aligned, else element by element.
__global__ void __launch_bounds__(kCopyThreads)
k_copy(Cols c, int nnz) {
  const int nrows = c.order + (c.vbytes ? 1 : 0);
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  for (int m = 0; m < nrows; ++m) {
    const uint8_t* src;
    uint8_t* dst;
    int64_t bytes;
    if (m < c.order) {
      src = reinterpret_cast<const uint8_t*>(c.in + (int64_t)m * c.in_stride);
      dst = reinterpret_cast<uint8_t*>(c.out + (int64_t)m * c.out_stride);
      bytes = (int64_t)nnz * 4;
    } else {
      src = static_cast<const uint8_t*>(c.vin);
      dst = static_cast<uint8_t*>(c.vout);
      bytes = (int64_t)nnz * c.vbytes;
    }
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    int64_t done = 0;
    if (vec) {
      const int64_t n16 = bytes / 16;
      const int4* s4 = reinterpret_cast<const int4*>(src);
      int4* d4 = reinterpret_cast<int4*>(dst);
      for (int64_t i = tid; i < n16; i += nthr) d4[i] = __ldcs(s4 + i);
      done = n16 * 16;
    }
    const int64_t nw = (bytes - done) / 4;
    const uint32_t* s1 = reinterpret_cast<const uint32_t*>(src + done);
    uint32_t* d1 = reinterpret_cast<uint32_t*>(dst + done);
    for (int64_t i = tid; i < nw; i += nthr) d1[i] = s1[i];
  }
}

constexpr int kPackThreads = 256;

// Each thread takes four consecutive entries j0 .. j0 + 3.
__global__ void __launch_bounds__(kPackThreads)
k_pack(const __grid_constant__ Cols c, const __grid_constant__ KeyPack kp, int nnz) {
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const bool vin = (c.in_stride & 3) == 0 && (reinterpret_cast<uintptr_t>(c.in) & 15) == 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q * 4 < nnz; q += nthr) {
    const int j0 = (int)(q * 4);
    const bool full = j0 + 4 <= nnz;
    unsigned long long key[4] = {0, 0, 0, 0};
    for (int i = 0; i < kp.nkeys; ++i) {
      const int32_t* row = c.in + (int64_t)kp.mode[i] * c.in_stride + j0;
      uint32_t v[4];
      if (full && vin) {
        const uint4 x = __ldcs(reinterpret_cast<const uint4*>(row));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = j0 + e < nnz ? (uint32_t)__ldcs(row + e) : 0u;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) key[e] |= (unsigned long long)v[e] << kp.base[i];
    }
    // rows: key bits 0..31, key bits 32..63 (two-word keys), the entry index
    uint32_t* out = reinterpret_cast<uint32_t*>(c.out);
    const int64_t st = c.out_stride;  // a multiple of 4, 16-byte-aligned rows
    if (full) {
      *reinterpret_cast<uint4*>(out + j0) =
          make_uint4((uint32_t)key[0], (uint32_t)key[1], (uint32_t)key[2], (uint32_t)key[3]);
      if (kp.words == 2)
        *reinterpret_cast<uint4*>(out + st + j0) =
            make_uint4((uint32_t)(key[0] >> 32), (uint32_t)(key[1] >> 32),
                       (uint32_t)(key[2] >> 32), (uint32_t)(key[3] >> 32));
      *reinterpret_cast<uint4*>(out + kp.words * st + j0) = make_uint4(j0, j0 + 1, j0 + 2, j0 + 3);
    } else {
      for (int e = 0; e < 4 && j0 + e < nnz; ++e) {
        out[j0 + e] = (uint32_t)key[e];
        if (kp.words == 2) out[st + j0 + e] = (uint32_t)(key[e] >> 32);
        out[kp.words * st + j0 + e] = (uint32_t)(j0 + e);
      }
    }
  }
}

// Each thread takes four consecutive outputs j0 .. j0 + 3: their input
// indices, then per row four reads through them and one 16-byte store (or
// four stores where a row is not 16-byte aligned or at the end).
template <int VB>
__global__ void __launch_bounds__(kPackThreads)
k_gather(const __grid_constant__ Cols c, const int32_t* __restrict__ idx, int nnz) {
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const bool vout = (c.out_stride & 3) == 0 && (reinterpret_cast<uintptr_t>(c.out) & 15) == 0 &&
                    (VB == 0 || (reinterpret_cast<uintptr_t>(c.vout) & 15) == 0);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q * 4 < nnz; q += nthr) {
    const int j0 = (int)(q * 4);
    const bool full = j0 + 4 <= nnz;
    int src[4];
    if (full) {  // the index row is 16-byte aligned (workspace, stride a multiple of 4)
      const int4 x = __ldcs(reinterpret_cast<const int4*>(idx + j0));
      src[0] = x.x; src[1] = x.y; src[2] = x.z; src[3] = x.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) src[e] = j0 + e < nnz ? idx[j0 + e] : 0;
    }
    const bool vec = full && vout;
    for (int m = 0; m < c.order; ++m) {
      const int32_t* in = c.in + (int64_t)m * c.in_stride;
      int32_t* out = c.out + (int64_t)m * c.out_stride + j0;
      int32_t v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (full || j0 + e < nnz) ? __ldg(in + src[e]) : 0;
      if (vec) {
        __stcs(reinterpret_cast<int4*>(out), make_int4(v[0], v[1], v[2], v[3]));
      } else {
        for (int e = 0; e < 4 && j0 + e < nnz; ++e) out[e] = v[e];
      }
    }
    if constexpr (VB == 4) {
      const uint32_t* in = static_cast<const uint32_t*>(c.vin);
      uint32_t* out = static_cast<uint32_t*>(c.vout) + j0;
      uint32_t v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (full || j0 + e < nnz) ? __ldg(in + src[e]) : 0u;
      if (vec) {
        __stcs(reinterpret_cast<uint4*>(out), make_uint4(v[0], v[1], v[2], v[3]));
      } else {
        for (int e = 0; e < 4 && j0 + e < nnz; ++e) out[e] = v[e];
      }
    } else if constexpr (VB == 8) {
      const unsigned long long* in = static_cast<const unsigned long long*>(c.vin);
      unsigned long long* out = static_cast<unsigned long long*>(c.vout) + j0;
      unsigned long long v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (full || j0 + e < nnz) ? __ldg(in + src[e]) : 0ull;
      if (vec) {
        __stcs(reinterpret_cast<ulonglong2*>(out), make_ulonglong2(v[0], v[1]));
        __stcs(reinterpret_cast<ulonglong2*>(out) + 1, make_ulonglong2(v[2], v[3]));
      } else {
        for (int e = 0; e < 4 && j0 + e < nnz; ++e) out[e] = v[e];
      }
    }
  }
}

int grid_for(int nnz, int per_thread) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = ((int64_t)nnz / per_thread + kPackThreads) / kPackThreads;
  const int64_t cap = (int64_t)sms * 16;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_pack(const Cols& c, const KeyPack& kp, int nnz, cudaStream_t stream) {
  if (nnz <= 0) return cudaSuccess;
  k_pack<<<grid_for(nnz, 4), kPackThreads, 0, stream>>>(c, kp, nnz);
  return cudaGetLastError();
}

cudaError_t launch_gather(const Cols& c, const int32_t* idx, int nnz, cudaStream_t stream) {
  if (nnz <= 0) return cudaSuccess;
  const int grid = grid_for(nnz, 4);
  switch (c.vbytes) {
    case 0: k_gather<0><<<grid, kPackThreads, 0, stream>>>(c, idx, nnz); break;
    case 4: k_gather<4><<<grid, kPackThreads, 0, stream>>>(c, idx, nnz); break;
    case 8: k_gather<8><<<grid, kPackThreads, 0, stream>>>(c, idx, nnz); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_copy(const Cols& c, int nnz, cudaStream_t stream) {
  if (nnz <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = ((int64_t)nnz * 4 / 16 + kCopyThreads - 1) / kCopyThreads;
  int grid = (int)(want < sms * 8 ? want : sms * 8);
  if (grid < 1) grid = 1;
  k_copy<<<grid, kCopyThreads, 0, stream>>>(c, nnz);
  return cudaGetLastError();
}

}  // namespace qsd
