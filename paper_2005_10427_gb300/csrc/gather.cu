// Row copy / gather kernels: move every coordinate row and the values of a
// COO tensor through a permutation (or the identity), with 128-bit accesses
// where the rows are 16-byte aligned.
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

}  // namespace

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
