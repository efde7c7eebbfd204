// Reference oracle for sparse COO tensor transposition.
//
// TEST INFRASTRUCTURE ONLY. This file is never linked into the product
// library; it is loaded by the tests, by the smoke check and by the bench's
// CPU-baseline leg, and by nothing else. It shares no code, header, table or
// helper with the CUDA path.
//
// What it computes (Section 2, "Background" and "Transposition"): a COO
// tensor is a list of r-tuples with values; transposing it to the complete
// ordering sigma means re-sorting the list into lexicographic order under
// sigma, where i <_sigma i' iff i[sigma_1] < i'[sigma_1], or the two agree
// there and i <_(sigma_2, ...) i'. The histogram partial sorts the method is
// built from are stable (Section 3.1, and Section 3.6 notes any stable sort
// may replace them), so entries with equal coordinates keep their input
// order. The result is therefore exactly the STABLE sort of the input under
// the sigma-lexicographic comparator, which is what this file writes out
// with std::stable_sort (a library sort used as a single step).
//
// Layout: coordinates are structure-of-arrays int32: mode m of entry j is
// coords[m * stride + j]. Values are opaque 4- or 8-byte payloads moved
// bit-for-bit (memcpy), so NaN payloads and -0.0 survive unchanged.
//
// Pins (tests/test_oracle.py): a dense brute-force transpose on tiny tensors,
// numpy.lexsort, the worked example of Section 3.3, and the invariants
// (permutation of the input multiset, sigma-sorted, ties in input order).

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

struct SigmaLess {
  int order;
  const int32_t* coords;
  int64_t stride;
  const int* sigma;
  bool operator()(int64_t a, int64_t b) const {
    // Lexicographic comparison under sigma (Section 2): the first mode of
    // sigma decides unless equal, then the next, and so on.
    for (int p = 0; p < order; ++p) {
      const int32_t* col = coords + (int64_t)sigma[p] * stride;
      int32_t x = col[a], y = col[b];
      if (x < y) return true;
      if (x > y) return false;
    }
    return false;  // equal under every mode: not less
  }
};

bool valid_perm(int order, const int* p) {
  if (order < 1 || order > 64) return false;
  std::vector<int> seen(order, 0);
  for (int i = 0; i < order; ++i) {
    if (p[i] < 0 || p[i] >= order || seen[p[i]]) return false;
    seen[p[i]] = 1;
  }
  return true;
}

}  // namespace

extern "C" {

// Writes into perm_out[0..nnz) the input index of each output entry of the
// stable sigma-lexicographic sort. Returns 0 on success, -1 on bad arguments.
int qsd_oracle_permutation(int order, int64_t nnz, const int32_t* coords,
                           int64_t stride, const int* sigma,
                           int64_t* perm_out) {
  if (nnz < 0 || !valid_perm(order, sigma)) return -1;
  if (nnz == 0) return 0;
  if (!coords || !perm_out || stride < nnz) return -1;
  std::iota(perm_out, perm_out + nnz, (int64_t)0);
  std::stable_sort(perm_out, perm_out + nnz,
                   SigmaLess{order, coords, stride, sigma});
  return 0;
}

// Transposes (coords, vals) into (out_coords, out_vals): the entries of the
// input re-sorted stably into sigma-lexicographic order. Mode labels are kept:
// out_coords row m is still mode m. val_bytes is 4 or 8 (or 0: no values).
// Returns 0 on success, -1 on bad arguments.
int qsd_oracle_transpose(int order, int64_t nnz, const int32_t* coords,
                         int64_t stride, const void* vals, int val_bytes,
                         const int* sigma, int32_t* out_coords,
                         int64_t out_stride, void* out_vals) {
  if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return -1;
  if (nnz < 0 || !valid_perm(order, sigma)) return -1;
  if (nnz == 0) return 0;
  if (!out_coords || out_stride < nnz) return -1;
  if (val_bytes && (!vals || !out_vals)) return -1;
  std::vector<int64_t> perm((size_t)nnz);
  int rc = qsd_oracle_permutation(order, nnz, coords, stride, sigma,
                                  perm.data());
  if (rc) return rc;
  for (int m = 0; m < order; ++m) {
    const int32_t* src = coords + (int64_t)m * stride;
    int32_t* dst = out_coords + (int64_t)m * out_stride;
    for (int64_t j = 0; j < nnz; ++j) dst[j] = src[perm[(size_t)j]];
  }
  if (val_bytes) {
    const unsigned char* src = (const unsigned char*)vals;
    unsigned char* dst = (unsigned char*)out_vals;
    for (int64_t j = 0; j < nnz; ++j)
      std::memcpy(dst + j * val_bytes, src + perm[(size_t)j] * val_bytes,
                  (size_t)val_bytes);
  }
  return 0;
}

}  // extern "C"
