// The paper's CPU method, restated in C++ for timing on the host cores (bench
// and test infrastructure; it shares no code with the CUDA library). It is
// not the oracle: the oracle is the stable sort of the definition, and the
// tests check this method against it.
//
// Algorithm 3 (QuesadillaSort) gives the PartialSort calls; each call runs as
//   - no prefix (l = 0): Algorithm 1, a stable counting sort of the whole
//     tensor by one mode. In parallel, as Section 3.2 describes: every thread
//     counts its contiguous block with private counts, the counts are summed
//     per value in (value, thread) order, and every thread places its block.
//   - prefix of length l > 0: Algorithm 2, the same stable sort inside every
//     bucket of equal prefix coordinates. In parallel along bucket
//     boundaries (Section 3.2): threads take whole buckets; each bucket is
//     counting-sorted over the range of coordinates it holds.
// The sorts permute an index array; the rows and values are gathered once at
// the end.
//
// Top-K-sadilla (Section 3.6), qsd_cpu_method_transpose_topk: the calls of
// Algorithm 3 that sort to the order of the first K target modes (the other
// modes in their input order), then every bucket of equal (sigma_1..sigma_K)
// sorted completely by the remaining target modes with a comparison sort,
// buckets spread over the threads. The section's quicksort is not stable;
// std::stable_sort stands in so that duplicate coordinates keep their input
// order here as on every other path.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Call {
  int prefix_len;
  int mode;
};

// Algorithm 3's calls for input order tau and target sigma (0-based): the
// scan runs over sigma_{l+1}.. while the mode needs sorting (Section 3.4:
// f(sigma, m) is not a subset of f(tau, m)), and the calls of one prefix are
// made from sigma_k down to sigma_{l+1}.
std::vector<Call> quesadilla_calls(int r, const int* tau, const int* sigma) {
  unsigned f_tau[16] = {0}, f_sigma[16] = {0};
  for (int i = 0; i < r; ++i)
    for (int j = i + 1; j < r; ++j) {
      f_tau[tau[i]] |= 1u << tau[j];
      f_sigma[sigma[i]] |= 1u << sigma[j];
    }
  auto needs = [&](int m) { return (f_sigma[m] & ~f_tau[m]) != 0; };
  std::vector<Call> calls;
  int l = 0;
  while (l < r) {
    int k = l;
    while (k + 1 < r && needs(sigma[k])) ++k;  // sigma[k] is sigma_{k+1} (1-based)
    for (int kk = k; kk > l; --kk) calls.push_back({l, sigma[kk - 1]});
    l = k + 1;
  }
  return calls;
}

int nthreads_of(int want) {
#ifdef _OPENMP
  return want > 0 ? want : omp_get_max_threads();
#else
  (void)want;
  return 1;
#endif
}

// Algorithm 1 in parallel: stable counting sort of idx by key[idx[j]].
void counting_sort_all(const int32_t* key, int64_t dim, std::vector<uint32_t>& idx,
                       std::vector<uint32_t>& tmp, int T) {
  const int64_t n = (int64_t)idx.size();
  std::vector<std::vector<uint32_t>> cnt(T, std::vector<uint32_t>(dim, 0));
#pragma omp parallel num_threads(T)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num();
#else
    const int t = 0;
#endif
    const int64_t lo = n * t / T, hi = n * (t + 1) / T;
    std::vector<uint32_t>& c = cnt[t];
    for (int64_t j = lo; j < hi; ++j) ++c[key[idx[j]]];
#pragma omp barrier
#pragma omp single
    {
      uint32_t run = 0;  // exclusive sum in (value, thread) order
      for (int64_t v = 0; v < dim; ++v)
        for (int u = 0; u < T; ++u) {
          const uint32_t x = cnt[u][v];
          cnt[u][v] = run;
          run += x;
        }
    }
    for (int64_t j = lo; j < hi; ++j) tmp[c[key[idx[j]]]++] = idx[j];
  }
  idx.swap(tmp);
}

// Bucket starts of idx under the prefix modes (entries whose prefix differs
// from the entry before), with n appended.
std::vector<int64_t> bucket_starts(const int32_t* const* prefix, int plen,
                                   const std::vector<uint32_t>& idx) {
  const int64_t n = (int64_t)idx.size();
  std::vector<int64_t> starts;
  for (int64_t j = 0; j < n; ++j) {
    bool s = j == 0;
    for (int q = 0; q < plen && !s; ++q) s = prefix[q][idx[j]] != prefix[q][idx[j - 1]];
    if (s) starts.push_back(j);
  }
  starts.push_back(n);
  return starts;
}

// Algorithm 2 in parallel: the same sort inside every bucket of equal prefix.
void counting_sort_buckets(const int32_t* const* prefix, int plen, const int32_t* key,
                           std::vector<uint32_t>& idx, std::vector<uint32_t>& tmp, int T) {
  const std::vector<int64_t> starts = bucket_starts(prefix, plen, idx);
  const int64_t nb = (int64_t)starts.size() - 1;
#pragma omp parallel num_threads(T)
  {
    std::vector<int64_t> c;
#pragma omp for schedule(dynamic, 64)
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t a = starts[b], e = starts[b + 1];
      if (e - a < 2) {
        if (e > a) tmp[a] = idx[a];
        continue;
      }
      int32_t vmin = key[idx[a]], vmax = vmin;
      for (int64_t j = a; j < e; ++j) {
        vmin = std::min(vmin, key[idx[j]]);
        vmax = std::max(vmax, key[idx[j]]);
      }
      if ((int64_t)vmax - vmin > 4 * (e - a) + 1024) {
        // a few entries over a wide range: counting would mostly clear empty
        // bins, so a stable comparison sort stands in (Section 3.6: any
        // stable sort may replace the histogram sort)
        std::copy(idx.begin() + a, idx.begin() + e, tmp.begin() + a);
        std::stable_sort(tmp.begin() + a, tmp.begin() + e,
                         [&](uint32_t x, uint32_t y) { return key[x] < key[y]; });
        continue;
      }
      c.assign((size_t)(vmax - vmin) + 1, 0);
      for (int64_t j = a; j < e; ++j) ++c[key[idx[j]] - vmin];
      int64_t run = a;
      for (auto& x : c) {
        const int64_t y = x;
        x = run;
        run += y;
      }
      for (int64_t j = a; j < e; ++j) tmp[c[key[idx[j]] - vmin]++] = idx[j];
    }
  }
  idx.swap(tmp);
}

}  // namespace

extern "C" {

// Transposes (rows: mode m at coords + m * stride, sorted under tau) into
// sigma order with the paper's method on `nthreads` threads (0 = all):
// Quesadilla for top_k = 0 or top_k >= r - 1, else Top-K-sadilla with
// K = top_k. Returns 0, or -1 on bad arguments.
int qsd_cpu_method_transpose_topk(int r, int64_t nnz, const int32_t* coords, int64_t stride,
                                  const void* vals, int vb, const int64_t* dims, const int* tau,
                                  const int* sigma, int top_k, int nthreads, int32_t* out_coords,
                                  int64_t out_stride, void* out_vals) {
  if (r < 1 || r > 16 || nnz < 0 || nnz > 0xffffffffLL || (vb != 0 && vb != 4 && vb != 8) ||
      top_k < 0)
    return -1;
  const int T = nthreads_of(nthreads);
  // the ordering Algorithm 3 sorts to: sigma itself, or for Top-K the first
  // K target modes followed by the others in their tau order
  const int K = top_k > 0 && top_k < r - 1 ? top_k : r;
  int target[16];
  {
    unsigned head = 0;
    int m = 0;
    for (int i = 0; i < K && i < r; ++i) {
      target[m++] = sigma[i];
      head |= 1u << sigma[i];
    }
    for (int i = 0; i < r && K < r; ++i)
      if (!(head >> tau[i] & 1u)) target[m++] = tau[i];
  }
  bool complete_sort = false;
  for (int i = 0; i < r; ++i) complete_sort |= target[i] != sigma[i];
  std::vector<uint32_t> idx((size_t)nnz), tmp((size_t)nnz);
  for (int64_t j = 0; j < nnz; ++j) idx[j] = (uint32_t)j;
  for (const Call& c : quesadilla_calls(r, tau, target)) {
    const int32_t* key = coords + (int64_t)c.mode * stride;
    if (c.prefix_len == 0) {
      counting_sort_all(key, dims[c.mode], idx, tmp, T);
    } else {
      const int32_t* prefix[16];
      for (int q = 0; q < c.prefix_len; ++q) prefix[q] = coords + (int64_t)sigma[q] * stride;
      counting_sort_buckets(prefix, c.prefix_len, key, idx, tmp, T);
    }
  }
  if (complete_sort) {  // Top-K-sadilla's second stage
    const int32_t* prefix[16];
    for (int q = 0; q < K; ++q) prefix[q] = coords + (int64_t)sigma[q] * stride;
    const std::vector<int64_t> starts = bucket_starts(prefix, K, idx);
    const int64_t nb = (int64_t)starts.size() - 1;
    auto less = [&](uint32_t x, uint32_t y) {
      for (int q = K; q < r; ++q) {
        const int32_t* row = coords + (int64_t)sigma[q] * stride;
        if (row[x] != row[y]) return row[x] < row[y];
      }
      return false;
    };
    // buckets over the threads: dynamic scheduling for K = 1, guided for
    // K > 1 (more and smaller buckets), as the paper's evaluation does
    if (K == 1) {
#pragma omp parallel for num_threads(T) schedule(dynamic, 64)
      for (int64_t b = 0; b < nb; ++b)
        std::stable_sort(idx.begin() + starts[b], idx.begin() + starts[b + 1], less);
    } else {
#pragma omp parallel for num_threads(T) schedule(guided)
      for (int64_t b = 0; b < nb; ++b)
        std::stable_sort(idx.begin() + starts[b], idx.begin() + starts[b + 1], less);
    }
  }
#pragma omp parallel for num_threads(T)
  for (int64_t j = 0; j < nnz; ++j) {
    for (int m = 0; m < r; ++m) out_coords[(int64_t)m * out_stride + j] = coords[(int64_t)m * stride + idx[j]];
    if (vb)
      std::memcpy(static_cast<uint8_t*>(out_vals) + (size_t)j * vb,
                  static_cast<const uint8_t*>(vals) + (size_t)idx[j] * vb, vb);
  }
  return 0;
}

int qsd_cpu_method_transpose(int r, int64_t nnz, const int32_t* coords, int64_t stride,
                             const void* vals, int vb, const int64_t* dims, const int* tau,
                             const int* sigma, int nthreads, int32_t* out_coords,
                             int64_t out_stride, void* out_vals) {
  return qsd_cpu_method_transpose_topk(r, nnz, coords, stride, vals, vb, dims, tau, sigma, 0,
                                       nthreads, out_coords, out_stride, out_vals);
}

int qsd_cpu_method_threads(int nthreads) { return nthreads_of(nthreads); }

}  // extern "C"
