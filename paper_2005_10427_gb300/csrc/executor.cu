// Executor: runs a plan's groups in order (Algorithm 3's outer loop) on the
// caller's double buffers, and the C-ABI entry points around it.
//
// Per group (prefix P, key K, passes p):
//   P empty, nnz <= local capacity: one block-local sort of the whole tensor;
//   P empty otherwise: digit histogram, digit scan, p global passes;
//   P non-empty: bucket discovery over the P rows, classification, a
//     block-local sort of every small bucket and the global passes over the
//     large buckets. Buckets found once per group serve all of its passes
//     (the paper's conclusion: discover the buckets once per prefix).
// The group's result lands in the buffer the global passes end in; the
// block-local sort writes straight there (in place when that is the input
// buffer). No step synchronises with the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include "kernels.cuh"

namespace qsd {
int seg_lookback_words(int nnz);
}

namespace {

using namespace qsd;

constexpr size_t kAlign = 256;
constexpr int64_t kMaxNnz = (int64_t(1) << 30) - 1;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  size_t status, counters, seg_start, seg_lb, large, chunk_base, group_base, chunk_owner,
      group_owner, chunk_hist, group_sum, keyrows, total;
  int max_large, max_chunks, max_groups, max_passes;
  int64_t key_stride;  // elements per (key, index) row: nnz rounded up to 4
};

// Rows of a group in (key, index) form: its key words and the index.
int key_rows(const Group& g) { return g.key_words + 1; }

bool plan_has_prefix_group(const qsd_plan_s* p) {
  for (int g = 0; g < p->ngroups; ++g)
    if (p->groups[g].npasses > 0 && p->groups[g].prefix_len > 0) return true;
  return false;
}

Layout layout_for(const qsd_plan_s* p, int64_t nnz, int vbytes) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  const int CH = digit_chunk(p->order, vbytes, p->opts.tile, p->opts.chunk_tiles);
  const int C = local_sort_capacity(p->local_capacity, p->order, vbytes);
  int maxp = 0;
  for (int g = 0; g < p->ngroups; ++g) maxp = std::max(maxp, p->groups[g].npasses);
  L.max_passes = std::max(maxp, 1);
  const int64_t n = std::max<int64_t>(nnz, 1);
  const bool segs = plan_has_prefix_group(p);
  L.max_large = segs ? (int)(n / (C + 1) + 1) : 1;
  L.max_chunks = (int)((n + CH - 1) / CH + L.max_large);
  int krows = 0;  // (key, index) groups: rows and their own chunk length
  for (int g = 0; g < p->ngroups; ++g) {
    if (!p->groups[g].key_index) continue;
    const int W = key_rows(p->groups[g]);
    krows = std::max(krows, W);
    const int CHk = digit_chunk(W, 0, p->opts.tile, p->opts.chunk_tiles);
    L.max_chunks = std::max(L.max_chunks, (int)((n + CHk - 1) / CHk + 1));
  }
  L.key_stride = (n + 3) & ~int64_t(3);
  L.max_groups = (L.max_chunks + kGroupChunks - 1) / kGroupChunks + L.max_large;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align_up(bytes);
    return o;
  };
  L.status = take(sizeof(unsigned));
  L.counters = take(sizeof(int) * kNumCounters);
  L.seg_start = take(segs ? sizeof(int) * (size_t)(n + 2) : 0);
  L.seg_lb = take(segs ? sizeof(uint32_t) * (size_t)seg_lookback_words((int)n) : 0);
  L.large = take(segs ? sizeof(int2) * (size_t)L.max_large : 0);
  L.chunk_base = take(segs ? sizeof(int) * (size_t)L.max_large : 0);
  L.group_base = take(segs ? sizeof(int) * (size_t)L.max_large : 0);
  L.chunk_owner = take(segs ? sizeof(int) * (size_t)L.max_chunks : 0);
  L.group_owner = take(segs ? sizeof(int) * (size_t)L.max_groups : 0);
  L.chunk_hist = take(sizeof(uint32_t) * (size_t)L.max_chunks * kRadix);
  L.group_sum = take(sizeof(uint32_t) * (size_t)L.max_passes * L.max_groups * kRadix);
  // two sets of (key, index) rows the passes alternate between
  L.keyrows = take(sizeof(int32_t) * 2 * (size_t)krows * (size_t)L.key_stride);
  L.total = off;
  return L;
}

#define QSD_CUDA(call)                      \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return QSD_ERR_CUDA; \
  } while (0)

qsd_status check_buffers(const qsd_coords* coords, const qsd_values* vals,
                         int64_t nnz, const qsd_plan_s* plan) {
  if (!coords || !plan) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > kMaxNnz) return QSD_ERR_UNSUPPORTED;
  if (coords->selector != 0 && coords->selector != 1) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > 0 && (!coords->buf[0] || !coords->buf[1])) return QSD_ERR_INVALID_ARGUMENT;
  if (coords->stride < nnz) return QSD_ERR_INVALID_ARGUMENT;
  if (vals && vals->elem_bytes != 0) {
    if (vals->elem_bytes != 4 && vals->elem_bytes != 8) return QSD_ERR_INVALID_ARGUMENT;
    if (vals->selector != 0 && vals->selector != 1) return QSD_ERR_INVALID_ARGUMENT;
    if (nnz > 0 && (!vals->buf[0] || !vals->buf[1])) return QSD_ERR_INVALID_ARGUMENT;
  }
  return QSD_OK;
}

// Where a group reads its input: one of the double buffers (idx 0/1) or a
// caller's read-only input (idx -1).
struct Src {
  const int32_t* c;
  const void* v;
  int64_t stride;
  int idx;
};

qsd_status run_plan(qsd_coords* coords, qsd_values* vals, const Src* ext,
                    int64_t nnz64, const qsd_plan_s* plan, void* ws, const Layout& L,
                    cudaStream_t st, const LevOut* lv = nullptr) {
  const int nnz = (int)nnz64;
  uint8_t* base = static_cast<uint8_t*>(ws);
  unsigned* status = reinterpret_cast<unsigned*>(base + L.status);
  int* counters = reinterpret_cast<int*>(base + L.counters);
  int* seg_start = reinterpret_cast<int*>(base + L.seg_start);
  uint32_t* seg_lb = reinterpret_cast<uint32_t*>(base + L.seg_lb);
  int2* large = reinterpret_cast<int2*>(base + L.large);
  int* chunk_base = reinterpret_cast<int*>(base + L.chunk_base);
  int* group_base = reinterpret_cast<int*>(base + L.group_base);
  int* chunk_owner = reinterpret_cast<int*>(base + L.chunk_owner);
  int* group_owner = reinterpret_cast<int*>(base + L.group_owner);
  uint32_t* chunk_hist = reinterpret_cast<uint32_t*>(base + L.chunk_hist);
  uint32_t* group_sum = reinterpret_cast<uint32_t*>(base + L.group_sum);

  QSD_CUDA(cudaMemsetAsync(base, 0, L.counters + sizeof(int) * kNumCounters, st));
  const bool has_vals = vals && vals->elem_bytes != 0;
  // values follow the coordinates buffer for buffer (selectors may differ)
  const int flipv = (!ext && has_vals) ? (vals->selector ^ coords->selector) : 0;
  auto buf_src = [&](int idx) {
    Src s;
    s.c = coords->buf[idx];
    s.v = has_vals ? vals->buf[idx ^ flipv] : nullptr;
    s.stride = coords->stride;
    s.idx = idx;
    return s;
  };
  auto cols = [&](const Src& src, int dst) {
    Cols c;
    c.in = src.c;
    c.vin = src.v;
    c.in_stride = src.stride;
    c.out = coords->buf[dst];
    c.vout = has_vals ? vals->buf[dst ^ flipv] : nullptr;
    c.out_stride = coords->stride;
    c.order = plan->order;
    c.vbytes = has_vals ? vals->elem_bytes : 0;
    return c;
  };
  Src cur = ext ? *ext : buf_src(coords->selector);
  const int64_t R = 4 * plan->order + (has_vals ? vals->elem_bytes : 0);  // bytes per entry
  auto tag = [&](const char* k, int gi, int pass, int64_t entries, int64_t bpe,
                 int complement = 0) {
    ProfTag t;
    t.kernel = k;
    t.group = gi;
    t.pass = pass;
    t.entries = entries;
    t.dev_entries = entries < 0 ? counters + kCntLargeEntries : nullptr;
    t.complement = complement;
    t.total = nnz;
    t.bytes_per_entry = bpe;
    return t;
  };
#define QSD_LAUNCH(TAG, CALL)                                     \
  do {                                                            \
    const int rec_ = prof_enabled() ? prof_begin((TAG), st) : -1; \
    const cudaError_t e_ = (CALL);                                \
    prof_end(rec_, st);                                           \
    if (e_ != cudaSuccess) return QSD_ERR_CUDA;                   \
  } while (0)
  if (plan->opts.validate)
    QSD_LAUNCH(tag("validate", -1, -1, nnz, 4 * plan->order),
               launch_validate(cur.c, cur.stride, plan->order, plan->dims, plan->tau, nnz,
                               status, st));
  const int vb = has_vals ? vals->elem_bytes : 0;
  const int T = digit_tile(plan->order, vb, plan->opts.tile);
  const int CH = digit_chunk(plan->order, vb, plan->opts.tile, plan->opts.chunk_tiles);
  const int C = local_sort_capacity(plan->local_capacity, plan->order, vb);
  // one tensor: no batch tables
  PassBatch pb1;
  std::memset(&pb1, 0, sizeof(pb1));
  LsBatch lb1;
  std::memset(&lb1, 0, sizeof(lb1));
  ClassifyBatch cb1;
  std::memset(&cb1, 0, sizeof(cb1));

  // the group whose movement leaves the entries in their final places: it
  // also writes the CSF levels when asked (lv)
  int last_moving = -1;
  for (int gi = 0; gi < plan->ngroups; ++gi)
    if (plan->groups[gi].npasses > 0) last_moving = gi;
  for (int gi = 0; gi < plan->ngroups && nnz > 0; ++gi) {
    const Group& g = plan->groups[gi];
    if (g.npasses == 0) continue;
    const LevOut* glv = gi == last_moving ? lv : nullptr;
    PassList pl;
    pl.npasses = g.npasses;
    for (int p = 0; p < g.npasses; ++p) pl.pass[p] = g.pass[p];
    const int P = g.npasses;
    const bool internal = cur.idx >= 0;

    if (g.key_index && nnz > C) {
      // (key, index) form: pack every entry's key and index into rows, sort
      // the rows with the group's digit passes, then move the coordinates
      // and values once, gathered through the sorted index.
      const int W = key_rows(g);
      const int64_t ks = L.key_stride;
      int32_t* krow[2] = {reinterpret_cast<int32_t*>(base + L.keyrows), nullptr};
      krow[1] = krow[0] + (size_t)W * ks;
      const int F = internal ? cur.idx ^ 1 : 0;
      KeyPack kp;
      std::memset(&kp, 0, sizeof(kp));
      kp.nkeys = g.nkeys;
      kp.words = g.key_words;
      for (int i = 0; i < g.nkeys; ++i) {
        kp.mode[i] = g.key_modes[i];
        kp.base[i] = g.kbase[i];
      }
      auto kcols = [&](const int32_t* in, const void* vin, int64_t in_stride, int32_t* out,
                       void* vout, int64_t out_stride, int order, int vbytes) {
        Cols c;
        c.in = in;
        c.vin = vin;
        c.in_stride = in_stride;
        c.out = out;
        c.vout = vout;
        c.out_stride = out_stride;
        c.order = order;
        c.vbytes = vbytes;
        return c;
      };
      QSD_LAUNCH(tag("pack", gi, -1, nnz, 4 * g.nkeys + 4 * W),
                 launch_pack(kcols(cur.c, nullptr, cur.stride, krow[0], nullptr, ks, plan->order,
                                   0),
                             kp, nnz, st));
      QSD_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * kNumCounters, st));
      LargeSegs ls;
      std::memset(&ls, 0, sizeof(ls));
      ls.single = 1;
      ls.nnz = nnz;
      ls.tile = digit_tile(W, 0, plan->opts.tile);
      ls.chunk = digit_chunk(W, 0, plan->opts.tile, plan->opts.chunk_tiles);
      ls.counters = counters;
      const int max_chunks = (nnz + ls.chunk - 1) / ls.chunk;
      const int max_groups = (max_chunks + kGroupChunks - 1) / kGroupChunks;
      for (int p = 0; p < P; ++p)
        QSD_CUDA(cudaMemsetAsync(group_sum + (size_t)p * L.max_groups * kRadix, 0,
                                 sizeof(uint32_t) * (size_t)max_groups * kRadix, st));
      for (int p = 0; p < P; ++p) {
        const Cols kc = kcols(krow[p & 1], nullptr, ks, krow[(p + 1) & 1], nullptr, ks, W, 0);
        uint32_t* gs = group_sum + (size_t)p * L.max_groups * kRadix;
        QSD_LAUNCH(tag("chunk_hist", gi, p, nnz, 4 * g.kpass[p].nfields),
                   launch_chunk_hist(kc, ls, g.kpass[p], chunk_hist, gs,
                                     counters + kCntClaim + 2 * p, max_chunks, pb1, st));
        QSD_LAUNCH(tag("chunk_scan", gi, p, nnz, 0),
                   launch_chunk_scan(ls, chunk_hist, gs, max_groups, pb1, st));
        QSD_LAUNCH(tag("digit_move", gi, p, nnz, 2 * 4 * W),
                   launch_digit_move(kc, ls, g.kpass[p], chunk_hist,
                                     counters + kCntClaim + 2 * p + 1, max_chunks, status, pb1,
                                     st));
      }
      const int32_t* idx = krow[P & 1] + (size_t)g.key_words * ks;
      QSD_LAUNCH(tag("gather", gi, -1, nnz, 2 * R + 4),
                 launch_gather(kcols(cur.c, cur.v, cur.stride, coords->buf[F],
                                     has_vals ? vals->buf[F ^ flipv] : nullptr, coords->stride,
                                     plan->order, has_vals ? vals->elem_bytes : 0),
                               idx, nnz, st));
      cur = buf_src(F);
      continue;
    }
    if (g.prefix_len == 0 && nnz <= C) {
      const int F = internal ? cur.idx ^ 1 : 0;
      QSD_LAUNCH(tag("local_sort", gi, -1, nnz, 2 * R),
                 launch_local_sort(cols(cur, F), pl, nullptr, counters, 1, nnz, C, status, lb1,
                                   st, glv));
      cur = buf_src(F);
      continue;
    }
    // F: the buffer the group ends in; pass p writes dst(p), the last one F.
    const int F = internal ? cur.idx ^ (P & 1) : 0;
    auto dst = [&](int p) { return F ^ ((P - 1 - p) & 1); };
    QSD_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * kNumCounters, st));
    LargeSegs ls;
    std::memset(&ls, 0, sizeof(ls));
    ls.nnz = nnz;
    ls.tile = T;
    ls.chunk = CH;
    ls.counters = counters;
    int max_chunks, max_groups;
    int64_t large_entries;  // -1: known on the device only
    if (g.prefix_len == 0) {
      ls.single = 1;
      max_chunks = (nnz + CH - 1) / CH;
      max_groups = (max_chunks + kGroupChunks - 1) / kGroupChunks;
      large_entries = nnz;
      for (int p = 0; p < P; ++p)
        QSD_CUDA(cudaMemsetAsync(group_sum + (size_t)p * L.max_groups * kRadix, 0,
                                 sizeof(uint32_t) * (size_t)max_groups * kRadix, st));
    } else {
      const int32_t* pcols[kMaxOrder];
      for (int i = 0; i < g.prefix_len; ++i)
        pcols[i] = cur.c + (int64_t)g.prefix_modes[i] * cur.stride;
      QSD_LAUNCH(tag("seg_discover", gi, -1, nnz, 4 * g.prefix_len),
                 launch_seg_discover(pcols, g.prefix_len, nnz, seg_start, seg_lb, counters,
                                     status, st));
      QSD_LAUNCH(tag("seg_classify", gi, -1, nnz, 0),
                 launch_seg_classify(seg_start, counters, nnz, C, CH, large, chunk_base,
                                     group_base, chunk_owner, group_owner, group_sum, P,
                                     L.max_groups, cb1, st));
      // small buckets: straight into F (in place when F is the input buffer)
      QSD_LAUNCH(tag("local_sort", gi, -1, -1, 2 * R, 1),
                 launch_local_sort(cols(cur, F), pl, seg_start, counters, 0, nnz, C, status,
                                   lb1, st, glv));
      ls.single = 0;
      ls.seg = large;
      ls.chunk_base = chunk_base;
      ls.group_base = group_base;
      ls.chunk_owner = chunk_owner;
      ls.group_owner = group_owner;
      max_chunks = L.max_chunks;
      max_groups = L.max_groups;
      large_entries = -1;
    }
    // Global passes over the large buckets (or the whole tensor).
    for (int p = 0; p < P; ++p) {
      const Src in = p == 0 ? cur : buf_src(dst(p - 1));
      uint32_t* gs = group_sum + (size_t)p * L.max_groups * kRadix;
      int nf = 0;  // key rows the digit is read from
      for (int k = 0; k < g.pass[p].nfields; ++k) {
        bool seen = false;
        for (int j = 0; j < k; ++j) seen |= g.pass[p].f[j].mode == g.pass[p].f[k].mode;
        nf += seen ? 0 : 1;
      }
      QSD_LAUNCH(tag("chunk_hist", gi, p, large_entries, 4 * nf),
                 launch_chunk_hist(cols(in, dst(p)), ls, g.pass[p], chunk_hist, gs,
                                   counters + kCntClaim + 2 * p, max_chunks, pb1, st));
      QSD_LAUNCH(tag("chunk_scan", gi, p, large_entries, 0),
                 launch_chunk_scan(ls, chunk_hist, gs, max_groups, pb1, st));
      QSD_LAUNCH(tag("digit_move", gi, p, large_entries, 2 * R),
                 launch_digit_move(cols(in, dst(p)), ls, g.pass[p], chunk_hist,
                                   counters + kCntClaim + 2 * p + 1, max_chunks, status, pb1,
                                   st, p == P - 1 ? glv : nullptr));
    }
    cur = buf_src(F);
  }
  if (cur.idx < 0) {  // no group moved anything: the caller wants a distinct copy
    QSD_LAUNCH(tag("copy", -1, -1, nnz, 2 * R), launch_copy(cols(cur, 0), nnz, st));
    cur = buf_src(0);
  }
#undef QSD_LAUNCH
  QSD_CUDA(launch_fold_status(status, st));
  coords->selector = cur.idx;
  if (has_vals) vals->selector = cur.idx ^ flipv;
  return QSD_OK;
}

}  // namespace

extern "C" {

qsd_status qsd_workspace_bytes(qsd_plan_t plan, int64_t nnz, size_t* bytes) {
  if (!plan || !bytes || nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > kMaxNnz) return QSD_ERR_UNSUPPORTED;
  // the tile size depends on the value width: take the largest layout
  size_t b = 0;
  for (int vb : {0, 4, 8}) b = std::max(b, layout_for(plan, nnz, vb).total);
  *bytes = b;
  return QSD_OK;
}

qsd_status qsd_transpose_ws(qsd_coords* coords, qsd_values* vals, int64_t nnz,
                            qsd_plan_t plan, void* workspace, size_t workspace_bytes,
                            void* stream) {
  qsd_status s = check_buffers(coords, vals, nnz, plan);
  if (s != QSD_OK) return s;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)))
    return QSD_ERR_INVALID_ARGUMENT;
  const Layout L = layout_for(plan, nnz, vals ? vals->elem_bytes : 0);
  if (workspace_bytes < L.total) return QSD_ERR_WORKSPACE_TOO_SMALL;
  return run_plan(coords, vals, nullptr, nnz, plan, workspace, L, (cudaStream_t)stream);
}

qsd_status qsd_transpose_from_ws(const int32_t* in_coords, int64_t in_stride,
                                 const void* in_vals, qsd_coords* out_coords,
                                 qsd_values* out_vals, int64_t nnz, qsd_plan_t plan,
                                 void* workspace, size_t workspace_bytes, void* stream) {
  qsd_status s = check_buffers(out_coords, out_vals, nnz, plan);
  if (s != QSD_OK) return s;
  const bool has_vals = out_vals && out_vals->elem_bytes != 0;
  if (nnz > 0 && (!in_coords || in_stride < nnz)) return QSD_ERR_INVALID_ARGUMENT;
  if (has_vals && nnz > 0 && !in_vals) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > 0 && (in_coords == out_coords->buf[0] || in_coords == out_coords->buf[1]))
    return QSD_ERR_INVALID_ARGUMENT;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)))
    return QSD_ERR_INVALID_ARGUMENT;
  const Layout L = layout_for(plan, nnz, has_vals ? out_vals->elem_bytes : 0);
  if (workspace_bytes < L.total) return QSD_ERR_WORKSPACE_TOO_SMALL;
  Src ext;
  ext.c = in_coords;
  ext.v = has_vals ? in_vals : nullptr;
  ext.stride = in_stride;
  ext.idx = -1;
  if (nnz == 0) {
    out_coords->selector = 0;
    if (has_vals) out_vals->selector = 0;
  }
  return run_plan(out_coords, out_vals, nnz > 0 ? &ext : nullptr, nnz, plan, workspace, L,
                  (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Transposition followed by the CSF levels of its result, the levels'
// comparisons done by the transposition's last movement.
namespace {
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

qsd_status qsd_transpose_csf_workspace_bytes(qsd_plan_t plan, int64_t nnz, size_t* bytes) {
  if (!plan || !bytes || nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > kMaxNnz) return QSD_ERR_UNSUPPORTED;
  size_t t = 0, c = 0;
  qsd_status s = qsd_workspace_bytes(plan, nnz, &t);
  if (s == QSD_OK) s = qsd_csf_workspace_bytes(plan->order, nnz, &c);
  if (s != QSD_OK) return s;
  *bytes = align256(t) + align256((size_t)nnz + 16) + c;
  return QSD_OK;
}

qsd_status qsd_transpose_csf_from_ws(const int32_t* in_coords, int64_t in_stride,
                                     const void* in_vals, qsd_coords* out_coords,
                                     qsd_values* out_vals, int64_t nnz, qsd_plan_t plan,
                                     const qsd_csf* csf, int32_t* nodes, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  if (!plan || !csf || !nodes) return QSD_ERR_INVALID_ARGUMENT;
  const int r = plan->order;
  for (int l = 0; l <= r; ++l) {
    if (!csf->ptr[l]) return QSD_ERR_INVALID_ARGUMENT;
    if (l < r && nnz > 0 && !csf->ids[l]) return QSD_ERR_INVALID_ARGUMENT;
  }
  size_t need = 0;
  qsd_status s = qsd_transpose_csf_workspace_bytes(plan, nnz, &need);
  if (s != QSD_OK) return s;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)))
    return QSD_ERR_INVALID_ARGUMENT;
  if (workspace_bytes < need) return QSD_ERR_WORKSPACE_TOO_SMALL;
  size_t tbytes = 0;
  qsd_workspace_bytes(plan, nnz, &tbytes);
  uint8_t* base = static_cast<uint8_t*>(workspace);
  uint8_t* lev = base + align256(tbytes);
  uint32_t* tile_count = reinterpret_cast<uint32_t*>(lev + align256((size_t)nnz + 16));
  cudaStream_t st = (cudaStream_t)stream;
  s = check_buffers(out_coords, out_vals, nnz, plan);
  if (s != QSD_OK) return s;
  const bool has_vals = out_vals && out_vals->elem_bytes != 0;
  if (nnz > 0 && (!in_coords || in_stride < nnz)) return QSD_ERR_INVALID_ARGUMENT;
  if (has_vals && nnz > 0 && !in_vals) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > 0 && (in_coords == out_coords->buf[0] || in_coords == out_coords->buf[1]))
    return QSD_ERR_INVALID_ARGUMENT;
  const Layout L = layout_for(plan, nnz, has_vals ? out_vals->elem_bytes : 0);
  Src ext;
  ext.c = in_coords;
  ext.v = has_vals ? in_vals : nullptr;
  ext.stride = in_stride;
  ext.idx = -1;
  if (nnz == 0) {
    out_coords->selector = 0;
    if (has_vals) out_vals->selector = 0;
  }
  // every level byte the last movement does not write stays 0 (unknown)
  if (nnz > 0) QSD_CUDA(cudaMemsetAsync(lev, 0, (size_t)nnz, st));
  LevOut lv;
  std::memset(&lv, 0, sizeof(lv));
  lv.lev = lev;
  lv.order = r;
  for (int l = 0; l < r; ++l) lv.sigma[l] = plan->sigma[l];
  s = run_plan(out_coords, out_vals, nnz > 0 ? &ext : nullptr, nnz, plan, workspace, L, st, &lv);
  if (s != QSD_OK) return s;
  const int32_t* res = out_coords->buf[out_coords->selector];
  const int32_t* rows[QSD_MAX_ORDER];
  for (int l = 0; l < r; ++l) rows[l] = nnz > 0 ? res + (int64_t)plan->sigma[l] * out_coords->stride
                                                : nullptr;
  CsfOut o;
  for (int l = 0; l < kMaxOrder; ++l) o.ids[l] = l < r ? csf->ids[l] : nullptr;
  for (int l = 0; l <= kMaxOrder; ++l) o.ptr[l] = l <= r ? csf->ptr[l] : nullptr;
  QSD_CUDA(launch_csf(rows, r, (int)nnz, o, nodes, tile_count, st, lev));
  return QSD_OK;
}

// ---------------------------------------------------------------------------
// A transposition captured once into a CUDA graph (qsd_exec_*): its launches
// replayed by one graph launch, which removes the host's per-launch cost and
// most of the gaps between dependent kernels.
struct qsd_exec_s {
  cudaGraphExec_t exec = nullptr;
  int selector = 0;
  int vselector = 0;
};

qsd_status qsd_exec_create(const int32_t* in_coords, int64_t in_stride, const void* in_vals,
                           const qsd_coords* out_coords, const qsd_values* out_vals,
                           int64_t nnz, qsd_plan_t plan, void* workspace,
                           size_t workspace_bytes, qsd_exec_t* out) {
  if (!out || !out_coords) return QSD_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  qsd_coords oc = *out_coords;
  qsd_values ov;
  std::memset(&ov, 0, sizeof(ov));
  if (out_vals) ov = *out_vals;
  qsd_status s = check_buffers(&oc, out_vals ? &ov : nullptr, nnz, plan);
  if (s != QSD_OK) return s;
  const bool has_vals = out_vals && out_vals->elem_bytes != 0;
  if (nnz > 0 && (!in_coords || in_stride < nnz)) return QSD_ERR_INVALID_ARGUMENT;
  if (has_vals && nnz > 0 && !in_vals) return QSD_ERR_INVALID_ARGUMENT;
  if (nnz > 0 && (in_coords == oc.buf[0] || in_coords == oc.buf[1]))
    return QSD_ERR_INVALID_ARGUMENT;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)))
    return QSD_ERR_INVALID_ARGUMENT;
  const Layout L = layout_for(plan, nnz, has_vals ? ov.elem_bytes : 0);
  if (workspace_bytes < L.total) return QSD_ERR_WORKSPACE_TOO_SMALL;
  // the launch profiler records events of its own: nothing to capture it into
  if (prof_enabled()) return QSD_ERR_UNSUPPORTED;
  Src ext;
  ext.c = in_coords;
  ext.v = has_vals ? in_vals : nullptr;
  ext.stride = in_stride;
  ext.idx = -1;
  if (nnz == 0) {
    oc.selector = 0;
    ov.selector = 0;
  }
  qsd_exec_s* e = new (std::nothrow) qsd_exec_s;
  if (!e) return QSD_ERR_OUT_OF_MEMORY;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return QSD_ERR_CUDA;
  }
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(cs);
    delete e;
    return QSD_ERR_CUDA;
  }
  s = run_plan(&oc, has_vals ? &ov : nullptr, nnz > 0 ? &ext : nullptr, nnz, plan, workspace, L,
               cs);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (s == QSD_OK && (ce != cudaSuccess || !g)) s = QSD_ERR_CUDA;
  if (s == QSD_OK && cudaGraphInstantiate(&e->exec, g, 0) != cudaSuccess) {
    e->exec = nullptr;
    s = QSD_ERR_CUDA;
  }
  if (g) cudaGraphDestroy(g);
  if (s != QSD_OK) {
    cudaGetLastError();
    delete e;
    return s;
  }
  e->selector = oc.selector;
  e->vselector = ov.selector;
  *out = e;
  return QSD_OK;
}

qsd_status qsd_exec_launch(qsd_exec_t e, void* stream, int* selector, int* vals_selector) {
  if (!e || !e->exec) return QSD_ERR_INVALID_ARGUMENT;
  QSD_CUDA(cudaGraphLaunch(e->exec, (cudaStream_t)stream));
  if (selector) *selector = e->selector;
  if (vals_selector) *vals_selector = e->vselector;
  return QSD_OK;
}

void qsd_exec_destroy(qsd_exec_t e) {
  if (!e) return;
  if (e->exec) cudaGraphExecDestroy(e->exec);
  delete e;
}

qsd_status qsd_transpose(qsd_coords* coords, qsd_values* vals, int64_t nnz,
                         qsd_plan_t plan, void* stream) {
  qsd_status s = check_buffers(coords, vals, nnz, plan);
  if (s != QSD_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = layout_for(plan, nnz, vals ? vals->elem_bytes : 0);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, L.total, st) != cudaSuccess) {
    cudaGetLastError();
    return QSD_ERR_OUT_OF_MEMORY;
  }
  s = run_plan(coords, vals, nullptr, nnz, plan, ws, L, st);
  if (cudaFreeAsync(ws, st) != cudaSuccess && s == QSD_OK) s = QSD_ERR_CUDA;
  return s;
}

qsd_status qsd_transpose_host_async(const int32_t* host_coords, int64_t host_stride,
                                    const void* host_vals, int32_t* host_out_coords,
                                    int64_t host_out_stride, void* host_out_vals, int64_t nnz,
                                    qsd_plan_t plan, qsd_coords* dev_coords,
                                    qsd_values* dev_vals, void* workspace,
                                    size_t workspace_bytes, void* stream) {
  qsd_status s = check_buffers(dev_coords, dev_vals, nnz, plan);
  if (s != QSD_OK) return s;
  const bool has_vals = dev_vals && dev_vals->elem_bytes != 0;
  if (nnz > 0 && (!host_coords || !host_out_coords)) return QSD_ERR_INVALID_ARGUMENT;
  if (host_stride < nnz || host_out_stride < nnz) return QSD_ERR_INVALID_ARGUMENT;
  if (has_vals && nnz > 0 && (!host_vals || !host_out_vals)) return QSD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = (cudaStream_t)stream;
  const int r = plan->order;
  if (nnz > 0) {
    QSD_CUDA(cudaMemcpy2DAsync(dev_coords->buf[dev_coords->selector],
                               sizeof(int32_t) * dev_coords->stride, host_coords,
                               sizeof(int32_t) * host_stride, sizeof(int32_t) * nnz, r,
                               cudaMemcpyHostToDevice, st));
    if (has_vals)
      QSD_CUDA(cudaMemcpyAsync(dev_vals->buf[dev_vals->selector], host_vals,
                               (size_t)dev_vals->elem_bytes * nnz, cudaMemcpyHostToDevice,
                               st));
  }
  s = qsd_transpose_ws(dev_coords, dev_vals, nnz, plan, workspace, workspace_bytes, stream);
  if (s != QSD_OK) return s;
  if (nnz > 0) {
    QSD_CUDA(cudaMemcpy2DAsync(host_out_coords, sizeof(int32_t) * host_out_stride,
                               dev_coords->buf[dev_coords->selector],
                               sizeof(int32_t) * dev_coords->stride, sizeof(int32_t) * nnz,
                               r, cudaMemcpyDeviceToHost, st));
    if (has_vals)
      QSD_CUDA(cudaMemcpyAsync(host_out_vals, dev_vals->buf[dev_vals->selector],
                               (size_t)dev_vals->elem_bytes * nnz, cudaMemcpyDeviceToHost,
                               st));
  }
  return QSD_OK;
}

qsd_status qsd_transpose_host(const int32_t* host_coords, int64_t host_stride,
                              const void* host_vals, int32_t* host_out_coords,
                              int64_t host_out_stride, void* host_out_vals, int64_t nnz,
                              qsd_plan_t plan, qsd_coords* dev_coords,
                              qsd_values* dev_vals, void* workspace,
                              size_t workspace_bytes, void* stream) {
  qsd_status s = qsd_transpose_host_async(host_coords, host_stride, host_vals, host_out_coords,
                                          host_out_stride, host_out_vals, nnz, plan, dev_coords,
                                          dev_vals, workspace, workspace_bytes, stream);
  if (s != QSD_OK) return s;
  qsd_status dev_status = QSD_OK;
  s = qsd_workspace_status(workspace, stream, &dev_status);
  if (s != QSD_OK) return s;
  return dev_status;
}

// ---------------------------------------------------------------------------
// Transposition that allocates nothing. Its scratch is this file-scope device
// array, reserved when the library is loaded onto a GPU and held until the
// process exits; every call on a device shares it.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (the host-side
// symbol is only a stand-in). Resolved once per device.
qsd_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QSD_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return QSD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return QSD_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return QSD_OK;
}
}  // namespace

qsd_status qsd_transpose_noalloc(qsd_coords* coords, qsd_values* vals, int64_t nnz,
                                 qsd_plan_t plan, void* stream) {
  qsd_status s = check_buffers(coords, vals, nnz, plan);
  if (s != QSD_OK) return s;
  const Layout L = layout_for(plan, nnz, vals ? vals->elem_bytes : 0);
  if (L.total > kNoAllocScratchBytes) return QSD_ERR_WORKSPACE_TOO_SMALL;
  // the launch profiler allocates pinned host memory and events of its own
  if (prof_enabled()) return QSD_ERR_UNSUPPORTED;
  void* ws = nullptr;
  s = noalloc_scratch(&ws);
  if (s != QSD_OK) return s;
  // run_plan clears the status word and counters it relies on before use
  return run_plan(coords, vals, nullptr, nnz, plan, ws, L, (cudaStream_t)stream);
}

qsd_status qsd_workspace_status(const void* workspace, void* stream, qsd_status* out) {
  if (!workspace || !out) return QSD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned v = 0;
  QSD_CUDA(cudaMemcpyAsync(&v, workspace, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  QSD_CUDA(cudaStreamSynchronize(st));
  *out = (qsd_status)v;
  return QSD_OK;
}

// ---------------------------------------------------------------------------
// Test-only knobs of the bounded waits (no counterpart in the paper).
namespace {
std::mutex g_debug_mu;
unsigned long long g_debug_limit = 0;  // 0 = the default limit
int g_debug_stall_on = 0;

qsd_status push_debug_words() {
  const unsigned long long lim = g_debug_limit ? g_debug_limit : 2000000000ull;  // default 2 s
  if (qsd::debug_words_digit_pass(lim, g_debug_stall_on) != cudaSuccess ||
      qsd::debug_words_local_sort(lim, g_debug_stall_on) != cudaSuccess) {
    cudaGetLastError();
    return QSD_ERR_CUDA;
  }
  return QSD_OK;
}
}  // namespace

qsd_status qsd_debug_set_spin_limit_ns(uint64_t limit_ns) {
  if (limit_ns > 60ull * 1000000000ull) return QSD_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(g_debug_mu);
  g_debug_limit = limit_ns;
  return push_debug_words();
}

qsd_status qsd_debug_set_stall(int stall) {
  if (stall != 0 && stall != 1) return QSD_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(g_debug_mu);
  g_debug_stall_on = stall;
  return push_debug_words();
}

qsd_status qsd_get_async_status(void* stream, qsd_status* out) {
  if (!out) return QSD_ERR_INVALID_ARGUMENT;
  unsigned v = 0;
  QSD_CUDA(qsd::read_and_clear_sticky(&v, (cudaStream_t)stream));
  *out = (qsd_status)v;
  return QSD_OK;
}

}  // extern "C"
