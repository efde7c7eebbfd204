// Batched transposition (qsd_batch_*): many tensors, one launch per stage.
//
// Each tensor keeps its own plan (Algorithm 3 and its groups); what the
// batch shares is the launches. Round r runs the r-th group (that has
// passes) of every tensor that has one: the tensors of the round are laid
// end to end in one index space, bucket discovery, classification and the
// shared-memory bucket sort run once over all of them, and each radix pass
// runs its count, offset and move kernels once over the chunks of every
// tensor that has that pass (tensors are ordered by pass count, so the
// tensors of pass p are a prefix of the round's). The work tables that tell
// a kernel which tensor an item belongs to (its buffers, digits and place in
// the index space) are built on the host when the batch is created and stay
// on the device; the data-dependent lists (buckets, chunks, per-pass chunk
// lists) are built on the device during the run, so a run never
// synchronises with the host and can be captured in a CUDA graph.
//
// The autotuner times whole runs under candidate execution options and
// keeps the fastest per batch shape in a process-wide cache.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch_internal.h"

struct qsd_batch_s {
  qsd::BatchCore core;
  void* dtab = nullptr;  // device allocation of the tables
  cudaGraphExec_t exec = nullptr;
  void* exec_ws = nullptr;
};

namespace qsd {

namespace {

// p moved back by `elems` elements of `esz` bytes: element J of the result is
// element J - elems of p (only ever dereferenced at J >= elems).
template <typename T>
T* shifted(T* p, int64_t elems, int esz) {
  if (!p) return nullptr;
  return reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) - (uintptr_t)(elems * esz));
}

// Re-plans a tensor when the batch's digit width differs from its plan's
// (the pass schedule depends on it).
qsd_status replan(BatchTensor& t, const qsd_batch_options& o) {
  const int want = o.digit_bits ? o.digit_bits
                                : (t.base_opts.digit_bits ? t.base_opts.digit_bits : kRadixBits);
  if (want == t.plan.digit_bits) return QSD_OK;
  qsd_plan_options po = t.base_opts;
  po.digit_bits = want;
  qsd_plan_t p = nullptr;
  const qsd_plan_s& src = t.plan;
  qsd_status s = qsd_plan_ex(src.order, src.dims, src.tau, src.sigma, &po, &p);
  if (s != QSD_OK) return s;
  t.plan = *p;
  qsd_plan_destroy(p);
  return QSD_OK;
}

}  // namespace

qsd_status batch_prepare(BatchCore& b) {
  for (BatchTensor& t : b.t) {
    qsd_status s = replan(t, b.opts);
    if (s != QSD_OK) return s;
  }
  // per tensor: the groups that have passes
  std::vector<std::vector<int>> eff(b.n);
  int nrounds = 0;
  b.max_order = 1;
  b.copies.clear();
  for (int i = 0; i < b.n; ++i) {
    const BatchTensor& t = b.t[i];
    for (int g = 0; g < t.plan.ngroups; ++g)
      if (t.plan.groups[g].npasses > 0) eff[i].push_back(g);
    if (t.nnz > 0 && !eff[i].empty()) {
      nrounds = std::max(nrounds, (int)eff[i].size());
      b.max_order = std::max(b.max_order, t.plan.order);
    }
    if (t.nnz > 0 && eff[i].empty()) b.copies.push_back(i);
  }
  b.C = local_sort_capacity(b.opts.local_capacity ? b.opts.local_capacity : 4096, b.max_order,
                            b.vbytes);
  b.T = digit_tile(b.max_order, b.vbytes, b.opts.tile);
  b.CH = digit_chunk(b.max_order, b.vbytes, b.opts.tile, b.opts.chunk_tiles);
  const int seg_tile = seg_tile_entries();

  std::vector<int> cur(b.n, -1);
  b.rounds.assign(nrounds, BatchRound());
  int maxN = 0, maxTiles = 0, maxP = 1, maxChunks = 1, maxGroups = 1, maxLarge = 1;
  for (int r = 0; r < nrounds; ++r) {
    BatchRound& R = b.rounds[r];
    for (int i = 0; i < b.n; ++i) {
      if (b.t[i].nnz == 0 || (int)eff[i].size() <= r) continue;
      BatchMember m;
      m.tensor = i;
      m.group = eff[i][r];
      m.P = b.t[i].plan.groups[m.group].npasses;
      m.cur = cur[i];
      m.F = cur[i] < 0 ? 0 : cur[i] ^ (m.P & 1);
      cur[i] = m.F;
      R.m.push_back(m);
    }
    std::stable_sort(R.m.begin(), R.m.end(),
                     [](const BatchMember& a, const BatchMember& c) { return a.P > c.P; });
    R.n = (int)R.m.size();
    int64_t N = 0, tiles = 0;
    for (const BatchMember& m : R.m) {
      N += b.t[m.tensor].nnz;
      tiles += (b.t[m.tensor].nnz + seg_tile - 1) / seg_tile;
    }
    R.N = (int)N;
    R.ntiles = (int)tiles;
    R.maxP = R.n ? R.m[0].P : 0;
    R.max_large = (int)(N / (b.C + 1) + 1);
    R.max_chunks = (int)((N + b.CH - 1) / b.CH + R.max_large);
    R.max_groups = (R.max_chunks + kGroupChunks - 1) / kGroupChunks + R.max_large;
    maxN = std::max(maxN, R.N);
    maxTiles = std::max(maxTiles, R.ntiles);
    maxP = std::max(maxP, R.maxP);
    maxChunks = std::max(maxChunks, R.max_chunks);
    maxGroups = std::max(maxGroups, R.max_groups);
    maxLarge = std::max(maxLarge, R.max_large);
  }
  for (int i = 0; i < b.n; ++i) b.t[i].result = cur[i] < 0 ? 0 : cur[i];

  // workspace
  BatchLayout& L = b.L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += ws_align_up(bytes);
    return o;
  };
  L.max_chunks = maxChunks;
  L.max_groups = maxGroups;
  L.max_passes = maxP;
  L.status = take(sizeof(unsigned));
  L.counters = take(sizeof(int) * kNumCounters);
  L.seg_start = take(sizeof(int) * ((size_t)maxN + 2));
  L.seg_lb = take(sizeof(uint32_t) *
                  ((size_t)maxTiles + 1 + (size_t)maxTiles * (seg_tile / 32) + 32));
  L.large = take(sizeof(int2) * (size_t)maxLarge);
  L.chunk_base = take(sizeof(int) * (size_t)maxLarge);
  L.group_base = take(sizeof(int) * (size_t)maxLarge);
  L.large_tensor = take(sizeof(int) * (size_t)maxLarge);
  L.chunk_owner = take(sizeof(int) * (size_t)maxChunks);
  L.group_owner = take(sizeof(int) * (size_t)maxGroups);
  L.chunk_hist = take(sizeof(uint32_t) * (size_t)maxChunks * kRadix);
  L.group_sum = take(sizeof(uint32_t) * (size_t)maxP * maxGroups * kRadix);
  L.pass_chunks = take(sizeof(int) * (size_t)maxP * maxChunks);
  L.pass_groups = take(sizeof(int) * (size_t)maxP * maxGroups);
  L.total = off;

  // table offsets
  size_t toff = 0;
  auto ttake = [&](size_t bytes) {
    const size_t o = toff;
    toff += (bytes + 15) & ~size_t(15);
    return o;
  };
  for (BatchRound& R : b.rounds) {
    R.jbase = ttake(sizeof(int) * (R.n + 1));
    R.tile_base = ttake(sizeof(int) * (R.n + 1));
    R.seg = ttake(sizeof(SegTensor) * R.n);
    R.ls = ttake(sizeof(LsTensor) * R.n);
    int pool = 0;
    for (const BatchMember& m : R.m) pool += m.P;
    R.pool = ttake(sizeof(PassDesc) * pool);
    for (int p = 0; p < R.maxP; ++p) {
      int np = 0;
      for (const BatchMember& m : R.m) np += m.P > p ? 1 : 0;
      R.pass[p] = ttake(sizeof(PassTensor) * np);
    }
  }
  b.table_bytes = toff;
  return QSD_OK;
}

void batch_fill_tables(const BatchCore& b, const void* dev_base, uint8_t* img) {
  std::memset(img, 0, b.table_bytes);
  const uint8_t* const dbase = static_cast<const uint8_t*>(dev_base);
  const int vb = b.vbytes;
  const int seg_tile = seg_tile_entries();
  for (const BatchRound& R : b.rounds) {
    int* jb = reinterpret_cast<int*>(img + R.jbase);
    int* tb = reinterpret_cast<int*>(img + R.tile_base);
    SegTensor* sg = reinterpret_cast<SegTensor*>(img + R.seg);
    LsTensor* lt = reinterpret_cast<LsTensor*>(img + R.ls);
    PassDesc* pool = reinterpret_cast<PassDesc*>(img + R.pool);
    const PassDesc* dpool = reinterpret_cast<const PassDesc*>(dbase + R.pool);
    int j = 0, tile = 0, pi = 0;
    for (int k = 0; k < R.n; ++k) {
      const BatchMember& m = R.m[k];
      const BatchTensor& t = b.t[m.tensor];
      const Group& g = t.plan.groups[m.group];
      jb[k] = j;
      tb[k] = tile;
      // rows and values of buffer idx (-1 = the input), shifted by j
      auto rows = [&](int idx) -> const int32_t* {
        return idx < 0 ? shifted(t.in, j, 4) : shifted<const int32_t>(t.out[idx], j, 4);
      };
      auto stride = [&](int idx) { return idx < 0 ? t.in_stride : t.out_stride; };
      auto vals = [&](int idx) -> const void* {
        if (!vb) return nullptr;
        return idx < 0 ? shifted(t.in_vals, j, vb) : shifted<const void>(t.out_vals[idx], j, vb);
      };
      auto cols = [&](int src, int dst) {
        Cols c;
        c.in = rows(src);
        c.vin = vals(src);
        c.in_stride = stride(src);
        c.out = shifted(t.out[dst], j, 4);
        c.vout = vb ? shifted(t.out_vals[dst], j, vb) : nullptr;
        c.out_stride = t.out_stride;
        c.order = t.plan.order;
        c.vbytes = vb;
        return c;
      };
      sg[k].n = g.prefix_len;
      for (int q = 0; q < g.prefix_len; ++q)
        sg[k].col[q] = rows(m.cur) + (int64_t)g.prefix_modes[q] * stride(m.cur);
      lt[k].c = cols(m.cur, m.F);
      lt[k].npasses = m.P;
      lt[k].pass = dpool + pi;
      for (int p = 0; p < m.P; ++p) pool[pi + p] = g.pass[p];
      pi += m.P;
      for (int p = 0; p < m.P; ++p) {
        // pass p reads the group's input (p = 0) or the previous pass's
        // output, and writes dst(p); the last pass writes F
        const int dst = m.F ^ ((m.P - 1 - p) & 1);
        const int src = p == 0 ? m.cur : (m.F ^ ((m.P - p) & 1));
        PassTensor* pt = reinterpret_cast<PassTensor*>(img + R.pass[p]);
        pt[k].c = cols(src, dst);
        pt[k].pd = g.pass[p];
      }
      j += (int)t.nnz;
      tile += (int)((t.nnz + seg_tile - 1) / seg_tile);
    }
    jb[R.n] = j;
    tb[R.n] = tile;
  }
}

#define QSD_CUDA(call)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return QSD_ERR_CUDA; \
  } while (0)

qsd_status batch_issue(const BatchCore& b, void* ws, cudaStream_t st) {
  const BatchLayout& L = b.L;
  uint8_t* base = static_cast<uint8_t*>(ws);
  unsigned* status = reinterpret_cast<unsigned*>(base + L.status);
  int* counters = reinterpret_cast<int*>(base + L.counters);
  int* seg_start = reinterpret_cast<int*>(base + L.seg_start);
  uint32_t* seg_lb = reinterpret_cast<uint32_t*>(base + L.seg_lb);
  int2* large = reinterpret_cast<int2*>(base + L.large);
  int* chunk_base = reinterpret_cast<int*>(base + L.chunk_base);
  int* group_base = reinterpret_cast<int*>(base + L.group_base);
  int* large_tensor = reinterpret_cast<int*>(base + L.large_tensor);
  int* chunk_owner = reinterpret_cast<int*>(base + L.chunk_owner);
  int* group_owner = reinterpret_cast<int*>(base + L.group_owner);
  uint32_t* chunk_hist = reinterpret_cast<uint32_t*>(base + L.chunk_hist);
  uint32_t* group_sum = reinterpret_cast<uint32_t*>(base + L.group_sum);
  int* pass_chunks = reinterpret_cast<int*>(base + L.pass_chunks);
  int* pass_groups = reinterpret_cast<int*>(base + L.pass_groups);
  const uint8_t* dt = static_cast<const uint8_t*>(b.dtab);

  QSD_CUDA(cudaMemsetAsync(base, 0, L.counters + sizeof(int) * kNumCounters, st));
  Cols lay;  // the staging layout: largest order, the batch's value width
  std::memset(&lay, 0, sizeof(lay));
  lay.order = b.max_order;
  lay.vbytes = b.vbytes;
  PassDesc pd0;
  std::memset(&pd0, 0, sizeof(pd0));
  PassList pl0;
  std::memset(&pl0, 0, sizeof(pl0));
  for (const BatchRound& R : b.rounds) {
    if (R.n == 0) continue;
    const int* jbase = reinterpret_cast<const int*>(dt + R.jbase);
    const LsTensor* lt = reinterpret_cast<const LsTensor*>(dt + R.ls);
    QSD_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * kNumCounters, st));
    SegBatch sb;
    sb.n = R.n;
    sb.jbase = jbase;
    sb.tile_base = reinterpret_cast<const int*>(dt + R.tile_base);
    sb.t = reinterpret_cast<const SegTensor*>(dt + R.seg);
    QSD_CUDA(launch_seg_discover_batch(sb, R.ntiles, R.N, seg_start, seg_lb, counters, st));
    ClassifyBatch cb;
    cb.n = R.n;
    cb.jbase = jbase;
    cb.t = lt;
    cb.large_tensor = large_tensor;
    cb.pass_chunks = pass_chunks;
    cb.pass_groups = pass_groups;
    cb.max_chunks = L.max_chunks;
    QSD_CUDA(launch_seg_classify(seg_start, counters, R.N, b.C, b.CH, large, chunk_base,
                                 group_base, chunk_owner, group_owner, group_sum, R.maxP,
                                 L.max_groups, cb, st));
    LsBatch lb;
    lb.n = R.n;
    lb.jbase = jbase;
    lb.t = lt;
    QSD_CUDA(launch_local_sort(lay, pl0, seg_start, counters, 0, R.N, b.C, status, lb, st));
    LargeSegs ls;
    std::memset(&ls, 0, sizeof(ls));
    ls.single = 0;
    ls.nnz = R.N;
    ls.tile = b.T;
    ls.chunk = b.CH;
    ls.counters = counters;
    ls.seg = large;
    ls.chunk_base = chunk_base;
    ls.group_base = group_base;
    ls.chunk_owner = chunk_owner;
    ls.group_owner = group_owner;
    for (int p = 0; p < R.maxP; ++p) {
      PassBatch pb;
      pb.t = reinterpret_cast<const PassTensor*>(dt + R.pass[p]);
      pb.large_tensor = large_tensor;
      pb.chunks = pass_chunks + (size_t)p * L.max_chunks;
      pb.groups = pass_groups + (size_t)p * L.max_groups;
      pb.counters = counters;
      pb.pass = p;
      uint32_t* gs = group_sum + (size_t)p * L.max_groups * kRadix;
      QSD_CUDA(launch_chunk_hist(lay, ls, pd0, chunk_hist, gs, counters + kCntClaim + 2 * p,
                                 R.max_chunks, pb, st));
      QSD_CUDA(launch_chunk_scan(ls, chunk_hist, gs, R.max_groups, pb, st));
      QSD_CUDA(launch_digit_move(lay, ls, pd0, chunk_hist, counters + kCntClaim + 2 * p + 1,
                                 R.max_chunks, status, pb, st));
    }
  }
  for (int i : b.copies) {  // no pass: the result is the input, copied
    const BatchTensor& t = b.t[i];
    Cols c;
    c.in = t.in;
    c.vin = b.vbytes ? t.in_vals : nullptr;
    c.in_stride = t.in_stride;
    c.out = t.out[0];
    c.vout = b.vbytes ? t.out_vals[0] : nullptr;
    c.out_stride = t.out_stride;
    c.order = t.plan.order;
    c.vbytes = b.vbytes;
    QSD_CUDA(launch_copy(c, (int)t.nnz, st));
  }
  QSD_CUDA(launch_fold_status(status, st));
  return QSD_OK;
}

}  // namespace qsd

namespace {

using namespace qsd;

void free_exec(qsd_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->exec_ws = nullptr;
}

// (Re)builds the schedule and the device tables for the batch's current
// options. The previous tables are freed (the caller makes sure no run still
// uses them).
qsd_status build(qsd_batch_s* b) {
  free_exec(b);
  if (b->dtab) {
    cudaFree(b->dtab);
    b->dtab = nullptr;
    b->core.dtab = nullptr;
  }
  qsd_status s = batch_prepare(b->core);
  if (s != QSD_OK) return s;
  if (b->core.table_bytes == 0) return QSD_OK;  // nothing to sort
  if (cudaMalloc(&b->dtab, b->core.table_bytes) != cudaSuccess) {
    cudaGetLastError();
    b->dtab = nullptr;
    return QSD_ERR_OUT_OF_MEMORY;
  }
  b->core.dtab = b->dtab;
  std::vector<uint8_t> img(b->core.table_bytes);
  batch_fill_tables(b->core, b->dtab, img.data());
  if (cudaMemcpy(b->dtab, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return QSD_ERR_CUDA;
  }
  return QSD_OK;
}

// Captures one run into a graph bound to `ws`.
qsd_status capture(qsd_batch_s* b, void* ws) {
  free_exec(b);
  cudaStream_t cs = nullptr;
  QSD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(cs);
    return QSD_ERR_CUDA;
  }
  const qsd_status s = batch_issue(b->core, ws, cs);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (s != QSD_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return s != QSD_OK ? s : QSD_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    b->exec = nullptr;
    cudaGetLastError();
    return QSD_ERR_CUDA;
  }
  b->exec_ws = ws;
  return QSD_OK;
}

qsd_status run(qsd_batch_s* b, void* ws, cudaStream_t st) {
  if (b->core.opts.no_graph) return batch_issue(b->core, ws, st);
  if (!b->exec || b->exec_ws != ws) {
    const qsd_status s = capture(b, ws);
    if (s != QSD_OK) return s;
  }
  QSD_CUDA(cudaGraphLaunch(b->exec, st));
  return QSD_OK;
}

// ---------------------------------------------------------------------------
// Tuning cache: batch shape -> execution options.
std::mutex g_tune_mu;
std::map<std::string, qsd_batch_options> g_tune_cache;

// The shape a tuned choice is reused for: tensor count, value width,
// largest order, total entries (to a quarter octave) and total passes of the
// plans under their own options.
std::string shape_key(const BatchCore& b, const std::vector<int>& own_passes) {
  int64_t N = 0;
  int P = 0;
  for (int i = 0; i < b.n; ++i) {
    N += b.t[i].nnz;
    P += own_passes[i];
  }
  const int lgN = N > 0 ? (int)std::lround(4.0 * std::log2((double)N)) : -1;
  char buf[128];
  std::snprintf(buf, sizeof(buf), "n=%d,vb=%d,r=%d,lgN4=%d,P=%d", b.n, b.vbytes, b.max_order,
                lgN, P);
  return buf;
}

std::vector<int> own_passes(const BatchCore& b) {
  std::vector<int> out(b.n, 0);
  for (int i = 0; i < b.n; ++i) {
    qsd_plan_t p = nullptr;
    const qsd_plan_s& s = b.t[i].plan;
    if (qsd_plan_ex(s.order, s.dims, s.tau, s.sigma, &b.t[i].base_opts, &p) != QSD_OK) continue;
    for (int g = 0; g < p->ngroups; ++g) out[i] += p->groups[g].npasses;
    qsd_plan_destroy(p);
  }
  return out;
}

bool valid_options(const qsd_batch_options& o) {
  if (o.digit_bits < 0 || o.digit_bits > kRadixBits) return false;
  if (o.local_capacity != 0 && o.local_capacity != 1024 && o.local_capacity != 2048 &&
      o.local_capacity != 4096 && o.local_capacity != 8192)
    return false;
  if (o.tile != 0 && o.tile != 1024 && o.tile != 2048 && o.tile != 3584 && o.tile != 4096) return false;
  if (o.chunk_tiles < 0 || o.chunk_tiles > 256) return false;
  return true;
}

}  // namespace

namespace qsd {

// Checks batch items (shared with the serving engine, which builds its own).
qsd_status check_batch_items(const qsd_batch_item* items, int n, int val_bytes) {
  if (!items || n < 1) return QSD_ERR_INVALID_ARGUMENT;
  if (val_bytes != 0 && val_bytes != 4 && val_bytes != 8) return QSD_ERR_INVALID_ARGUMENT;
  int64_t total = 0;
  for (int i = 0; i < n; ++i) {
    const qsd_batch_item& it = items[i];
    if (!it.plan || it.nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
    total += it.nnz;
    if (it.nnz > kMaxBatchNnz || total > kMaxBatchNnz) return QSD_ERR_UNSUPPORTED;
    if (it.nnz == 0) continue;
    if (!it.in || !it.out[0] || !it.out[1]) return QSD_ERR_INVALID_ARGUMENT;
    if (it.in_stride < it.nnz || it.out_stride < it.nnz) return QSD_ERR_INVALID_ARGUMENT;
    if (val_bytes && (!it.in_vals || !it.out_vals[0] || !it.out_vals[1]))
      return QSD_ERR_INVALID_ARGUMENT;
    // the input is read while results are written: no overlap
    const int r = it.plan->order;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(it.in);
    const uintptr_t a1 = a0 + 4 * (uintptr_t)((r - 1) * it.in_stride + it.nnz);
    for (int s = 0; s < 2; ++s) {
      const uintptr_t b0 = reinterpret_cast<uintptr_t>(it.out[s]);
      const uintptr_t b1 = b0 + 4 * (uintptr_t)((r - 1) * it.out_stride + it.nnz);
      if (a0 < b1 && b0 < a1) return QSD_ERR_INVALID_ARGUMENT;
    }
  }
  return QSD_OK;
}

void fill_batch_tensor(BatchTensor& t, const qsd_batch_item& it) {
  t.plan = *it.plan;
  t.base_opts = it.plan->opts;  // batches sort whole entries (no (key, index) form)
  t.nnz = it.nnz;
  t.in = it.in;
  t.in_stride = it.in_stride;
  t.in_vals = it.in_vals;
  t.out[0] = it.out[0];
  t.out[1] = it.out[1];
  t.out_stride = it.out_stride;
  t.out_vals[0] = it.out_vals[0];
  t.out_vals[1] = it.out_vals[1];
  t.result = 0;
}

}  // namespace qsd

extern "C" {

qsd_status qsd_batch_create(const qsd_batch_item* items, int n, int val_bytes,
                            const qsd_batch_options* opts, qsd_batch_t* out) {
  if (!out) return QSD_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  qsd_batch_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (!valid_options(o)) return QSD_ERR_INVALID_ARGUMENT;
  qsd_status s = check_batch_items(items, n, val_bytes);
  if (s != QSD_OK) return s;
  qsd_batch_s* b = new (std::nothrow) qsd_batch_s;
  if (!b) return QSD_ERR_OUT_OF_MEMORY;
  BatchCore& c = b->core;
  c.n = n;
  c.vbytes = val_bytes;
  c.opts = o;
  c.t.resize(n);
  for (int i = 0; i < n; ++i) fill_batch_tensor(c.t[i], items[i]);
  s = build(b);
  if (s == QSD_OK && o.use_tuned) {
    const std::string key = shape_key(c, own_passes(c));
    bool hit = false;
    qsd_batch_options tuned;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto f = g_tune_cache.find(key);
      if (f != g_tune_cache.end()) {
        tuned = f->second;
        hit = true;
      }
    }
    if (hit) {
      tuned.no_graph = o.no_graph;
      tuned.use_tuned = 1;
      c.opts = tuned;
      s = build(b);
    }
  }
  if (s != QSD_OK) {
    qsd_batch_destroy(b);
    return s;
  }
  *out = b;
  return QSD_OK;
}

qsd_status qsd_batch_workspace_bytes(qsd_batch_t b, size_t* bytes) {
  if (!b || !bytes) return QSD_ERR_INVALID_ARGUMENT;
  *bytes = b->core.L.total;
  return QSD_OK;
}

qsd_status qsd_batch_run(qsd_batch_t b, void* workspace, size_t workspace_bytes, void* stream) {
  if (!b || !workspace || (reinterpret_cast<uintptr_t>(workspace) & (kWsAlign - 1)))
    return QSD_ERR_INVALID_ARGUMENT;
  if (workspace_bytes < b->core.L.total) return QSD_ERR_WORKSPACE_TOO_SMALL;
  return run(b, workspace, (cudaStream_t)stream);
}

qsd_status qsd_batch_result(qsd_batch_t b, int i, int* selector) {
  if (!b || !selector || i < 0 || i >= b->core.n) return QSD_ERR_INVALID_ARGUMENT;
  *selector = b->core.t[i].result;
  return QSD_OK;
}

qsd_status qsd_batch_get_options(qsd_batch_t b, qsd_batch_options* out) {
  if (!b || !out) return QSD_ERR_INVALID_ARGUMENT;
  *out = b->core.opts;
  return QSD_OK;
}

qsd_status qsd_batch_tune(qsd_batch_t b, void* workspace, size_t workspace_bytes, void* stream,
                          int reps, qsd_batch_options* best_out) {
  if (!b || !workspace || (reinterpret_cast<uintptr_t>(workspace) & (kWsAlign - 1)))
    return QSD_ERR_INVALID_ARGUMENT;
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  BatchCore& c = b->core;
  const std::vector<int> own = own_passes(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  QSD_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return QSD_ERR_CUDA;
  }
  // ms per run under options o (< 0: not runnable within the workspace)
  auto measure = [&](const qsd_batch_options& o, float* ms) -> qsd_status {
    *ms = -1.f;
    if (cudaStreamSynchronize(st) != cudaSuccess) return QSD_ERR_CUDA;
    c.opts = o;
    qsd_status s = build(b);
    if (s != QSD_OK) return s;
    if (c.L.total > workspace_bytes) return QSD_OK;
    s = run(b, workspace, st);  // warm-up (and graph capture)
    if (s != QSD_OK) return s;
    QSD_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) {
      s = run(b, workspace, st);
      if (s != QSD_OK) return s;
    }
    QSD_CUDA(cudaEventRecord(e1, st));
    QSD_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    QSD_CUDA(cudaEventElapsedTime(&t, e0, e1));
    *ms = t / reps;
    return QSD_OK;
  };
  qsd_batch_options best = c.opts;
  if (!best.local_capacity) best.local_capacity = 4096;
  if (!best.tile) best.tile = c.T;
  if (!best.chunk_tiles) best.chunk_tiles = 2;
  if (!best.digit_bits) best.digit_bits = kRadixBits;
  float best_ms = -1.f;
  qsd_status s = measure(best, &best_ms);
  // coordinate search: one option at a time, keeping the fastest
  const int tiles[] = {4096, 3584, 2048, 1024};
  const int bits[] = {8, 7, 6};
  const int caps[] = {4096, 2048, 8192, 1024};
  const int chunks[] = {2, 4, 1, 8};
  for (int dim = 0; dim < 4 && s == QSD_OK; ++dim) {
    const int* vals = dim == 0 ? tiles : dim == 1 ? bits : dim == 2 ? caps : chunks;
    const int nv = dim == 1 ? 3 : 4;
    for (int k = 0; k < nv && s == QSD_OK; ++k) {
      qsd_batch_options o = best;
      int& field = dim == 0 ? o.tile
                   : dim == 1 ? o.digit_bits
                   : dim == 2 ? o.local_capacity
                              : o.chunk_tiles;
      if (field == vals[k]) continue;
      field = vals[k];
      if (dim == 0 && digit_tile(c.max_order, c.vbytes, vals[k]) != vals[k]) continue;
      float ms = -1.f;
      s = measure(o, &ms);
      if (s == QSD_OK && ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best = o;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // adopt the winner
  if (cudaStreamSynchronize(st) != cudaSuccess && s == QSD_OK) s = QSD_ERR_CUDA;
  best.no_graph = c.opts.no_graph;
  c.opts = best;
  const qsd_status sb = build(b);
  if (s == QSD_OK) s = sb;
  if (s == QSD_OK) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[shape_key(c, own)] = best;
  }
  if (best_out) *best_out = best;
  return s;
}

qsd_status qsd_tune_cache_save(const char* path) {
  if (!path) return QSD_ERR_INVALID_ARGUMENT;
  FILE* f = std::fopen(path, "w");
  if (!f) return QSD_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : g_tune_cache)
    std::fprintf(f, "%s %d %d %d %d\n", kv.first.c_str(), kv.second.digit_bits,
                 kv.second.local_capacity, kv.second.tile, kv.second.chunk_tiles);
  std::fclose(f);
  return QSD_OK;
}

qsd_status qsd_tune_cache_load(const char* path) {
  if (!path) return QSD_ERR_INVALID_ARGUMENT;
  FILE* f = std::fopen(path, "r");
  if (!f) return QSD_ERR_INVALID_ARGUMENT;
  char key[128];
  qsd_batch_options o;
  qsd_status s = QSD_OK;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (true) {
    std::memset(&o, 0, sizeof(o));
    const int got = std::fscanf(f, "%127s %d %d %d %d", key, &o.digit_bits, &o.local_capacity,
                                &o.tile, &o.chunk_tiles);
    if (got == EOF) break;
    if (got != 5 || !valid_options(o)) {
      s = QSD_ERR_INVALID_ARGUMENT;
      break;
    }
    g_tune_cache[key] = o;
  }
  std::fclose(f);
  return s;
}

void qsd_batch_destroy(qsd_batch_t b) {
  if (!b) return;
  free_exec(b);
  if (b->dtab) cudaFree(b->dtab);
  delete b;
}

}  // extern "C"
