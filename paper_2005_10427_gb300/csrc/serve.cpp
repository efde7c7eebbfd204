// Serving engine (qsd_server_*): continuous batching of transposition
// requests over resident tensors under a device memory budget.
//
// One engine thread owns the device work. Each iteration it
//   1. reaps finished steps (a CUDA event per step): their requests become
//      results, the spare half of each result's double buffer and the
//      step's scratch go back to the budget;
//   2. for every idle stream, admits requests from the head of the queue (in
//      arrival order) while the in-flight limit and the memory budget allow,
//      builds one batch over them (each request's own plan; tables uploaded
//      from pinned memory on the stream) and launches it.
// The memory budget is one device reservation carved by a first-fit
// allocator; a request is admitted only when its result buffers fit, and a
// step only when its scratch fits too. Launches happen outside the lock, so
// submitting never waits for the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_internal.h"

namespace qsd {
qsd_status check_batch_items(const qsd_batch_item* items, int n, int val_bytes);
void fill_batch_tensor(BatchTensor& t, const qsd_batch_item& it);
}  // namespace qsd

namespace {

using namespace qsd;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over [0, size): 256-byte aligned blocks, neighbours
// merged on release.
class Arena {
 public:
  void init(size_t size) {
    size_ = size;
    free_.clear();
    free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = ws_align_up(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes, next = it->first + bytes;
      free_.erase(it);
      if (rest) free_[next] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = ws_align_up(std::max<size_t>(bytes, 1));
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

struct Block {
  size_t off = 0, bytes = 0;
  bool live = false;
};

struct Resident {
  int order;
  int64_t dims[QSD_MAX_ORDER];
  int tau[QSD_MAX_ORDER];
  const int32_t* coords;
  int64_t stride;
  const void* vals;
  int64_t nnz;
};

enum class State { kQueued, kInflight, kDone, kReleased };

struct Request {
  int64_t id;
  int tensor;
  qsd_plan_t plan;
  State state = State::kQueued;
  int status = QSD_OK;
  double arrival = 0, admit = 0, done = 0;
  Block c[2], v[2];  // result double buffers
  int sel = 0;
  bool delivered = false;
};

struct Step {
  bool busy = false;
  std::vector<int64_t> reqs;
  Block ws, tables;
  cudaEvent_t done = nullptr;
  unsigned* status_host = nullptr;  // pinned word the step's status is copied to
  uint8_t* staging = nullptr;       // pinned table image
  size_t staging_bytes = 0;
  double admit = 0;
};

}  // namespace

struct qsd_server_s {
  qsd_server_options opts;
  int device = 0;
  uint8_t* base = nullptr;  // the budget's device reservation
  Arena arena;
  std::vector<Resident> tensors;
  std::map<std::string, qsd_plan_t> plans;  // (tensor, sigma) -> plan
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> queue;
  std::deque<int64_t> completed;  // not yet polled
  std::vector<cudaStream_t> streams;
  std::vector<Step> steps;
  cudaEvent_t epoch = nullptr;
  double epoch_host = 0;
  int64_t next_id = 0;
  int inflight = 0;
  qsd_server_stats stats;
  std::mutex mu;
  std::condition_variable work_cv, done_cv;
  bool stop = false;
  std::thread engine;
};

namespace {

size_t rows_bytes(const Resident& t) { return (size_t)t.order * (size_t)t.nnz * 4; }

void free_block(qsd_server_s* s, Block& b) {
  if (!b.live) return;
  s->arena.release(b.off, b.bytes);
  b.live = false;
}

bool alloc_block(qsd_server_s* s, size_t bytes, Block* b) {
  size_t off = 0;
  if (!s->arena.alloc(bytes, &off)) return false;
  b->off = off;
  b->bytes = bytes;
  b->live = true;
  return true;
}

// Result buffers of a request: two row blocks and two value blocks.
bool alloc_result(qsd_server_s* s, Request& r) {
  const Resident& t = s->tensors[r.tensor];
  const size_t cb = rows_bytes(t), vb = (size_t)t.nnz * s->opts.val_bytes;
  Block* all[4] = {&r.c[0], &r.c[1], &r.v[0], &r.v[1]};
  const size_t sz[4] = {cb, cb, vb, vb};
  for (int k = 0; k < 4; ++k) {
    if (sz[k] == 0) continue;
    if (!alloc_block(s, sz[k], all[k])) {
      for (int q = 0; q < k; ++q) free_block(s, *all[q]);
      return false;
    }
  }
  return true;
}

size_t result_bytes(const qsd_server_s* s, const Resident& t) {
  return 2 * ws_align_up(std::max<size_t>(rows_bytes(t), 1)) +
         (s->opts.val_bytes ? 2 * ws_align_up((size_t)t.nnz * s->opts.val_bytes) : 0);
}

void finish(qsd_server_s* s, Request& r, int status, double done) {
  r.state = State::kDone;
  r.status = status;
  r.done = done;
  s->completed.push_back(r.id);
  s->stats.completed++;
  if (status == QSD_OK) s->stats.entries_completed += s->tensors[r.tensor].nnz;
}

// Moves finished steps' requests to the completed list (lock held).
void reap(qsd_server_s* s) {
  bool any = false;
  for (Step& st : s->steps) {
    if (!st.busy) continue;
    const cudaError_t q = cudaEventQuery(st.done);
    if (q == cudaErrorNotReady) continue;
    float ms = 0.f;
    double done = now_s();
    if (q == cudaSuccess && cudaEventElapsedTime(&ms, s->epoch, st.done) == cudaSuccess)
      done = s->epoch_host + ms / 1e3;
    const int status = q != cudaSuccess ? QSD_ERR_CUDA : (int)*st.status_host;
    if (q != cudaSuccess) cudaGetLastError();
    for (int64_t id : st.reqs) {
      Request& r = *s->reqs[id];
      free_block(s, r.c[r.sel ^ 1]);  // the spare half of the double buffers
      free_block(s, r.v[r.sel ^ 1]);
      finish(s, r, status, done);
      s->inflight--;
    }
    free_block(s, st.ws);
    free_block(s, st.tables);
    st.reqs.clear();
    st.busy = false;
    any = true;
  }
  if (any) s->done_cv.notify_all();
}

// A plan per (tensor, sigma), made on first use (lock held).
qsd_status plan_for(qsd_server_s* s, int tensor, const int* sigma, qsd_plan_t* out) {
  const Resident& t = s->tensors[tensor];
  std::string key = std::to_string(tensor) + ":";
  for (int i = 0; i < t.order; ++i) key += (char)('0' + sigma[i]);
  auto it = s->plans.find(key);
  if (it != s->plans.end()) {
    *out = it->second;
    return QSD_OK;
  }
  qsd_plan_t p = nullptr;
  qsd_status st = qsd_plan(t.order, t.dims, t.tau, sigma, &p);
  if (st != QSD_OK) return st;
  s->plans[key] = p;
  *out = p;
  return QSD_OK;
}

void fill_item(const qsd_server_s* s, const Request& r, qsd_batch_item* it) {
  const Resident& t = s->tensors[r.tensor];
  std::memset(it, 0, sizeof(*it));
  it->plan = r.plan;
  it->nnz = t.nnz;
  it->in = t.coords;
  it->in_stride = t.stride;
  it->in_vals = s->opts.val_bytes ? t.vals : nullptr;
  for (int k = 0; k < 2; ++k) {
    it->out[k] = reinterpret_cast<int32_t*>(s->base + r.c[k].off);
    it->out_vals[k] = s->opts.val_bytes ? s->base + r.v[k].off : nullptr;
  }
  it->out_stride = t.nnz;
}

// One engine step on idle stream k: admission, batch, launch. Called with
// the lock held; releases it around the launches.
void launch_step(qsd_server_s* s, int k, std::unique_lock<std::mutex>& lk) {
  Step& st = s->steps[k];
  std::vector<int64_t> take;
  // admission in arrival order: stop at the first request that does not fit
  while (!s->queue.empty() && (int)take.size() < s->opts.max_batch &&
         s->inflight + (int)take.size() < s->opts.max_inflight) {
    Request& r = *s->reqs[s->queue.front()];
    const Resident& t = s->tensors[r.tensor];
    if (result_bytes(s, t) > s->arena.size()) {  // can never fit
      s->queue.pop_front();
      s->stats.rejected++;
      finish(s, r, QSD_ERR_BUDGET, now_s());
      s->done_cv.notify_all();
      continue;
    }
    if (!alloc_result(s, r)) break;
    s->queue.pop_front();
    take.push_back(r.id);
  }
  // the step's scratch and tables; give requests back until they fit
  BatchCore core;
  while (!take.empty()) {
    std::vector<qsd_batch_item> items(take.size());
    for (size_t i = 0; i < take.size(); ++i) fill_item(s, *s->reqs[take[i]], &items[i]);
    core = BatchCore();
    core.n = (int)take.size();
    core.vbytes = s->opts.val_bytes;
    core.opts = s->opts.batch;
    core.opts.no_graph = 1;
    core.t.resize(core.n);
    for (int i = 0; i < core.n; ++i) fill_batch_tensor(core.t[i], items[i]);
    if (batch_prepare(core) == QSD_OK && alloc_block(s, core.L.total, &st.ws)) {
      if (core.table_bytes == 0 || alloc_block(s, core.table_bytes, &st.tables)) break;
      free_block(s, st.ws);
    }
    Request& last = *s->reqs[take.back()];  // back to the head of the queue
    for (Block* b : {&last.c[0], &last.c[1], &last.v[0], &last.v[1]}) free_block(s, *b);
    s->queue.push_front(last.id);
    take.pop_back();
  }
  if (take.empty()) return;
  const double admit = now_s();
  for (int64_t id : take) {
    Request& r = *s->reqs[id];
    r.state = State::kInflight;
    r.admit = admit;
  }
  s->inflight += (int)take.size();
  s->stats.admitted += (int64_t)take.size();
  s->stats.steps++;
  s->stats.max_inflight_seen = std::max(s->stats.max_inflight_seen, s->inflight);
  st.busy = true;
  st.reqs = take;
  st.admit = admit;
  core.dtab = core.table_bytes ? s->base + st.tables.off : nullptr;
  uint8_t* ws = s->base + st.ws.off;
  const bool grow = core.table_bytes > st.staging_bytes;
  lk.unlock();
  cudaStream_t stream = s->streams[k];
  bool ok = true;
  if (grow) {  // the stream is idle, so its staging buffer is free
    if (st.staging) cudaFreeHost(st.staging);
    st.staging = nullptr;
    st.staging_bytes = 0;
    const size_t want = std::max<size_t>(core.table_bytes * 2, 1 << 20);
    if (cudaHostAlloc(reinterpret_cast<void**>(&st.staging), want, cudaHostAllocDefault) ==
        cudaSuccess)
      st.staging_bytes = want;
    else
      ok = false;
  }
  if (ok && core.table_bytes) {
    batch_fill_tables(core, core.dtab, st.staging);
    ok = cudaMemcpyAsync(const_cast<void*>(core.dtab), st.staging, core.table_bytes,
                         cudaMemcpyHostToDevice, stream) == cudaSuccess;
  }
  if (ok) ok = batch_issue(core, ws, stream) == QSD_OK;
  if (ok)
    ok = cudaMemcpyAsync(st.status_host, ws + core.L.status, sizeof(unsigned),
                         cudaMemcpyDeviceToHost, stream) == cudaSuccess;
  if (ok) ok = cudaEventRecord(st.done, stream) == cudaSuccess;
  lk.lock();
  for (int i = 0; i < core.n; ++i) s->reqs[take[i]]->sel = core.t[i].result;
  if (!ok) {  // nothing more will be enqueued: finish the requests now
    cudaGetLastError();
    cudaStreamSynchronize(stream);
    for (int64_t id : take) {
      Request& r = *s->reqs[id];
      finish(s, r, QSD_ERR_CUDA, now_s());
      s->inflight--;
    }
    free_block(s, st.ws);
    free_block(s, st.tables);
    st.reqs.clear();
    st.busy = false;
    s->done_cv.notify_all();
  }
}

void engine_main(qsd_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    reap(s);
    if (s->stop) break;
    for (int k = 0; k < (int)s->steps.size(); ++k)
      if (!s->steps[k].busy && !s->queue.empty()) launch_step(s, k, lk);
    s->stats.queue_depth = (int)s->queue.size();
    s->stats.inflight = s->inflight;
    bool busy = false;
    for (const Step& st : s->steps) busy |= st.busy;
    if (busy)  // poll the steps' events
      s->work_cv.wait_for(lk, std::chrono::microseconds(20));
    else
      s->work_cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
  }
  // stopping: wait for the steps in flight
  for (Step& st : s->steps)
    if (st.busy) {
      lk.unlock();
      cudaEventSynchronize(st.done);
      lk.lock();
    }
  reap(s);
}

}  // namespace

extern "C" {

double qsd_server_clock(void) { return now_s(); }

qsd_status qsd_server_create(const qsd_server_options* opts, qsd_server_t* out) {
  if (!opts || !out) return QSD_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  qsd_server_options o = *opts;
  if (o.memory_budget == 0 || o.max_inflight < 0 || o.streams < 0 || o.max_batch < 0)
    return QSD_ERR_INVALID_ARGUMENT;
  if (o.val_bytes != 0 && o.val_bytes != 4 && o.val_bytes != 8) return QSD_ERR_INVALID_ARGUMENT;
  if (!o.max_inflight) o.max_inflight = 1024;
  if (!o.streams) o.streams = 2;
  if (!o.max_batch) o.max_batch = 256;
  if (o.streams > 16) return QSD_ERR_UNSUPPORTED;
  qsd_server_s* s = new (std::nothrow) qsd_server_s;
  if (!s) return QSD_ERR_OUT_OF_MEMORY;
  s->opts = o;
  std::memset(&s->stats, 0, sizeof(s->stats));
  cudaGetDevice(&s->device);
  qsd_status st = QSD_OK;
  if (cudaMalloc(reinterpret_cast<void**>(&s->base), o.memory_budget) != cudaSuccess) {
    cudaGetLastError();
    s->base = nullptr;
    st = QSD_ERR_OUT_OF_MEMORY;
  }
  s->arena.init(o.memory_budget);
  s->steps.resize(o.streams);
  for (int k = 0; k < o.streams && st == QSD_OK; ++k) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      st = QSD_ERR_CUDA;
      break;
    }
    s->streams.push_back(cs);
    if (cudaEventCreate(&s->steps[k].done) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s->steps[k].status_host), sizeof(unsigned),
                      cudaHostAllocDefault) != cudaSuccess)
      st = QSD_ERR_CUDA;
  }
  if (st == QSD_OK) {  // the epoch the device completion times are measured from
    if (cudaEventCreate(&s->epoch) != cudaSuccess ||
        cudaEventRecord(s->epoch, s->streams[0]) != cudaSuccess ||
        cudaEventSynchronize(s->epoch) != cudaSuccess)
      st = QSD_ERR_CUDA;
    s->epoch_host = now_s();
  }
  if (st != QSD_OK) {
    cudaGetLastError();
    qsd_server_destroy(s);
    return st;
  }
  s->engine = std::thread(engine_main, s);
  *out = s;
  return QSD_OK;
}

qsd_status qsd_server_add_tensor(qsd_server_t s, int order, const int64_t* dims,
                                 const int* input_mode_order, const int32_t* coords,
                                 int64_t stride, const void* vals, int64_t nnz, int* tensor_id) {
  if (!s || !dims || !tensor_id || order < 1 || nnz < 0) return QSD_ERR_INVALID_ARGUMENT;
  if (order > QSD_MAX_ORDER) return QSD_ERR_UNSUPPORTED;
  if (nnz > kMaxBatchNnz) return QSD_ERR_UNSUPPORTED;
  if (nnz > 0 && (!coords || stride < nnz || (s->opts.val_bytes && !vals)))
    return QSD_ERR_INVALID_ARGUMENT;
  Resident t;
  t.order = order;
  for (int i = 0; i < order; ++i) {
    if (dims[i] < 1) return QSD_ERR_INVALID_ARGUMENT;
    t.dims[i] = dims[i];
    t.tau[i] = input_mode_order ? input_mode_order[i] : i;
  }
  // the identity target checks the dims and the input order once
  qsd_plan_t probe = nullptr;
  qsd_status st = qsd_plan(order, t.dims, t.tau, t.tau, &probe);
  if (st != QSD_OK) return st;
  qsd_plan_destroy(probe);
  t.coords = coords;
  t.stride = stride;
  t.vals = vals;
  t.nnz = nnz;
  std::lock_guard<std::mutex> lk(s->mu);
  s->tensors.push_back(t);
  *tensor_id = (int)s->tensors.size() - 1;
  return QSD_OK;
}

qsd_status qsd_server_submit(qsd_server_t s, int tensor_id, const int* target_perm,
                             double arrival_s, int64_t* request_id) {
  if (!s || !target_perm || !request_id) return QSD_ERR_INVALID_ARGUMENT;
  std::unique_lock<std::mutex> lk(s->mu);
  if (tensor_id < 0 || tensor_id >= (int)s->tensors.size()) return QSD_ERR_INVALID_ARGUMENT;
  qsd_plan_t plan = nullptr;
  qsd_status st = plan_for(s, tensor_id, target_perm, &plan);
  if (st != QSD_OK) return st;
  auto r = std::make_unique<Request>();
  r->id = s->next_id++;
  r->tensor = tensor_id;
  r->plan = plan;
  r->arrival = arrival_s > 0 ? arrival_s : now_s();
  const int64_t id = r->id;
  *request_id = id;
  s->stats.submitted++;
  if (s->tensors[tensor_id].nnz == 0) {  // nothing to move
    s->reqs[id] = std::move(r);
    finish(s, *s->reqs[id], QSD_OK, now_s());
    s->done_cv.notify_all();
    return QSD_OK;
  }
  s->reqs[id] = std::move(r);
  s->queue.push_back(id);
  s->stats.max_queue_depth = std::max(s->stats.max_queue_depth, (int)s->queue.size());
  lk.unlock();
  s->work_cv.notify_one();
  return QSD_OK;
}

qsd_status qsd_server_poll(qsd_server_t s, qsd_server_result* out, int max_results,
                           int wait_ms, int* n) {
  if (!s || !n || max_results < 0 || (max_results > 0 && !out)) return QSD_ERR_INVALID_ARGUMENT;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->completed.empty() && wait_ms > 0)
    s->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms),
                        [&] { return !s->completed.empty(); });
  int k = 0;
  while (k < max_results && !s->completed.empty()) {
    Request& r = *s->reqs[s->completed.front()];
    s->completed.pop_front();
    const Resident& t = s->tensors[r.tensor];
    qsd_server_result& o = out[k++];
    std::memset(&o, 0, sizeof(o));
    o.request = r.id;
    o.tensor = r.tensor;
    o.status = r.status;
    o.nnz = t.nnz;
    o.stride = t.nnz;
    if (r.status == QSD_OK && t.nnz > 0) {
      o.coords = reinterpret_cast<const int32_t*>(s->base + r.c[r.sel].off);
      o.vals = s->opts.val_bytes ? s->base + r.v[r.sel].off : nullptr;
    }
    o.arrival_s = r.arrival;
    o.admit_s = r.admit;
    o.done_s = r.done;
    r.delivered = true;
  }
  *n = k;
  return QSD_OK;
}

qsd_status qsd_server_copy_result(qsd_server_t s, int64_t request_id, int32_t* dst_coords,
                                  int64_t dst_stride, void* dst_vals, void* stream) {
  if (!s) return QSD_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end() || it->second->state != State::kDone) return QSD_ERR_INVALID_ARGUMENT;
  const Request& r = *it->second;
  if (r.status != QSD_OK) return (qsd_status)r.status;
  const Resident& t = s->tensors[r.tensor];
  if (t.nnz == 0) return QSD_OK;
  if (!dst_coords || dst_stride < t.nnz || (s->opts.val_bytes && !dst_vals))
    return QSD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpy2DAsync(dst_coords, sizeof(int32_t) * dst_stride, s->base + r.c[r.sel].off,
                        sizeof(int32_t) * t.nnz, sizeof(int32_t) * t.nnz, t.order,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return QSD_ERR_CUDA;
  if (s->opts.val_bytes &&
      cudaMemcpyAsync(dst_vals, s->base + r.v[r.sel].off, (size_t)t.nnz * s->opts.val_bytes,
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return QSD_ERR_CUDA;
  return QSD_OK;
}

qsd_status qsd_server_release(qsd_server_t s, int64_t request_id) {
  if (!s) return QSD_ERR_INVALID_ARGUMENT;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end() || it->second->state != State::kDone) return QSD_ERR_INVALID_ARGUMENT;
    Request& r = *it->second;
    for (Block* b : {&r.c[0], &r.c[1], &r.v[0], &r.v[1]}) free_block(s, *b);
    if (!r.delivered)  // still in the completed list: drop it from there
      s->completed.erase(std::remove(s->completed.begin(), s->completed.end(), request_id),
                         s->completed.end());
    s->reqs.erase(it);
    s->stats.released++;
  }
  s->work_cv.notify_one();  // memory came back: queued requests may fit now
  return QSD_OK;
}

qsd_status qsd_server_get_stats(qsd_server_t s, qsd_server_stats* out) {
  if (!s || !out) return QSD_ERR_INVALID_ARGUMENT;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queue_depth = (int)s->queue.size();
  out->inflight = s->inflight;
  out->bytes_in_use = s->arena.used();
  out->peak_bytes = s->arena.peak();
  return QSD_OK;
}

void qsd_server_destroy(qsd_server_t s) {
  if (!s) return;
  if (s->engine.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      s->queue.clear();
    }
    s->work_cv.notify_all();
    s->engine.join();
  }
  for (Step& st : s->steps) {
    if (st.done) cudaEventDestroy(st.done);
    if (st.status_host) cudaFreeHost(st.status_host);
    if (st.staging) cudaFreeHost(st.staging);
  }
  for (cudaStream_t cs : s->streams) cudaStreamDestroy(cs);
  if (s->epoch) cudaEventDestroy(s->epoch);
  for (auto& kv : s->plans) qsd_plan_destroy(kv.second);
  if (s->base) cudaFree(s->base);
  delete s;
}

}  // extern "C"
