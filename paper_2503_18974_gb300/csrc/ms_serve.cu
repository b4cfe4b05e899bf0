// Serving loop for streams of detection requests: admission by a device
// memory budget, resident input buffers, continuous batching over several
// streams.  Host code only; the device work is ms_batch (ms.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/ms.h"

namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing, 256-byte granules.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  size_t size_;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;
};

size_t input_bytes(const ms_matrix& m) {
  const size_t elem = m.fmt == MS_U8 ? 1 : 4;
  const int64_t row = m.fmt == MS_U8 ? m.n : (m.n + 31) / 32;
  // rows are stored densely on the device, padded to 16 bytes
  const size_t ld = ((size_t)row * elem + 15) & ~(size_t)15;
  return (size_t)m.m * ld;
}

struct Request {
  uint64_t id;
  ms_matrix host;  // caller's host matrix
  const void* host_dev = nullptr;  // the same memory's device address when the GPU can
                                   // read it directly (pinned, mapped), else null
  ms_matrix dev;   // resident copy
  size_t off = 0, bytes = 0;
  double t_submit = 0, t_admit = 0, t_launch = 0, t_done = 0;
  cudaEvent_t copied = nullptr;      // owned: recorded after this request's copy round
  cudaEvent_t round_done = nullptr;  // the copy round's event (owned by its last request)
  ms_result result{};
};

// Gather copy of admitted inputs: the GPU reads each request's rows straight
// from pinned (mapped) host memory into its arena slot, so that a round of
// admissions costs a few kernel launches instead of one host call per
// request.  Descriptors travel as kernel parameters.
struct CopyDesc {
  const unsigned char* src;  // device address of the host rows
  unsigned char* dst;
  int64_t rows;
  int32_t row_bytes, src_ld, dst_ld, blocks;  // strides in bytes; blocks sharing it
};
constexpr int kCopyDescs = 48;  // per launch (the parameters stay below 4 KB)
struct CopyBatch {
  CopyDesc d[kCopyDescs];
  int32_t n;
};
static_assert(sizeof(CopyBatch) <= 4000, "kernel parameter size");

__global__ void k_gather_copy(const CopyBatch b) {
  const int k = blockIdx.y;
  if (k >= b.n) return;
  const CopyDesc c = b.d[k];
  if ((int)blockIdx.x >= c.blocks) return;
  // 4-byte words when every address and stride allows, else bytes
  const bool words = ((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst) |
                       (uintptr_t)c.row_bytes | (uintptr_t)c.src_ld | (uintptr_t)c.dst_ld) & 3u) == 0;
  const int64_t per_row = words ? c.row_bytes / 4 : c.row_bytes;
  const int64_t total = c.rows * per_row;
  const int64_t stride = (int64_t)c.blocks * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t r = t / per_row, e = t - r * per_row;
    if (words)
      *reinterpret_cast<uint32_t*>(c.dst + r * c.dst_ld + 4 * e) =
          *reinterpret_cast<const uint32_t*>(c.src + r * c.src_ld + 4 * e);
    else
      c.dst[r * c.dst_ld + e] = c.src[r * c.src_ld + e];
  }
}

struct Lane {  // one compute stream with its context and result buffers
  cudaStream_t stream = nullptr;
  ms_ctx* ctx = nullptr;
  ms_result* d_res = nullptr;
  ms_result* h_res = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<Request*> batch;
  bool busy = false;
  bool failed = false;  // the batch could not be launched; results already set
};

}  // namespace

struct ms_server {
  int device = 0;
  ms_server_config cfg{};
  unsigned char* d_arena = nullptr;
  Arena* arena = nullptr;
  cudaStream_t copy_stream = nullptr;
  std::vector<Lane> lanes;
  std::vector<cudaEvent_t> event_pool;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;   // submitted, not admitted (arrival order)
  std::deque<Request*> admitted;  // copy issued, not launched
  std::deque<ms_server_completion> done;
  uint64_t next_id = 1;
  int64_t launches = 0;           // batch launches attempted (scheduler thread only)
  int64_t outstanding = 0;        // submitted and not completed
  bool stop = false;
  ms_server_stats stats{};
  double host_copy_s = 0, host_batch_s = 0;
  std::thread worker;
  std::condition_variable idle_cv;
};

namespace {

cudaEvent_t take_event(ms_server* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void finish_request(ms_server* s, Request* r, std::vector<ms_server_completion>& out) {
  ms_server_completion c;
  c.id = r->id;
  c.result = r->result;
  c.t_submit = r->t_submit;
  c.t_admit = r->t_admit;
  c.t_launch = r->t_launch;
  c.t_done = r->t_done;
  out.push_back(c);
  s->arena->release(r->off, r->bytes);
  if (r->copied) s->event_pool.push_back(r->copied);
  delete r;
}

// One scheduler round; returns true if it made progress.  The lock guards the
// queues and statistics only: copies and batch launches are issued without
// it, so submissions never wait for the scheduler's CUDA calls.  Lanes,
// their batches and the admitted queue are touched by the scheduler thread
// alone.
bool schedule_round(ms_server* s) {
  bool progress = false;
  std::vector<ms_server_completion> finished;
  std::vector<Request*> newly;
  double copy_s = 0, batch_s = 0;
  // 1. completions
  for (Lane& ln : s->lanes) {
    if (!ln.busy || ln.failed) continue;
    const cudaError_t q = cudaEventQuery(ln.done);
    if (q == cudaErrorNotReady) continue;
    const double t = now_s();
    for (size_t k = 0; k < ln.batch.size(); ++k) {
      Request* r = ln.batch[k];
      r->result = q == cudaSuccess ? ln.h_res[k] : ms_result{0, -1, -1, (int32_t)MS_ERR_CUDA};
      r->t_done = t;
    }
    if (q != cudaSuccess) cudaGetLastError();
    progress = true;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Lane& ln : s->lanes) {
      if (!ln.busy || ln.batch.empty() || ln.batch[0]->t_done == 0) continue;
      for (Request* r : ln.batch) finish_request(s, r, finished);
      ln.batch.clear();
      ln.busy = false;
      ln.failed = false;
    }
    // 2. admission in arrival order while the arena has room
    while (!s->pending.empty()) {
      Request* r = s->pending.front();
      size_t off = 0;
      if (!s->arena->alloc(r->bytes, &off)) break;
      s->pending.pop_front();
      r->off = off;
      r->t_admit = now_s();
      newly.push_back(r);
      s->stats.peak_bytes = std::max<int64_t>(s->stats.peak_bytes, (int64_t)s->arena->used());
    }
    for (const ms_server_completion& c : finished) s->done.push_back(c);
    s->stats.completed += (int64_t)finished.size();
    s->outstanding -= (int64_t)finished.size();
  }
  if (!finished.empty()) s->idle_cv.notify_all();
  // copies of the newly admitted requests: one contiguous copy when the host
  // rows are already packed like the device rows, one event per round
  if (!newly.empty()) {
    const double t0 = now_s();
    CopyBatch cb;
    cb.n = 0;
    auto flush = [&]() {
      if (cb.n == 0) return;
      int most = 1;
      for (int k = 0; k < cb.n; ++k) most = std::max(most, cb.d[k].blocks);
      k_gather_copy<<<dim3((unsigned)most, (unsigned)cb.n), 256, 0, s->copy_stream>>>(cb);
      cb.n = 0;
    };
    for (Request* r : newly) {
      const ms_matrix& h = r->host;
      const size_t elem = h.fmt == MS_U8 ? 1 : 4;
      const int64_t row = h.fmt == MS_U8 ? h.n : (h.n + 31) / 32;
      const size_t dld_bytes = ((size_t)row * elem + 15) & ~(size_t)15;
      r->dev = h;
      r->dev.data = s->d_arena + r->off;
      r->dev.ld = (int64_t)(dld_bytes / elem);
      if (h.m <= 0 || row <= 0) continue;
      const size_t row_bytes = (size_t)row * elem, src_ld = (size_t)h.ld * elem;
      if (r->host_dev && row_bytes < (1u << 30) && src_ld < (1u << 30)) {
        CopyDesc& d = cb.d[cb.n++];
        d.src = static_cast<const unsigned char*>(r->host_dev);
        d.dst = s->d_arena + r->off;
        d.rows = h.m;
        d.row_bytes = (int32_t)row_bytes;
        d.src_ld = (int32_t)src_ld;
        d.dst_ld = (int32_t)dld_bytes;
        // about 64 KB per block, at most 64 blocks per request
        d.blocks = (int32_t)std::min<int64_t>(64, std::max<int64_t>(1, (h.m * (int64_t)row_bytes) >> 16));
        if (cb.n == kCopyDescs) flush();
      } else if (src_ld == dld_bytes) {
        cudaMemcpyAsync(s->d_arena + r->off, h.data, dld_bytes * (size_t)h.m,
                        cudaMemcpyHostToDevice, s->copy_stream);
      } else {
        cudaMemcpy2DAsync(s->d_arena + r->off, dld_bytes, h.data, src_ld, row_bytes, (size_t)h.m,
                          cudaMemcpyHostToDevice, s->copy_stream);
      }
    }
    flush();
    cudaEvent_t e = take_event(s);
    if (e) cudaEventRecord(e, s->copy_stream);
    for (size_t k = 0; k < newly.size(); ++k) {
      newly[k]->copied = (k + 1 == newly.size()) ? e : nullptr;  // the round's last owns it
      newly[k]->round_done = e;
      s->admitted.push_back(newly[k]);
    }
    copy_s += now_s() - t0;
    progress = true;
  }
  // 3. continuous batching: each free lane takes the copied requests
  for (Lane& ln : s->lanes) {
    if (ln.busy || s->admitted.empty()) continue;
    const double t0 = now_s();
    std::vector<ms_matrix> descs;
    cudaEvent_t last_ok = nullptr;
    while (!s->admitted.empty() && (int)ln.batch.size() < s->cfg.max_batch) {
      Request* r = s->admitted.front();
      if (r->round_done && r->round_done != last_ok) {
        if (cudaEventQuery(r->round_done) == cudaErrorNotReady) break;
        last_ok = r->round_done;
      }
      s->admitted.pop_front();
      ln.batch.push_back(r);
      descs.push_back(r->dev);
    }
    if (ln.batch.empty()) continue;
    const double t = now_s();
    for (Request* r : ln.batch) {
      r->t_launch = t;
      r->t_done = 0;
    }
    const int64_t ordinal = ++s->launches;
    ms_status st = (s->cfg.test_fail_batch > 0 && ordinal == s->cfg.test_fail_batch)
                       ? MS_ERR_CUDA  // test hook: this launch counts as failed
                       : ms_batch(ln.ctx, descs.data(), (int32_t)descs.size(), ln.d_res,
                                  reinterpret_cast<ms_stream_t>(ln.stream));
    if (st == MS_OK &&
        cudaMemcpyAsync(ln.h_res, ln.d_res, descs.size() * sizeof(ms_result),
                        cudaMemcpyDeviceToHost, ln.stream) != cudaSuccess)
      st = MS_ERR_CUDA;
    if (st == MS_OK && cudaEventRecord(ln.done, ln.stream) != cudaSuccess) st = MS_ERR_CUDA;
    if (st != MS_OK) {
      cudaGetLastError();
      for (Request* r : ln.batch) {
        r->result = ms_result{0, -1, -1, (int32_t)st};
        r->t_done = now_s();
      }
      ln.failed = true;
    }
    ln.busy = true;  // a failed batch completes at the next round
    int inflight = 0;
    for (const Lane& l2 : s->lanes) inflight += l2.busy ? 1 : 0;
    batch_s += now_s() - t0;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (st == MS_OK) s->stats.batches++;
      s->stats.peak_inflight = std::max(s->stats.peak_inflight, inflight);
    }
    progress = true;
  }
  if (copy_s > 0 || batch_s > 0) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->host_copy_s += copy_s;
    s->host_batch_s += batch_s;
  }
  return progress;
}

void worker_main(ms_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->outstanding == 0) return;
      if (s->outstanding == 0)
        s->cv.wait(lk, [&] { return s->stop || s->outstanding > 0; });
      if (s->stop && s->outstanding == 0) return;
    }
    if (!schedule_round(s)) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

double ms_server_now(void) { return now_s(); }

ms_status ms_server_create(ms_server** out, int device, const ms_server_config* cfg) {
  if (!out || !cfg || cfg->memory_budget_bytes == 0) return MS_ERR_INVALID;
  *out = nullptr;
  ms_server* s = new (std::nothrow) ms_server();
  if (!s) return MS_ERR_OOM;
  s->device = device;
  s->cfg = *cfg;
  if (s->cfg.streams <= 0) s->cfg.streams = 2;
  if (s->cfg.max_batch <= 0) s->cfg.max_batch = 512;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  ms_status st = MS_OK;
  if (cudaMalloc(&s->d_arena, cfg->memory_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    st = MS_ERR_OOM;
  }
  if (st == MS_OK) {
    s->arena = new Arena(cfg->memory_budget_bytes);
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      st = MS_ERR_CUDA;
  }
  for (int k = 0; st == MS_OK && k < s->cfg.streams; ++k) {
    Lane ln;
    if (cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&ln.d_res, sizeof(ms_result) * s->cfg.max_batch) != cudaSuccess ||
        cudaMallocHost(&ln.h_res, sizeof(ms_result) * s->cfg.max_batch) != cudaSuccess) {
      cudaGetLastError();
      st = MS_ERR_CUDA;
    } else if ((st = ms_create(&ln.ctx, device, 0)) != MS_OK) {
    }
    s->lanes.push_back(ln);
  }
  cudaSetDevice(prev);
  if (st != MS_OK) {
    ms_server_destroy(s);
    return st;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return MS_OK;
}

ms_status ms_server_submit(ms_server* s, const ms_matrix* host, double t_arrival, uint64_t* id) {
  if (!s || !host || !id) return MS_ERR_INVALID;
  if (host->m < 0 || host->n < 0 || (host->fmt != MS_U8 && host->fmt != MS_BITS32) ||
      host->reserved != 0)
    return MS_ERR_INVALID;
  if (host->m > 0 && host->n > 0 && !host->data) return MS_ERR_INVALID;
  const int64_t row = host->fmt == MS_U8 ? host->n : (host->n + 31) / 32;
  if (host->m > 0 && host->ld < row) return MS_ERR_INVALID;
  Request* r = new (std::nothrow) Request();
  if (!r) return MS_ERR_OOM;
  r->host = *host;
  if (host->m > 0 && host->n > 0) {
    // pinned host memory that the device maps is copied by the gather kernel
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, host->data) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr && pa.device == s->device)
      r->host_dev = pa.devicePointer;
    else
      cudaGetLastError();
  }
  r->bytes = std::max<size_t>(input_bytes(*host), 256);
  if (r->bytes > s->arena->size()) {
    delete r;
    return MS_ERR_BUDGET;
  }
  r->t_submit = t_arrival >= 0 ? t_arrival : now_s();
  uint64_t rid;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    rid = r->id = s->next_id++;
    s->pending.push_back(r);
    s->outstanding++;
    s->stats.submitted++;
  }
  // (r belongs to the scheduler from here on: it may already be finished
  // and freed, so only the local copy of its id is read)
  s->cv.notify_one();
  *id = rid;
  return MS_OK;
}

ms_status ms_server_poll(ms_server* s, ms_server_completion* out, int32_t max, int32_t* n_out) {
  if (!s || !n_out || (max > 0 && !out)) return MS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  int32_t n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  *n_out = n;
  return MS_OK;
}

ms_status ms_server_cancel(ms_server* s, uint64_t id) {
  if (!s) return MS_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = std::find_if(s->pending.begin(), s->pending.end(),
                           [&](const Request* r) { return r->id == id; });
    if (it == s->pending.end()) return MS_ERR_INVALID;  // unknown, or admitted already
    Request* r = *it;
    s->pending.erase(it);
    ms_server_completion c;
    c.id = r->id;
    c.result = ms_result{0, -1, -1, (int32_t)MS_ERR_CANCELLED};
    c.t_submit = r->t_submit;
    c.t_admit = c.t_launch = 0.0;
    c.t_done = now_s();
    delete r;  // never admitted: it holds no arena space or event
    s->done.push_back(c);
    s->stats.completed++;
    s->outstanding--;
  }
  s->idle_cv.notify_all();
  return MS_OK;
}

ms_status ms_server_wait_all(ms_server* s) {
  if (!s) return MS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  s->idle_cv.wait(lk, [&] { return s->outstanding == 0; });
  return MS_OK;
}

ms_status ms_server_stats_get(ms_server* s, ms_server_stats* out) {
  if (!s || !out) return MS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->host_batch_s = s->host_batch_s;
  out->host_copy_s = s->host_copy_s;
  return MS_OK;
}

ms_status ms_server_destroy(ms_server* s) {
  if (!s) return MS_ERR_INVALID;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv.notify_all();
    s->worker.join();
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (Lane& ln : s->lanes) {
    if (ln.ctx) ms_destroy(ln.ctx);
    if (ln.stream) cudaStreamDestroy(ln.stream);
    if (ln.done) cudaEventDestroy(ln.done);
    if (ln.d_res) cudaFree(ln.d_res);
    if (ln.h_res) cudaFreeHost(ln.h_res);
  }
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  for (Request* r : s->pending) delete r;
  for (Request* r : s->admitted) {
    if (r->copied) cudaEventDestroy(r->copied);
    delete r;
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->d_arena) cudaFree(s->d_arena);
  delete s->arena;
  cudaSetDevice(prev);
  delete s;
  return MS_OK;
}

}  // extern "C"
