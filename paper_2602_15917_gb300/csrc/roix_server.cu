// Serving loop: continuous batching of compression requests under an HBM
// budget (roix_server_*). Host code only; the work is roix_compress_batch.
//
// The server owns one device arena of hbm_budget bytes, allocated at
// creation, and `lanes` contexts, each with a CUDA stream. A batch's
// workspace (the device state of its requests: masks, pixel sections,
// symbols, records, code tables) is carved out of the arena when the batch is
// admitted (first fit, 256-byte aligned) and given back when it completes, so
// one large volume may use most of the budget while many small projections
// share it. A scheduler thread loops:
//   1. reap: lanes whose completion event has fired hand their requests' sizes
//      and status (copied to pinned host memory behind the batch) to the
//      completion queue, free their region of the arena and become free;
//   2. admit: while a lane is free, the oldest pending request opens a batch
//      if its workspace fits the largest free region of the arena (otherwise
//      it waits, and so do the requests behind it), and every later pending
//      request with the same settings joins it in arrival order while the
//      batch has fewer than max_batch items and its workspace still fits that
//      region;
//   3. otherwise wait for a submission or a short poll interval.
// Requests that arrive while other batches run are admitted as soon as a lane
// and the memory they need free up, and batches on different lanes overlap on
// the device.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "roix_internal.cuh"
#include "roix_regions.h"

using namespace roix;

namespace {

using Clock = std::chrono::steady_clock;

bool same_settings(const roix_request& a, const roix_request& b) {
  // field by field: the structs may carry padding bytes of any value
  const roix_roi &ra = a.roi, &rb = b.roi;
  return a.dtype == b.dtype && ra.cmp == rb.cmp && ra.keep == rb.keep &&
         ra.connectivity == rb.connectivity && ra.dilate == rb.dilate &&
         std::memcmp(&ra.threshold, &rb.threshold, 8) == 0 &&
         std::memcmp(&ra.dark, &rb.dark, 8) == 0 && a.eb.mode == b.eb.mode &&
         std::memcmp(&a.eb.value, &b.eb.value, 8) == 0 && a.params.radius == b.params.radius &&
         a.params.chunk == b.params.chunk && std::memcmp(&a.params.fill, &b.params.fill, 8) == 0 &&
         (a.params.predictor == 2) == (b.params.predictor == 2);
}

struct Pending {
  roix_request req;
  double t_submit;
};

struct Lane {
  roix_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  u64* sizes_dev = nullptr;   // [max_batch]
  u64* sizes_host = nullptr;  // pinned
  u32* status_host = nullptr; // pinned
  bool busy = false;
  std::vector<Pending> batch;
  double t_admit = 0.0;
  u64 ws_off = 0, ws_size = 0;  // the batch's region of the arena
};

constexpr u64 kArenaAlign = 256;

}  // namespace

struct roix_server {
  int device = 0;
  roix_server_config cfg{};
  char* arena = nullptr;  // hbm_budget bytes of device memory
  Regions regions;        // its regions in use (scheduler thread, under mu)
  std::vector<Lane> lanes;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> pending;
  std::deque<roix_completion> done;
  std::thread thread;
  std::atomic<bool> stop{false};
  Clock::time_point t0;
  u64 submitted = 0, completed = 0, batches = 0, bytes_in = 0, max_queue = 0;
  std::string err;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

u64 request_bytes(const roix_request& r) {
  return r.dims.nx * r.dims.ny * r.dims.nz * (r.dtype == ROIX_F32 ? 4u : 2u);
}

size_t request_workspace(const roix_request& r, u32 n, const roix_request* more) {
  Desc c;
  const roix_dims one{1, 1, 1};
  if (make_desc(nullptr, r.dtype, one, &r.roi, &r.eb, &r.params, &c) != ROIX_OK) return ~size_t(0);
  std::vector<roix_item> items(n);
  for (u32 i = 0; i < n; ++i) {
    const roix_request& q = i == 0 ? r : more[i - 1];
    items[i] = roix_item{q.in, q.dims, q.out, q.cap, nullptr};
  }
  return batch_workspace(c, items.data(), n);
}

u64 round_up(u64 v, u64 a) { return (v + a - 1) / a * a; }

// Lane finished: completions out, region back to the arena, lane free
// (scheduler thread).
void reap(roix_server* s, Lane& L) {
  const double t = s->now();
  const u32 st = *L.status_host;
  std::lock_guard<std::mutex> lock(s->mu);
  for (size_t i = 0; i < L.batch.size(); ++i) {
    const Pending& p = L.batch[i];
    roix_completion c{};
    c.tag = p.req.tag;
    c.size = L.sizes_host[i];
    c.status = st ? (int32_t)st : (c.size > p.req.cap ? ROIX_ECAPACITY : ROIX_OK);
    c.t_submit = p.t_submit;
    c.t_admit = L.t_admit;
    c.t_done = t;
    s->done.push_back(c);
    ++s->completed;
  }
  if (L.ws_size) {
    s->regions.give(L.ws_off);
    L.ws_size = 0;
  }
  L.batch.clear();
  L.busy = false;
}

// Forms a batch from the pending queue for a free lane (scheduler thread).
bool admit(roix_server* s, Lane& L) {
  std::vector<Pending> batch;
  u64 need = 0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->pending.empty()) return false;
    const u64 room = s->regions.largest_gap();
    need = request_workspace(s->pending.front().req, 1, nullptr);
    if (need > room) return false;  // the oldest request waits for memory
    batch.push_back(s->pending.front());
    s->pending.pop_front();
    std::vector<roix_request> reqs{batch[0].req};
    for (auto it = s->pending.begin(); it != s->pending.end() && batch.size() < s->cfg.max_batch;) {
      if (!same_settings(it->req, batch[0].req)) {
        ++it;
        continue;
      }
      reqs.push_back(it->req);
      const u64 grown = request_workspace(reqs[0], (u32)reqs.size(), reqs.data() + 1);
      if (grown > room) {
        reqs.pop_back();
        break;  // arrival order is kept: later requests wait for the next batch
      }
      need = grown;
      batch.push_back(*it);
      it = s->pending.erase(it);
    }
    L.ws_size = round_up(need, kArenaAlign);  // (room is a multiple of kArenaAlign)
    L.ws_off = s->regions.take(L.ws_size);   // fits: need <= the largest gap
  }
  const u32 n = (u32)batch.size();
  std::vector<roix_item> items(n);
  for (u32 i = 0; i < n; ++i) {
    const roix_request& r = batch[i].req;
    items[i] = roix_item{r.in, r.dims, r.out, r.cap, (uint64_t*)(L.sizes_dev + i)};
  }
  const roix_request& r0 = batch[0].req;
  L.t_admit = s->now();
  // the batch works in its region; the context status word starts clear
  borrow_ws(L.ctx, s->arena + L.ws_off, L.ws_size);
  cudaMemsetAsync(s->arena + L.ws_off, 0, 4, L.stream);
  roix_status st = roix_compress_batch(L.ctx, n, items.data(), r0.dtype, &r0.roi, &r0.eb,
                                       &r0.params, L.stream);
  if (st == ROIX_OK) {
    cudaMemcpyAsync(L.sizes_host, L.sizes_dev, 8 * n, cudaMemcpyDeviceToHost, L.stream);
    cudaMemcpyAsync(L.status_host, L.ctx->ws, 4, cudaMemcpyDeviceToHost, L.stream);
    cudaMemsetAsync(L.ctx->ws, 0, 4, L.stream);
    cudaEventRecord(L.done, L.stream);
  }
  L.batch = std::move(batch);
  L.busy = true;
  s->batches++;
  if (st != ROIX_OK) {  // refused on the host: every request of the batch fails with it
    *L.status_host = (u32)st;
    for (u32 i = 0; i < n; ++i) L.sizes_host[i] = 0;
    reap(s, L);
  }
  return true;
}

void scheduler(roix_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    bool progress = false;
    for (Lane& L : s->lanes) {
      if (!L.busy) continue;
      const cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaSuccess) {
        reap(s, L);
        progress = true;
      } else {
        cudaGetLastError();  // "not ready" must not surface in a later launch check
      }
    }
    for (Lane& L : s->lanes)
      if (!L.busy && admit(s, L)) progress = true;
    if (progress) continue;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->stop && s->pending.empty()) {
      bool idle = true;
      for (Lane& L : s->lanes) idle = idle && !L.busy;
      if (idle) break;
    }
    s->cv.wait_for(lock, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" {

roix_status roix_server_create(int device, const roix_server_config* cfg, roix_server** out) {
  if (!cfg || !out || cfg->lanes == 0 || cfg->max_batch == 0 || cfg->max_batch > kMaxBatch ||
      cfg->hbm_budget < cfg->lanes * (u64)4096)
    return ROIX_EINVAL;
  *out = nullptr;
  roix_server* s = new roix_server();
  s->device = device;
  s->cfg = *cfg;
  s->regions.size = cfg->hbm_budget / kArenaAlign * kArenaAlign;
  s->t0 = Clock::now();
  s->lanes.resize(cfg->lanes);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  roix_status st = ROIX_OK;
  if (cudaMalloc(&s->arena, cfg->hbm_budget) != cudaSuccess) {
    cudaGetLastError();
    s->arena = nullptr;
    st = ROIX_ENOMEM;
  }
  for (Lane& L : s->lanes) {
    if (st != ROIX_OK) break;
    if ((st = roix_ctx_create(device, &L.ctx)) != ROIX_OK) break;
    if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&L.sizes_dev, 8 * cfg->max_batch) != cudaSuccess ||
        cudaMallocHost(&L.sizes_host, 8 * cfg->max_batch) != cudaSuccess ||
        cudaMallocHost(&L.status_host, 4) != cudaSuccess) {
      cudaGetLastError();
      st = ROIX_ENOMEM;
      break;
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (st != ROIX_OK) {
    roix_server_destroy(s);
    return st;
  }
  s->thread = std::thread(scheduler, s);
  *out = s;
  return ROIX_OK;
}

roix_status roix_server_submit(roix_server* s, const roix_request* r) {
  if (!s || !r) return ROIX_EINVAL;
  // a request must fit the budget on its own, and be a valid call
  Desc c;
  if (make_desc(nullptr, r->dtype, r->dims, &r->roi, &r->eb, &r->params, &c) != ROIX_OK)
    return ROIX_EINVAL;
  const u64 N = r->dims.nx * r->dims.ny * r->dims.nz;
  if ((N && !r->in) || !r->out || ((uintptr_t)r->out & 15)) return ROIX_EINVAL;
  if (request_workspace(*r, 1, nullptr) > s->cfg.hbm_budget) return ROIX_ENOMEM;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return ROIX_EBUSY;
    s->pending.push_back(Pending{*r, s->now()});
    s->submitted++;
    s->bytes_in += request_bytes(*r);
    if (s->pending.size() > s->max_queue) s->max_queue = s->pending.size();
  }
  s->cv.notify_one();
  return ROIX_OK;
}

uint32_t roix_server_poll(roix_server* s, roix_completion* out, uint32_t max) {
  if (!s || !out) return 0;
  std::lock_guard<std::mutex> lock(s->mu);
  uint32_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

roix_status roix_server_drain(roix_server* s, double timeout_s) {
  if (!s) return ROIX_EINVAL;
  const auto until = Clock::now() + std::chrono::duration<double>(timeout_s);
  while (Clock::now() < until) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      if (s->completed == s->submitted) return ROIX_OK;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  return ROIX_ETIMEOUT;
}

roix_status roix_server_get_stats(roix_server* s, roix_server_stats* out) {
  if (!s || !out) return ROIX_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->bytes_in = s->bytes_in;
  out->max_queue = s->max_queue;
  out->pending = s->pending.size();
  out->budget_bytes = s->cfg.hbm_budget;
  out->in_use_bytes = s->regions.in_use;
  return ROIX_OK;
}

roix_status roix_server_destroy(roix_server* s) {
  if (!s) return ROIX_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->thread.joinable()) s->thread.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (Lane& L : s->lanes) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.sizes_dev) cudaFree(L.sizes_dev);
    if (L.sizes_host) cudaFreeHost(L.sizes_host);
    if (L.status_host) cudaFreeHost(L.status_host);
    if (L.ctx) roix_ctx_destroy(L.ctx);
  }
  if (s->arena) cudaFree(s->arena);
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
  return ROIX_OK;
}

}  // extern "C"
