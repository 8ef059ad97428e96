// kdb_serve.cu -- a build server on one GPU: requests are accepted as they
// arrive and built by continuous batching.
//
// A worker thread owns a few CUDA streams ("slots").  Whenever a slot is free
// it takes the requests waiting in the queue that share the head request's
// record layout (k, stride, split mode), as many as the device-memory budget
// and the batch cap allow, and enqueues on that slot: one copy in per
// request, one batched build of all of them (kdb_build_batched_async: every
// set is the paper's build, Sec. 3.2, and equals a build of that set alone),
// one copy out per request, and a host callback that marks the slot done.
// Requests that arrive while batches are running are admitted into the next
// free slot, so their work overlaps the running batches on the device.
// Device memory comes from a pool reserved for the server; a batch is charged
// its points and workspace when it is launched and released when it ends.
// If a batch fails on the device (a request with a NaN coordinate, say), the
// build leaves every record as it was and each of its requests runs again
// alone, so one bad request fails by itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "kdb.h"

namespace {

using Clock = std::chrono::steady_clock;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Req {
  int64_t id = 0;
  const unsigned char* h_in = nullptr;
  unsigned char* h_out = nullptr;
  int64_t n = 0;
  int k = 0, stride = 0, mode = 0;
  bool solo = false;  // its batch failed: it runs alone
  double t_submit = 0, t_admit = 0;
};

struct Server;

struct Slot {
  Server* srv = nullptr;
  cudaStream_t st = nullptr;
  uint32_t* h_err = nullptr;  // pinned: the batch's device error word
  std::vector<Req> reqs;
  size_t charged = 0;
  kdb_status launch_status = KDB_OK;
  bool busy = false;
  bool done = false;
  double t_done = 0;
};

struct Server {
  int dev = 0;
  size_t budget = 0;
  int max_inflight = 0;
  int64_t max_batch_points = 0;
  int max_batch_requests = 0;
  cudaMemPool_t pool = nullptr;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable wake;     // the worker: new request, finished batch, stop
  std::condition_variable results_cv;
  std::deque<Req> queue;
  std::deque<kdb_request_result> results;
  size_t used = 0;
  int busy = 0;
  bool stop = false;
  int64_t next_id = 0;
  kdb_server_stats stats{};
  std::thread worker;
  Clock::time_point t0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

// Workspace of a batch with these set sizes (0 if it cannot be built).
size_t batch_workspace(const std::vector<int64_t>& offs, int k, int stride, int mode) {
  return kdb_batched_workspace_size(offs.data(), (int)offs.size() - 1, k, stride,
                                    (kdb_split_mode)mode);
}

// Device bytes a batch is charged: points, workspace, error word.
size_t batch_charge(const std::vector<int64_t>& offs, int stride, size_t ws) {
  return align256((size_t)offs.back() * stride) + align256(ws) + 256;
}

void CUDART_CB on_batch_done(void* p) {
  Slot* sl = static_cast<Slot*>(p);
  Server* S = sl->srv;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    sl->done = true;
    sl->t_done = S->now();
  }
  S->wake.notify_all();
}

void push_result(Server& S, const Req& r, kdb_status st, double t_done) {
  kdb_request_result res{};
  res.id = r.id;
  res.status = st;
  res.n = r.n;
  res.submit_s = r.t_submit;
  res.admit_s = r.t_admit;
  res.done_s = t_done;
  S.results.push_back(res);
  ++S.stats.completed;
  if (st != KDB_OK) ++S.stats.failed;
}

// Finished batches: results out, memory back.  Called with the lock held.
bool reap(Server& S) {
  bool any = false;
  for (Slot& sl : S.slots) {
    if (!sl.busy || !sl.done) continue;
    any = true;
    const kdb_status st =
        sl.launch_status != KDB_OK ? sl.launch_status : kdb_error_word_status(*sl.h_err);
    if (st != KDB_OK && sl.reqs.size() > 1 && sl.launch_status == KDB_OK) {
      // the records of every set were left untouched: run each request
      // alone, ahead of the queue, in its original order
      for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) {
        Req r = *it;
        r.solo = true;
        S.queue.push_front(r);
      }
      S.stats.retried_alone += (int64_t)sl.reqs.size();
    } else {
      for (const Req& r : sl.reqs) push_result(S, r, st, sl.t_done);
    }
    S.used -= sl.charged;
    sl.charged = 0;
    sl.reqs.clear();
    sl.busy = false;
    sl.done = false;
    --S.busy;
  }
  if (any) S.results_cv.notify_all();
  return any;
}

// Takes the next batch from the queue: the head request and the later ones
// with the same layout, in arrival order, within the free budget and the
// caps.  Returns false (queue unchanged) if even the head does not fit yet.
// Called with the lock held.
bool form_batch(Server& S, std::vector<Req>& batch, std::vector<int64_t>& offs, size_t& ws,
                size_t& charge) {
  batch.clear();
  if (S.queue.empty()) return false;
  const Req head = S.queue.front();
  const size_t room = S.budget - S.used;
  std::vector<size_t> picked;
  int64_t pts = 0;
  size_t est = 0;
  for (size_t i = 0; i < S.queue.size(); ++i) {
    const Req& r = S.queue[i];
    if (r.k != head.k || r.stride != head.stride || r.mode != head.mode) continue;
    if (i > 0 && (head.solo || r.solo)) continue;
    if ((int)picked.size() >= S.max_batch_requests) break;
    if (!picked.empty() && pts + r.n > S.max_batch_points) break;
    // estimate: the request built alone
    const size_t one = align256((size_t)r.n * r.stride) +
                       kdb_workspace_size(r.n, r.k, r.stride, (kdb_split_mode)r.mode) + 1024;
    if (!picked.empty() && est + one > room) break;
    picked.push_back(i);
    pts += r.n;
    est += one;
    if (head.solo) break;
  }
  // exact charge; drop requests from the tail until it fits
  for (;;) {
    offs.assign(1, 0);
    for (size_t i : picked) offs.push_back(offs.back() + S.queue[i].n);
    ws = batch_workspace(offs, head.k, head.stride, head.mode);
    charge = batch_charge(offs, head.stride, ws);
    if (charge <= room) break;
    if (picked.size() == 1) return false;
    picked.pop_back();
  }
  std::deque<Req> rest;
  size_t j = 0;
  for (size_t i = 0; i < S.queue.size(); ++i) {
    if (j < picked.size() && picked[j] == i) {
      batch.push_back(S.queue[i]);
      ++j;
    } else {
      rest.push_back(S.queue[i]);
    }
  }
  S.queue.swap(rest);
  return true;
}

// Enqueues one batch on its slot's stream (lock not held).
void launch(Server& S, Slot& sl, const std::vector<int64_t>& offs, size_t ws_bytes) {
  const Req& h = sl.reqs.front();
  const size_t stride = (size_t)h.stride;
  unsigned char* buf = nullptr;
  kdb_status st = KDB_OK;
  if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&buf), sl.charged, S.pool, sl.st) != cudaSuccess) {
    cudaGetLastError();
    buf = nullptr;
    st = KDB_ERR_OUT_OF_MEMORY;
  }
  if (buf) {
    unsigned char* pts = buf;
    unsigned char* ws = buf + align256((size_t)offs.back() * stride);
    uint32_t* err = reinterpret_cast<uint32_t*>(ws + align256(ws_bytes));
    for (size_t b = 0; b < sl.reqs.size() && st == KDB_OK; ++b) {
      const Req& r = sl.reqs[b];
      if (r.n > 0 && cudaMemcpyAsync(pts + (size_t)offs[b] * stride, r.h_in, (size_t)r.n * stride,
                                     cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
        st = KDB_ERR_CUDA;
    }
    if (st == KDB_OK)
      st = kdb_build_batched_async(pts, offs.data(), (int)sl.reqs.size(), h.k, h.stride,
                                   (kdb_split_mode)h.mode, ws, ws_bytes, err,
                                   reinterpret_cast<kdb_stream_t>(sl.st));
    if (st == KDB_OK &&
        cudaMemcpyAsync(sl.h_err, err, 4, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
      st = KDB_ERR_CUDA;
    for (size_t b = 0; b < sl.reqs.size() && st == KDB_OK; ++b) {
      const Req& r = sl.reqs[b];
      if (r.h_out && r.n > 0 &&
          cudaMemcpyAsync(r.h_out, pts + (size_t)offs[b] * stride, (size_t)r.n * stride,
                          cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
        st = KDB_ERR_CUDA;
    }
    cudaFreeAsync(buf, sl.st);
  }
  if (st != KDB_OK) cudaGetLastError();
  sl.launch_status = st;
  if (cudaLaunchHostFunc(sl.st, on_batch_done, &sl) != cudaSuccess) {
    // no callback: wait here and complete the slot directly
    cudaGetLastError();
    cudaStreamSynchronize(sl.st);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(S.mu);
    sl.launch_status = sl.launch_status != KDB_OK ? sl.launch_status : KDB_ERR_CUDA;
    sl.done = true;
    sl.t_done = S.now();
  }
}

void worker_main(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.dev);
  std::unique_lock<std::mutex> lk(S.mu);
  std::vector<Req> batch;
  std::vector<int64_t> offs;
  for (;;) {
    reap(S);
    bool launched = false;
    for (Slot& sl : S.slots) {
      if (sl.busy) continue;
      size_t ws = 0, charge = 0;
      if (!form_batch(S, batch, offs, ws, charge)) break;
      const double t = S.now();
      for (Req& r : batch) r.t_admit = t;
      sl.reqs = batch;
      sl.charged = charge;
      sl.busy = true;
      sl.done = false;
      ++S.busy;
      S.used += charge;
      ++S.stats.batches;
      S.stats.max_batch_requests = std::max<int64_t>(S.stats.max_batch_requests, (int64_t)batch.size());
      S.stats.max_inflight_batches = std::max<int64_t>(S.stats.max_inflight_batches, S.busy);
      S.stats.max_used_bytes = std::max(S.stats.max_used_bytes, S.used);
      const std::vector<int64_t> o = offs;
      lk.unlock();
      launch(S, sl, o, ws);
      lk.lock();
      launched = true;
    }
    if (launched) continue;
    if (S.stop && S.queue.empty() && S.busy == 0) break;
    bool ready = false;
    for (const Slot& sl : S.slots) ready = ready || (sl.busy && sl.done);
    if (!ready) S.wake.wait_for(lk, std::chrono::milliseconds(50));
  }
}

}  // namespace

struct kdb_server_st {
  Server s;
};

extern "C" {

kdb_status kdb_server_create(const kdb_server_config* cfg, kdb_server* out) {
  if (!out) return KDB_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (!cfg || cfg->budget_bytes == 0 || cfg->max_inflight_batches < 1 ||
      cfg->max_inflight_batches > 16 || cfg->max_batch_points < 1 || cfg->max_batch_requests < 1)
    return KDB_ERR_INVALID_ARGUMENT;
  kdb_server_st* h = new (std::nothrow) kdb_server_st();
  if (!h) return KDB_ERR_OUT_OF_MEMORY;
  Server& S = h->s;
  S.t0 = Clock::now();
  S.budget = cfg->budget_bytes;
  S.max_inflight = cfg->max_inflight_batches;
  S.max_batch_points = std::min<int64_t>(cfg->max_batch_points, 2147483647LL);
  S.max_batch_requests = cfg->max_batch_requests;
  kdb_status st = KDB_OK;
  size_t free_b = 0, total_b = 0;
  if (cudaGetDevice(&S.dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return KDB_ERR_CUDA;
  }
  if (S.budget > free_b) {  // admission is by memory the device really has
    delete h;
    return KDB_ERR_OUT_OF_MEMORY;
  }
  cudaMemPoolProps props;
  memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = S.dev;
  if (cudaMemPoolCreate(&S.pool, &props) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return KDB_ERR_CUDA;
  }
  uint64_t keep = ~0ull;  // the pool keeps its memory: buffers stay resident
  int no = 0;             // an allocation never waits on another slot's stream
  cudaMemPoolSetAttribute(S.pool, cudaMemPoolAttrReleaseThreshold, &keep);
  cudaMemPoolSetAttribute(S.pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  S.slots.resize(S.max_inflight);
  for (Slot& sl : S.slots) {
    sl.srv = &S;
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&sl.h_err), 4) != cudaSuccess) {
      cudaGetLastError();
      st = KDB_ERR_CUDA;
      break;
    }
  }
  // reserve the budget once, so that admitted batches find their memory
  if (st == KDB_OK) {
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, S.budget, S.pool, S.slots[0].st) != cudaSuccess) {
      cudaGetLastError();
      st = KDB_ERR_OUT_OF_MEMORY;
    } else {
      cudaFreeAsync(p, S.slots[0].st);
      if (cudaStreamSynchronize(S.slots[0].st) != cudaSuccess) st = KDB_ERR_CUDA;
    }
  }
  // one small build per record layout the benchmarks serve (k = 3, float3
  // and float4 records) and per split mode, on zero points: the first launch
  // of a kernel loads it, which can stall the host thread that launches it,
  // so it happens here and not in the worker while batches are in flight
  if (st == KDB_OK) {
    const int64_t offs[3] = {0, 20000, 20100};
    const size_t ws_b = kdb_batched_workspace_size(offs, 2, 3, 16, KDB_SPLIT_WIDEST_EXTENT);
    const size_t ws_r = kdb_batched_workspace_size(offs, 2, 3, 16, KDB_SPLIT_ROUND_ROBIN);
    const size_t ws_bytes = std::max(std::max(ws_b, ws_r),
                                     std::max(kdb_batched_workspace_size(offs, 2, 3, 12, KDB_SPLIT_WIDEST_EXTENT),
                                              kdb_batched_workspace_size(offs, 2, 3, 12, KDB_SPLIT_ROUND_ROBIN)));
    const size_t pts_bytes = align256((size_t)offs[2] * 16);
    unsigned char* buf = nullptr;
    cudaStream_t s0 = S.slots[0].st;
    if (cudaMalloc(reinterpret_cast<void**>(&buf), pts_bytes + ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      st = KDB_ERR_OUT_OF_MEMORY;
    } else {
      for (int stride = 12; stride <= 16 && st == KDB_OK; stride += 4)
        for (int mode = 0; mode < 2 && st == KDB_OK; ++mode) {
          if (cudaMemsetAsync(buf, 0, pts_bytes, s0) != cudaSuccess) st = KDB_ERR_CUDA;
          if (st == KDB_OK)
            st = kdb_build_batched_async(buf, offs, 2, 3, stride, (kdb_split_mode)mode, buf + pts_bytes,
                                         ws_bytes, nullptr, reinterpret_cast<kdb_stream_t>(s0));
        }
      if (cudaStreamSynchronize(s0) != cudaSuccess && st == KDB_OK) st = KDB_ERR_CUDA;
      cudaFree(buf);
      cudaGetLastError();
    }
  }
  if (st != KDB_OK) {
    for (Slot& sl : S.slots) {
      if (sl.st) cudaStreamDestroy(sl.st);
      if (sl.h_err) cudaFreeHost(sl.h_err);
    }
    cudaMemPoolDestroy(S.pool);
    cudaGetLastError();
    delete h;
    return st;
  }
  S.stats.budget_bytes = S.budget;
  S.worker = std::thread(worker_main, &S);
  *out = h;
  return KDB_OK;
}

kdb_status kdb_server_submit(kdb_server srv, const void* h_points, void* h_out, int64_t n, int k,
                             int stride_bytes, kdb_split_mode mode, int64_t* out_id) {
  if (!srv || !out_id) return KDB_ERR_INVALID_ARGUMENT;
  Server& S = srv->s;
  if (n < 0 || n > 2147483647LL || k < 1 || k > 8 || stride_bytes < 4 * k || stride_bytes % 4 ||
      ((int)mode & ~(0xFF | KDB_COORDS_INT32 | KDB_COORDS_UINT32)) != 0 ||
      (((int)mode & KDB_COORDS_INT32) && ((int)mode & KDB_COORDS_UINT32)) || (n > 0 && !h_points))
    return KDB_ERR_INVALID_ARGUMENT;
  Req r;
  r.h_in = static_cast<const unsigned char*>(h_points);
  r.h_out = static_cast<unsigned char*>(h_out);
  r.n = n;
  r.k = k;
  r.stride = stride_bytes;
  r.mode = mode;
  if (n > 1) {
    const std::vector<int64_t> offs{0, n};
    const size_t ws = batch_workspace(offs, k, stride_bytes, mode);
    if (ws == 0) return KDB_ERR_INVALID_ARGUMENT;
    if (batch_charge(offs, stride_bytes, ws) > S.budget) return KDB_ERR_OUT_OF_MEMORY;
  }
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.stop) return KDB_ERR_INVALID_ARGUMENT;
    r.id = S.next_id++;
    r.t_submit = S.now();
    *out_id = r.id;
    ++S.stats.submitted;
    if (n <= 1) {  // already a tree
      if (n == 1 && r.h_out && r.h_out != r.h_in) memcpy(r.h_out, r.h_in, (size_t)stride_bytes);
      push_result(S, r, KDB_OK, r.t_submit);
      S.results_cv.notify_all();
      return KDB_OK;
    }
    S.queue.push_back(r);
  }
  S.wake.notify_all();
  return KDB_OK;
}

int kdb_server_poll(kdb_server srv, kdb_request_result* out, int max_results, int timeout_ms) {
  if (!srv || !out || max_results < 1) return -1;
  Server& S = srv->s;
  std::unique_lock<std::mutex> lk(S.mu);
  if (S.results.empty() && timeout_ms != 0) {
    auto has = [&] { return !S.results.empty(); };
    if (timeout_ms < 0) S.results_cv.wait(lk, has);
    else S.results_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), has);
  }
  int n = 0;
  while (n < max_results && !S.results.empty()) {
    out[n++] = S.results.front();
    S.results.pop_front();
  }
  return n;
}

kdb_status kdb_server_get_stats(kdb_server srv, kdb_server_stats* out) {
  if (!srv || !out) return KDB_ERR_INVALID_ARGUMENT;
  Server& S = srv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  *out = S.stats;
  out->queued = (int64_t)S.queue.size();
  int64_t inflight = 0;
  for (const Slot& sl : S.slots) inflight += sl.busy ? (int64_t)sl.reqs.size() : 0;
  out->inflight_requests = inflight;
  out->used_bytes = S.used;
  return KDB_OK;
}

kdb_status kdb_server_destroy(kdb_server srv) {
  if (!srv) return KDB_OK;
  Server& S = srv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.wake.notify_all();
  if (S.worker.joinable()) S.worker.join();
  kdb_status st = KDB_OK;
  for (Slot& sl : S.slots) {
    if (sl.st) {
      if (cudaStreamSynchronize(sl.st) != cudaSuccess) st = KDB_ERR_CUDA;
      cudaStreamDestroy(sl.st);
    }
    if (sl.h_err) cudaFreeHost(sl.h_err);
  }
  cudaMemPoolDestroy(S.pool);
  cudaGetLastError();
  delete srv;
  return st;
}

}  // extern "C"
