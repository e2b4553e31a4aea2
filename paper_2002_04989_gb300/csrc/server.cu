// Serving loop: continuous batching of eigenvector-component requests on one GPU.
//
// Requests (a host matrix A and the component columns j wanted, rows = all i)
// arrive on caller threads.  A scheduler thread admits them in arrival order while
// the device budget allows, and merges the waiting requests of one cost band (see
// cost_band) into one batched launch: all tridiagonalisations, bisections and
// identity evaluations of the batch share the persistent kernels of
// eeid_components_batched.  Up to `max_inflight` batches are on the GPU at once, each
// on its own stream with its own context (workspace), so requests that arrive while
// a batch runs are launched as soon as a slot and memory free up.  The contexts cut
// each reduction into launches of one round of the grid, so the other batch's
// kernels get SMs between them: a large request delays a small one by about one
// round of its reductions, not by its whole run.
// A request's matrix, output and eigenvalues stay resident on the device from
// admission until its results are copied back.  Device buffers come from the
// stream-ordered allocator; results go through pinned host buffers.
//
// Every kernel a batch runs depends only on the sizes of its own matrices, so a
// request's result is bitwise the same alone and in any mix.
#include "eeid.h"
#include "host_plan.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace eeid {
void set_last_error(const char* msg);
eeid_status set_round_launches(eeid_ctx* ctx, int enable);
eeid_status set_sm_reserve(eeid_ctx* ctx, int sms);
eeid_status reserve_workspace(eeid_ctx* ctx, size_t device_bytes, size_t staging_bytes);
}

namespace {

using Clock = std::chrono::steady_clock;

eeid_status sfail(eeid_status s, const std::string& m) {
  eeid::set_last_error(m.c_str());
  return s;
}

struct Request {
  uint64_t ticket = 0;
  int n = 0;
  std::vector<int64_t> cols;   // empty + all_cols = every column
  bool all_cols = true;
  int64_t ncols = 0;
  double* h_out = nullptr;     // caller's result buffers (n x ncols, n)
  double* h_lambda = nullptr;
  char* pinned = nullptr;      // [A n*n | out n*ncols | lambda n] host staging
  bool pooled = false;         // pinned comes from the server's pool (else cudaMallocHost)
  size_t bytes_a = 0, bytes_out = 0, bytes_lam = 0;
  size_t dev_bytes = 0;
  char* dev = nullptr;         // same layout on the device
  enum State { PENDING, RUNNING, DONE, CANCELLED } state = PENDING;
  eeid_status status = EEID_OK;
  Clock::time_point t_submit, t_launch, t_done;
  int64_t batch_id = -1, batch_size = 0;
};

struct Slot {
  eeid_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Request*> reqs;
  int64_t batch_id = -1;
};

}  // namespace

struct eeid_server {
  int device = 0;
  int sms = 1;
  size_t budget = 0;        // device bytes for resident requests
  size_t used = 0;
  int max_batch = 64;
  int max_pending = 4096;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_space;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> all;
  std::vector<Slot> slots;
  std::thread th;
  bool stop = false;
  uint64_t next_ticket = 1;
  int64_t next_batch = 0;
  int64_t batches_launched = 0;
  int64_t max_overlap = 0;  // most batches seen on the GPU at once
  eeid::PinnedPool pool;   // pinned staging (see host_plan.h), guarded by mu
  char* pool_mem = nullptr;
  // The server's own stream-ordered device pool for request buffers: warmed to the
  // request budget at creation and never trimmed, so no allocation maps new memory
  // while batches run, and without cross-stream reuse dependencies, so one slot's
  // allocation never waits for the other slot's frees.
  cudaMemPool_t mempool = nullptr;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t staging_bytes(const Request* r) { return r->bytes_a + r->bytes_out + r->bytes_lam; }

// Return a request's staging buffer (the pool part under the server mutex).
void release_staging(eeid_server* S, Request* r) {
  if (!r->pinned) return;
  if (r->pooled) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->pool.give(r->pinned, staging_bytes(r));
  } else {
    cudaFreeHost(r->pinned);
  }
  r->pinned = nullptr;
}

// Copy results to the callers' buffers, release device memory, mark done.
void finalize(eeid_server* S, Slot& sl, std::unique_lock<std::mutex>& lk, cudaError_t qerr) {
  std::vector<Request*> reqs;
  reqs.swap(sl.reqs);
  sl.busy = false;
  lk.unlock();
  eeid_status st = EEID_OK;
  if (qerr == cudaSuccess) {
    st = eeid_sync(sl.ctx, sl.stream);   // deferred warnings of this batch
    for (Request* r : reqs) {
      const double* out = (const double*)(r->pinned + r->bytes_a);
      memcpy(r->h_out, out, r->bytes_out);
      if (r->h_lambda) memcpy(r->h_lambda, r->pinned + r->bytes_a + r->bytes_out, r->bytes_lam);
    }
  } else {
    st = sfail(EEID_ERR_CUDA, std::string("serving batch failed: ") + cudaGetErrorString(qerr));
  }
  for (Request* r : reqs)
    if (r->dev) cudaFreeAsync(r->dev, sl.stream);
  lk.lock();
  const auto now = Clock::now();
  for (Request* r : reqs) {
    S->used -= r->dev_bytes;
    r->dev = nullptr;
    r->status = st;
    r->state = Request::DONE;
    r->t_done = now;
  }
  S->cv_done.notify_all();
}

// Batches from this band up (about 0.2 s of reductions and more) leave 1/16 of the SMs
// free of their persistent reduction CTAs, which take a whole SM each: a smaller batch
// launched meanwhile runs there at once instead of waiting for round boundaries.  The
// reserve is kept only while other work is around (requests waiting, or another batch on
// the GPU); a costly batch that arrives to an idle server takes every SM, and a request
// that arrives later waits at most for the end of one of its rounds.
constexpr int kReserveBand = 3;
// Pinned staging pool for requests, and each slot's pinned metadata stage.
constexpr size_t kPinnedPoolBytes = (size_t)1 << 30;
constexpr size_t kStageBytes = (size_t)64 << 20;
// A batch holds requests of one cost band only (eeid::cost_band), so a small request
// never waits for the reductions of a much larger one that happens to be queued with it.
int cost_band(const Request* r) { return eeid::cost_band(r->n, r->ncols); }

// Form a batch from the waiting requests that fit, upload, launch, download.  The
// batch is the longest run of waiting requests, in arrival order, that share the first
// one's cost band and fit the device budget.
bool launch(eeid_server* S, Slot& sl, std::unique_lock<std::mutex>& lk) {
  std::vector<Request*> batch;
  int band = -1;
  while (!S->pending.empty() && (int)batch.size() < S->max_batch) {
    Request* r = S->pending.front();
    if (!batch.empty() && cost_band(r) != band) break;
    if (S->used + r->dev_bytes > S->budget) {
      bool idle = batch.empty() && S->used == 0;
      if (idle) {  // can never fit
        S->pending.pop_front();
        r->status = sfail(EEID_ERR_NOMEM, "request exceeds the server's device budget");
        r->state = Request::DONE;
        r->t_done = Clock::now();
        S->cv_done.notify_all();
        S->cv_space.notify_all();
        continue;
      }
      break;  // wait for memory to free up (arrival order is kept)
    }
    S->pending.pop_front();
    S->used += r->dev_bytes;
    r->state = Request::RUNNING;
    if (batch.empty()) band = cost_band(r);
    batch.push_back(r);
  }
  if (batch.empty()) return false;
  bool others = !S->pending.empty();
  for (auto& x : S->slots) others |= (&x != &sl && x.busy);
  S->cv_space.notify_all();
  const int64_t bid = S->next_batch++;
  const auto now = Clock::now();
  for (Request* r : batch) {
    r->t_launch = now;
    r->batch_id = bid;
    r->batch_size = (int64_t)batch.size();
  }
  sl.busy = true;
  sl.reqs = batch;
  sl.batch_id = bid;
  int busy = 0;
  for (auto& x : S->slots) busy += x.busy;
  S->max_overlap = std::max<int64_t>(S->max_overlap, busy);
  S->batches_launched++;
  lk.unlock();

  cudaError_t e = cudaSuccess;
  std::vector<eeid_problem> probs(batch.size());
  for (size_t q = 0; q < batch.size() && e == cudaSuccess; ++q) {
    Request* r = batch[q];
    e = cudaMallocFromPoolAsync((void**)&r->dev, r->dev_bytes, S->mempool, sl.stream);
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(r->dev, r->pinned, r->bytes_a, cudaMemcpyHostToDevice, sl.stream);
    eeid_problem& p = probs[q];
    p.dA = (const double*)r->dev;
    p.lda = r->n;
    p.n = r->n;
    p.h_rows = nullptr;
    p.nrows = r->n;
    p.h_cols = r->all_cols ? nullptr : r->cols.data();
    p.ncols = r->ncols;
    p.d_out = (double*)(r->dev + r->bytes_a);
    p.d_lambda = (double*)(r->dev + r->bytes_a + r->bytes_out);
  }
  eeid_status st = EEID_OK;
  if (e == cudaSuccess && S->slots.size() > 1)
    st = eeid::set_sm_reserve(sl.ctx,
                              band >= kReserveBand && others ? std::max(1, S->sms / 16) : 0);
  if (e == cudaSuccess && st == EEID_OK)
    st = eeid_components_batched(sl.ctx, probs.data(), (int64_t)probs.size(), sl.stream);
  if (e == cudaSuccess && st >= 0)
    for (Request* r : batch) {
      e = cudaMemcpyAsync(r->pinned + r->bytes_a, r->dev + r->bytes_a, r->bytes_out + r->bytes_lam,
                          cudaMemcpyDeviceToHost, sl.stream);
      if (e != cudaSuccess) break;
    }
  if (e == cudaSuccess && st >= 0) e = cudaEventRecord(sl.done, sl.stream);
  lk.lock();
  if (e != cudaSuccess || st < 0) {
    // nothing usable was enqueued: fail the batch now
    finalize(S, sl, lk, e != cudaSuccess ? e : cudaErrorUnknown);
    for (Request* r : batch) r->status = (st < 0) ? st : EEID_ERR_CUDA;
  }
  return true;
}

void scheduler(eeid_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progress = false;
    for (auto& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      finalize(S, sl, lk, q);
      progress = true;
    }
    for (auto& sl : S->slots) {
      if (sl.busy || S->pending.empty()) continue;
      if (launch(S, sl, lk)) progress = true;
    }
    bool busy = false;
    for (auto& sl : S->slots) busy |= sl.busy;
    if (S->stop && S->pending.empty() && !busy) break;
    if (!progress) S->cv_sched.wait_for(lk, std::chrono::microseconds(busy ? 50 : 2000));
  }
}

}  // namespace

extern "C" {

eeid_status eeid_server_create(int device, const eeid_server_opts* opts, eeid_server** out) {
  if (!out) return sfail(EEID_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return sfail(EEID_ERR_CUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return sfail(EEID_ERR_INVALID, "device out of range");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return sfail(EEID_ERR_CUDA, cudaGetErrorString(e));
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  eeid_server* S = new eeid_server();
  S->device = device;
  cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, device);
  const size_t total = (opts && opts->hbm_budget_bytes) ? opts->hbm_budget_bytes : fr / 2;
  const int inflight = (opts && opts->max_inflight > 0) ? opts->max_inflight : 2;
  S->max_batch = (opts && opts->max_batch > 0) ? opts->max_batch : 64;
  S->max_pending = (opts && opts->max_pending > 0) ? opts->max_pending : 4096;
  // half of the budget for resident requests, the rest split over the batch workspaces
  S->budget = total / 2;
  const size_t ws_budget = (total - S->budget) / (size_t)inflight;
  S->slots.resize(inflight);
  for (auto& sl : S->slots) {
    eeid_status st = eeid_ctx_create(device, ws_budget, &sl.ctx);
    if (st == EEID_OK) st = eeid_set_graphs(sl.ctx, 0);
    // reductions in round-sized launches: the other slot's kernels get SMs in between
    if (st == EEID_OK) st = eeid::set_round_launches(sl.ctx, 1);
    // the whole workspace and a metadata stage now, so no batch allocates later (an
    // allocation would serialise the other slot's work with this one)
    if (st == EEID_OK) st = eeid::reserve_workspace(sl.ctx, ws_budget, kStageBytes);
    if (st == EEID_OK) {
      e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
      if (e != cudaSuccess) st = sfail(EEID_ERR_CUDA, cudaGetErrorString(e));
    }
    if (st != EEID_OK) {
      eeid_server_destroy(S);
      return st;
    }
  }
  if (cudaMallocHost((void**)&S->pool_mem, kPinnedPoolBytes) != cudaSuccess) {
    cudaGetLastError();   // no pool: every request allocates its own staging
    S->pool_mem = nullptr;
  }
  S->pool.init(S->pool_mem, kPinnedPoolBytes);
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&S->mempool, &props);
    uint64_t keep = UINT64_MAX;
    int no = 0;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(S->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess)
      e = cudaMemPoolSetAttribute(S->mempool, cudaMemPoolReuseAllowInternalDependencies, &no);
    void* warm = nullptr;
    cudaStream_t s0 = S->slots[0].stream;
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&warm, S->budget, S->mempool, s0);
    if (e == cudaSuccess) e = cudaFreeAsync(warm, s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) {
      eeid_server_destroy(S);
      return sfail(EEID_ERR_NOMEM, std::string("device pool: ") + cudaGetErrorString(e));
    }
  }
  S->th = std::thread(scheduler, S);
  *out = S;
  return EEID_OK;
}

void eeid_server_destroy(eeid_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (Request* r : S->pending) {
      r->state = Request::CANCELLED;
      r->status = EEID_ERR_CANCELLED;
    }
    S->pending.clear();
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_done.notify_all();
  S->cv_space.notify_all();
  if (S->th.joinable()) S->th.join();
  for (auto& kv : S->all) {
    if (kv.second->pinned && !kv.second->pooled) cudaFreeHost(kv.second->pinned);
    delete kv.second;
  }
  for (auto& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) eeid_ctx_destroy(sl.ctx);
  }
  if (S->pool_mem) cudaFreeHost(S->pool_mem);
  if (S->mempool) cudaMemPoolDestroy(S->mempool);
  delete S;
}

eeid_status eeid_server_submit(eeid_server* S, const double* hA, int64_t lda, int64_t n,
                               const int64_t* h_cols, int64_t ncols, double* h_out,
                               double* h_lambda_opt, int nonblocking, uint64_t* ticket) {
  if (!S || !ticket) return sfail(EEID_ERR_INVALID, "null server or ticket pointer");
  if (n < 1 || n > 4096) return sfail(EEID_ERR_INVALID, "n must be in [1, 4096]");
  if (!hA || lda < n || !h_out) return sfail(EEID_ERR_INVALID, "bad matrix or output pointer");
  const int64_t nc = h_cols ? ncols : n;
  if (nc < 1 || nc > n || (!h_cols && ncols != n)) return sfail(EEID_ERR_INVALID, "bad column count");
  Request* r = new Request();
  r->n = (int)n;
  r->all_cols = (h_cols == nullptr);
  r->ncols = nc;
  if (h_cols) {
    std::vector<char> seen(n, 0);
    r->cols.assign(h_cols, h_cols + nc);
    for (int64_t c : r->cols)
      if (c < 0 || c >= n || seen[c]++) {
        delete r;
        return sfail(EEID_ERR_INVALID, "column index out of range or repeated");
      }
  }
  r->h_out = h_out;
  r->h_lambda = h_lambda_opt;
  r->bytes_a = sizeof(double) * (size_t)n * n;
  r->bytes_out = sizeof(double) * (size_t)n * nc;
  r->bytes_lam = sizeof(double) * (size_t)n;
  r->dev_bytes = ((r->bytes_a + r->bytes_out + r->bytes_lam + 255) / 256) * 256;
  if (r->dev_bytes > S->budget) {
    delete r;
    return sfail(EEID_ERR_NOMEM, "request larger than the server's device budget");
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->pinned = S->pool.take(staging_bytes(r));
    r->pooled = r->pinned != nullptr;
  }
  if (!r->pinned) {
    cudaError_t e = cudaMallocHost((void**)&r->pinned, staging_bytes(r));
    if (e != cudaSuccess) {
      r->pinned = nullptr;
      delete r;
      return sfail(EEID_ERR_NOMEM, std::string("pinned staging: ") + cudaGetErrorString(e));
    }
  }
  double* pa = (double*)r->pinned;
  for (int64_t i = 0; i < n; ++i) memcpy(pa + i * n, hA + i * lda, sizeof(double) * n);
  r->t_submit = Clock::now();
  {
    std::unique_lock<std::mutex> lk(S->mu);
    if ((int)S->pending.size() >= S->max_pending) {
      if (nonblocking) {
        lk.unlock();
        release_staging(S, r);
        delete r;
        return sfail(EEID_ERR_BUSY, "server queue is full");
      }
      S->cv_space.wait(lk, [&] { return S->stop || (int)S->pending.size() < S->max_pending; });
      if (S->stop) {
        lk.unlock();
        release_staging(S, r);
        delete r;
        return sfail(EEID_ERR_CANCELLED, "server is shutting down");
      }
    }
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->all[r->ticket] = r;
    S->pending.push_back(r);
  }
  S->cv_sched.notify_one();
  return EEID_OK;
}

eeid_status eeid_server_wait(eeid_server* S, uint64_t ticket, int64_t timeout_ms,
                             eeid_req_stats* stats) {
  if (!S) return sfail(EEID_ERR_INVALID, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return sfail(EEID_ERR_NOT_FOUND, "unknown ticket");
  Request* r = it->second;
  auto ready = [&] { return r->state == Request::DONE || r->state == Request::CANCELLED; };
  if (timeout_ms < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return sfail(EEID_ERR_TIMEOUT, "request not finished within the timeout");
  }
  if (stats) {
    stats->queue_ms = r->state == Request::DONE && r->batch_id >= 0 ? ms_between(r->t_submit, r->t_launch) : 0.0;
    stats->total_ms = ms_between(r->t_submit, r->state == Request::DONE ? r->t_done : Clock::now());
    stats->batch_id = r->batch_id;
    stats->batch_requests = r->batch_size;
  }
  eeid_status st = r->state == Request::CANCELLED ? EEID_ERR_CANCELLED : r->status;
  S->all.erase(it);
  lk.unlock();
  release_staging(S, r);
  delete r;
  if (st == EEID_ERR_CANCELLED) return sfail(st, "request cancelled before it ran");
  return st;
}

eeid_status eeid_server_cancel(eeid_server* S, uint64_t ticket) {
  if (!S) return sfail(EEID_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return sfail(EEID_ERR_NOT_FOUND, "unknown ticket");
  Request* r = it->second;
  if (r->state != Request::PENDING) return sfail(EEID_ERR_BUSY, "request already running or done");
  S->pending.erase(std::find(S->pending.begin(), S->pending.end(), r));
  r->state = Request::CANCELLED;
  S->cv_done.notify_all();
  S->cv_space.notify_all();
  return EEID_OK;
}

eeid_status eeid_server_info(eeid_server* S, eeid_server_info_t* info) {
  if (!S || !info) return sfail(EEID_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  info->pending = (int64_t)S->pending.size();
  int busy = 0;
  for (auto& sl : S->slots) busy += sl.busy;
  info->inflight_batches = busy;
  info->batches_launched = S->batches_launched;
  info->max_overlapping_batches = S->max_overlap;
  info->device_bytes_in_use = (int64_t)S->used;
  info->device_budget_bytes = (int64_t)S->budget;
  return EEID_OK;
}

}  // extern "C"
