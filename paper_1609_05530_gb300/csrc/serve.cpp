// serve.cpp -- the serving loop: continuous batching of fit requests.
//
// Requests (one dataset each: columns u, v in host memory, subset offsets,
// family, options) arrive at any time through copula_server_submit.  A
// scheduler thread admits them in arrival order while a batch slot and room
// in the device arena are free, packs everything admitted together into one
// batched fit (copula_fit_batch: one launch sequence over all their subsets,
// longest first), and runs up to `streams` such batches at once on separate
// CUDA streams, so requests that arrive while others are on the GPU overlap
// with them.  A subset's result does not depend on which other requests
// share its batch.  Completions are detected with CUDA events; each request
// records its arrival, admission and completion times for the latency
// statistics.
//
// Device memory comes from a caller-owned arena (the HBM budget) managed by
// a first-fit allocator with coalescing; nothing is allocated on the device
// after creation.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "copula.h"
#include "internal.h"

// ---------------------------------------------------------------------------
// Arena: first-fit allocation of offsets inside [0, size), 256-byte granules,
// free neighbours coalesced.  Pure host bookkeeping.
// ---------------------------------------------------------------------------
struct copula_arena {
  size_t size = 0;
  size_t used = 0, peak = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> bytes
  std::map<size_t, size_t> live;         // offset -> bytes
};

extern "C" int copula_arena_create(copula_arena** a, size_t bytes) {
  if (!a || bytes < 256) return COPULA_ERR_ARG;
  copula_arena* r = new copula_arena();
  r->size = bytes & ~size_t(255);
  r->free_blocks[0] = r->size;
  *a = r;
  return COPULA_SUCCESS;
}

extern "C" int copula_arena_destroy(copula_arena* a) {
  if (!a) return COPULA_ERR_ARG;
  delete a;
  return COPULA_SUCCESS;
}

extern "C" int copula_arena_alloc(copula_arena* a, size_t bytes, size_t* offset) {
  if (!a || !offset) return COPULA_ERR_ARG;
  const size_t need = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
  for (auto it = a->free_blocks.begin(); it != a->free_blocks.end(); ++it) {
    if (it->second >= need) {
      const size_t off = it->first, len = it->second;
      a->free_blocks.erase(it);
      if (len > need) a->free_blocks[off + need] = len - need;
      a->live[off] = need;
      a->used += need;
      a->peak = std::max(a->peak, a->used);
      *offset = off;
      return COPULA_SUCCESS;
    }
  }
  return COPULA_ERR_WORKSPACE;  // no free block large enough
}

extern "C" int copula_arena_free(copula_arena* a, size_t offset) {
  if (!a) return COPULA_ERR_ARG;
  auto it = a->live.find(offset);
  if (it == a->live.end()) return COPULA_ERR_ARG;
  size_t off = it->first, len = it->second;
  a->live.erase(it);
  a->used -= len;
  auto nx = a->free_blocks.lower_bound(off);
  if (nx != a->free_blocks.end() && nx->first == off + len) {
    len += nx->second;
    nx = a->free_blocks.erase(nx);
  }
  if (nx != a->free_blocks.begin()) {
    auto pv = std::prev(nx);
    if (pv->first + pv->second == off) {
      pv->second += len;
      return COPULA_SUCCESS;
    }
  }
  a->free_blocks[off] = len;
  return COPULA_SUCCESS;
}

extern "C" int copula_arena_stats(copula_arena* a, size_t* used, size_t* peak, size_t* largest_free) {
  if (!a) return COPULA_ERR_ARG;
  size_t big = 0;
  for (const auto& kv : a->free_blocks) big = std::max(big, kv.second);
  if (used) *used = a->used;
  if (peak) *peak = a->peak;
  if (largest_free) *largest_free = big;
  return COPULA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Server.
// ---------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kStagingReserve = 4u << 20;  // pinned schedule staging per stream (no regrowth in service)
constexpr size_t kResultReserve = 4u << 20;   // pinned result buffer per stream: 200K subsets before any regrowth

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

struct Request {
  uint64_t ticket = 0;
  copula_request req;
  std::vector<int64_t> offsets;  // copy of the subset offsets
  Clock::time_point t_arrive, t_admit, t_done;
  int state = COPULA_REQ_PENDING;
  int rc = COPULA_SUCCESS;
  double combined = 0.0;
  size_t bytes = 0;  // device bytes of its inputs + outputs
};

struct Batch {
  std::vector<std::shared_ptr<Request>> reqs;
  size_t arena_off = 0;
  int stream = 0;
  cudaEvent_t done = nullptr;
  char* host = nullptr;  // pinned results
  size_t host_bytes = 0;
  int64_t S = 0;
  int32_t B = 0;
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct copula_server {
  int device = 0;
  char* arena_base = nullptr;
  copula_arena* arena = nullptr;
  int max_slots = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<char*> pinned;  // per stream: pinned result buffer
  std::vector<size_t> pinned_bytes;
  std::vector<bool> stream_busy;
  copula_ctx* ctx = nullptr;        // size queries
  std::vector<copula_ctx*> sctx;    // per stream: its own pinned schedule staging, so that a
                                    // batch never waits for another stream's upload

  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<Batch> inflight;
  uint64_t next_ticket = 1;
  int slots_used = 0;
  bool stop = false;
  std::thread worker;

  // statistics
  std::vector<double> latencies, queue_waits;
  Clock::time_point t_first{};
  Clock::time_point t_last{};
  bool any = false;
  int64_t fits_done = 0, batches = 0, batched_requests = 0, errors = 0;
  int max_inflight = 0;
};

namespace {

bool same_kind(const copula_request& a, const copula_request& b) {
  return a.dtype == b.dtype && a.opts.precision == b.opts.precision && a.opts.weight == b.opts.weight &&
         a.opts.max_iter == b.opts.max_iter && a.opts.rtol == b.opts.rtol && a.opts.block == b.opts.block;
}

// Try to form and launch one batch.  Called with the lock held.
bool launch_batch(copula_server* s) {
  if (s->pending.empty()) return false;
  int st = -1;
  for (size_t i = 0; i < s->stream_busy.size(); ++i)
    if (!s->stream_busy[i]) {
      st = (int)i;
      break;
    }
  if (st < 0) return false;
  // gather requests of the head's kind, in arrival order, while slots last
  std::vector<std::shared_ptr<Request>> take;
  const copula_request& kind = s->pending.front()->req;
  for (auto& r : s->pending) {
    if (s->slots_used + (int)take.size() >= s->max_slots) break;
    if (!same_kind(r->req, kind)) continue;
    take.push_back(r);
  }
  // shrink until the batch fits the arena
  while (!take.empty()) {
    const size_t es = kind.dtype == COPULA_DTYPE_F32 ? 4 : 8;
    int64_t n = 0, S = 0;
    std::vector<int64_t> doff(1, 0), soff(1, 0), dss(1, 0);
    std::vector<int32_t> fam;
    for (auto& r : take) {
      for (int64_t k = 1; k <= r->req.K; ++k) soff.push_back(n + r->offsets[k]);
      n += r->req.n;
      S += r->req.K;
      doff.push_back(n);
      dss.push_back(S);
      fam.push_back(r->req.family);
    }
    size_t ws = 0;
    int rc = copula_fit_batch_workspace_size(s->ctx, kind.dtype, &kind.opts, (int32_t)take.size(), fam.data(),
                                             doff.data(), soff.data(), dss.data(), &ws);
    if (rc != COPULA_SUCCESS) {
      // reject the first request of the batch; the rest stay pending
      auto bad = take.front();
      bad->rc = rc;
      bad->state = COPULA_REQ_ERROR;
      bad->t_done = Clock::now();
      s->pending.erase(std::find(s->pending.begin(), s->pending.end(), bad));
      ++s->errors;
      s->cv_done.notify_all();
      return true;
    }
    const size_t bytes = 2 * a256((size_t)n * es) + 3 * a256((size_t)S * 8) + a256((size_t)take.size() * 8) + a256(ws);
    size_t off = 0;
    if (copula_arena_alloc(s->arena, bytes, &off) != COPULA_SUCCESS) {
      if (take.size() == 1) return false;  // wait for memory to free up
      take.pop_back();
      continue;
    }
    char* base = s->arena_base + off;
    char* du = base;
    char* dv = du + a256((size_t)n * es);
    double* dth = (double*)(dv + a256((size_t)n * es));
    double* dvar = (double*)((char*)dth + a256((size_t)S * 8));
    int32_t* dst = (int32_t*)((char*)dvar + a256((size_t)S * 8));
    double* dcomb = (double*)((char*)dst + a256((size_t)S * 8));
    char* dws = (char*)dcomb + a256((size_t)take.size() * 8);
    cudaStream_t stream = s->streams[st];
    // pinned result buffer for this stream
    const size_t hb = (size_t)S * (8 + 8 + 4) + take.size() * 8;
    if (s->pinned_bytes[st] < hb) {
      if (s->pinned[st]) cudaFreeHost(s->pinned[st]);
      s->pinned[st] = nullptr;
      s->pinned_bytes[st] = 0;
      if (cudaHostAlloc((void**)&s->pinned[st], std::max(hb, (size_t)1 << 20), cudaHostAllocDefault) != cudaSuccess) {
        copula_arena_free(s->arena, off);
        return false;
      }
      s->pinned_bytes[st] = std::max(hb, (size_t)1 << 20);
    }
    size_t pos = 0;
    bool ok = true;
    for (auto& r : take) {
      ok = ok && cudaMemcpyAsync(du + pos * es, r->req.u, (size_t)r->req.n * es, cudaMemcpyHostToDevice, stream) ==
                     cudaSuccess;
      ok = ok && cudaMemcpyAsync(dv + pos * es, r->req.v, (size_t)r->req.n * es, cudaMemcpyHostToDevice, stream) ==
                     cudaSuccess;
      pos += (size_t)r->req.n;
    }
    rc = ok ? copula_fit_batch(s->sctx[st], (int32_t)take.size(), fam.data(), kind.dtype, du, dv, doff.data(), soff.data(),
                               dss.data(), dth, dvar, dst, dcomb, &kind.opts, dws, ws, stream)
            : COPULA_ERR_CUDA;
    char* h = s->pinned[st];
    if (rc == COPULA_SUCCESS) {
      ok = cudaMemcpyAsync(h, dth, (size_t)S * 8, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
           cudaMemcpyAsync(h + S * 8, dvar, (size_t)S * 8, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
           cudaMemcpyAsync(h + S * 16, dst, (size_t)S * 4, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
           cudaMemcpyAsync(h + S * 20, dcomb, take.size() * 8, cudaMemcpyDeviceToHost, stream) == cudaSuccess &&
           cudaEventRecord(s->events[st], stream) == cudaSuccess;
      if (!ok) rc = COPULA_ERR_CUDA;
    }
    const auto now = Clock::now();
    for (auto& r : take) s->pending.erase(std::find(s->pending.begin(), s->pending.end(), r));
    if (rc != COPULA_SUCCESS) {
      cudaStreamSynchronize(stream);
      copula_arena_free(s->arena, off);
      for (auto& r : take) {
        r->rc = rc;
        r->state = COPULA_REQ_ERROR;
        r->t_done = now;
        ++s->errors;
      }
      s->cv_done.notify_all();
      return true;
    }
    Batch b;
    b.reqs = take;
    b.arena_off = off;
    b.stream = st;
    b.done = s->events[st];
    b.host = h;
    b.S = S;
    b.B = (int32_t)take.size();
    for (auto& r : take) {
      r->state = COPULA_REQ_RUNNING;
      r->t_admit = now;
    }
    s->stream_busy[st] = true;
    s->slots_used += (int)take.size();
    s->inflight.push_back(b);
    s->max_inflight = std::max(s->max_inflight, (int)s->inflight.size());
    ++s->batches;
    s->batched_requests += (int64_t)take.size();
    return true;
  }
  return false;
}

// Retire finished batches.  Called with the lock held.
bool retire(copula_server* s) {
  bool any = false;
  for (size_t i = 0; i < s->inflight.size();) {
    Batch& b = s->inflight[i];
    const cudaError_t q = cudaEventQuery(b.done);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    const auto now = Clock::now();
    const double* th = (const double*)b.host;
    const double* var = (const double*)(b.host + b.S * 8);
    const int32_t* st = (const int32_t*)(b.host + b.S * 16);
    const double* comb = (const double*)(b.host + b.S * 20);
    int64_t base = 0;
    for (int32_t j = 0; j < b.B; ++j) {
      auto& r = b.reqs[j];
      r->t_done = now;
      if (q != cudaSuccess) {
        r->rc = COPULA_ERR_CUDA;
        r->state = COPULA_REQ_ERROR;
        ++s->errors;
      } else {
        if (r->req.theta_out) std::memcpy(r->req.theta_out, th + base, (size_t)r->req.K * 8);
        if (r->req.var_out) std::memcpy(r->req.var_out, var + base, (size_t)r->req.K * 8);
        if (r->req.status_out) std::memcpy(r->req.status_out, st + base, (size_t)r->req.K * 4);
        r->combined = comb[j];
        r->state = COPULA_REQ_DONE;
        ++s->fits_done;
        s->latencies.push_back(secs(r->t_arrive, r->t_done));
        s->queue_waits.push_back(secs(r->t_arrive, r->t_admit));
        s->t_last = now;
      }
      base += r->req.K;
    }
    copula_arena_free(s->arena, b.arena_off);
    s->stream_busy[b.stream] = false;
    s->slots_used -= b.B;
    s->inflight.erase(s->inflight.begin() + (long)i);
    any = true;
  }
  if (any) s->cv_done.notify_all();
  return any;
}

void scheduler(copula_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop || !s->pending.empty() || !s->inflight.empty()) {
    bool progress = retire(s);
    while (launch_batch(s)) progress = true;
    if (!progress) {
      // nothing to do right now: wake on a submit, or poll the GPU shortly
      s->cv_sched.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 2000 : 20));
    }
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p * (double)(v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int copula_server_create(copula_server** out, void* arena, size_t arena_bytes, int32_t max_slots, int32_t streams) {
  if (!out || !arena || arena_bytes < (1u << 20) || max_slots < 1 || streams < 1 || streams > 16)
    return COPULA_ERR_ARG;
  copula_server* s = new copula_server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return COPULA_ERR_CUDA;
  }
  s->arena_base = (char*)arena;
  copula_arena_create(&s->arena, arena_bytes);
  s->max_slots = max_slots;
  int rc = copula_ctx_create(&s->ctx);
  if (rc != COPULA_SUCCESS) {
    copula_arena_destroy(s->arena);
    delete s;
    return rc;
  }
  for (int i = 0; i < streams; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    copula_ctx* c = nullptr;
    const bool ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
                    copula_ctx_create(&c) == COPULA_SUCCESS &&
                    cop::ctx_reserve_staging(c, kStagingReserve) == COPULA_SUCCESS;
    if (!ok) {
      if (c) copula_ctx_destroy(c);
      if (ev) cudaEventDestroy(ev);
      if (st) cudaStreamDestroy(st);
      copula_server_destroy(s);  // releases the streams and contexts made so far (no worker yet)
      return COPULA_ERR_CUDA;
    }
    // (regrowing a pinned buffer in service would synchronise the device)
    char* pinned = nullptr;
    if (cudaHostAlloc((void**)&pinned, kResultReserve, cudaHostAllocDefault) != cudaSuccess) {
      copula_ctx_destroy(c);
      cudaEventDestroy(ev);
      cudaStreamDestroy(st);
      copula_server_destroy(s);
      return COPULA_ERR_CUDA;
    }
    s->sctx.push_back(c);
    s->streams.push_back(st);
    s->events.push_back(ev);
    s->pinned.push_back(pinned);
    s->pinned_bytes.push_back(kResultReserve);
    s->stream_busy.push_back(false);
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return COPULA_SUCCESS;
}

int copula_server_submit(copula_server* s, const copula_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return COPULA_ERR_ARG;
  if (req->family < 0 || req->family > 2 || !req->u || !req->v || !req->subset_offsets || req->K < 1 || req->n < 2)
    return COPULA_ERR_ARG;
  if (req->subset_offsets[0] != 0 || req->subset_offsets[req->K] != req->n) return COPULA_ERR_ARG;
  {
    size_t ws = 0;
    const int rc = copula_fit_workspace_size(nullptr, req->dtype, &req->opts, req->subset_offsets, req->K, &ws);
    if (rc != COPULA_SUCCESS) return rc;
    const size_t es = req->dtype == COPULA_DTYPE_F32 ? 4 : 8;
    const size_t need = 2 * a256((size_t)req->n * es) + 3 * a256((size_t)req->K * 8) + a256(8) + a256(ws);
    if (need > s->arena->size) return COPULA_ERR_WORKSPACE;
  }
  auto r = std::make_shared<Request>();
  r->req = *req;
  if (r->req.opts.max_iter <= 0) r->req.opts.max_iter = 64;
  if (!(r->req.opts.rtol > 0.0)) r->req.opts.rtol = r->req.opts.precision == COPULA_PREC_F64 ? 1e-13 : 1e-6;
  r->offsets.assign(req->subset_offsets, req->subset_offsets + req->K + 1);
  r->req.subset_offsets = nullptr;
  r->t_arrive = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return COPULA_ERR_ARG;
    r->ticket = s->next_ticket++;
    if (!s->any) {
      s->t_first = r->t_arrive;
      s->any = true;
    }
    s->pending.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv_sched.notify_one();
  return COPULA_SUCCESS;
}

static void fill_result(const Request& r, copula_result* res) {
  res->state = r.state;
  res->rc = r.rc;
  res->theta_combined = r.combined;
  res->latency_s = r.state == COPULA_REQ_DONE || r.state == COPULA_REQ_ERROR ? secs(r.t_arrive, r.t_done) : 0.0;
  res->queue_s = r.state != COPULA_REQ_PENDING ? secs(r.t_arrive, r.t_admit) : 0.0;
}

int copula_server_poll(copula_server* s, uint64_t ticket, copula_result* res) {
  if (!s || !res) return COPULA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return COPULA_ERR_ARG;
  fill_result(*it->second, res);
  if (res->state == COPULA_REQ_DONE || res->state == COPULA_REQ_ERROR) s->all.erase(it);
  return COPULA_SUCCESS;
}

int copula_server_wait(copula_server* s, uint64_t ticket, double timeout_s, copula_result* res) {
  if (!s || !res) return COPULA_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return COPULA_ERR_ARG;
  auto r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                           timeout_s > 0 ? timeout_s : 1e9));
  while (r->state == COPULA_REQ_PENDING || r->state == COPULA_REQ_RUNNING) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
  }
  fill_result(*r, res);
  if (res->state == COPULA_REQ_DONE || res->state == COPULA_REQ_ERROR) s->all.erase(r->ticket);
  return COPULA_SUCCESS;
}

int copula_server_stats(copula_server* s, copula_server_statistics* st) {
  if (!s || !st) return COPULA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->fits_done = s->fits_done;
  st->errors = s->errors;
  st->batches = s->batches;
  st->mean_batch = s->batches ? (double)s->batched_requests / (double)s->batches : 0.0;
  st->max_inflight_batches = s->max_inflight;
  const double span = s->any ? secs(s->t_first, s->t_last) : 0.0;
  st->fits_per_s = span > 0 ? (double)s->fits_done / span : 0.0;
  st->p50_s = percentile(s->latencies, 0.50);
  st->p99_s = percentile(s->latencies, 0.99);
  st->mean_queue_s = 0.0;
  for (double q : s->queue_waits) st->mean_queue_s += q;
  if (!s->queue_waits.empty()) st->mean_queue_s /= (double)s->queue_waits.size();
  size_t used = 0, peak = 0, big = 0;
  copula_arena_stats(s->arena, &used, &peak, &big);
  st->arena_peak_bytes = peak;
  st->pending = (int64_t)s->pending.size();
  return COPULA_SUCCESS;
}

int copula_server_reset_stats(copula_server* s) {
  if (!s) return COPULA_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->queue_waits.clear();
  s->fits_done = s->batches = s->batched_requests = s->errors = 0;
  s->max_inflight = 0;
  s->any = false;
  return COPULA_SUCCESS;
}

int copula_server_destroy(copula_server* s) {
  if (!s) return COPULA_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (size_t i = 0; i < s->streams.size(); ++i) {
    cudaStreamSynchronize(s->streams[i]);
    cudaStreamDestroy(s->streams[i]);
    cudaEventDestroy(s->events[i]);
    if (s->pinned[i]) cudaFreeHost(s->pinned[i]);
  }
  for (copula_ctx* c : s->sctx) copula_ctx_destroy(c);
  copula_ctx_destroy(s->ctx);
  copula_arena_destroy(s->arena);
  delete s;
  return COPULA_SUCCESS;
}

}  // extern "C"
