// knnm_server.cu -- the serving loop: J-Merge (Alg. 2, Sec. 3.2) applied to
// a stream of raw batches against a graph kept resident on the device.
//
// Resident state: vectors [capacity][d], lists ids/dists [capacity][K]; rows
// 0..n_committed-1 are live.  Each worker slot owns a library context (its
// own stream and scratch) and buffers for one batch: a copy of the resident
// lists taken at admission (the snapshot), the batch rows, and the merged
// lists of snapshot + batch.  A slot takes the oldest queued batch when the
// memory that batch needs is free, runs J-Merge on it with a seed derived
// from the request id, and commits on the server's commit stream:
//   - batch vectors are appended at commit_base, and batch ids in the result
//     are moved there;
//   - every snapshot row's list becomes the first K distinct entries of
//     (resident list, result list); batch rows are written as they are.
// Snapshots and commits are issued on one stream under the server lock, so a
// snapshot is exactly the state after the commits issued before it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/knnm.h"
#include "knnm_internal.cuh"

using namespace knnm;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Request {
  uint64_t id = 0;
  const float* batch = nullptr;
  int64_t rows = 0;
  ReqState state = QUEUED;
  Clock::time_point t_submit, t_admit, t_done;
  knnm_request_info info{};
  std::vector<int32_t> ids;  // [rows][K], ids in the snapshot's numbering
  std::vector<float> dists;
};

struct Slot {
  int index = 0;
  knnm_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_snap = nullptr, ev_commit = nullptr;
  int32_t* snap_ids = nullptr;  // [snap_rows][K]
  float* batch = nullptr;       // [batch_rows][d]
  int32_t* out_ids = nullptr;   // [out_rows][K]
  float* out_dists = nullptr;
  int64_t snap_rows = 0, batch_rows = 0, out_rows = 0;
  bool busy = false;
  std::thread worker;
};

// Host side of the library hash (chained SplitMix64 steps): H(seed, t,
// stream, owner, member).
uint64_t hash5(uint64_t seed, uint64_t t, uint64_t stream, uint64_t owner, uint64_t member) {
  return mix_step(hash_prefix(seed, t, stream, owner) ^ member);
}

constexpr uint64_t STREAM_SERVE = 4;

}  // namespace

struct knnm_server {
  int device = 0;
  int d = 0, K = 0;
  knnm_params params{};
  knnm_server_config cfg{};
  float* X = nullptr;       // resident vectors [capacity][d]
  int32_t* ids = nullptr;   // resident lists [capacity][K]
  float* dists = nullptr;
  cudaStream_t cstream = nullptr;  // snapshots and commits, in issue order
  std::mutex mu;
  std::condition_variable cv;  // queue, slot and completion changes
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Slot*> slots;
  int64_t n_committed = 0;    // live resident rows
  int64_t n_commits = 0;      // commits issued
  int64_t rows_reserved = 0;  // live rows + rows of queued or running batches
  int64_t inflight_rows = 0;  // rows of running batches (not yet committed)
  int in_flight = 0;
  bool stopping = false;
  int64_t submitted = 0, completed = 0, failed = 0, rows_completed = 0, max_concurrent = 0;
  std::vector<double> latencies;
  bool any_admit = false;
  Clock::time_point t_first_admit, t_last_done;
  char err[512] = {0};
};

namespace {

int sfail(knnm_server* S, int code, const char* fmt, ...) {
  if (S) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(S->err, sizeof(S->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define SRV_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return sfail(S, KNNM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// Device bytes one batch needs on a slot: the merge scratch plus the slot's
// snapshot, batch and output buffers.
struct Need {
  uint64_t scratch = 0;
  int64_t snap_rows = 0, batch_rows = 0, out_rows = 0;
};

int size_batch(knnm_server* S, Slot* sl, int64_t rows, int64_t snap_bound, Need* n) {
  int rc = knnm_merge_scratch_bytes(sl->ctx, 1, snap_bound, rows, S->d, &S->params, &n->scratch);
  if (rc) return sfail(S, rc, "batch of %lld rows: %s", (long long)rows, knnm_last_error(sl->ctx));
  n->snap_rows = snap_bound;
  n->batch_rows = rows;
  n->out_rows = snap_bound + rows;
  return KNNM_OK;
}

// Extra device memory the slot must allocate to hold `n` (buffers grow with
// 1/8 headroom; the old buffer is released before the new one is taken).
uint64_t extra_bytes(const knnm_server* S, const Slot* sl, const Need& n) {
  uint64_t extra = 0;
  const uint64_t held_scratch = ctx_scratch_bytes(sl->ctx);
  if (n.scratch > held_scratch) extra += n.scratch + (n.scratch >> 4) - held_scratch;
  auto grow = [&](int64_t want, int64_t have, uint64_t row_bytes) {
    if (want > have) extra += (uint64_t)(want + (want >> 3) - have) * row_bytes;
  };
  grow(n.snap_rows, sl->snap_rows, (uint64_t)S->K * 4);
  grow(n.batch_rows, sl->batch_rows, (uint64_t)S->d * 4);
  grow(n.out_rows, sl->out_rows, (uint64_t)S->K * 8);
  return extra;
}

bool fits(const knnm_server* S, uint64_t extra) {
  if (extra == 0) return true;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return extra + S->cfg.hbm_reserve_bytes <= (uint64_t)free_b;
}

template <typename T>
int grow_buffer(knnm_server* S, Slot* sl, T** p, int64_t* have, int64_t want, size_t row_elems) {
  if (want <= *have) return KNNM_OK;
  const int64_t rows = want + (want >> 3);
  if (*p) SRV_CUDA(cudaFreeAsync(*p, sl->stream));
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMallocAsync((void**)p, (size_t)rows * row_elems * sizeof(T), sl->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return sfail(S, KNNM_ERR_NOMEM, "slot %d: cannot allocate %lld rows: %s", sl->index,
                 (long long)rows, cudaGetErrorString(e));
  }
  *have = rows;
  return KNNM_OK;
}

// Grows the slot's scratch and buffers to hold `n` (slot idle).
int prepare_slot(knnm_server* S, Slot* sl, const Need& n) {
  int rc = ctx_reserve(sl->ctx, n.scratch);
  if (rc) return sfail(S, rc, "slot %d: %s", sl->index, knnm_last_error(sl->ctx));
  if ((rc = grow_buffer(S, sl, &sl->snap_ids, &sl->snap_rows, n.snap_rows, S->K))) return rc;
  if ((rc = grow_buffer(S, sl, &sl->batch, &sl->batch_rows, n.batch_rows, S->d))) return rc;
  if (n.out_rows > sl->out_rows) {
    int64_t have_i = sl->out_rows, have_d = sl->out_rows;
    rc = grow_buffer(S, sl, &sl->out_ids, &have_i, n.out_rows, S->K);
    if (!rc) rc = grow_buffer(S, sl, &sl->out_dists, &have_d, n.out_rows, S->K);
    sl->out_rows = rc ? 0 : have_i;
    if (rc) return rc;
  }
  // the buffers are used on the commit stream too
  SRV_CUDA(cudaStreamSynchronize(sl->stream));
  return KNNM_OK;
}

// Takes the snapshot of an admitted batch (server lock held): the resident
// lists as the commits issued so far leave them.
int take_snapshot(knnm_server* S, Slot* sl, Request* r) {
  const int64_t n_snap = S->n_committed;
  r->info.snapshot_rows = n_snap;
  r->info.snapshot_commits = S->n_commits;
  SRV_CUDA(cudaMemcpyAsync(sl->snap_ids, S->ids, (size_t)n_snap * S->K * 4,
                           cudaMemcpyDeviceToDevice, S->cstream));
  SRV_CUDA(cudaEventRecord(sl->ev_snap, S->cstream));
  return KNNM_OK;
}

// Runs one admitted batch on slot `sl` (server lock not held).  Returns the
// batch status; on success the commit has been issued and has completed.
int run_batch(knnm_server* S, Slot* sl, Request* r) {
  const int64_t n_snap = r->info.snapshot_rows;
  int rc;
  SRV_CUDA(cudaStreamWaitEvent(sl->stream, sl->ev_snap, 0));
  SRV_CUDA(cudaMemcpyAsync(sl->batch, r->batch, (size_t)r->rows * S->d * 4, cudaMemcpyDefault,
                           sl->stream));
  knnm_params p = S->params;
  p.seed = hash5(S->params.seed, 0, STREAM_SERVE, r->id, 0);
  knnm_stats st;
  const auto t_merge = Clock::now();
  rc = knnm_merge_joint(sl->ctx, S->X, n_snap, sl->snap_ids, sl->batch, r->rows, S->d, &p,
                        sl->out_ids, reinterpret_cast<float*>(sl->out_dists), &st);
  if (rc) return sfail(S, rc, "request %llu: %s", (unsigned long long)r->id,
                       knnm_last_error(sl->ctx));
  r->info.merge_ms = ms_between(t_merge, Clock::now());
  r->info.init_ms = st.ms_init;
  r->info.rounds_ms = st.ms_rounds;
  r->info.final_ms = st.ms_final;
  r->info.rounds = st.rounds;
  int64_t evals = 0;
  for (int t = 0; t < st.rounds; ++t) evals += st.dist_evals[t];
  r->info.dist_evals = evals;
  r->ids.resize((size_t)r->rows * S->K);
  r->dists.resize((size_t)r->rows * S->K);
  SRV_CUDA(cudaMemcpyAsync(r->ids.data(), sl->out_ids + (size_t)n_snap * S->K,
                           r->ids.size() * 4, cudaMemcpyDeviceToHost, sl->stream));
  SRV_CUDA(cudaMemcpyAsync(r->dists.data(), sl->out_dists + (size_t)n_snap * S->K,
                           r->dists.size() * 4, cudaMemcpyDeviceToHost, sl->stream));
  SRV_CUDA(cudaStreamSynchronize(sl->stream));
  const auto t_commit = Clock::now();
  {
    std::lock_guard<std::mutex> g(S->mu);
    const int64_t base = S->n_committed;
    r->info.commit_base = base;
    r->info.commit_seq = S->n_commits;
    SRV_CUDA(cudaMemcpyAsync(S->X + (size_t)base * S->d, sl->batch, (size_t)r->rows * S->d * 4,
                             cudaMemcpyDeviceToDevice, S->cstream));
    SRV_CUDA(launch_commit(n_snap, r->rows, S->K, S->ids, S->dists, sl->out_ids, sl->out_dists,
                           base, S->cstream));
    SRV_CUDA(cudaEventRecord(sl->ev_commit, S->cstream));
    S->n_committed += r->rows;
    S->n_commits += 1;
    S->inflight_rows -= r->rows;
  }
  SRV_CUDA(cudaEventSynchronize(sl->ev_commit));
  r->info.commit_ms = ms_between(t_commit, Clock::now());
  return KNNM_OK;
}

void worker_main(knnm_server* S, Slot* sl) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    if (S->queue.empty()) {
      if (S->stopping) return;
      S->cv.wait(lk);
      continue;
    }
    Request* r = S->queue.front();
    const int64_t bound = S->n_committed;  // the snapshot is taken right at admission
    Need need;
    int rc = size_batch(S, sl, r->rows, bound, &need);
    bool admit = rc == KNNM_OK && fits(S, extra_bytes(S, sl, need));
    if (rc == KNNM_OK && !admit) {
      // Leave the batch to another idle slot that can hold it, or to this one
      // once running batches finish; fail it if nothing can ever hold it.
      bool other = false;
      for (Slot* o : S->slots) {
        if (o == sl || o->busy) continue;
        Need on;
        if (size_batch(S, o, r->rows, bound, &on) == KNNM_OK && fits(S, extra_bytes(S, o, on)))
          other = true;
      }
      if (other || S->in_flight > 0) {
        S->cv.wait(lk);
        continue;
      }
      rc = sfail(S, KNNM_ERR_NOMEM, "request %llu (%lld rows) needs more device memory than "
                 "is free", (unsigned long long)r->id, (long long)r->rows);
    }
    S->queue.pop_front();
    if (rc == KNNM_OK) {
      // Device allocation with the lock held keeps admission, growth and the
      // snapshot one step; growth is rare (buffers keep 1/8 headroom).
      rc = prepare_slot(S, sl, need);
      if (rc == KNNM_OK) rc = take_snapshot(S, sl, r);
    }
    if (rc != KNNM_OK) {
      r->state = DONE;
      r->info.status = rc;
      r->t_done = Clock::now();
      S->rows_reserved -= r->rows;
      S->failed += 1;
      S->cv.notify_all();
      continue;
    }
    r->state = RUNNING;
    r->t_admit = Clock::now();
    r->info.slot = sl->index;
    if (!S->any_admit) {
      S->any_admit = true;
      S->t_first_admit = r->t_admit;
    }
    sl->busy = true;
    S->in_flight += 1;
    S->inflight_rows += r->rows;
    if (S->in_flight > S->max_concurrent) S->max_concurrent = S->in_flight;
    lk.unlock();
    rc = run_batch(S, sl, r);
    lk.lock();
    r->t_done = Clock::now();
    r->info.status = rc;
    r->info.queue_ms = ms_between(r->t_submit, r->t_admit);
    r->info.run_ms = ms_between(r->t_admit, r->t_done);
    r->info.latency_ms = ms_between(r->t_submit, r->t_done);
    if (rc == KNNM_OK) {
      S->completed += 1;
      S->rows_completed += r->rows;
      S->latencies.push_back(r->info.latency_ms);
    } else {
      S->failed += 1;
      if (r->info.commit_seq < 0) {  // never committed
        S->inflight_rows -= r->rows;
        S->rows_reserved -= r->rows;
      }
    }
    S->t_last_done = r->t_done;
    r->state = DONE;
    sl->busy = false;
    S->in_flight -= 1;
    S->cv.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  size_t rank = (size_t)(q * (double)v.size() + 0.999999);  // nearest rank
  if (rank < 1) rank = 1;
  if (rank > v.size()) rank = v.size();
  return v[rank - 1];
}

void free_server(knnm_server* S) {
  for (Slot* sl : S->slots) {
    if (sl->worker.joinable()) sl->worker.join();
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    cudaFree(sl->snap_ids);
    cudaFree(sl->batch);
    cudaFree(sl->out_ids);
    cudaFree(sl->out_dists);
    if (sl->ev_snap) cudaEventDestroy(sl->ev_snap);
    if (sl->ev_commit) cudaEventDestroy(sl->ev_commit);
    if (sl->ctx) knnm_destroy(sl->ctx);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    delete sl;
  }
  S->slots.clear();
  if (S->cstream) {
    cudaStreamSynchronize(S->cstream);
    cudaStreamDestroy(S->cstream);
  }
  cudaFree(S->X);
  cudaFree(S->ids);
  cudaFree(S->dists);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}

}  // namespace

extern "C" int knnm_server_create(int device, const float* Sv, int64_t n, const int32_t* G, int d,
                                  const knnm_params* params, const knnm_server_config* cfg,
                                  knnm_server** out) {
  if (!out || !Sv || !G || !params || !cfg) return KNNM_ERR_INVALID;
  *out = nullptr;
  if (params->k < 1 || params->k > 32 || d < 1 || n < params->k + 1 || cfg->slots < 1 ||
      cfg->slots > 64 || cfg->capacity_rows < n || cfg->capacity_rows > 0x7FFFFFFFLL ||
      cfg->max_batch_rows < 1 || params->metric < 0 ||
      params->metric > 4)  // dense rows only: the Jaccard metric takes set rows
    return KNNM_ERR_INVALID;
  knnm_server* S = new knnm_server();
  S->device = device;
  S->d = d;
  S->K = params->k;
  S->params = *params;
  S->cfg = *cfg;
  auto bail = [&](int rc) {
    free_server(S);
    return rc;
  };
  if (cudaSetDevice(device) != cudaSuccess) return bail(KNNM_ERR_CUDA);
  if (cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(KNNM_ERR_CUDA);
  const size_t cap = (size_t)cfg->capacity_rows;
  if (cudaMalloc(&S->X, cap * d * 4) != cudaSuccess ||
      cudaMalloc(&S->ids, cap * S->K * 4) != cudaSuccess ||
      cudaMalloc(&S->dists, cap * S->K * 4) != cudaSuccess) {
    cudaGetLastError();
    return bail(KNNM_ERR_NOMEM);
  }
  for (int i = 0; i < cfg->slots; ++i) {
    Slot* sl = new Slot();
    sl->index = i;
    S->slots.push_back(sl);
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl->ev_snap, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl->ev_commit, cudaEventDisableTiming) != cudaSuccess)
      return bail(KNNM_ERR_CUDA);
    if (knnm_create(&sl->ctx, device, sl->stream) != KNNM_OK) return bail(KNNM_ERR_CUDA);
    knnm_set_option(sl->ctx, KNNM_OPT_GRAPHS, cfg->use_graphs ? 1 : 0);
  }
  // The parameters and the largest batch must make a valid J-Merge.
  uint64_t probe = 0;
  int rc = knnm_merge_scratch_bytes(S->slots[0]->ctx, 1, n, cfg->max_batch_rows, d, params, &probe);
  if (rc) return bail(rc);

  // Resident rows and their lists (canonical distances, sorted).
  cudaStream_t st = S->cstream;
  int32_t* Gd = nullptr;
  float* norms = nullptr;
  DevCounters* ctr = nullptr;
  DevCounters hc;
  bool ok = cudaMemcpyAsync(S->X, Sv, (size_t)n * d * 4, cudaMemcpyDefault, st) == cudaSuccess &&
            cudaMalloc(&Gd, (size_t)n * S->K * 4) == cudaSuccess &&
            cudaMemcpyAsync(Gd, G, (size_t)n * S->K * 4, cudaMemcpyDefault, st) == cudaSuccess &&
            cudaMalloc(&ctr, sizeof(DevCounters)) == cudaSuccess &&
            cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st) == cudaSuccess &&
            cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st) == cudaSuccess;
  Rows rows{S->X, S->X, n, d};
  if (ok && params->metric == KNNM_COS)
    ok = cudaMalloc(&norms, (size_t)n * 4) == cudaSuccess &&
         launch_norms(rows, n, norms, st) == cudaSuccess;
  ok = ok && launch_list_dists(rows, n, Gd, S->K, params->metric, norms, S->ids, S->dists, ctr,
                               st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(Gd);
  cudaFree(norms);
  cudaFree(ctr);
  if (!ok) {
    cudaGetLastError();
    return bail(KNNM_ERR_CUDA);
  }
  if (hc.err) return bail(KNNM_ERR_INVALID);
  S->n_committed = n;
  S->rows_reserved = n;
  for (Slot* sl : S->slots) sl->worker = std::thread(worker_main, S, sl);
  *out = S;
  return KNNM_OK;
}

extern "C" int knnm_server_submit(knnm_server* S, const float* batch, int64_t rows,
                                  uint64_t req_id) {
  if (!S) return KNNM_ERR_INVALID;
  const int Kr = S->K - (int)((double)S->params.keep_ratio * (double)S->K);
  if (!batch || rows < 1 || rows < Kr)
    return sfail(S, KNNM_ERR_INVALID, "batch needs at least %d rows", Kr > 1 ? Kr : 1);
  std::lock_guard<std::mutex> g(S->mu);
  if (S->stopping) return sfail(S, KNNM_ERR_INVALID, "server is shutting down");
  if (S->reqs.count(req_id))
    return sfail(S, KNNM_ERR_INVALID, "request id %llu is in use", (unsigned long long)req_id);
  if (rows > S->cfg.max_batch_rows || S->rows_reserved + rows > S->cfg.capacity_rows)
    return sfail(S, KNNM_ERR_NOMEM, "batch of %lld rows exceeds the batch limit or capacity",
                 (long long)rows);
  Request* r = new Request();
  r->id = req_id;
  r->batch = batch;
  r->rows = rows;
  r->t_submit = Clock::now();
  r->info.req_id = req_id;
  r->info.rows = rows;
  r->info.commit_seq = -1;
  r->info.commit_base = -1;
  r->info.slot = -1;
  S->reqs[req_id] = r;
  S->queue.push_back(r);
  S->rows_reserved += rows;
  S->submitted += 1;
  S->cv.notify_all();
  return KNNM_OK;
}

extern "C" int knnm_server_wait(knnm_server* S, uint64_t req_id, int timeout_ms,
                                int32_t* ids_out, float* dists_out, knnm_request_info* info) {
  if (!S) return KNNM_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(req_id);
  if (it == S->reqs.end())
    return sfail(S, KNNM_ERR_INVALID, "unknown request id %llu", (unsigned long long)req_id);
  Request* r = it->second;
  auto done = [&] { return r->state == DONE; };
  if (timeout_ms < 0)
    S->cv.wait(lk, done);
  else if (!S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
    return KNNM_ERR_TIMEOUT;
  S->reqs.erase(it);
  lk.unlock();
  const int status = r->info.status;
  if (info) *info = r->info;
  if (status == KNNM_OK && (ids_out || dists_out)) {
    const int64_t n_snap = r->info.snapshot_rows, base = r->info.commit_base;
    std::vector<int32_t> ids(r->ids);
    for (auto& v : ids)
      if (v >= n_snap) v = (int32_t)(base + (v - n_snap));
    const size_t bytes = ids.size() * 4;
    if (ids_out) {
      if (cudaMemcpy(ids_out, ids.data(), bytes, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return sfail(S, KNNM_ERR_CUDA, "copying request %llu's ids out failed",
                     (unsigned long long)req_id);
      }
    }
    if (dists_out) {
      if (cudaMemcpy(dists_out, r->dists.data(), bytes, cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return sfail(S, KNNM_ERR_CUDA, "copying request %llu's distances out failed",
                     (unsigned long long)req_id);
      }
    }
  }
  delete r;
  return status;
}

extern "C" int knnm_server_drain(knnm_server* S, int timeout_ms) {
  if (!S) return KNNM_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  auto idle = [&] { return S->queue.empty() && S->in_flight == 0; };
  if (timeout_ms < 0)
    S->cv.wait(lk, idle);
  else if (!S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
    return KNNM_ERR_TIMEOUT;
  return KNNM_OK;
}

extern "C" int knnm_server_get_stats(knnm_server* S, knnm_server_stats* out) {
  if (!S || !out) return KNNM_ERR_INVALID;
  std::lock_guard<std::mutex> g(S->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->resident_rows = S->n_committed;
  out->rows_completed = S->rows_completed;
  out->max_concurrent = S->max_concurrent;
  out->p50_ms = percentile(S->latencies, 0.50);
  out->p99_ms = percentile(S->latencies, 0.99);
  out->busy_s = S->any_admit ? ms_between(S->t_first_admit, S->t_last_done) / 1000.0 : 0.0;
  if (out->busy_s < 0) out->busy_s = 0;
  return KNNM_OK;
}

extern "C" int knnm_server_resident(knnm_server* S, int64_t* rows, float* vectors, int32_t* ids,
                                    float* dists) {
  if (!S || !rows) return KNNM_ERR_INVALID;
  std::lock_guard<std::mutex> g(S->mu);
  int64_t n = S->n_committed;
  if (*rows >= 0 && *rows < n) n = *rows;
  *rows = n;
  SRV_CUDA(cudaStreamSynchronize(S->cstream));
  if (vectors) SRV_CUDA(cudaMemcpy(vectors, S->X, (size_t)n * S->d * 4, cudaMemcpyDefault));
  if (ids) SRV_CUDA(cudaMemcpy(ids, S->ids, (size_t)n * S->K * 4, cudaMemcpyDefault));
  if (dists) SRV_CUDA(cudaMemcpy(dists, S->dists, (size_t)n * S->K * 4, cudaMemcpyDefault));
  return KNNM_OK;
}

extern "C" const char* knnm_server_last_error(const knnm_server* S) {
  return S ? S->err : "no server";
}

extern "C" int knnm_server_destroy(knnm_server* S) {
  if (!S) return KNNM_ERR_INVALID;
  knnm_server_drain(S, -1);
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stopping = true;
    S->cv.notify_all();
  }
  free_server(S);
  return KNNM_OK;
}
