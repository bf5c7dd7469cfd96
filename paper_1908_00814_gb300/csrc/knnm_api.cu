// knnm_api.cu -- the C ABI of libknnm.so (include/knnm.h): argument checks,
// scratch management, host/device pointer handling and the round loop that
// drives the kernels of S-Merge (Alg. 1), J-Merge (Alg. 2) and the build.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/knnm.h"
#include "knnm_internal.cuh"

using namespace knnm;

struct knnm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  DevCounters* host_ctr = nullptr;  // pinned
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t rev[4] = {nullptr, nullptr, nullptr, nullptr};  // per-round phases
  int use_graphs = 0;  // replay each round as one captured CUDA graph
  int bucket_cap = 0;         // proposal slots per target and round (0: from K)
  uint32_t wait_polls = WAIT_LIMIT;  // polls before a device wait of the join gives up
  int fail_alloc = 0;         // scratch reservations still to fail (host-side injection)
  int tc_choice = 0;          // tensor-core precisions: 0 per-round choice, 1 always TC, 2 never
  cudaStream_t cap_stream = nullptr;  // private stream the round graph is captured on
  char err[512] = {0};
};

namespace {

int fail(knnm_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define KNNM_CUDA(call)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, KNNM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

// Bump allocator over the context's arena; sizes are rounded to 256 bytes.
struct Carver {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

int ensure_arena(knnm_ctx* ctx, size_t bytes) {
  if (ctx->fail_alloc > 0) {
    --ctx->fail_alloc;
    return fail(ctx, KNNM_ERR_NOMEM, "cannot reserve %zu bytes of device scratch (injected failure)",
                bytes);
  }
  if (bytes <= ctx->arena_bytes) return KNNM_OK;
  if (ctx->arena) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
  }
  size_t want = bytes + (bytes >> 4);
  cudaError_t e = cudaMalloc(&ctx->arena, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->arena = nullptr;
    return fail(ctx, KNNM_ERR_NOMEM, "cannot allocate %zu bytes of device scratch: %s", want,
                cudaGetErrorString(e));
  }
  ctx->arena_bytes = want;
  return KNNM_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct Derived {
  int K, K_keep, Kr, s, cap_new, cap_old;
};

int derive(knnm_ctx* ctx, const knnm_params* p, int mode, int64_t n1, Derived* out) {
  if (!p) return fail(ctx, KNNM_ERR_INVALID, "params is NULL");
  if (p->k < 1 || p->k > 32) return fail(ctx, KNNM_ERR_INVALID, "k=%d outside 1..32", p->k);
  if (p->metric < 0 || p->metric > 5) return fail(ctx, KNNM_ERR_INVALID, "bad metric %d", p->metric);
  if (p->precision < KNNM_FP32 || p->precision > KNNM_FP16_RERANK)
    return fail(ctx, KNNM_ERR_INVALID, "bad precision %d", p->precision);
  if (p->max_iters < 0 || p->max_iters > KNNM_MAX_ROUNDS)
    return fail(ctx, KNNM_ERR_INVALID, "max_iters=%d outside 0..%d", p->max_iters, KNNM_MAX_ROUNDS);
  if (!(p->sample_rate > 0.f) || !(p->keep_ratio >= 0.f) || !(p->keep_ratio <= 1.f) ||
      !(p->delta >= 0.f))
    return fail(ctx, KNNM_ERR_INVALID, "sample_rate, keep_ratio or delta out of range");
  Derived d;
  d.K = p->k;
  d.K_keep = (int)((double)p->keep_ratio * (double)d.K);
  if (mode == JOINT && n1 == 0) d.K_keep = d.K;
  d.Kr = d.K - d.K_keep;
  double sd = (double)p->sample_rate * (double)d.K;
  d.s = sd >= (double)d.K ? d.K : (int)sd;
  if (d.s < 1) d.s = 1;
  d.cap_new = 2 * d.s;
  d.cap_old = d.K + d.s;
  *out = d;
  return KNNM_OK;
}

// The join kernel a merge uses: the pipelined one when the shapes fit it,
// else the single-stage one (long rows, large candidate sets, unaligned rows).
struct JoinPath {
  bool pipe = false;
  JoinPlan plan;
  PipeArgs pa;
  size_t smem = 0;
  int grid = 0;
};

int choose_join(knnm_ctx* ctx, int precision, int metric, int cap_new, int cap_old, int d,
                bool rows_aligned, JoinPath* jp) {
  const bool tc = precision != KNNM_FP32 && metric != KNNM_L1 && metric != KNNM_CHI2;
  if (tc || rows_aligned) {
    if (plan_pipe(precision, metric, cap_new, cap_old, d, &jp->pa, &jp->smem, &jp->grid) ==
        cudaSuccess) {
      jp->pipe = true;
      return KNNM_OK;
    }
    cudaGetLastError();
  }
  cudaError_t e = plan_join(precision, metric, cap_new, cap_old, d, &jp->plan);
  if (e != cudaSuccess)
    return fail(ctx, KNNM_ERR_INVALID, "no join configuration for cap %d+%d, d=%d: %s", cap_new,
                cap_old, d, cudaGetErrorString(e));
  return KNNM_OK;
}

// Bucket slots per target and round for the join's proposals: enough that
// only targets offered far more than the average (hubs) spill into direct
// inserts.
int proposal_slots(const knnm_ctx* ctx, int K) {
  if (ctx->bucket_cap > 0) return ctx->bucket_cap;
  int b = (24 * K + 31) & ~31;
  return b < 64 ? 64 : (b > 1024 ? 1024 : b);
}

}  // namespace

// ---------------------------------------------------------------------------
// The merge driver shared by the three whole-merge entry points.
// ---------------------------------------------------------------------------
namespace {

struct MergeIn {
  int mode;
  const float* S1;
  int64_t n1;  // rows of S1 (= set split)
  const int32_t* G1;
  const float* S2;
  int64_t n2;
  const int32_t* G2;
  int d;
  // sets (JACCARD): all n1 + n2 rows as one CSR array on the device
  const int64_t* set_off = nullptr;
  const int32_t* set_items = nullptr;
  int64_t set_nnz = 0;  // entries of set_items
};

// With size_only set, nothing runs: the scratch the call would take (every
// array on the device) is written there.
int run_merge(knnm_ctx* ctx, const MergeIn& in, const knnm_params* params, int32_t* out_ids,
              float* out_dists, knnm_stats* stats, uint64_t* size_only = nullptr) {
  auto t_wall0 = std::chrono::steady_clock::now();
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  Derived D{};
  int rc = derive(ctx, params, in.mode, in.n1, &D);
  if (rc) return rc;
  const int64_t N = in.n1 + in.n2;
  const bool sets = in.set_off != nullptr;
  const int d = sets ? 1 : in.d;
  const int K = D.K;
  if (d < 1) return fail(ctx, KNNM_ERR_INVALID, "d=%d", d);
  if (sets != (params->metric == KNNM_JACCARD))
    return fail(ctx, KNNM_ERR_INVALID, sets ? "set rows take the Jaccard metric"
                                            : "the Jaccard metric takes set rows (knnm_*_sets)");
  if (sets && !size_only &&
      (!is_device_ptr(in.set_off) ||
       (in.set_nnz > 0 && (!in.set_items || !is_device_ptr(in.set_items)))))
    return fail(ctx, KNNM_ERR_INVALID, "set rows must be device arrays");
  if (in.n1 < 0 || in.n2 < 0 || N > 0x7FFFFFFFLL)
    return fail(ctx, KNNM_ERR_INVALID, "row counts out of range");
  if (!size_only && (!out_ids || !out_dists))
    return fail(ctx, KNNM_ERR_INVALID, "output arrays are NULL");
  if (in.mode == SYMMETRIC) {
    if (in.n1 < K + 1 || in.n2 < K + 1)
      return fail(ctx, KNNM_ERR_INVALID, "S-Merge needs n1, n2 >= k+1 (n1=%lld n2=%lld k=%d)",
                  (long long)in.n1, (long long)in.n2, K);
    if (in.n1 < D.Kr || in.n2 < D.Kr)
      return fail(ctx, KNNM_ERR_INVALID, "each set needs at least k - floor(r*k) = %d rows", D.Kr);
    if (!size_only && ((!sets && (!in.S1 || !in.S2)) || !in.G1 || !in.G2))
      return fail(ctx, KNNM_ERR_INVALID, "NULL input array");
  } else {
    if (N < K + 1) return fail(ctx, KNNM_ERR_INVALID, "n1+n2 must be >= k+1");
    if (in.n1 > 0 && (in.n1 < K + 1 || in.n2 < D.Kr ||
                      (!size_only && (!in.G1 || (!sets && !in.S1)))))
      return fail(ctx, KNNM_ERR_INVALID,
                  "J-Merge needs n1 >= k+1, n2 >= k - floor(r*k) and G1 when n1 > 0");
    if (in.n2 > 0 && !sets && !in.S2 && !size_only)
      return fail(ctx, KNNM_ERR_INVALID, "S_new is NULL");
  }
  // L1 has no tensor-core form
  const int precision = params->metric != KNNM_L1 && params->metric != KNNM_CHI2 &&
                                params->metric != KNNM_JACCARD
                            ? params->precision
                            : KNNM_FP32;
  if (precision != KNNM_FP32 && d % 8 != 0)
    return fail(ctx, KNNM_ERR_INVALID, "the tensor-core paths need d %% 8 == 0 (d=%d)", d);

  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));

  // Where does each array live?
  const bool s1_dev = size_only || sets || in.n1 == 0 || is_device_ptr(in.S1);
  const bool s2_dev = size_only || sets || in.n2 == 0 || is_device_ptr(in.S2);
  const bool g1_dev = size_only || !in.G1 || is_device_ptr(in.G1);
  const bool g2_dev = size_only || !in.G2 || is_device_ptr(in.G2);
  const bool oi_dev = size_only || is_device_ptr(out_ids);
  const bool od_dev = size_only || is_device_ptr(out_dists);

  // rows staged from the caller's device arrays need 16-byte alignment for bulk copies
  const bool rows_aligned = !sets && d % 4 == 0 && (size_only || !s1_dev || !s2_dev ||
                                           ((in.n1 == 0 || aligned16(in.S1)) &&
                                            (in.n2 == 0 || aligned16(in.S2))));
  JoinPath jp;
  rc = choose_join(ctx, precision, params->metric, D.cap_new, D.cap_old, d, rows_aligned, &jp);
  if (rc) return rc;
  const bool tc = precision != KNNM_FP32;
  // The tensor-core join settles a pair without FP32 work only when its
  // estimate proves the pair is no proposal (or the rows are small integers);
  // every other pair is re-ranked in canonical FP32 from global memory.  On
  // rounds where most pairs are proposals the FP32 join is faster with the
  // same result, so with a tensor-core precision both joins are planned and
  // each round takes one (see the choice after each round below).
  JoinPath jp32;
  const bool adaptive = tc && choose_join(ctx, KNNM_FP32, params->metric, D.cap_new, D.cap_old,
                                          d, rows_aligned, &jp32) == KNNM_OK;
  if (tc && !adaptive) ctx->err[0] = 0;

  const int bcap = proposal_slots(ctx, K);
  // candidate records (and the per-node entry fields) whenever a ring join runs
  const bool with_rec = jp.pipe || (adaptive && jp32.pipe);
  // Carve the scratch (two passes: size, then pointers).
  struct Ptrs {
    float* X;
    int32_t *G1, *G2, *oi;
    float* od;
    uint64_t *keys, *prev, *rear, *rev_new, *rev_old;
    uint8_t* flags;
    int32_t *new_ids, *new_cnt, *old_ids, *old_cnt;
    float* norms;
    __nv_bfloat16* Xb;
    float4* aux;
    float* rmax;
    __nv_bfloat16* Xe;
    float* wx;
    unsigned char* rec;
    DevCounters* ctr;
    int32_t* pcnt;
    uint64_t* bucket;
    int32_t* rcnt;
    unsigned long long *roffs, *rtile, *rtotal;
    int32_t* rbucket;
    int* tdev;
    uint4* info;
  } P;
  auto carve = [&](Carver& c) {
    P.X = (!s1_dev || !s2_dev) ? c.take<float>((size_t)N * d) : nullptr;
    P.G1 = (in.G1 && !g1_dev) ? c.take<int32_t>((size_t)in.n1 * K) : nullptr;
    P.G2 = (in.G2 && !g2_dev) ? c.take<int32_t>((size_t)in.n2 * K) : nullptr;
    P.oi = !oi_dev ? c.take<int32_t>((size_t)N * K) : nullptr;
    P.od = !od_dev ? c.take<float>((size_t)N * K) : nullptr;
    P.keys = c.take<uint64_t>((size_t)N * K);
    P.prev = c.take<uint64_t>((size_t)N * K);
    P.rear = c.take<uint64_t>((size_t)N * (D.Kr > 0 ? D.Kr : 1));
    P.rcnt = c.take<int32_t>((size_t)2 * N);
    P.roffs = c.take<unsigned long long>((size_t)2 * N + 1);
    P.rbucket = c.take<int32_t>((size_t)N * K);
    P.rtile = c.take<unsigned long long>((size_t)(2 * N + 1023) / 1024 + 1);
    P.rtotal = c.take<unsigned long long>(1);
    P.tdev = c.take<int>(1);
    P.info = with_rec ? c.take<uint4>((size_t)N) : nullptr;
    P.flags = c.take<uint8_t>((size_t)N * K);
    P.new_ids = c.take<int32_t>((size_t)N * D.cap_new);
    P.new_cnt = c.take<int32_t>((size_t)N);
    P.old_ids = c.take<int32_t>((size_t)N * D.cap_old);
    P.old_cnt = c.take<int32_t>((size_t)N);
    P.norms = params->metric == KNNM_COS ? c.take<float>((size_t)N) : nullptr;
    P.Xb = tc && !jp.pipe ? c.take<__nv_bfloat16>((size_t)N * d) : nullptr;
    P.aux = tc && !jp.pipe ? c.take<float4>((size_t)N) : nullptr;
    P.rmax = tc && !jp.pipe ? c.take<float>((size_t)N) : nullptr;
    P.Xe = tc && jp.pipe ? c.take<__nv_bfloat16>((size_t)N * jp.pa.dx) : nullptr;
    P.wx = tc && jp.pipe ? c.take<float>((size_t)N) : nullptr;
    P.rec = with_rec
                ? c.take<unsigned char>((size_t)N * rec_bytes(jp.pipe ? jp.pa.cap : jp32.pa.cap))
                : nullptr;
    P.ctr = c.take<DevCounters>(1);
    P.pcnt = c.take<int32_t>((size_t)N);
    P.bucket = c.take<uint64_t>((size_t)N * bcap);
  };
  Carver sizer;
  carve(sizer);
  if (size_only) {
    *size_only = sizer.off;
    return KNNM_OK;
  }
  rc = ensure_arena(ctx, sizer.off);
  if (rc) return rc;
  Carver real;
  real.base = (char*)ctx->arena;
  carve(real);

  // Stage host inputs.
  const float* X1 = in.S1;
  const float* X2 = in.S2;
  int64_t nx1 = in.n1;
  if (P.X) {
    if (in.n1 > 0)
      KNNM_CUDA(cudaMemcpyAsync(P.X, in.S1, (size_t)in.n1 * d * 4,
                                s1_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (in.n2 > 0)
      KNNM_CUDA(cudaMemcpyAsync(P.X + (size_t)in.n1 * d, in.S2, (size_t)in.n2 * d * 4,
                                s2_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    X1 = P.X;
    X2 = P.X + (size_t)in.n1 * d;
    nx1 = N;
  }
  if (in.n1 == 0) {  // build: every row lives in S_new
    X1 = X2;
    nx1 = N;
  }
  const int32_t* G1 = in.G1;
  const int32_t* G2 = in.G2;
  if (P.G1) {
    KNNM_CUDA(cudaMemcpyAsync(P.G1, in.G1, (size_t)in.n1 * K * 4, cudaMemcpyHostToDevice, st));
    G1 = P.G1;
  }
  if (P.G2) {
    KNNM_CUDA(cudaMemcpyAsync(P.G2, in.G2, (size_t)in.n2 * K * 4, cudaMemcpyHostToDevice, st));
    G2 = P.G2;
  }
  Rows rows{X1, X2 ? X2 : X1, nx1, d};
  rows.off = in.set_off;
  rows.items = in.set_items;
  const bool use_bulk = !sets && d % 4 == 0 && aligned16(rows.X1) && aligned16(rows.X2) &&
                        (nx1 == N || aligned16(rows.X2));

  int launches = 1;
  KNNM_CUDA(cudaEventRecord(ctx->ev[0], st));
  KNNM_CUDA(cudaMemsetAsync(P.ctr, 0, sizeof(DevCounters), st));
  KNNM_CUDA(cudaMemsetAsync(&P.ctr->err_row, 0xFF, 8, st));
  if (sets) {  // CSR offsets non-decreasing from 0, items ascending without repeats
    KNNM_CUDA(launch_check_sets(in.set_off, in.set_items, in.set_nnz, N, P.ctr, st));
    KNNM_CUDA(cudaMemcpyAsync(ctx->host_ctr, P.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                              st));
    KNNM_CUDA(cudaStreamSynchronize(st));
    if (ctx->host_ctr->err)
      return fail(ctx, KNNM_ERR_INVALID, "set row %llu is malformed (offsets or item order)",
                  (unsigned long long)ctx->host_ctr->err_row);
    ++launches;
  }
  if (P.norms) {
    KNNM_CUDA(launch_norms(rows, N, P.norms, st));
    ++launches;
  }
  if (P.Xb) {
    KNNM_CUDA(launch_bf16_prep(rows, N, P.Xb, P.aux, P.rmax, precision == KNNM_FP16_RERANK,
                               &P.ctr->inexact, st));
    ++launches;
  }
  if (P.Xe) {
    KNNM_CUDA(launch_bf16_ext(rows, N, jp.pa.dx, P.Xe, P.wx, precision == KNNM_FP16_RERANK,
                              &P.ctr->inexact, st));
    ++launches;
  }
  // the per-node entry fields: widths and norms into their words of P.info
  // (the sampler writes the k-th keys each round)
  if (P.info) {
    KNNM_CUDA(launch_fill_info(N, P.wx, P.norms, P.info, st));
    ++launches;
  }

  InitArgs ia;
  ia.mode = in.mode;
  ia.rows = rows;
  ia.N = N;
  ia.n1 = in.n1;
  ia.G1 = G1;
  ia.G2 = G2;
  ia.K = K;
  ia.K_keep = D.K_keep;
  ia.metric = params->metric;
  ia.seed = params->seed;
  ia.norms = P.norms;
  ia.vec4 = (!sets && d % 4 == 0 && aligned16(rows.X1) && aligned16(rows.X2)) ? 1 : 0;
  ia.keys = P.keys;
  ia.flags = P.flags;
  ia.rear = P.rear;
  ia.ctr = P.ctr;
  if (P.Xe) {
    // every row exact in its 16-bit copy: init reads the 16-bit rows
    KNNM_CUDA(cudaMemcpyAsync(ctx->host_ctr, P.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                              st));
    KNNM_CUDA(cudaStreamSynchronize(st));
    if (ctx->host_ctr->inexact == 0) {
      ia.Xe = P.Xe;
      ia.dx = jp.pa.dx;
      ia.half = precision == KNNM_FP16_RERANK ? 1 : 0;
    }
  }
  KNNM_CUDA(launch_init(ia, st));
  KNNM_CUDA(cudaMemcpyAsync(ctx->host_ctr, P.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  KNNM_CUDA(cudaEventRecord(ctx->ev[1], st));
  KNNM_CUDA(cudaStreamSynchronize(st));
  if (ctx->host_ctr->err)
    return fail(ctx, KNNM_ERR_INVALID, "input graph row %llu is malformed (%s)",
                (unsigned long long)ctx->host_ctr->err_row,
                (ctx->host_ctr->err & DERR_DUP_ID) ? "repeated id" : "id out of range or self");

  knnm_stats local;
  memset(&local, 0, sizeof(local));
  SampleArgs sa;
  sa.N = N;
  sa.K = K;
  sa.s = D.s;
  sa.seed = params->seed;
  sa.keys = P.keys;
  sa.flags = P.flags;
  sa.prev_keys = P.prev;
  sa.rev_new = nullptr;
  sa.rev_old = nullptr;
  sa.rcnt = P.rcnt;
  sa.roffs = P.roffs;
  sa.rbucket = P.rbucket;
  sa.tile_sum = P.rtile;
  sa.total = P.rtotal;
  sa.cap_new = D.cap_new;
  sa.cap_old = D.cap_old;
  sa.new_ids = P.new_ids;
  sa.new_cnt = P.new_cnt;
  sa.old_ids = P.old_ids;
  sa.old_cnt = P.old_cnt;
  sa.ctr = P.ctr;
  // The merge only needs old(u) where new(u) is not empty; skipping the rest
  // pays once few lists change (its extra counting pass costs more while most
  // nodes are active), so direct launches turn it on after a round with fewer
  // than N*K/8 updates; captured rounds always use it.
  sa.active_only = ctx->use_graphs ? 1 : 0;
  if (P.rec) {
    sa.rec = P.rec;
    sa.rec_cap = jp.pipe ? jp.pa.cap : jp32.pa.cap;
    sa.norms = P.norms;
    sa.K_list = K;
    sa.info = P.info;
    jp.pa.rec = P.rec;
    jp.pa.Xe = P.Xe;
    jp32.pa.rec = P.rec;
    jp32.pa.Xe = nullptr;
  }
  JoinArgs ja;
  ja.mode = in.mode;
  ja.rows = rows;
  ja.N = N;
  ja.n1 = in.n1;
  ja.K = K;
  ja.metric = params->metric;
  ja.norms = P.norms;
  ja.keys = P.keys;
  ja.cap_new = D.cap_new;
  ja.cap_old = D.cap_old;
  ja.new_ids = P.new_ids;
  ja.new_cnt = P.new_cnt;
  ja.old_ids = P.old_ids;
  ja.old_cnt = P.old_cnt;
  ja.bucket = P.bucket;
  ja.bcnt = P.pcnt;
  ja.bcap = bcap;
  ja.live_keys = P.keys;
  ja.ctr = P.ctr;
  ja.Xb = P.Xb;
  ja.aux = P.aux;
  ja.rmax = P.rmax;
  ja.use_bulk = use_bulk ? 1 : 0;
  ja.wait_polls = ctx->wait_polls;
  MergeArgs ma{N, K, P.keys, P.prev, P.flags, P.pcnt, bcap, P.bucket, P.ctr};
  KNNM_CUDA(cudaMemsetAsync(P.pcnt, 0, (size_t)N * 4, st));
  KNNM_CUDA(cudaMemsetAsync(P.rcnt, 0, (size_t)N * 8, st));

  const double stop_at = (double)params->delta * (double)N * (double)K;
  // One round: counters reset, sampler, join, bucketed update (plus, in graph
  // mode, the round-index bump that the next replay reads).
  // Phase events are recorded only when launching directly; a replayed graph
  // is timed as a whole.
  auto enqueue_round = [&](int t, cudaStream_t rs, bool use_tc) -> int {
    const bool timed = t > 0;
    KNNM_CUDA(cudaMemsetAsync(P.ctr, 0, sizeof(DevCounters), rs));
    KNNM_CUDA(cudaMemsetAsync(&P.ctr->err_row, 0xFF, 8, rs));
    sa.t = t;
    const bool alt = adaptive && !use_tc;  // a tensor-core precision taking the FP32 join
    const JoinPath& j = alt ? jp32 : jp;
    // the ring join reads its candidates from the records alone; their third
    // column is the rows' exactness width for the tensor-core ring join and
    // the cosine norm (or nothing) for the FP32 one
    sa.records_only = (P.rec && j.pipe) ? 1 : 0;
    sa.info_c = (tc && !alt && jp.pipe) ? 0 : (P.norms ? 1 : -1);
    sa.norms = (tc && !alt && jp.pipe) ? P.wx : P.norms;  // the same column without info
    if (timed) KNNM_CUDA(cudaEventRecord(ctx->rev[0], rs));
    KNNM_CUDA(launch_sample(sa, rs));
    if (timed) KNNM_CUDA(cudaEventRecord(ctx->rev[1], rs));
    const int jprec = alt ? KNNM_FP32 : precision;
    if (j.pipe)
      KNNM_CUDA(launch_pipe(jprec, ja, j.pa, j.smem, j.grid, rs));
    else
      KNNM_CUDA(launch_join(jprec, ja, j.plan, rs));
    if (timed) KNNM_CUDA(cudaEventRecord(ctx->rev[2], rs));
    ma.prefetch = sa.active_only;  // few proposals: the update waits on loads
    KNNM_CUDA(launch_bucket_update(ma, rs));
    if (timed) KNNM_CUDA(cudaEventRecord(ctx->rev[3], rs));
    if (sa.t_dev) KNNM_CUDA(launch_bump_int(P.tdev, rs));
    KNNM_CUDA(cudaMemcpyAsync(ctx->host_ctr, P.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                              rs));
    return KNNM_OK;
  };
  // Which join each round takes: with a tensor-core precision, the tensor-core
  // join while it pays (all rows small integers, or the last round re-ranked
  // under 10% of its pairs), else the FP32 join.  A round that ran the FP32
  // join predicts the re-rank share from its proposal share.
  const bool all_exact = tc && ctx->host_ctr->inexact == 0;
  bool use_tc = tc && (!adaptive || all_exact);
  if (adaptive && ctx->tc_choice == 1) use_tc = true;
  if (adaptive && ctx->tc_choice == 2) use_tc = false;
  // In graph mode each join gets its own captured round, made when first used.
  cudaGraphExec_t round_exec[2] = {nullptr, nullptr};
  auto drop_graphs = [&]() {
    for (auto& g : round_exec)
      if (g) cudaGraphExecDestroy(g);
  };
  auto capture = [&](bool path_tc, cudaGraphExec_t* out) -> int {
    cudaGraph_t graph = nullptr;
    // captured on the context's own stream (the caller's may be the legacy
    // default stream, which cannot capture); replayed on the caller's stream
    if (!ctx->cap_stream)
      KNNM_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    KNNM_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int crc = enqueue_round(0, ctx->cap_stream, path_tc);  // t is read from P.tdev
    cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (crc) {
      if (graph) cudaGraphDestroy(graph);
      return crc;
    }
    if (ce != cudaSuccess) return fail(ctx, KNNM_ERR_CUDA, "round capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess)
      return fail(ctx, KNNM_ERR_CUDA, "round graph instantiate: %s", cudaGetErrorString(ce));
    return KNNM_OK;
  };
  const bool graphs = ctx->use_graphs && params->max_iters > 0;
  if (graphs) {
    sa.t_dev = P.tdev;
    KNNM_CUDA(launch_set_int(P.tdev, 1, st));
  }
  for (int t = 1; t <= params->max_iters; ++t) {
    if (!graphs && t > 1)
      sa.active_only = (double)local.updates[t - 2] < (double)N * (double)K / 8.0 ? 1 : 0;
    if (graphs) {
      cudaGraphExec_t& g = round_exec[use_tc ? 1 : 0];
      if (!g) {
        rc = capture(use_tc, &g);
        if (rc) {
          drop_graphs();
          return rc;
        }
      }
      cudaEventRecord(ctx->rev[0], st);
      cudaError_t le = cudaGraphLaunch(g, st);
      cudaEventRecord(ctx->rev[3], st);
      if (le != cudaSuccess) {
        drop_graphs();
        return fail(ctx, KNNM_ERR_CUDA, "round graph launch: %s", cudaGetErrorString(le));
      }
    } else {
      rc = enqueue_round(t, st, use_tc);
      if (rc) return rc;
    }
    launches += 12;
    cudaError_t se = cudaStreamSynchronize(st);
    if (se != cudaSuccess) {
      drop_graphs();
      return fail(ctx, KNNM_ERR_CUDA, "round %d: %s", t, cudaGetErrorString(se));
    }
    const DevCounters& h = *ctx->host_ctr;
    if (h.err) {
      drop_graphs();
      return fail(ctx, KNNM_ERR_DEVICE, "round %d: device error bits 0x%llx (row %llu)", t,
                  (unsigned long long)h.err, (unsigned long long)h.err_row);
    }
    local.updates[t - 1] = (int64_t)h.updates;
    local.dist_evals[t - 1] = (int64_t)h.dist_evals;
    local.proposals[t - 1] = (int64_t)h.proposals;
    local.reranked[t - 1] = (int64_t)h.reranked;
    local.gathered[t - 1] = (int64_t)h.gathered;
    local.spilled[t - 1] = (int64_t)h.overflow;
    if (use_tc) local.tc_rounds |= 1ull << (t - 1);
    if (graphs) {
      cudaEventElapsedTime(&local.ms_join[t - 1], ctx->rev[0], ctx->rev[3]);
    } else {
      cudaEventElapsedTime(&local.ms_sample[t - 1], ctx->rev[0], ctx->rev[1]);
      cudaEventElapsedTime(&local.ms_join[t - 1], ctx->rev[1], ctx->rev[2]);
      cudaEventElapsedTime(&local.ms_update[t - 1], ctx->rev[2], ctx->rev[3]);
    }
    cudaGetLastError();  // a timing query that failed leaves no error behind
    local.rounds = t;
    if ((double)h.updates <= stop_at) break;
    if (adaptive && !all_exact && ctx->tc_choice == 0) {
      const double ev = h.dist_evals > 0 ? (double)h.dist_evals : 1.0;
      use_tc = use_tc ? (double)h.reranked / ev < 0.10
                      : (double)h.proposals / (2.0 * ev) < 0.03;
    }
  }
  drop_graphs();
  KNNM_CUDA(cudaEventRecord(ctx->ev[2], st));
  int32_t* oi = P.oi ? P.oi : out_ids;
  float* od = P.od ? P.od : out_dists;
  KNNM_CUDA(launch_final(N, K, P.keys, D.Kr, P.rear, oi, od, true, st));
  ++launches;
  KNNM_CUDA(cudaEventRecord(ctx->ev[3], st));
  if (P.oi)
    KNNM_CUDA(cudaMemcpyAsync(out_ids, P.oi, (size_t)N * K * 4, cudaMemcpyDeviceToHost, st));
  if (P.od)
    KNNM_CUDA(cudaMemcpyAsync(out_dists, P.od, (size_t)N * K * 4, cudaMemcpyDeviceToHost, st));
  KNNM_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    local.ms_init = ms;
    cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
    local.ms_rounds = ms;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    local.ms_final = ms;
    local.kernel_launches = launches;
    local.ms_total = (float)std::chrono::duration<double, std::milli>(
                         std::chrono::steady_clock::now() - t_wall0)
                         .count();
    *stats = local;
  }
  return KNNM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

extern "C" int knnm_create(knnm_ctx** out, int device, void* cuda_stream) {
  if (!out) return KNNM_ERR_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return KNNM_ERR_INVALID;
  }
  if (cudaSetDevice(device) != cudaSuccess) return KNNM_ERR_CUDA;
  knnm_ctx* c = new (std::nothrow) knnm_ctx();
  if (!c) return KNNM_ERR_NOMEM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaMallocHost(&c->host_ctr, sizeof(DevCounters)) != cudaSuccess) {
    delete c;
    return KNNM_ERR_NOMEM;
  }
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      knnm_destroy(c);
      return KNNM_ERR_CUDA;
    }
  for (auto& e : c->rev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      knnm_destroy(c);
      return KNNM_ERR_CUDA;
    }
  *out = c;
  return KNNM_OK;
}

extern "C" int knnm_destroy(knnm_ctx* c) {
  if (!c) return KNNM_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->arena) cudaFree(c->arena);
  if (c->host_ctr) cudaFreeHost(c->host_ctr);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : c->rev)
    if (e) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
  return KNNM_OK;
}

extern "C" int knnm_set_stream(knnm_ctx* c, void* s) {
  if (!c) return KNNM_ERR_INVALID;
  c->stream = (cudaStream_t)s;
  return KNNM_OK;
}

extern "C" const char* knnm_last_error(const knnm_ctx* c) { return c ? c->err : "no context"; }

extern "C" int knnm_set_option(knnm_ctx* c, int option, int value) {
  if (!c) return KNNM_ERR_INVALID;
  if (option == KNNM_OPT_GRAPHS) {
    c->use_graphs = value ? 1 : 0;
    return KNNM_OK;
  }
  if (option == KNNM_OPT_BUCKET_CAP && value >= 0 && value <= 4096) {
    c->bucket_cap = value;
    return KNNM_OK;
  }
  if (option == KNNM_OPT_WAIT_POLLS && value >= -1) {
    c->wait_polls = value < 0 ? WAIT_LIMIT : (uint32_t)value;
    return KNNM_OK;
  }
  if (option == KNNM_OPT_FAIL_ALLOC && value >= 0) {
    c->fail_alloc = value;
    return KNNM_OK;
  }
  if (option == KNNM_OPT_TC_JOIN && value >= 0 && value <= 2) {
    c->tc_choice = value;
    return KNNM_OK;
  }
  return KNNM_ERR_INVALID;
}

extern "C" int knnm_list_widths(const knnm_params* params, int mode, int64_t set_split,
                                int* K_keep, int* Kr, int* s) {
  if (mode != SYMMETRIC && mode != JOINT) return KNNM_ERR_INVALID;
  Derived D{};
  const int rc = derive(nullptr, params, mode, set_split, &D);
  if (rc) return rc;
  if (K_keep) *K_keep = D.K_keep;
  if (Kr) *Kr = D.Kr;
  if (s) *s = D.s;
  return KNNM_OK;
}

extern "C" uint64_t knnm_hash64(uint64_t seed, uint64_t t, uint64_t stream, uint64_t owner,
                                uint64_t member) {
  return mix_step(hash_prefix(seed, t, stream, owner) ^ member);
}

extern "C" const char* knnm_strerror(int code) {
  switch (code) {
    case KNNM_OK: return "ok";
    case KNNM_ERR_INVALID: return "invalid argument";
    case KNNM_ERR_NOMEM: return "out of memory";
    case KNNM_ERR_CUDA: return "CUDA error";
    case KNNM_ERR_TIMEOUT: return "timeout";
    case KNNM_ERR_NOT_READY: return "not ready";
    case KNNM_ERR_DEVICE: return "device-side error";
    default: return "unknown error";
  }
}

extern "C" void knnm_default_params(knnm_params* p) {
  if (!p) return;
  p->k = 20;
  p->metric = KNNM_L2;
  p->precision = KNNM_FP32;
  p->max_iters = 10;
  p->sample_rate = 0.5f;
  p->keep_ratio = 0.5f;
  p->delta = 0.001f;
  p->seed = 0;
}

// ---------------------------------------------------------------------------
// Whole merges
// ---------------------------------------------------------------------------

extern "C" int knnm_merge_symmetric(knnm_ctx* ctx, const float* S1, int64_t n1, const int32_t* G1,
                                    const float* S2, int64_t n2, const int32_t* G2, int d,
                                    const knnm_params* params, int32_t* out_ids, float* out_dists,
                                    knnm_stats* stats) {
  MergeIn in{SYMMETRIC, S1, n1, G1, S2, n2, G2, d};
  return run_merge(ctx, in, params, out_ids, out_dists, stats);
}

extern "C" int knnm_merge_joint(knnm_ctx* ctx, const float* S1, int64_t n1, const int32_t* G1,
                                const float* S_new, int64_t n2, int d, const knnm_params* params,
                                int32_t* out_ids, float* out_dists, knnm_stats* stats) {
  MergeIn in{JOINT, S1, n1, G1, S_new, n2, nullptr, d};
  return run_merge(ctx, in, params, out_ids, out_dists, stats);
}

extern "C" int knnm_build(knnm_ctx* ctx, const float* S, int64_t n, int d,
                          const knnm_params* params, int32_t* out_ids, float* out_dists,
                          knnm_stats* stats) {
  MergeIn in{JOINT, nullptr, 0, nullptr, S, n, nullptr, d};
  return run_merge(ctx, in, params, out_ids, out_dists, stats);
}

extern "C" int knnm_merge_symmetric_sets(knnm_ctx* ctx, const int64_t* offsets,
                                         const int32_t* items, int64_t nnz, int64_t n1,
                                         int64_t n2, const int32_t* G1, const int32_t* G2,
                                         const knnm_params* params, int32_t* out_ids,
                                         float* out_dists, knnm_stats* stats) {
  if (!offsets || nnz < 0) return fail(ctx, KNNM_ERR_INVALID, "bad set rows");
  MergeIn in{SYMMETRIC, nullptr, n1, G1, nullptr, n2, G2, 1, offsets, items, nnz};
  return run_merge(ctx, in, params, out_ids, out_dists, stats);
}

extern "C" int knnm_merge_joint_sets(knnm_ctx* ctx, const int64_t* offsets, const int32_t* items,
                                     int64_t nnz, int64_t n1, int64_t n2, const int32_t* G1,
                                     const knnm_params* params, int32_t* out_ids,
                                     float* out_dists, knnm_stats* stats) {
  if (!offsets || nnz < 0) return fail(ctx, KNNM_ERR_INVALID, "bad set rows");
  MergeIn in{JOINT, nullptr, n1, G1, nullptr, n2, nullptr, 1, offsets, items, nnz};
  return run_merge(ctx, in, params, out_ids, out_dists, stats);
}

extern "C" int knnm_build_sets(knnm_ctx* ctx, const int64_t* offsets, const int32_t* items,
                               int64_t nnz, int64_t n, const knnm_params* params,
                               int32_t* out_ids, float* out_dists, knnm_stats* stats) {
  if (!offsets || nnz < 0) return fail(ctx, KNNM_ERR_INVALID, "bad set rows");
  MergeIn in{JOINT, nullptr, 0, nullptr, nullptr, n, nullptr, 1, offsets, items, nnz};
  return run_merge(ctx, in, params, out_ids, out_dists, stats);
}

extern "C" int knnm_merge_tree(knnm_ctx* ctx, const float* S, int64_t n, int d, int parts,
                               const int64_t* part_rows, const int32_t* G,
                               const knnm_params* params, int32_t* out_ids, float* out_dists,
                               knnm_stats* stats) {
  auto t_wall0 = std::chrono::steady_clock::now();
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (!S || !G || !part_rows || !out_ids || !out_dists || parts < 1 || d < 1 || !params ||
      n > 0x7FFFFFFFLL)
    return fail(ctx, KNNM_ERR_INVALID, "bad merge-tree arguments");
  const int K = params->k;
  if (K < 1 || K > 32) return fail(ctx, KNNM_ERR_INVALID, "k=%d outside 1..32", K);
  int64_t total = 0;
  for (int p = 0; p < parts; ++p) {
    if (part_rows[p] < K + 1)
      return fail(ctx, KNNM_ERR_INVALID, "part %d has %lld rows (< k+1)", p,
                  (long long)part_rows[p]);
    total += part_rows[p];
  }
  if (total != n) return fail(ctx, KNNM_ERR_INVALID, "part rows sum to %lld, not n=%lld",
                              (long long)total, (long long)n);
  KNNM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  // device copies: vectors (if on the host), two id buffers, distances
  const bool s_dev = is_device_ptr(S), od_dev = is_device_ptr(out_dists),
             oi_dev = is_device_ptr(out_ids);
  float* Sd = nullptr;
  int32_t* ids[2] = {nullptr, nullptr};
  float* dists = nullptr;
  DevCounters* ctr = nullptr;
  auto release = [&]() {
    cudaStreamSynchronize(st);
    if (!s_dev) cudaFree(Sd);
    cudaFree(ids[0]);
    cudaFree(ids[1]);
    cudaFree(dists);
    cudaFree(ctr);
  };
  if ((!s_dev && cudaMalloc(&Sd, (size_t)n * d * 4) != cudaSuccess) ||
      cudaMalloc(&ids[0], (size_t)n * K * 4) != cudaSuccess ||
      cudaMalloc(&ids[1], (size_t)n * K * 4) != cudaSuccess ||
      cudaMalloc(&dists, (size_t)n * K * 4) != cudaSuccess ||
      cudaMalloc(&ctr, sizeof(DevCounters)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(ctx, KNNM_ERR_NOMEM, "cannot allocate the merge-tree buffers");
  }
  int rc = KNNM_OK;
  auto cuda_ok = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    rc = fail(ctx, KNNM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return false;
  };
  if (s_dev) Sd = const_cast<float*>(S);
  else if (!cuda_ok(cudaMemcpyAsync(Sd, S, (size_t)n * d * 4, cudaMemcpyHostToDevice, st), "copy S")) {
    release();
    return rc;
  }
  if (!cuda_ok(cudaMemcpyAsync(ids[0], G, (size_t)n * K * 4, cudaMemcpyDefault, st), "copy G")) {
    release();
    return rc;
  }
  knnm_stats total_st;
  memset(&total_st, 0, sizeof(total_st));
  struct Block {
    int64_t start, rows;
  };
  std::vector<Block> blocks;
  int64_t off = 0;
  for (int p = 0; p < parts; ++p) {
    blocks.push_back({off, part_rows[p]});
    off += part_rows[p];
  }
  int cur = 0, level = 0;
  if (parts == 1) {
    // one part: its own lists, canonical distances, sorted
    Rows rows{Sd, Sd, n, d};
    float* norms = nullptr;
    bool ok = cuda_ok(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st), "memset") &&
              cuda_ok(cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st), "memset");
    if (ok && params->metric == KNNM_COS)
      ok = cuda_ok(cudaMalloc(&norms, (size_t)n * 4), "norms") &&
           cuda_ok(launch_norms(rows, n, norms, st), "norms");
    ok = ok && cuda_ok(launch_list_dists(rows, n, ids[0], K, params->metric, norms, ids[1],
                                         dists, ctr, st), "list distances");
    ok = ok && cuda_ok(cudaMemcpyAsync(ctx->host_ctr, ctr, sizeof(DevCounters),
                                       cudaMemcpyDeviceToHost, st), "counters") &&
         cuda_ok(cudaStreamSynchronize(st), "sync");
    cudaFree(norms);
    if (!ok) {
      release();
      return rc;
    }
    if (ctx->host_ctr->err) {
      release();
      return fail(ctx, KNNM_ERR_INVALID, "input graph row %llu is malformed",
                  (unsigned long long)ctx->host_ctr->err_row);
    }
    cur = 1;
  }
  while (blocks.size() > 1) {
    if (level >= KNNM_MAX_ROUNDS) {
      release();
      return fail(ctx, KNNM_ERR_INVALID, "too many levels");
    }
    std::vector<Block> next;
    const int nxt = cur ^ 1;
    for (size_t j = 0; j < blocks.size(); j += 2) {
      const Block a = blocks[j];
      if (j + 1 == blocks.size()) {  // odd block: carried to the next level as it is
        if (!cuda_ok(cudaMemcpyAsync(ids[nxt] + (size_t)a.start * K, ids[cur] + (size_t)a.start * K,
                                     (size_t)a.rows * K * 4, cudaMemcpyDeviceToDevice, st),
                     "carry")) {
          release();
          return rc;
        }
        next.push_back(a);
        continue;
      }
      const Block b = blocks[j + 1];
      knnm_params p = *params;
      p.seed = mix_step(hash_prefix(params->seed, (uint64_t)level, 6, (uint64_t)(j / 2)) ^ 0ull);
      MergeIn in{SYMMETRIC, Sd + (size_t)a.start * d, a.rows, ids[cur] + (size_t)a.start * K,
                 Sd + (size_t)b.start * d, b.rows, ids[cur] + (size_t)b.start * K, d};
      knnm_stats ms;
      rc = run_merge(ctx, in, &p, ids[nxt] + (size_t)a.start * K, dists + (size_t)a.start * K,
                     &ms);
      if (rc) {
        release();
        return rc;
      }
      for (int t = 0; t < ms.rounds; ++t) {
        total_st.updates[level] += ms.updates[t];
        total_st.dist_evals[level] += ms.dist_evals[t];
        total_st.proposals[level] += ms.proposals[t];
        total_st.reranked[level] += ms.reranked[t];
        total_st.gathered[level] += ms.gathered[t];
        total_st.spilled[level] += ms.spilled[t];
        total_st.ms_sample[level] += ms.ms_sample[t];
        total_st.ms_join[level] += ms.ms_join[t];
        total_st.ms_update[level] += ms.ms_update[t];
      }
      total_st.kernel_launches += ms.kernel_launches;
      total_st.ms_init += ms.ms_init;
      total_st.ms_rounds += ms.ms_rounds;
      total_st.ms_final += ms.ms_final;
      next.push_back({a.start, a.rows + b.rows});
    }
    blocks.swap(next);
    cur ^= 1;
    ++level;
  }
  total_st.rounds = level;
  bool ok = cuda_ok(cudaMemcpyAsync(out_ids, ids[cur], (size_t)n * K * 4,
                                    oi_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st),
                    "copy out ids") &&
            cuda_ok(cudaMemcpyAsync(out_dists, dists, (size_t)n * K * 4,
                                    od_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st),
                    "copy out dists") &&
            cuda_ok(cudaStreamSynchronize(st), "sync");
  release();
  if (!ok) return rc;
  total_st.ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() -
                                                               t_wall0).count();
  if (stats) *stats = total_st;
  return KNNM_OK;
}

extern "C" int knnm_hmerge(knnm_ctx* ctx, const float* S, int64_t n, int d, int64_t first_rows,
                           const knnm_params* params, int32_t* perm_out, int32_t* out_ids,
                           float* out_dists, int n_layers, const int64_t* layer_rows,
                           int32_t* layer_ids, knnm_stats* stats) {
  auto t_wall0 = std::chrono::steady_clock::now();
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (!S || !params || !perm_out || !out_ids || !out_dists || d < 1 || n > 0x7FFFFFFFLL ||
      n_layers < 0 || (n_layers > 0 && (!layer_rows || !layer_ids)))
    return fail(ctx, KNNM_ERR_INVALID, "bad H-Merge arguments");
  const int K = params->k;
  if (K < 2 || K > 32) return fail(ctx, KNNM_ERR_INVALID, "k=%d outside 2..32", K);
  const int half = K / 2;
  if (first_rows < K + 1 || first_rows > n)
    return fail(ctx, KNNM_ERR_INVALID, "first_rows=%lld must be in k+1..n", (long long)first_rows);
  // each step joins as many raw rows as the graph has, and the whole rest when
  // what would be left after it is too small for a J-Merge of its own
  auto block_after = [&](int64_t m) {
    int64_t b = std::min(m, n - m);
    if (n - m - b > 0 && n - m - b < K + 1) b = n - m;
    return b;
  };
  for (int l = 0; l < n_layers; ++l) {
    bool ok = false;
    for (int64_t m = first_rows; m < n; m += block_after(m)) ok = ok || m == layer_rows[l];
    if (!ok)
      return fail(ctx, KNNM_ERR_INVALID, "layer of %lld rows is not produced",
                  (long long)layer_rows[l]);
  }
  KNNM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  float *Xs = nullptr, *Xp = nullptr, *dists = nullptr;
  int32_t *perm = nullptr, *ids[2] = {nullptr, nullptr};
  const bool s_dev = is_device_ptr(S);
  auto release = [&]() {
    cudaStreamSynchronize(st);
    cudaFree(Xs);
    cudaFree(Xp);
    cudaFree(dists);
    cudaFree(perm);
    cudaFree(ids[0]);
    cudaFree(ids[1]);
  };
  if ((!s_dev && cudaMalloc(&Xs, (size_t)n * d * 4) != cudaSuccess) ||
      cudaMalloc(&Xp, (size_t)n * d * 4) != cudaSuccess ||
      cudaMalloc(&dists, (size_t)n * K * 4) != cudaSuccess ||
      cudaMalloc(&perm, (size_t)n * 4) != cudaSuccess ||
      cudaMalloc(&ids[0], (size_t)n * K * 4) != cudaSuccess ||
      cudaMalloc(&ids[1], (size_t)n * K * 4) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(ctx, KNNM_ERR_NOMEM, "cannot allocate the H-Merge buffers");
  }
  int rc = KNNM_OK;
  auto cuda_ok = [&](cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    rc = fail(ctx, KNNM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return false;
  };
  const float* X = S;
  if (!s_dev) {
    if (!cuda_ok(cudaMemcpyAsync(Xs, S, (size_t)n * d * 4, cudaMemcpyHostToDevice, st), "copy S")) {
      release();
      return rc;
    }
    X = Xs;
  }
  if (!cuda_ok(launch_permute(n, params->seed, perm, st), "permute") ||
      !cuda_ok(launch_gather_rows(X, perm, n, d, Xp, st), "gather")) {
    release();
    return rc;
  }
  knnm_stats total;
  memset(&total, 0, sizeof(total));
  auto add_stats = [&](const knnm_stats& ms, int level) {
    for (int t = 0; t < ms.rounds; ++t) {
      total.updates[level] += ms.updates[t];
      total.dist_evals[level] += ms.dist_evals[t];
      total.proposals[level] += ms.proposals[t];
      total.reranked[level] += ms.reranked[t];
      total.gathered[level] += ms.gathered[t];
      total.spilled[level] += ms.spilled[t];
      total.ms_sample[level] += ms.ms_sample[t];
      total.ms_join[level] += ms.ms_join[t];
      total.ms_update[level] += ms.ms_update[t];
    }
    total.kernel_launches += ms.kernel_launches;
    total.ms_init += ms.ms_init;
    total.ms_rounds += ms.ms_rounds;
    total.ms_final += ms.ms_final;
  };
  // layer outputs: copy the k/2 lists of an m-row layer when it is asked for
  auto save_layer = [&](int64_t m, const int32_t* lists) {
    int64_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
      if (layer_rows[l] == m)  // the first k/2 entries of each list
        return cuda_ok(cudaMemcpy2DAsync(layer_ids + off, (size_t)half * 4, lists, (size_t)K * 4,
                                         (size_t)half * 4, (size_t)m, cudaMemcpyDefault, st),
                       "copy layer");
      off += layer_rows[l] * half;
    }
    return true;
  };
  int64_t m = first_rows;
  int cur = 0, level = 0;
  {
    knnm_params p = *params;
    p.seed = mix_step(hash_prefix(params->seed, 0, 8, 0) ^ 0ull);
    MergeIn in{JOINT, nullptr, 0, nullptr, Xp, m, nullptr, d};
    knnm_stats ms;
    rc = run_merge(ctx, in, &p, ids[cur], dists, &ms);
    if (rc) {
      release();
      return rc;
    }
    add_stats(ms, 0);
    if (m < n && !save_layer(m, ids[cur])) {
      release();
      return rc;
    }
  }
  while (m < n) {
    ++level;
    if (level >= KNNM_MAX_ROUNDS) {
      release();
      return fail(ctx, KNNM_ERR_INVALID, "too many H-Merge steps");
    }
    const int64_t b = block_after(m);
    const bool last = m + b == n;
    knnm_params p = *params;
    p.seed = mix_step(hash_prefix(params->seed, (uint64_t)level, 8, 0) ^ 0ull);
    MergeIn in{JOINT, Xp, m, ids[cur], Xp + (size_t)m * d, b, nullptr, d};
    knnm_stats ms;
    rc = run_merge(ctx, in, &p, ids[cur ^ 1], dists, &ms);
    if (rc) {
      release();
      return rc;
    }
    add_stats(ms, level);
    cur ^= 1;
    m += b;
    if (!last && !save_layer(m, ids[cur])) {
      release();
      return rc;
    }
  }
  total.rounds = level + 1;
  bool ok = cuda_ok(cudaMemcpyAsync(out_ids, ids[cur], (size_t)n * K * 4, cudaMemcpyDefault, st),
                    "copy ids") &&
            cuda_ok(cudaMemcpyAsync(out_dists, dists, (size_t)n * K * 4, cudaMemcpyDefault, st),
                    "copy dists") &&
            cuda_ok(cudaMemcpyAsync(perm_out, perm, (size_t)n * 4, cudaMemcpyDefault, st),
                    "copy perm") &&
            cuda_ok(cudaStreamSynchronize(st), "sync");
  release();
  if (!ok) return rc;
  total.ms_total = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() -
                                                            t_wall0).count();
  if (stats) *stats = total;
  return KNNM_OK;
}

extern "C" int knnm_merge_scratch_bytes(knnm_ctx* ctx, int mode, int64_t n1, int64_t n2, int d,
                                        const knnm_params* params, uint64_t* bytes) {
  if (!ctx || !bytes || (mode != SYMMETRIC && mode != JOINT)) return KNNM_ERR_INVALID;
  // the sizes are what count; the arrays are taken to be on the device
  MergeIn in{mode, nullptr, n1, nullptr, nullptr, n2, nullptr, d};
  return run_merge(ctx, in, params, nullptr, nullptr, nullptr, bytes);
}

namespace knnm {

int ctx_reserve(knnm_ctx* ctx, uint64_t bytes) { return ensure_arena(ctx, (size_t)bytes); }

uint64_t ctx_scratch_bytes(const knnm_ctx* ctx) { return ctx ? ctx->arena_bytes : 0; }

}  // namespace knnm

// ---------------------------------------------------------------------------
// Round steps (device pointers)
// ---------------------------------------------------------------------------

namespace {

int check_rows(knnm_ctx* ctx, const float* X1, int64_t nx1, const float* X2, int64_t N, int d) {
  if (!X1 || d < 1 || N < 1 || nx1 < 1 || nx1 > N || (nx1 < N && !X2) || N > 0x7FFFFFFFLL)
    return fail(ctx, KNNM_ERR_INVALID, "bad row arrays");
  return KNNM_OK;
}

int read_counters(knnm_ctx* ctx, DevCounters* dev) {
  KNNM_CUDA(cudaMemcpyAsync(ctx->host_ctr, dev, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                            ctx->stream));
  KNNM_CUDA(cudaStreamSynchronize(ctx->stream));
  return KNNM_OK;
}

}  // namespace

extern "C" int knnm_step_init(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1,
                              const float* X2, int64_t N, int64_t set_split, int d,
                              const int32_t* G1, const int32_t* G2, const knnm_params* params,
                              int32_t* ids, float* dists, uint8_t* flags, int32_t* rear_ids,
                              float* rear_dists) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  int rc = check_rows(ctx, X1, nx1, X2, N, d);
  if (rc) return rc;
  Derived D{};
  rc = derive(ctx, params, mode, set_split, &D);
  if (rc) return rc;
  if (mode != SYMMETRIC && mode != JOINT) return fail(ctx, KNNM_ERR_INVALID, "bad mode");
  if (set_split < 0 || set_split > N || (set_split > 0 && !G1) ||
      (mode == SYMMETRIC && (!G2 || set_split == 0 || set_split == N)))
    return fail(ctx, KNNM_ERR_INVALID, "bad graphs or split");
  const int K = D.K;
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));
  Carver c0;
  auto carve = [&](Carver& c, uint64_t*& keys, uint64_t*& rear, float*& norms, DevCounters*& ctr) {
    keys = c.take<uint64_t>((size_t)N * K);
    rear = c.take<uint64_t>((size_t)N * (D.Kr > 0 ? D.Kr : 1));
    norms = c.take<float>((size_t)N);
    ctr = c.take<DevCounters>(1);
  };
  uint64_t *keys, *rear;
  float* norms;
  DevCounters* ctr;
  carve(c0, keys, rear, norms, ctr);
  rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1, keys, rear, norms, ctr);
  Rows rows{X1, X2 ? X2 : X1, nx1, d};
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st));
  KNNM_CUDA(cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st));
  if (params->metric == KNNM_COS) KNNM_CUDA(launch_norms(rows, N, norms, st));
  InitArgs ia;
  ia.mode = mode;
  ia.rows = rows;
  ia.N = N;
  ia.n1 = set_split;
  ia.G1 = G1;
  ia.G2 = G2;
  ia.K = K;
  ia.K_keep = D.K_keep;
  ia.metric = params->metric;
  ia.seed = params->seed;
  ia.norms = params->metric == KNNM_COS ? norms : nullptr;
  ia.vec4 = (d % 4 == 0 && aligned16(rows.X1) && aligned16(rows.X2)) ? 1 : 0;
  ia.keys = keys;
  ia.flags = flags;
  ia.rear = rear;
  ia.ctr = ctr;
  KNNM_CUDA(launch_init(ia, st));
  KNNM_CUDA(launch_unpack((int64_t)N * K, keys, ids, dists, st));
  if (D.Kr > 0) KNNM_CUDA(launch_unpack((int64_t)N * D.Kr, rear, rear_ids, rear_dists, st));
  rc = read_counters(ctx, ctr);
  if (rc) return rc;
  if (ctx->host_ctr->err)
    return fail(ctx, KNNM_ERR_INVALID, "input graph row %llu is malformed",
                (unsigned long long)ctx->host_ctr->err_row);
  return KNNM_OK;
}

extern "C" int knnm_step_sample(knnm_ctx* ctx, int64_t N, int K, const int32_t* ids,
                                const float* dists, uint8_t* flags, uint64_t seed, int t, int s,
                                int cap_new, int cap_old, int32_t* new_ids, int32_t* new_cnt,
                                int32_t* old_ids, int32_t* old_cnt) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (N < 1 || K < 1 || K > 32 || s < 1 || s > K || cap_new < 2 * s || cap_old < K + s || !ids ||
      !dists || !flags || !new_ids || !new_cnt || !old_ids || !old_cnt)
    return fail(ctx, KNNM_ERR_INVALID, "bad sampling arguments");
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));
  uint64_t* keys;
  int32_t* rbucket;
  int32_t* rcnt;
  unsigned long long *roffs, *rtile, *rtotal;
  DevCounters* ctr;
  auto carve = [&](Carver& c) {
    keys = c.take<uint64_t>((size_t)N * K);
    rcnt = c.take<int32_t>((size_t)2 * N);
    roffs = c.take<unsigned long long>((size_t)2 * N + 1);
    rbucket = c.take<int32_t>((size_t)N * K);
    rtile = c.take<unsigned long long>((size_t)(2 * N + 1023) / 1024 + 1);
    rtotal = c.take<unsigned long long>(1);
    ctr = c.take<DevCounters>(1);
  };
  Carver c0;
  carve(c0);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  KNNM_CUDA(launch_pack((int64_t)N * K, ids, dists, keys, st));
  KNNM_CUDA(cudaMemsetAsync(rcnt, 0, (size_t)N * 8, st));
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st));
  SampleArgs sa;
  sa.N = N;
  sa.K = K;
  sa.s = s;
  sa.seed = seed;
  sa.t = t;
  sa.keys = keys;
  sa.flags = flags;
  sa.prev_keys = nullptr;
  sa.rev_new = nullptr;
  sa.rev_old = nullptr;
  sa.rcnt = rcnt;
  sa.roffs = roffs;
  sa.rbucket = rbucket;
  sa.tile_sum = rtile;
  sa.total = rtotal;
  sa.cap_new = cap_new;
  sa.cap_old = cap_old;
  sa.new_ids = new_ids;
  sa.new_cnt = new_cnt;
  sa.old_ids = old_ids;
  sa.old_cnt = old_cnt;
  sa.ctr = ctr;
  KNNM_CUDA(launch_sample(sa, st));
  return read_counters(ctx, ctr);
}

namespace {

// The join and UpdateNN of one round for the nodes u in [row_lo, row_hi)
// (every node for the full range): only pairs of those nodes' candidate sets
// are compared; their proposals update every target's list.
int step_join_rows(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1, const float* X2,
                   int64_t N, int64_t set_split, int d, const knnm_params* params, int32_t* ids,
                   float* dists, uint8_t* flags, int cap_new, int cap_old,
                   const int32_t* new_ids, const int32_t* new_cnt_in, const int32_t* old_ids,
                   const int32_t* old_cnt_in, int64_t row_lo, int64_t row_hi, int64_t* updates,
                   int64_t* dist_evals) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  int rc = check_rows(ctx, X1, nx1, X2, N, d);
  if (rc) return rc;
  if (!params || params->k < 1 || params->k > 32 || params->metric < 0 || params->metric > 4)
    return fail(ctx, KNNM_ERR_INVALID, "bad params");
  if (cap_new < 1 || cap_old < 1 || cap_new + cap_old > 96 || set_split < 0 || set_split > N ||
      (mode != SYMMETRIC && mode != JOINT))
    return fail(ctx, KNNM_ERR_INVALID, "bad capacities, split or mode");
  const int K = params->k;
  const int precision = params->metric != KNNM_L1 && params->metric != KNNM_CHI2 &&
                                params->metric != KNNM_JACCARD
                            ? params->precision
                            : KNNM_FP32;
  if (precision != KNNM_FP32 && d % 8 != 0)
    return fail(ctx, KNNM_ERR_INVALID, "the tensor-core paths need d %% 8 == 0");
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));
  JoinPath jp;
  rc = choose_join(ctx, precision, params->metric, cap_new, cap_old, d,
                   d % 4 == 0 && aligned16(X1) && aligned16(X2 ? X2 : X1), &jp);
  if (rc) return rc;
  if (row_lo < 0 || row_hi > N || row_lo > row_hi)
    return fail(ctx, KNNM_ERR_INVALID, "node range [%lld, %lld) outside 0..%lld", (long long)row_lo,
                (long long)row_hi, (long long)N);
  const bool tc = precision != KNNM_FP32;
  const bool masked = row_lo > 0 || row_hi < N;
  const int bcap = proposal_slots(ctx, K);
  uint64_t *keys, *prev, *bucket;
  int32_t *pcnt, *mnew = nullptr, *mold = nullptr;
  float* norms;
  __nv_bfloat16* Xb;
  float4* aux;
  float* rmax;
  __nv_bfloat16* Xe;
  float* wx;
  unsigned char* rec;
  DevCounters* ctr;
  auto carve = [&](Carver& c) {
    keys = c.take<uint64_t>((size_t)N * K);
    prev = c.take<uint64_t>((size_t)N * K);
    norms = c.take<float>((size_t)N);
    Xb = tc && !jp.pipe ? c.take<__nv_bfloat16>((size_t)N * d) : nullptr;
    aux = tc && !jp.pipe ? c.take<float4>((size_t)N) : nullptr;
    rmax = tc && !jp.pipe ? c.take<float>((size_t)N) : nullptr;
    ctr = c.take<DevCounters>(1);
    pcnt = c.take<int32_t>((size_t)N);
    bucket = c.take<uint64_t>((size_t)N * bcap);
    if (masked) {
      mnew = c.take<int32_t>((size_t)N);
      mold = c.take<int32_t>((size_t)N);
    }
    Xe = tc && jp.pipe ? c.take<__nv_bfloat16>((size_t)N * jp.pa.dx) : nullptr;
    wx = tc && jp.pipe ? c.take<float>((size_t)N) : nullptr;
    rec = jp.pipe ? c.take<unsigned char>((size_t)N * rec_bytes(jp.pa.cap)) : nullptr;
  };
  Carver c0;
  carve(c0);
  rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  Rows rows{X1, X2 ? X2 : X1, nx1, d};
  const int32_t* new_cnt = new_cnt_in;
  const int32_t* old_cnt = old_cnt_in;
  if (masked) {
    KNNM_CUDA(launch_mask_counts(N, row_lo, row_hi, new_cnt_in, old_cnt_in, mnew, mold, st));
    new_cnt = mnew;
    old_cnt = mold;
  }
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st));
  KNNM_CUDA(cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st));
  KNNM_CUDA(launch_pack((int64_t)N * K, ids, dists, keys, st));
  KNNM_CUDA(cudaMemcpyAsync(prev, keys, (size_t)N * K * 8, cudaMemcpyDeviceToDevice, st));
  if (params->metric == KNNM_COS) KNNM_CUDA(launch_norms(rows, N, norms, st));
  if (Xb)
    KNNM_CUDA(launch_bf16_prep(rows, N, Xb, aux, rmax, precision == KNNM_FP16_RERANK, nullptr, st));
  if (Xe)
    KNNM_CUDA(launch_bf16_ext(rows, N, jp.pa.dx, Xe, wx, precision == KNNM_FP16_RERANK, nullptr, st));
  JoinArgs ja;
  ja.mode = mode;
  ja.rows = rows;
  ja.N = N;
  ja.n1 = set_split;
  ja.K = K;
  ja.metric = params->metric;
  ja.norms = norms;
  ja.keys = keys;
  ja.cap_new = cap_new;
  ja.cap_old = cap_old;
  ja.new_ids = new_ids;
  ja.new_cnt = new_cnt;
  ja.old_ids = old_ids;
  ja.old_cnt = old_cnt;
  ja.bucket = bucket;
  ja.bcnt = pcnt;
  ja.bcap = bcap;
  ja.live_keys = keys;
  ja.ctr = ctr;
  ja.Xb = Xb;
  ja.aux = aux;
  ja.rmax = rmax;
  ja.use_bulk = (d % 4 == 0 && aligned16(rows.X1) && aligned16(rows.X2)) ? 1 : 0;
  ja.wait_polls = ctx->wait_polls;
  KNNM_CUDA(cudaMemsetAsync(pcnt, 0, (size_t)N * 4, st));
  if (jp.pipe) {
    // third record column: exactness widths (tensor-core join), cosine norms
    KNNM_CUDA(launch_build_records(N, K, keys,
                                   tc ? wx : (params->metric == KNNM_COS ? norms : nullptr),
                                   cap_new, cap_old, new_ids, new_cnt, old_ids, old_cnt, rec,
                                   jp.pa.cap, st));
    jp.pa.rec = rec;
    jp.pa.Xe = Xe;
    KNNM_CUDA(launch_pipe(precision, ja, jp.pa, jp.smem, jp.grid, st));
  } else {
    KNNM_CUDA(launch_join(precision, ja, jp.plan, st));
  }
  MergeArgs ma{N, K, keys, prev, flags, pcnt, bcap, bucket, ctr};
  KNNM_CUDA(launch_bucket_update(ma, st));
  KNNM_CUDA(launch_unpack((int64_t)N * K, keys, ids, dists, st));
  rc = read_counters(ctx, ctr);
  if (rc) return rc;
  if (ctx->host_ctr->err)
    return fail(ctx, KNNM_ERR_DEVICE, "device error bits 0x%llx (row %llu)",
                (unsigned long long)ctx->host_ctr->err,
                (unsigned long long)ctx->host_ctr->err_row);
  if (updates) *updates = (int64_t)ctx->host_ctr->updates;
  if (dist_evals) *dist_evals = (int64_t)ctx->host_ctr->dist_evals;
  return KNNM_OK;
}

}  // namespace

extern "C" int knnm_step_join(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1,
                              const float* X2, int64_t N, int64_t set_split, int d,
                              const knnm_params* params, int32_t* ids, float* dists,
                              uint8_t* flags, int cap_new, int cap_old, const int32_t* new_ids,
                              const int32_t* new_cnt, const int32_t* old_ids,
                              const int32_t* old_cnt, int64_t* updates, int64_t* dist_evals) {
  return step_join_rows(ctx, mode, X1, nx1, X2, N, set_split, d, params, ids, dists, flags,
                        cap_new, cap_old, new_ids, new_cnt, old_ids, old_cnt, 0, N, updates,
                        dist_evals);
}

extern "C" int knnm_step_join_rows(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1,
                                   const float* X2, int64_t N, int64_t set_split, int d,
                                   const knnm_params* params, int32_t* ids, float* dists,
                                   uint8_t* flags, int cap_new, int cap_old,
                                   const int32_t* new_ids, const int32_t* new_cnt,
                                   const int32_t* old_ids, const int32_t* old_cnt,
                                   int64_t row_lo, int64_t row_hi, int64_t* updates,
                                   int64_t* dist_evals) {
  return step_join_rows(ctx, mode, X1, nx1, X2, N, set_split, d, params, ids, dists, flags,
                        cap_new, cap_old, new_ids, new_cnt, old_ids, old_cnt, row_lo, row_hi,
                        updates, dist_evals);
}

extern "C" int knnm_step_union(knnm_ctx* ctx, int64_t n, int K, int parts,
                               const int32_t* part_ids, const float* part_dists,
                               const int32_t* start_ids, const float* start_dists,
                               const uint8_t* start_flags, int32_t* out_ids, float* out_dists,
                               uint8_t* out_flags, int64_t* updates) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (n < 0 || K < 1 || K > 32 || parts < 1 || (n > 0 && (!part_ids || !part_dists ||
      !start_ids || !start_dists || !start_flags || !out_ids || !out_dists || !out_flags)))
    return fail(ctx, KNNM_ERR_INVALID, "bad union arguments");
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));
  DevCounters* ctr = nullptr;
  auto carve = [&](Carver& c) { ctr = c.take<DevCounters>(1); };
  Carver c0;
  carve(c0);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(DevCounters), st));
  KNNM_CUDA(launch_union(n, K, parts, part_ids, part_dists, start_ids, start_dists, start_flags,
                         out_ids, out_dists, out_flags, ctr, st));
  rc = read_counters(ctx, ctr);
  if (rc) return rc;
  if (updates) *updates = (int64_t)ctx->host_ctr->updates;
  return KNNM_OK;
}

extern "C" int knnm_step_final(knnm_ctx* ctx, int64_t N, int K, const int32_t* ids,
                               const float* dists, int Kr, const int32_t* rear_ids,
                               const float* rear_dists, int32_t* out_ids, float* out_dists) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (N < 1 || K < 1 || K > 32 || Kr < 0 || Kr > 32 || !ids || !dists || !out_ids ||
      !out_dists || (Kr > 0 && (!rear_ids || !rear_dists)))
    return fail(ctx, KNNM_ERR_INVALID, "bad final-merge arguments");
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));
  uint64_t *keys, *rear;
  auto carve = [&](Carver& c) {
    keys = c.take<uint64_t>((size_t)N * K);
    rear = c.take<uint64_t>((size_t)N * (Kr > 0 ? Kr : 1));
  };
  Carver c0;
  carve(c0);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  KNNM_CUDA(launch_pack((int64_t)N * K, ids, dists, keys, st));
  if (Kr > 0) KNNM_CUDA(launch_pack((int64_t)N * Kr, rear_ids, rear_dists, rear, st));
  KNNM_CUDA(launch_final(N, K, keys, Kr, rear, out_ids, out_dists, false, st));
  KNNM_CUDA(cudaStreamSynchronize(st));
  return KNNM_OK;
}

extern "C" int knnm_step_tc_estimate(knnm_ctx* ctx, const float* X, int64_t n, int d, int metric,
                                     int precision, const int32_t* pi, const int32_t* pj,
                                     int64_t P, float* est, float* bound, float* canon) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (n < 1 || n > 0x7FFFFFFFLL || d < 8 || d > 2048 || d % 8 != 0 || P < 0 || !X ||
      (P > 0 && (!pi || !pj || !est || !bound || !canon)))
    return fail(ctx, KNNM_ERR_INVALID, "bad estimate arguments (n=%lld d=%d P=%lld)", (long long)n,
                d, (long long)P);
  if (metric != KNNM_L2 && metric != KNNM_IP && metric != KNNM_COS)
    return fail(ctx, KNNM_ERR_INVALID, "metric %d has no tensor-core form", metric);
  if (precision != KNNM_BF16_RERANK && precision != KNNM_FP16_RERANK)
    return fail(ctx, KNNM_ERR_INVALID, "precision %d is not a tensor-core precision", precision);
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaSetDevice(ctx->device));
  if (P == 0) return KNNM_OK;
  // every pair index must name a row: checked on the host before any launch
  std::vector<int32_t> hi((size_t)P), hj((size_t)P);
  KNNM_CUDA(cudaMemcpyAsync(hi.data(), pi, (size_t)P * 4, cudaMemcpyDeviceToHost, st));
  KNNM_CUDA(cudaMemcpyAsync(hj.data(), pj, (size_t)P * 4, cudaMemcpyDeviceToHost, st));
  KNNM_CUDA(cudaStreamSynchronize(st));
  for (int64_t r = 0; r < P; ++r)
    if (hi[r] < 0 || hi[r] >= n || hj[r] < 0 || hj[r] >= n)
      return fail(ctx, KNNM_ERR_INVALID, "pair %lld names a row outside 0..%lld", (long long)r,
                  (long long)(n - 1));
  const int dx = ((d + 15) & ~15) + 16;
  __nv_bfloat16* Xe = nullptr;
  auto carve = [&](Carver& c) { Xe = c.take<__nv_bfloat16>((size_t)n * dx); };
  Carver c0;
  carve(c0);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  Rows rows{X, X, n, d};
  KNNM_CUDA(launch_bf16_ext(rows, n, dx, Xe, nullptr, precision == KNNM_FP16_RERANK, nullptr, st));
  KNNM_CUDA(launch_tc_estimate(precision, metric, Xe, dx, rows, pi, pj, P, est, bound, canon, st));
  KNNM_CUDA(cudaStreamSynchronize(st));
  return KNNM_OK;
}

// ---------------------------------------------------------------------------
// Graph diversification (Alg. 3) and the top-down search (Sec. 3.4)
// ---------------------------------------------------------------------------

namespace {

int read_gd_counters(knnm_ctx* ctx, GdCounters* dev, GdCounters* host) {
  KNNM_CUDA(cudaMemcpyAsync(host, dev, sizeof(GdCounters), cudaMemcpyDeviceToHost, ctx->stream));
  KNNM_CUDA(cudaStreamSynchronize(ctx->stream));
  return KNNM_OK;
}

bool all_device(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (!p || !is_device_ptr(p)) return false;
  return true;
}

}  // namespace

extern "C" int knnm_gather_rows(knnm_ctx* ctx, const float* S, int64_t n_src, int d,
                                const int32_t* perm, int64_t n, float* out) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (n_src < 1 || n < 0 || d < 1 || n_src > 0x7FFFFFFFLL || !all_device({S, perm, out}))
    return fail(ctx, KNNM_ERR_INVALID, "bad gather arguments (device pointers only)");
  KNNM_CUDA(cudaSetDevice(ctx->device));
  Carver c0;
  c0.take<GdCounters>(1);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  GdCounters* ctr = reinterpret_cast<GdCounters*>(ctx->arena);
  cudaStream_t st = ctx->stream;
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(GdCounters), st));
  KNNM_CUDA(cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st));
  KNNM_CUDA(launch_gather_checked(S, n_src, perm, n, d, out, ctr, st));
  GdCounters h;
  rc = read_gd_counters(ctx, ctr, &h);
  if (rc) return rc;
  if (h.err)
    return fail(ctx, KNNM_ERR_INVALID, "perm[%llu] is outside the rows of S",
                (unsigned long long)h.err_row);
  return KNNM_OK;
}

extern "C" int knnm_diversify(knnm_ctx* ctx, const float* S, int64_t n, int d, const int32_t* G,
                              int k, int metric, int max_degree, int32_t* out_ids,
                              float* out_dists, int32_t* out_degree, knnm_gd_stats* stats) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (n < 2 || n > 0x7FFFFFFFLL || d < 1 || k < 1 || k > 32 || k >= n || metric < 0 ||
      metric > 4 || max_degree < 1 || max_degree > 256)
    return fail(ctx, KNNM_ERR_INVALID, "bad diversification arguments (n=%lld k=%d max_degree=%d)",
                (long long)n, k, max_degree);
  if (!all_device({S, G, out_ids, out_dists, out_degree}))
    return fail(ctx, KNNM_ERR_INVALID, "diversification takes device pointers only");
  KNNM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  GdArgs a;
  float* norms = nullptr;
  GdCounters* ctr = nullptr;
  auto carve = [&](Carver& c) {
    a.indeg = c.take<int32_t>((size_t)n);
    a.rev_fill = c.take<int32_t>((size_t)n);
    a.rev_off = c.take<unsigned long long>((size_t)n + 1);
    a.tile_sum = c.take<unsigned long long>((size_t)(n + 1023) / 1024 + 1);
    a.total = c.take<unsigned long long>(1);
    a.rev = c.take<uint64_t>((size_t)n * k);
    a.fwd = c.take<uint64_t>((size_t)n * k);
    a.fwd_cnt = c.take<int32_t>((size_t)n);
    norms = c.take<float>((size_t)n);
    ctr = c.take<GdCounters>(1);
  };
  Carver c0;
  carve(c0);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  a.X = S;
  a.n = n;
  a.d = d;
  a.vec4 = (d % 4 == 0 && aligned16(S)) ? 1 : 0;
  a.norms = metric == KNNM_COS ? norms : nullptr;
  a.G = G;
  a.K = k;
  a.M = max_degree;
  a.out_ids = out_ids;
  a.out_dists = out_dists;
  a.out_deg = out_degree;
  a.ctr = ctr;
  if (!plan_diversify(&a))
    return fail(ctx, KNNM_ERR_INVALID, "no diversification layout for d=%d max_degree=%d", d,
                max_degree);
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(GdCounters), st));
  KNNM_CUDA(cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st));
  KNNM_CUDA(cudaEventRecord(ctx->ev[0], st));
  if (metric == KNNM_COS) KNNM_CUDA(launch_norms(Rows{S, S, n, d}, n, norms, st));
  KNNM_CUDA(launch_diversify(a, metric, st));
  KNNM_CUDA(cudaEventRecord(ctx->ev[1], st));
  GdCounters h;
  rc = read_gd_counters(ctx, ctr, &h);
  if (rc) return rc;
  if (h.err)
    return fail(ctx, KNNM_ERR_INVALID, "input graph row %llu is malformed (%s)",
                (unsigned long long)h.err_row,
                (h.err & DERR_DUP_ID) ? "repeated id" : "id out of range or self");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->dist_evals = h.dist_evals;
    stats->edges = h.edges;
    stats->full_rows = (int64_t)h.full_rows;
    stats->max_in_degree = (int64_t)h.max_in;
    KNNM_CUDA(cudaEventElapsedTime(&stats->ms, ctx->ev[0], ctx->ev[1]));
  }
  return KNNM_OK;
}

extern "C" int knnm_search_prepare(knnm_ctx* ctx, const float* S, int64_t n, int d,
                                   float* row_aux) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (n < 1 || n > 0x7FFFFFFFLL || d < 1 || !all_device({S, row_aux}))
    return fail(ctx, KNNM_ERR_INVALID, "bad search_prepare arguments (device pointers only)");
  KNNM_CUDA(cudaSetDevice(ctx->device));
  KNNM_CUDA(launch_row_aux(S, n, d, row_aux, ctx->stream));
  KNNM_CUDA(cudaStreamSynchronize(ctx->stream));
  return KNNM_OK;
}

extern "C" int knnm_search(knnm_ctx* ctx, const float* S, int64_t n, int d, const float* row_aux,
                           int metric, int n_layers, const int64_t* layer_rows,
                           const int32_t* layer_width,
                           const int32_t* const* layer_ids, const float* Q, int64_t nq, int ef,
                           int k_out, uint64_t seed, int32_t* out_ids, float* out_dists,
                           uint32_t* out_evals, knnm_search_stats* stats) {
  if (!ctx) return KNNM_ERR_INVALID;
  ctx->err[0] = 0;
  if (n < 1 || n > 0x7FFFFFFFLL || d < 1 || nq < 0 || metric < 0 || metric > 4 || k_out < 1 ||
      ef < k_out || ef > 1024 || n_layers < 1 || n_layers > SEARCH_MAX_LAYERS || !layer_rows ||
      !layer_width || !layer_ids)
    return fail(ctx, KNNM_ERR_INVALID, "bad search arguments (ef=%d k_out=%d layers=%d)", ef,
                k_out, n_layers);
  SearchArgs a;
  memset(&a, 0, sizeof(a));
  for (int l = 0; l < n_layers; ++l) {
    if (layer_rows[l] < 1 || layer_rows[l] > n || (l > 0 && layer_rows[l] < layer_rows[l - 1]) ||
        layer_width[l] < 1 || layer_width[l] > 1024 || !layer_ids[l] ||
        !is_device_ptr(layer_ids[l]))
      return fail(ctx, KNNM_ERR_INVALID, "bad layer %d (rows, width or device pointer)", l);
    a.rows[l] = layer_rows[l];
    a.width[l] = layer_width[l];
    a.g[l] = layer_ids[l];
  }
  if (layer_rows[n_layers - 1] != n)
    return fail(ctx, KNNM_ERR_INVALID, "the bottom layer must cover all %lld rows", (long long)n);
  if (!all_device({S}) || (nq > 0 && !all_device({Q, out_ids, out_dists})) ||
      (nq > 0 && out_evals && !is_device_ptr(out_evals)) || (row_aux && !is_device_ptr(row_aux)))
    return fail(ctx, KNNM_ERR_INVALID, "search takes device pointers only");
  KNNM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  float* aux = nullptr;
  GdCounters* ctr = nullptr;
  auto carve = [&](Carver& c) {
    aux = c.take<float>(row_aux ? 1 : (size_t)n * 2);
    ctr = c.take<GdCounters>(1);
  };
  Carver c0;
  carve(c0);
  int rc = ensure_arena(ctx, c0.off);
  if (rc) return rc;
  Carver c1;
  c1.base = (char*)ctx->arena;
  carve(c1);
  a.X = S;
  a.n = n;
  a.d = d;
  a.vec4 = (d % 4 == 0 && aligned16(S)) ? 1 : 0;
  a.aux = row_aux ? row_aux : aux;
  a.n_layers = n_layers;
  a.Q = Q;
  a.nq = nq;
  a.ef = ef;
  a.k_out = k_out;
  a.seed = seed;
  a.out_ids = out_ids;
  a.out_dists = out_dists;
  a.out_evals = out_evals;
  a.ctr = ctr;
  size_t smem = 0;
  int grid = 0;
  cudaError_t pe = plan_search(&a, &smem, &grid);
  if (pe != cudaSuccess)
    return fail(ctx, KNNM_ERR_INVALID, "no search layout for d=%d ef=%d: %s", d, ef,
                cudaGetErrorString(pe));
  KNNM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(GdCounters), st));
  KNNM_CUDA(cudaMemsetAsync(&ctr->err_row, 0xFF, 8, st));
  KNNM_CUDA(cudaEventRecord(ctx->ev[0], st));
  if (!row_aux) KNNM_CUDA(launch_row_aux(S, n, d, aux, st));
  if (nq > 0) KNNM_CUDA(launch_search(a, metric, smem, grid, st));
  KNNM_CUDA(cudaEventRecord(ctx->ev[1], st));
  GdCounters h;
  rc = read_gd_counters(ctx, ctr, &h);
  if (rc) return rc;
  if (h.err)
    return fail(ctx, KNNM_ERR_INVALID, "a layer graph lists an id beyond its layer (row %llu)",
                (unsigned long long)h.err_row);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->dist_evals = h.dist_evals;
    stats->crowded_queries = (int64_t)h.overflow;
    KNNM_CUDA(cudaEventElapsedTime(&stats->ms, ctx->ev[0], ctx->ev[1]));
  }
  return KNNM_OK;
}
