// knnm_kernels.cu -- list kernels of the merge: init (Divide / Append /
// Initialize of Alg. 1 and Alg. 2), the sampler of each round (Reverse(G) and
// the new/old candidate sets), the top-k insert (UpdateNN), the flag/counter
// pass, the final Merge and Sort, and small conversion kernels.
//
// Lists are packed 64-bit keys (distance order bits << 32 | id), K <= 32, so a
// whole list fits one warp with one entry per lane.
#include <atomic>

#include "knnm_internal.cuh"

namespace knnm {

namespace {

constexpr int WARPS_PER_BLOCK = 8;
constexpr int BLOCK = WARPS_PER_BLOCK * 32;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void raise_err(DevCounters* c, unsigned bits, int64_t row) {
  atomicOr(&c->err, (unsigned long long)bits);
  atomicMin(&c->err_row, (unsigned long long)row);
}

int grid_for_warps(int64_t nwarps) {
  static std::atomic<int> sms_cached{0};  // launches come from several host threads
  int sms = sms_cached.load(std::memory_order_relaxed);
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
    sms_cached.store(sms, std::memory_order_relaxed);
  }
  int64_t blocks = (nwarps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
  int64_t cap = (int64_t)sms * 8;  // persistent: at most 8 resident blocks per SM
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// Adds a per-warp count into a 64-bit device counter with one atomic per block.
__device__ __forceinline__ void block_add(unsigned long long* dst, unsigned long long v,
                                          unsigned long long* red) {
  // v is warp-uniform; lane 0 of each warp contributes
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    if (s) atomicAdd(dst, s);
  }
}

// ---------------------------------------------------------------------------
// Init
// ---------------------------------------------------------------------------

template <int METRIC>
__device__ __forceinline__ float dist_rows(const Rows& R, int64_t i, int64_t j, const float* norms,
                                           int vec4) {
  if constexpr (METRIC == JACCARD) {
    return jaccard_rows(R, i, j);
  } else {
    float na = 0.f, nb = 0.f;
    if (METRIC == COS) {
      na = norms[i];
      nb = norms[j];
    }
    if (vec4) return canon_dist_global4<METRIC>(R.row(i), R.row(j), R.d, na, nb);
    return canon_dist_global<METRIC>(R.row(i), R.row(j), R.d, na, nb);
  }
}

// Draws `want` distinct ids from [base, base+n_src) \ {i}: candidate c is
// base + H(seed, 0, 3, i, c) mod n_src, taken in order of c, skipping self and
// repeats; after 32*K candidates the row is completed with the smallest
// unused ids.  Returns the id held by this lane (lane m holds draw m).
__device__ int32_t draw_random(uint64_t seed, int64_t i, int64_t base, int64_t n_src, int want,
                               int K) {
  const int lane = threadIdx.x & 31;
  int32_t chosen = -1;
  int got = 0;
  const uint64_t pre = hash_prefix(seed, 0, STREAM_INIT, (uint64_t)i);
  const int limit = 32 * K;
  {
    // First 32 candidates at once: with nothing chosen yet, candidate c is taken
    // iff it is not self and no earlier candidate drew the same id (an earlier
    // equal one was either taken, or rejected for the same reason).
    const int64_t j = base + (int64_t)(mix_step(pre ^ (uint64_t)lane) % (uint64_t)n_src);
    const bool valid = j != i;
    const unsigned same = __match_any_sync(FULL, valid ? j : -1 - (int64_t)lane);
    const unsigned acc = __ballot_sync(FULL, valid && (same & lanemask_lt()) == 0);
    got = min(want, __popc(acc));
    const int src = lane < got ? (int)__fns(acc, 0, lane + 1) : 0;
    const int64_t js = __shfl_sync(FULL, j, src);
    if (lane < got) chosen = (int32_t)js;
  }
  for (int c0 = 32; c0 < limit && got < want; c0 += 32) {
    int c = c0 + lane;
    int64_t j = base + (int64_t)(mix_step(pre ^ (uint64_t)c) % (uint64_t)n_src);
    bool valid = c < limit && j != i;
    for (int m = 0; m < 32 && got < want; ++m) {
      int64_t jm = __shfl_sync(FULL, j, m);
      bool vm = __shfl_sync(FULL, valid, m);
      if (!vm) continue;
      bool seen = __any_sync(FULL, lane < got && chosen == (int32_t)jm);
      if (!seen) {
        if (lane == got) chosen = (int32_t)jm;
        ++got;
      }
    }
  }
  for (int64_t j0 = base; j0 < base + n_src && got < want; j0 += 32) {
    int64_t j = j0 + lane;
    bool valid = j < base + n_src && j != i;
    for (int m = 0; m < 32 && got < want; ++m) {
      int64_t jm = __shfl_sync(FULL, j, m);
      bool vm = __shfl_sync(FULL, valid, m);
      if (!vm) continue;
      bool seen = __any_sync(FULL, lane < got && chosen == (int32_t)jm);
      if (!seen) {
        if (lane == got) chosen = (int32_t)jm;
        ++got;
      }
    }
  }
  return chosen;
}

// Canonical distances from row i to the rows g (one per lane, -1 for none) for
// 16-byte aligned rows with d % 4 == 0.  The warp stages INIT_CH dimensions of
// every listed row at a time in shared memory with coalesced 16-byte
// asynchronous copies (two rows per warp instruction), then each lane
// continues its own in-order accumulation from there: the same arithmetic as
// canon_dist_global4, with all rows' loads in flight at once.
constexpr int INIT_CH = 64;              // dimensions staged per pass
constexpr int INIT_STRIDE = INIT_CH + 4;  // floats per staged row (conflict-free float4 reads)
// Staged rows per warp: up to 32 listed rows, then the node's own row (read
// by every lane from shared memory: its loads never wait inside the chain).
constexpr int INIT_ROWS = 33;

__device__ __forceinline__ void init_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}

template <int METRIC>
__device__ __forceinline__ float staged_dist(const Rows& R, int64_t i, int32_t g, int rows,
                                             const float* norms, float* buf) {
  if constexpr (METRIC == JACCARD) {  // sets are never staged; kept for completeness
    return g >= 0 ? jaccard_rows(R, i, g) : 0.0f;
  } else {
  const int lane = threadIdx.x & 31, d = R.d;
  float* own = buf + 32 * INIT_STRIDE;
  const float* yj = buf + lane * INIT_STRIDE;
  float acc = 0.0f;
  for (int c = 0; c < d; c += INIT_CH) {
    const int q4 = min(INIT_CH, d - c) >> 2;  // float4 per row this pass
    for (int s0 = 0; s0 < rows; s0 += 2) {
      const int slot = s0 + (lane >> 4), o = lane & 15;
      const int32_t gs = __shfl_sync(FULL, g, slot & 31);
      if (slot < rows && gs >= 0 && o < q4)
        init_cp16(buf + slot * INIT_STRIDE + o * 4, R.row(gs) + c + o * 4);
    }
    if (lane < q4) init_cp16(own + lane * 4, R.row(i) + c + lane * 4);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    if (g >= 0) {
      for (int t = 0; t < q4; ++t) {
        const float4 x = *reinterpret_cast<const float4*>(own + 4 * t);
        const float4 y = *reinterpret_cast<const float4*>(yj + 4 * t);
        acc = Canon<METRIC>::step(acc, x.x, y.x);
        acc = Canon<METRIC>::step(acc, x.y, y.y);
        acc = Canon<METRIC>::step(acc, x.z, y.z);
        acc = Canon<METRIC>::step(acc, x.w, y.w);
      }
    }
    __syncwarp();
  }
  float na = 0.f, nb = 0.f;
  if (METRIC == COS) {
    na = norms[i];
    nb = g >= 0 ? norms[g] : 0.f;
  }
  return canon_finish<METRIC>(acc, na, nb);
  }
}

// staged_dist from the 16-bit extended rows (SRC 1: BF16, 2: FP16) of rows
// that hold their FP32 values exactly: each element converts back to the very
// FP32 value, and the accumulation is the same in-order canonical one.  128
// dimensions (256 bytes of a row) are staged per pass; d % 8 == 0.
template <int SRC>
__device__ __forceinline__ float e16_to_f32(uint32_t bits) {
  if (SRC == 1) return __uint_as_float(bits << 16);
  return __half2float(__ushort_as_half((unsigned short)bits));
}

template <int METRIC, int SRC>
__device__ __forceinline__ float staged_dist16(const InitArgs& a, int64_t i, int32_t g, int rows,
                                               float* bufF) {
  const int lane = threadIdx.x & 31, d = a.rows.d;
  constexpr int RS = INIT_STRIDE * 2;  // 16-bit elements between staged rows (272 bytes)
  uint16_t* buf = reinterpret_cast<uint16_t*>(bufF);
  const uint16_t* X = reinterpret_cast<const uint16_t*>(a.Xe);
  uint16_t* own = buf + 32 * RS;
  const uint16_t* yj = buf + lane * RS;
  float acc = 0.0f;
  for (int c = 0; c < d; c += 128) {
    const int q8 = min(128, d - c) >> 3;  // 16-byte chunks per row this pass
    for (int s0 = 0; s0 < rows; s0 += 2) {
      const int slot = s0 + (lane >> 4), o = lane & 15;
      const int32_t gs = __shfl_sync(FULL, g, slot & 31);
      if (slot < rows && gs >= 0 && o < q8)
        init_cp16(buf + slot * RS + o * 8, X + (size_t)gs * a.dx + c + o * 8);
    }
    if (lane < q8) init_cp16(own + lane * 8, X + (size_t)i * a.dx + c + lane * 8);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    if (g >= 0) {
      for (int t = 0; t < q8; ++t) {
        const uint4 xv = *reinterpret_cast<const uint4*>(own + 8 * t);
        const uint4 yv = *reinterpret_cast<const uint4*>(yj + 8 * t);
        const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w}, yw[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc = Canon<METRIC>::step(acc, e16_to_f32<SRC>(xw[q] & 0xFFFFu),
                                    e16_to_f32<SRC>(yw[q] & 0xFFFFu));
          acc = Canon<METRIC>::step(acc, e16_to_f32<SRC>(xw[q] >> 16),
                                    e16_to_f32<SRC>(yw[q] >> 16));
        }
      }
    }
    __syncwarp();
  }
  float na = 0.f, nb = 0.f;
  if (METRIC == COS) {
    na = a.norms[i];
    nb = g >= 0 ? a.norms[g] : 0.f;
  }
  return canon_finish<METRIC>(acc, na, nb);
}

template <int METRIC, int SRC>
__device__ __forceinline__ float staged_dist_src(const InitArgs& a, int64_t i, int32_t g, int rows,
                                                 float* buf) {
  if constexpr (SRC == 0 || METRIC == JACCARD || METRIC == L1 || METRIC == CHI2)
    return staged_dist<METRIC>(a.rows, i, g, rows, a.norms, buf);
  else
    return staged_dist16<METRIC, SRC>(a, i, g, rows, buf);
}

template <int METRIC, int SRC>
__global__ void __launch_bounds__(BLOCK) k_init(InitArgs a) {
  extern __shared__ __align__(16) float init_buf[];  // [warps][INIT_ROWS][INIT_STRIDE] when staged
  float* wbuf = init_buf + (threadIdx.x >> 5) * INIT_ROWS * INIT_STRIDE;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int K = a.K, Kk = a.K_keep, Kr = a.K - a.K_keep;
  for (int64_t i = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); i < a.N;
       i += nwarps) {
    const int32_t* in = nullptr;
    int64_t own_base = 0, own_n = 0;
    if (i < a.n1) {
      in = a.G1 + (size_t)i * K;
      own_n = a.n1;
    } else if (a.mode == SYMMETRIC) {
      in = a.G2 + (size_t)(i - a.n1) * K;
      own_base = a.n1;
      own_n = a.N - a.n1;
    }
    uint64_t kept = KEY_EMPTY;
    int want;
    int64_t base, n_src;
    uint64_t pre_dkey = KEY_EMPTY;  // the drawn members' keys when computed with the list
    bool have_dkey = false;
    if (in) {
      // Divide: recompute distances of the input list, sort, keep the top K_keep.
      int32_t loc = lane < K ? in[lane] : -1;
      bool bad = lane < K && (loc < 0 || loc >= own_n || own_base + loc == i);
      bool dup = false;
      for (int m = 0; m < K; ++m) {
        int32_t o = __shfl_sync(FULL, loc, m);
        dup |= (lane < K && m != lane && o == loc);
      }
      if (__any_sync(FULL, bad) && lane == 0) raise_err(a.ctr, DERR_BAD_ID, i);
      if (__any_sync(FULL, dup) && lane == 0) raise_err(a.ctr, DERR_DUP_ID, i);
      want = Kr;
      base = i < a.n1 ? a.n1 : 0;
      n_src = i < a.n1 ? a.N - a.n1 : a.n1;
      uint64_t key = KEY_EMPTY;
      if (a.vec4 && K + want <= 32) {
        // The random members do not depend on the list, so the listed rows
        // (lanes 0..K-1) and the drawn rows (lanes K..K+want-1) are staged and
        // compared in one pass.
        const int32_t drawn = draw_random(a.seed, i, base, n_src, want, K);
        const int32_t dsh = __shfl_sync(FULL, drawn, (lane - K) & 31);
        int32_t g = -1;
        if (lane < K) g = !bad ? (int32_t)(own_base + loc) : -1;
        else if (lane < K + want) g = dsh;
        const float dist = staged_dist_src<METRIC, SRC>(a, i, g, K + want, wbuf);
        const uint64_t kk = g >= 0 ? make_key(dist, g) : KEY_EMPTY;
        key = lane < K ? kk : KEY_EMPTY;
        const uint64_t dk = __shfl_sync(FULL, kk, (lane + K) & 31);
        pre_dkey = lane < want ? dk : KEY_EMPTY;
        have_dkey = true;
      } else if (a.vec4) {
        const int32_t g = (lane < K && !bad) ? (int32_t)(own_base + loc) : -1;
        const float dist = staged_dist_src<METRIC, SRC>(a, i, g, K, wbuf);
        if (g >= 0) key = make_key(dist, g);
      } else if (lane < K && !bad) {
        int64_t g = own_base + loc;
        key = make_key(dist_rows<METRIC>(a.rows, i, g, a.norms, a.vec4), (int32_t)g);
      }
      key = warp_sort32(key);
      if (lane >= Kk && lane < K) a.rear[(size_t)i * Kr + (lane - Kk)] = key;
      kept = lane < Kk ? key : KEY_EMPTY;
    } else {
      // Initialize (Alg. 2): K random members of S1 u S2.
      want = K;
      base = 0;
      n_src = a.N;
      if (Kr > 0 && lane < Kr) a.rear[(size_t)i * Kr + lane] = KEY_EMPTY;
    }
    uint64_t dkey = pre_dkey;
    if (!have_dkey) {
      const int32_t drawn = draw_random(a.seed, i, base, n_src, want, K);
      if (a.vec4) {
        const int32_t g = lane < want ? drawn : -1;
        const float dist = staged_dist_src<METRIC, SRC>(a, i, g, want, wbuf);
        if (g >= 0) dkey = make_key(dist, g);
      } else if (lane < want) {
        dkey = make_key(dist_rows<METRIC>(a.rows, i, drawn, a.norms, a.vec4), drawn);
      }
    }
    int first = in ? Kk : 0;
    uint64_t shifted = __shfl_sync(FULL, dkey, (lane - first) & 31);
    uint64_t v = lane < first ? kept : (lane < K ? shifted : KEY_EMPTY);
    v = warp_sort32(v);
    if (lane < K) {
      a.keys[(size_t)i * K + lane] = v;
      a.flags[(size_t)i * K + lane] = FLAG_NEW;
    }
  }
}

template <int METRIC>
__global__ void __launch_bounds__(BLOCK) k_list_dists(Rows R, int64_t n, const int32_t* G, int K,
                                                      const float* norms, int vec4, int32_t* ids,
                                                      float* dists, DevCounters* ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t i = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); i < n;
       i += nwarps) {
    const int32_t g = lane < K ? G[(size_t)i * K + lane] : -1;
    const bool bad = lane < K && (g < 0 || g >= n || g == i);
    uint64_t key = KEY_EMPTY;
    if (lane < K && !bad) key = make_key(dist_rows<METRIC>(R, i, g, norms, vec4), g);
    key = warp_sort32(key);
    // a repeated id has a bit-identical distance, so its copies end up adjacent
    const uint64_t prev = __shfl_up_sync(FULL, key, 1);
    const bool dup = lane > 0 && lane < K && key != KEY_EMPTY && key == prev;
    if (__any_sync(FULL, bad) && lane == 0) raise_err(ctr, DERR_BAD_ID, i);
    if (__any_sync(FULL, dup) && lane == 0) raise_err(ctr, DERR_DUP_ID, i);
    if (lane < K) {
      ids[(size_t)i * K + lane] = key_id(key);
      dists[(size_t)i * K + lane] = key_dist(key);
    }
  }
}

__global__ void k_norms(Rows R, int64_t N, float* norms) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) norms[i] = canon_norm_global(R.row(i), R.d);
}

// ---------------------------------------------------------------------------
// Sampler (round step 1)
// ---------------------------------------------------------------------------

// Forward sets of each node u and the pushes into the reverse slot arrays.
// Rank of every lane's key among the first n (even) of the warp's 32 keys
// (KEY_EMPTY never counts), read two keys at a time from a broadcast copy in
// `stage` (32 keys of the warp's shared memory).  Keys other than KEY_EMPTY are
// distinct.  All 32 lanes must call it together.
__device__ __forceinline__ int warp_rank(uint64_t x, int n, uint64_t* stage) {
  const int lane = threadIdx.x & 31;
  stage[lane] = x;
  __syncwarp();
  int rank = 0;
  const ulonglong2* st2 = (const ulonglong2*)stage;
  for (int m = 0; m < n; m += 2) {
    const ulonglong2 y = st2[m >> 1];
    rank += (y.x < x ? 1 : 0) + (y.y < x ? 1 : 0);
  }
  __syncwarp();
  return rank;
}

__global__ void __launch_bounds__(BLOCK) k_sample_fwd(SampleArgs a) {
  __shared__ __align__(16) uint64_t stage[WARPS_PER_BLOCK][32];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int K = a.K, s = a.s;
  const uint64_t t = (uint64_t)(a.t_dev ? *a.t_dev : a.t);
  // each node's list and flags are loaded one node ahead
  int64_t u = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  uint64_t key_next = u < a.N && lane < K ? a.keys[(size_t)u * K + lane] : KEY_EMPTY;
  uint8_t f_next = u < a.N && lane < K ? a.flags[(size_t)u * K + lane] : FLAG_OLD;
  for (; u < a.N; u += nwarps) {
    const uint64_t key = key_next;
    const uint8_t f = f_next;
    const int64_t un = u + nwarps;
    if (un < a.N && lane < K) {
      key_next = a.keys[(size_t)un * K + lane];
      f_next = a.flags[(size_t)un * K + lane];
    }
    if (a.prev_keys && lane < K) a.prev_keys[(size_t)u * K + lane] = key;
    if (a.info && lane == K - 1) reinterpret_cast<uint64_t*>(a.info + u)[1] = key;
    const int32_t v = key_id(key);
    const bool isnew = lane < K && f == FLAG_NEW;
    const bool isold = lane < K && f != FLAG_NEW;
    // at most s new entries: every one is drawn, whatever the keys
    bool sel = isnew;
    if (__popc(__ballot_sync(FULL, isnew)) > s) {
      const uint64_t pre = hash_prefix(a.seed, t, STREAM_FWD_NEW, (uint64_t)u);
      const uint64_t sk = isnew ? sampling_key(pre, v) : KEY_EMPTY;
      // every lane takes part: warp_rank writes the stage and syncs the warp
      const int rank = warp_rank(sk, (K + 1) & ~1, stage[threadIdx.x >> 5]);
      sel = isnew && rank < s;
    }
    if (sel) a.flags[(size_t)u * K + lane] = FLAG_OLD;
    const unsigned bs = __ballot_sync(FULL, sel), bo = __ballot_sync(FULL, isold);
    if (sel) a.new_ids[(size_t)u * a.cap_new + __popc(bs & lanemask_lt())] = v;
    if (isold) a.old_ids[(size_t)u * a.cap_old + __popc(bo & lanemask_lt())] = v;
    if (lane == 0) {
      a.new_cnt[u] = __popc(bs);
      a.old_cnt[u] = __popc(bo);
    }
    if (a.rcnt) {
      // bucketed reverse lists: count the in-edges of (target, stream) here
      // (old edges later, to active targets only, when active_only is set)
      if (sel) atomicAdd(&a.rcnt[2 * (size_t)v], 1);
      if (isold && !a.active_only) atomicAdd(&a.rcnt[2 * (size_t)v + 1], 1);
    } else {
      if (sel)
        slots_insert(a.rev_new + (size_t)v * s, s,
                     sampling_key(hash_prefix(a.seed, t, STREAM_REV_NEW, (uint64_t)v),
                                  (int32_t)u));
      if (isold)
        slots_insert(a.rev_old + (size_t)v * s, s,
                     sampling_key(hash_prefix(a.seed, t, STREAM_REV_OLD, (uint64_t)v),
                                  (int32_t)u));
    }
  }
}

// A node is active when its new set will not be empty: it drew forward-new
// entries, or some node drew it as one (a reverse-new in-edge).  Before the
// scan the in-edge count says so; after it (while the scatter consumes the
// counts) the bucket bounds do.
__device__ __forceinline__ bool active_by_count(const SampleArgs& a, int32_t v) {
  return a.new_cnt[v] > 0 || a.rcnt[2 * (size_t)v] > 0;
}
__device__ __forceinline__ bool active_by_bucket(const SampleArgs& a, int32_t v) {
  return a.new_cnt[v] > 0 || a.roffs[2 * (size_t)v + 1] > a.roffs[2 * (size_t)v];
}

// Old-stream in-edges of active targets (active_only), counted after every
// forward-new draw is known.
__global__ void __launch_bounds__(BLOCK) k_sample_count_old(SampleArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t u = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); u < a.N;
       u += nwarps) {
    const int of = a.old_cnt[u];
    if (lane < of) {
      const int32_t v = a.old_ids[(size_t)u * a.cap_old + lane];
      if (active_by_count(a, v)) atomicAdd(&a.rcnt[2 * (size_t)v + 1], 1);
    }
  }
}

// Moves each reverse edge's source id into its (target, stream) bucket (the
// reverse pass derives the sampling keys from the ids); the counts are
// consumed back to zero.
// Two nodes per warp and pass: each step's loads (counts, ids, bucket starts)
// and slot claims of both are in flight together, since every step waits
// on the one before.
constexpr int SCATTER_NODES = 2;

__global__ void __launch_bounds__(BLOCK) k_sample_scatter(SampleArgs a) {
  constexpr int U = SCATTER_NODES;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t u0 = ((int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5)) * U; u0 < a.N;
       u0 += nwarps * U) {
    int nf[U], of[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const bool in = u0 + j < a.N;
      nf[j] = in ? a.new_cnt[u0 + j] : 0;
      of[j] = in ? a.old_cnt[u0 + j] : 0;
    }
    // the id rows are read whole, beside the counts (entries past a count are
    // stale and unused)
    int32_t vn[U], vo[U];
    bool hn[U], ho[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const bool in = u0 + j < a.N;
      vn[j] = in && lane < a.cap_new ? a.new_ids[(size_t)(u0 + j) * a.cap_new + lane] : 0;
      vo[j] = in && lane < a.cap_old ? a.old_ids[(size_t)(u0 + j) * a.cap_old + lane] : 0;
    }
#pragma unroll
    for (int j = 0; j < U; ++j) hn[j] = lane < nf[j];
#pragma unroll
    for (int j = 0; j < U; ++j)
      ho[j] = lane < of[j] && (!a.active_only || active_by_bucket(a, vo[j]));
    unsigned long long bn[U], bo[U];
    int pn[U], po[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      bn[j] = hn[j] ? a.roffs[2 * (size_t)vn[j]] : 0ull;
      bo[j] = ho[j] ? a.roffs[2 * (size_t)vo[j] + 1] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      pn[j] = hn[j] ? atomicSub(&a.rcnt[2 * (size_t)vn[j]], 1) - 1 : 0;
      po[j] = ho[j] ? atomicSub(&a.rcnt[2 * (size_t)vo[j] + 1], 1) - 1 : 0;
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      if (hn[j]) a.rbucket[bn[j] + (uint64_t)pn[j]] = (int32_t)(u0 + j);
      if (ho[j]) a.rbucket[bo[j] + (uint64_t)po[j]] = (int32_t)(u0 + j);
    }
  }
}

// The s smallest of the c <= 32 keys x (lane j holding the j-th of a
// bucket, KEY_EMPTY beyond), ascending in lanes 0.. (KEY_EMPTY beyond).  Keys
// are distinct.  `stage` is 32 keys of the warp's shared memory.
__device__ __forceinline__ uint64_t select_sorted32(uint64_t x, int c, int s, uint64_t* stage) {
  const int lane = threadIdx.x & 31;
  const int rank = warp_rank(x, (c + 1) & ~1, stage);
  stage[lane] = KEY_EMPTY;
  __syncwarp();
  if (x != KEY_EMPTY && rank < s) stage[rank] = x;
  __syncwarp();
  const uint64_t best = stage[lane];
  __syncwarp();
  return best;
}

// As select_sorted32, in no particular order: every key when c <= s, else the
// keys of rank below s, packed into lanes 0..
__device__ __forceinline__ uint64_t select_any32(uint64_t x, int c, int s, uint64_t* stage) {
  if (c <= s) return x;
  const int lane = threadIdx.x & 31;
  const int rank = warp_rank(x, (c + 1) & ~1, stage);
  const unsigned sel = __ballot_sync(FULL, x != KEY_EMPTY && rank < s);
  const int src = lane < __popc(sel) ? (int)__fns(sel, 0, lane + 1) : lane;
  const uint64_t y = __shfl_sync(FULL, x, src);
  return lane < __popc(sel) ? y : KEY_EMPTY;
}

// The s smallest sampling keys of the source ids in bucket [b0, b1) with
// b1 - b0 > 32 (keys from the bucket owner's hash prefix), ascending, lane j
// holding the j-th (KEY_EMPTY beyond).  Ids in a bucket are distinct.
__device__ __forceinline__ uint64_t warp_smallest_long(const int32_t* bucket, uint64_t b0,
                                                       uint64_t b1, int s, uint64_t prefix) {
  const int lane = threadIdx.x & 31;
  uint64_t best = KEY_EMPTY;
  for (uint64_t c = b0; c < b1; c += 32) {
    uint64_t x = c + lane < b1 ? sampling_key(prefix, bucket[c + lane]) : KEY_EMPTY;
    const uint64_t kth = __shfl_sync(FULL, best, s - 1);
    if (x >= kth) x = KEY_EMPTY;
    unsigned live = __ballot_sync(FULL, x != KEY_EMPTY);
    if (!live) continue;
    if (__popc(live) <= 6) {
      while (live) {
        const int src = __ffs(live) - 1;
        live &= live - 1u;
        const uint64_t y = __shfl_sync(FULL, x, src);
        if (y >= __shfl_sync(FULL, best, s - 1)) continue;
        const int pos = __popc(__ballot_sync(FULL, best < y));
        const uint64_t up = __shfl_up_sync(FULL, best, 1);
        best = lane == pos ? y : (lane > pos ? up : best);
        if (lane >= s) best = KEY_EMPTY;
      }
    } else {
      best = warp_merge_lo32(best, warp_sort32(x));
      if (lane >= s) best = KEY_EMPTY;
    }
  }
  return best;
}

// new(u) = fwd_new u rev_new;  old(u) = (fwd_old u rev_old) \ new(u).
// Each node's loads come in two waves, all of a wave in flight together: its
// ids and bucket keys, then (once the sets are known) the records' gathers.
// The counts and bucket bounds they need are loaded one node ahead.
__global__ void __launch_bounds__(BLOCK) k_sample_rev(SampleArgs a) {
  __shared__ __align__(16) uint64_t stage[WARPS_PER_BLOCK][32];
  __shared__ __align__(16) int32_t sets[WARPS_PER_BLOCK][3][32];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int s = a.s;
  const bool buckets = a.rcnt != nullptr;
  // hash prefixes of the two reverse streams up to the owner (the same for
  // every node of the round); each node's own is one more mixing step
  const uint64_t t = (uint64_t)(a.t_dev ? *a.t_dev : a.t);
  const uint64_t h_new = mix_step(mix_step(mix_step(a.seed) ^ t) ^ STREAM_REV_NEW);
  const uint64_t h_old = mix_step(mix_step(mix_step(a.seed) ^ t) ^ STREAM_REV_OLD);
  uint64_t* st = stage[threadIdx.x >> 5];
  int32_t(*sw)[32] = sets[threadIdx.x >> 5];
  int64_t u = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  int nf_next = 0, of_next = 0;
  unsigned long long q0 = 0, q1 = 0, q2 = 0;
  if (u < a.N) {
    nf_next = a.new_cnt[u];
    of_next = a.old_cnt[u];
    if (buckets) {
      q0 = a.roffs[2 * u];
      q1 = a.roffs[2 * u + 1];
      q2 = a.roffs[2 * u + 2];
    }
  }
  for (; u < a.N; u += nwarps) {
    const int nf = nf_next, of = of_next;
    const unsigned long long r0 = q0, r1 = q1, r2 = q2;
    const int64_t un = u + nwarps;
    if (un < a.N) {
      nf_next = a.new_cnt[un];
      of_next = a.old_cnt[un];
      if (buckets) {
        q0 = a.roffs[2 * un];
        q1 = a.roffs[2 * un + 1];
        q2 = a.roffs[2 * un + 2];
      }
    }
    if (a.active_only && buckets && nf == 0 && r0 == r1) {
      // new(u) is empty: no pair of the join starts here
      if (lane == 0) {
        a.new_cnt[u] = 0;
        a.old_cnt[u] = 0;
        if (a.rec) {
          int32_t* h = (int32_t*)(a.rec + (size_t)u * rec_bytes(a.rec_cap));
          h[0] = h[1] = h[2] = h[3] = 0;
        }
      }
      continue;
    }
    // first wave: forward ids and the first 32 keys of both buckets
    const int32_t fn = lane < nf ? a.new_ids[(size_t)u * a.cap_new + lane] : -1;
    const int32_t fo = lane < of ? a.old_ids[(size_t)u * a.cap_old + lane] : -2;
    uint64_t xn, xo, pre_n = 0, pre_o = 0;
    if (buckets) {
      const int32_t yn = r0 + lane < r1 ? a.rbucket[r0 + lane] : -1;
      const int32_t yo = r1 + lane < r2 ? a.rbucket[r1 + lane] : -1;
      // a bucket the records take whole (at most s ids) is never ranked: its
      // ids travel as keys with an empty hash half
      const bool whole_n = a.records_only && r1 - r0 <= (uint64_t)s;
      const bool whole_o = a.records_only && r2 - r1 <= (uint64_t)s;
      if (!whole_n) pre_n = mix_step(h_new ^ (uint64_t)u);  // = hash_prefix(seed, t, STREAM_REV_NEW, u)
      if (!whole_o) pre_o = mix_step(h_old ^ (uint64_t)u);
      xn = yn < 0 ? KEY_EMPTY : (whole_n ? (uint64_t)(uint32_t)yn : sampling_key(pre_n, yn));
      xo = yo < 0 ? KEY_EMPTY : (whole_o ? (uint64_t)(uint32_t)yo : sampling_key(pre_o, yo));
    } else {
      xn = lane < s ? a.rev_new[(size_t)u * s + lane] : KEY_EMPTY;
      xo = lane < s ? a.rev_old[(size_t)u * s + lane] : KEY_EMPTY;
    }
    uint64_t rk = xn, ok = xo;
    if (buckets) {
      const uint64_t cn = r1 - r0, co = r2 - r1;
      if (a.records_only) {
        rk = cn > 32 ? warp_smallest_long(a.rbucket, r0, r1, s, pre_n)
                     : select_any32(xn, (int)cn, s, st);
        ok = co > 32 ? warp_smallest_long(a.rbucket, r1, r2, s, pre_o)
                     : select_any32(xo, (int)co, s, st);
      } else {
        rk = cn > 32 ? warp_smallest_long(a.rbucket, r0, r1, s, pre_n)
                     : select_sorted32(xn, (int)cn, s, st);
        ok = co > 32 ? warp_smallest_long(a.rbucket, r1, r2, s, pre_o)
                     : select_sorted32(xo, (int)co, s, st);
      }
    }
    const int32_t rn = rk != KEY_EMPTY ? key_id(rk) : -3;
    const int32_t ro = ok != KEY_EMPTY ? key_id(ok) : -4;
    // membership tests against broadcast copies of the three sets, four ids
    // a load; the markers of absent entries (-1, -2, -3, -4) never match
    sw[0][lane] = fn;
    sw[1][lane] = rn;
    sw[2][lane] = fo;
    __syncwarp();
    const int nr = 32 - __clz((int)__ballot_sync(FULL, rn >= 0));
    bool rn_dup = false, fo_in_rn = false, ro_drop = false;
    for (int m = 0; m < nf; m += 4) {
      const int4 x = *(const int4*)&sw[0][m];
      rn_dup |= (rn == x.x) | (rn == x.y) | (rn == x.z) | (rn == x.w);
      ro_drop |= (ro == x.x) | (ro == x.y) | (ro == x.z) | (ro == x.w);
    }
    for (int m = 0; m < nr; m += 4) {
      const int4 x = *(const int4*)&sw[1][m];
      fo_in_rn |= (fo == x.x) | (fo == x.y) | (fo == x.z) | (fo == x.w);
      ro_drop |= (ro == x.x) | (ro == x.y) | (ro == x.z) | (ro == x.w);
    }
    for (int m = 0; m < of; m += 4) {
      const int4 x = *(const int4*)&sw[2][m];
      ro_drop |= (ro == x.x) | (ro == x.y) | (ro == x.z) | (ro == x.w);
    }
    const bool has_fn = lane < nf;
    const bool add_rn = rn >= 0 && !rn_dup;
    const bool keep_fo = fo >= 0 && !fo_in_rn;
    const bool keep_ro = ro >= 0 && !ro_drop;
    const unsigned b1 = __ballot_sync(FULL, add_rn), b2 = __ballot_sync(FULL, keep_fo),
                   b3 = __ballot_sync(FULL, keep_ro);
    const int nn = nf + __popc(b1), no = __popc(b2) + __popc(b3);
    const int p_rn = nf + __popc(b1 & lanemask_lt());
    const int p_fo = __popc(b2 & lanemask_lt());
    const int p_ro = __popc(b2) + __popc(b3 & lanemask_lt());
    __syncwarp();
    if (!a.records_only) {
      if (add_rn) a.new_ids[(size_t)u * a.cap_new + p_rn] = rn;
      if (keep_fo) a.old_ids[(size_t)u * a.cap_old + p_fo] = fo;
      if (keep_ro) a.old_ids[(size_t)u * a.cap_old + p_ro] = ro;
    }
    if (lane == 0) {
      a.new_cnt[u] = nn;
      a.old_cnt[u] = no;
    }
    if (a.rec) {
      // second wave: every candidate's entry fields (one 16-byte gather each),
      // then the stores
      auto entry_of = [&](int32_t id) -> uint4 {
        if (a.info) {
          const uint4 f = __ldg(&a.info[id]);
          const uint32_t c = a.info_c == 0 ? f.x : (a.info_c == 1 ? f.y : 0u);
          return make_uint4((uint32_t)id, c, f.z, f.w);
        }
        return rec_entry(id, a.norms ? __ldg(&a.norms[id]) : 0.0f,
                         __ldg(&a.keys[(size_t)id * a.K_list + (a.K_list - 1)]));
      };
      const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
      const uint4 e_fn = has_fn ? entry_of(fn) : zero, e_rn = add_rn ? entry_of(rn) : zero,
                  e_fo = keep_fo ? entry_of(fo) : zero, e_ro = keep_ro ? entry_of(ro) : zero;
      unsigned char* R = a.rec + (size_t)u * rec_bytes(a.rec_cap);
      uint4* ent = (uint4*)(R + 16);
      if (has_fn) ent[lane] = e_fn;
      if (add_rn) ent[p_rn] = e_rn;
      if (keep_fo) ent[nn + p_fo] = e_fo;
      if (keep_ro) ent[nn + p_ro] = e_ro;
      if (lane == 0) {
        int32_t* h = (int32_t*)R;
        h[0] = nn;
        h[1] = no;
        h[2] = 0;
        h[3] = 0;
      }
    }
  }
}

__global__ void __launch_bounds__(BLOCK) k_build_records(int64_t N, int K, const uint64_t* keys,
                                                         const float* norms, int cap_new,
                                                         int cap_old, const int32_t* new_ids,
                                                         const int32_t* new_cnt,
                                                         const int32_t* old_ids,
                                                         const int32_t* old_cnt,
                                                         unsigned char* rec, int rec_cap) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t u = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); u < N;
       u += nwarps) {
    const int nn = min(new_cnt[u], cap_new), no = min(old_cnt[u], cap_old);
    unsigned char* R = rec + (size_t)u * rec_bytes(rec_cap);
    uint4* ent = (uint4*)(R + 16);
    for (int r = lane; r < nn + no; r += 32) {
      const int32_t id = r < nn ? new_ids[(size_t)u * cap_new + r]
                                : old_ids[(size_t)u * cap_old + (r - nn)];
      const int32_t safe = (id < 0 || id >= N) ? 0 : id;
      ent[r] = rec_entry(id, norms ? norms[safe] : 0.0f, keys[(size_t)safe * K + (K - 1)]);
    }
    if (lane == 0) {
      int32_t* h = (int32_t*)R;
      h[0] = nn;
      h[1] = no;
      h[2] = 0;
      h[3] = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Bucketed UpdateNN: the join put every proposal into its target's bucket (or,
// once the bucket was full, straight into the target's live list); one warp
// per node merges its list with its bucket (top-K distinct keys), sets the
// flags against the round-start snapshot and counts c_t.  The exclusive scan
// below serves the sampler's reverse buckets.
// ---------------------------------------------------------------------------

constexpr int SCAN_TILE = 1024;  // elements per scan block (256 threads x 4)

__global__ void __launch_bounds__(256) k_scan_tiles(const int32_t* cnt, int64_t n,
                                                    unsigned long long* tile_sum) {
  __shared__ unsigned long long red[8];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
  unsigned long long s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (base + q < n) s += (unsigned)cnt[base + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    tile_sum[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile sums in place (one block, running carry).
__global__ void __launch_bounds__(1024) k_scan_sums(unsigned long long* tile_sum, int64_t ntiles,
                                                    unsigned long long* total) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t b = 0; b < ntiles; b += 1024) {
    int64_t i = b + threadIdx.x;
    unsigned long long v = i < ntiles ? tile_sum[i] : 0ull;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long z = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(FULL, z, o);
        if (lane >= o) z += y;
      }
      wsum[lane] = z;
    }
    __syncthreads();
    unsigned long long incl = x + (w > 0 ? wsum[w - 1] : 0ull);
    if (i < ntiles) tile_sum[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(256) k_scan_apply(const int32_t* cnt, int64_t n,
                                                    const unsigned long long* tile_off,
                                                    unsigned long long* offs,
                                                    const unsigned long long* total) {
  __shared__ unsigned long long wsum[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * 4;
  unsigned long long v[4], s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = base + q < n ? (unsigned)cnt[base + q] : 0u;
    s += v[q];
  }
  unsigned long long x = s;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  unsigned long long before = tile_off[blockIdx.x];
  for (int q = 0; q < w; ++q) before += wsum[q];
  before += x - s;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (base + q < n) offs[base + q] = before;
    before += v[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) offs[n] = *total;
}

// The list `cur` (ascending, lanes >= K empty) after offering it the keys of
// `x` (one per lane, KEY_EMPTY for none): the first K distinct keys of both.
// Keys at or above the current K-th cannot enter (an equal key is already
// held); a few survivors are inserted one by one, more are sorted and merged.
__device__ __forceinline__ uint64_t offer_chunk(uint64_t cur, uint64_t x, int K, uint64_t* stage) {
  const int lane = threadIdx.x & 31;
  if (x >= __shfl_sync(FULL, cur, K - 1)) x = KEY_EMPTY;
  unsigned live = __ballot_sync(FULL, x != KEY_EMPTY);
  if (!live) return cur;
  if (__popc(live) <= 16) {
    // few survivors: insert them one by one (rank insertion across the warp;
    // each insertion lowers the K-th key, so later survivors often drop out;
    // below 17 this beats sorting the chunk on the 1M merge)
    while (live) {
      const int src = __ffs(live) - 1;
      live &= live - 1u;
      const uint64_t y = __shfl_sync(FULL, x, src);
      const uint64_t kk = __shfl_sync(FULL, cur, K - 1);
      if (y >= kk || __any_sync(FULL, cur == y)) continue;
      const int pos = __popc(__ballot_sync(FULL, cur < y));
      const uint64_t up = __shfl_up_sync(FULL, cur, 1);
      cur = lane == pos ? y : (lane > pos ? up : cur);
      if (lane >= K) cur = KEY_EMPTY;
    }
    return cur;
  }
  {
    // many survivors: sort the chunk and drop its repeats, keep the 32
    // smallest of (list, chunk) and remove keys the list already holds; that
    // is the answer unless repeats pushed distinct keys past 32
    const uint64_t xs = warp_sort32(x);
    const uint64_t xp = __shfl_up_sync(FULL, xs, 1);
    const bool keep_x = xs != KEY_EMPTY && (lane == 0 || xs != xp);
    const unsigned kx = __ballot_sync(FULL, keep_x);
    stage[lane] = KEY_EMPTY;
    __syncwarp();
    if (keep_x) stage[__popc(kx & lanemask_lt())] = xs;
    __syncwarp();
    const uint64_t xd = stage[lane];  // sorted, repeats dropped, KEY_EMPTY after
    __syncwarp();
    const uint64_t m = warp_merge_lo32(cur, xd);
    const uint64_t mp = __shfl_up_sync(FULL, m, 1);
    const bool keep = m != KEY_EMPTY && (lane == 0 || m != mp);
    const unsigned km = __ballot_sync(FULL, keep);
    if (__popc(km) >= K || __shfl_sync(FULL, m, 31) == KEY_EMPTY) {
      stage[lane] = KEY_EMPTY;
      __syncwarp();
      if (keep) stage[__popc(km & lanemask_lt())] = m;
      __syncwarp();
      cur = lane < K ? stage[lane] : KEY_EMPTY;
      __syncwarp();
      return cur;
    }
  }
  uint64_t e0 = cur, e1 = x;
  warp_sort64(e0, e1);
  uint64_t p0 = __shfl_up_sync(FULL, e0, 1);
  uint64_t p1 = __shfl_up_sync(FULL, e1, 1);
  const uint64_t last0 = __shfl_sync(FULL, e0, 31);
  if (lane == 0) p1 = last0;
  const bool k0 = e0 != KEY_EMPTY && (lane == 0 || e0 != p0);
  const bool k1 = e1 != KEY_EMPTY && e1 != p1;
  const unsigned m0 = __ballot_sync(FULL, k0), m1 = __ballot_sync(FULL, k1);
  const unsigned lt = (1u << lane) - 1u;
  const int pos0 = __popc(m0 & lt), pos1 = __popc(m0) + __popc(m1 & lt);
  stage[lane] = KEY_EMPTY;
  __syncwarp();
  if (k0 && pos0 < 32) stage[pos0] = e0;
  if (k1 && pos1 < 32) stage[pos1] = e1;
  __syncwarp();
  cur = lane < K ? stage[lane] : KEY_EMPTY;
  __syncwarp();
  return cur;
}

template <bool PF>
__global__ void __launch_bounds__(BLOCK) k_merge_lists(MergeArgs a) {
  __shared__ unsigned long long red[WARPS_PER_BLOCK];
  __shared__ uint64_t stage[WARPS_PER_BLOCK][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int K = a.K;
  unsigned long long cnt = 0;
  const int64_t passes = (a.N + nwarps - 1) / nwarps;
  const int64_t w0 = (int64_t)blockIdx.x * WARPS_PER_BLOCK + w;
  // With PF a node's list, count, snapshot, flags and first bucket chunk are
  // loaded one node ahead (more registers, fewer warps); without, each load
  // comes where it is first needed.
  uint64_t cur_n = KEY_EMPTY, pk_n = KEY_EMPTY, x0_n = KEY_EMPTY;
  uint8_t pf_n = FLAG_NEW;
  int cv_n = 0;
  const int first = min(a.bcap, 32);
  auto load = [&](int64_t v) {
    cur_n = lane < K ? a.keys[(size_t)v * K + lane] : KEY_EMPTY;
    cv_n = a.cnt[v];
    pk_n = lane < K ? a.prev_keys[(size_t)v * K + lane] : KEY_EMPTY;
    pf_n = lane < K ? a.flags[(size_t)v * K + lane] : (uint8_t)FLAG_NEW;
    x0_n = lane < first ? a.bucket[(size_t)v * a.bcap + lane] : KEY_EMPTY;
  };
  if (PF && w0 < a.N) load(w0);
  for (int64_t p = 0; p < passes; ++p) {
    const int64_t v = w0 + p * nwarps;
    if (v >= a.N) continue;
    uint64_t cur = PF ? cur_n : (lane < K ? a.keys[(size_t)v * K + lane] : KEY_EMPTY);
    const int cv = PF ? cv_n : a.cnt[v];
    const uint64_t x0 = x0_n, pk_ahead = pk_n;  // this node's, before the next load
    const uint8_t pf_ahead = pf_n;
    if (PF && v + nwarps < a.N) load(v + nwarps);
    const uint64_t b0 = (uint64_t)v * a.bcap, b1 = b0 + (uint64_t)min(cv, a.bcap);
    if (lane == 0 && cv) a.cnt[v] = 0;  // the next round's join starts from zero
    // The bucket in groups of four 32-key chunks: each lane's smallest key of
    // the group goes first (those are the likely winners), which lowers the
    // K-th key before the other three chunks are offered, so that most of
    // their keys are rejected by one compare.
    if (b1 - b0 <= 32) {
      cur = offer_chunk(cur, b0 + lane < b1 ? (PF ? x0 : a.bucket[b0 + lane]) : KEY_EMPTY, K,
                        stage[w]);
    } else for (uint64_t g = b0; g < b1; g += 128) {
      uint64_t x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t at = g + 32 * q + lane;
        x[q] = at < b1 ? a.bucket[at] : KEY_EMPTY;
      }
      uint64_t mn = x[0];
      int mi = 0;
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if (x[q] < mn) {
          mn = x[q];
          mi = q;
        }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q == mi) x[q] = KEY_EMPTY;
      cur = offer_chunk(cur, mn, K, stage[w]);
#pragma unroll
      for (int q = 0; q < 4; ++q) cur = offer_chunk(cur, x[q], K, stage[w]);
    }
    const uint64_t pk =
        PF ? pk_ahead : (lane < K ? a.prev_keys[(size_t)v * K + lane] : KEY_EMPTY);
    const uint8_t pf =
        PF ? pf_ahead : (lane < K ? a.flags[(size_t)v * K + lane] : (uint8_t)FLAG_NEW);
    // flags against the round-start snapshot: an entry is old when the same key
    // was in the list at round start.  The snapshot is sorted ascending (empty
    // places last), so each entry finds its place by a five-step binary search.
    int at = 0;  // number of snapshot keys <= cur among places 0..30
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint64_t probe = __shfl_sync(FULL, pk, at + step - 1);
      if (probe <= cur) at += step;
    }
    const uint64_t last = __shfl_sync(FULL, pk, 31);
    if (at == 31 && last <= cur) at = 32;
    const int idx = at > 0 ? at - 1 : 0;
    const uint64_t o = __shfl_sync(FULL, pk, idx);
    const uint8_t of = (uint8_t)__shfl_sync(FULL, (int)pf, idx);
    const uint64_t kth_prev = __shfl_sync(FULL, pk, K - 1);
    const bool found = cur == KEY_EMPTY ? kth_prev == KEY_EMPTY : (at > 0 && idx < K && o == cur);
    const uint8_t fl = found ? (cur == KEY_EMPTY ? (uint8_t)__shfl_sync(FULL, (int)pf, K - 1) : of)
                             : (uint8_t)FLAG_NEW;
    __syncwarp();
    if (lane < K) {
      a.keys[(size_t)v * K + lane] = cur;
      a.flags[(size_t)v * K + lane] = found ? fl : FLAG_NEW;
    }
    cnt += __popc(__ballot_sync(FULL, lane < K && !found));
  }
  block_add(&a.ctr->updates, cnt, red);
}

// Candidate counts of the nodes in [lo, hi) kept, all others zeroed (a join
// restricted to those nodes: every other node then has no pair).
__global__ void k_mask_counts(int64_t N, int64_t lo, int64_t hi, const int32_t* in_new,
                              const int32_t* in_old, int32_t* out_new, int32_t* out_old) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= N) return;
  const bool own = u >= lo && u < hi;
  out_new[u] = own ? in_new[u] : 0;
  out_old[u] = own ? in_old[u] : 0;
}

// Top-K union of `parts` lists per row (UpdateNN applied to the union of the
// proposals behind each partial list): the first K distinct keys of all parts,
// flags against the round-start list (an entry already there keeps its flag,
// any other is new), and c_t.  One warp per row.
__global__ void __launch_bounds__(BLOCK) k_union(int64_t n, int K, int parts,
                                                 const int32_t* part_ids, const float* part_dists,
                                                 const int32_t* start_ids,
                                                 const float* start_dists,
                                                 const uint8_t* start_flags, int32_t* out_ids,
                                                 float* out_dists, uint8_t* out_flags,
                                                 DevCounters* ctr) {
  __shared__ unsigned long long red[WARPS_PER_BLOCK];
  __shared__ uint64_t stage[WARPS_PER_BLOCK][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int64_t w0 = (int64_t)blockIdx.x * WARPS_PER_BLOCK + w;
  const int64_t passes = (n + nwarps - 1) / nwarps;
  unsigned long long cnt = 0;
  auto key_at = [&](const int32_t* I, const float* D, size_t at) {
    const int32_t id = I[at];
    return id < 0 ? KEY_EMPTY : make_key(D[at], id);
  };
  for (int64_t pass = 0; pass < passes; ++pass) {
    const int64_t v = w0 + pass * nwarps;
    if (v >= n) continue;  // warp-uniform
    uint64_t cur = KEY_EMPTY;
    for (int p = 0; p < parts; ++p) {
      uint64_t e0 = cur;
      uint64_t e1 = lane < K ? key_at(part_ids, part_dists, ((size_t)p * n + v) * K + lane)
                             : KEY_EMPTY;
      warp_sort64(e0, e1);
      uint64_t p0 = __shfl_up_sync(FULL, e0, 1);
      uint64_t p1 = __shfl_up_sync(FULL, e1, 1);
      const uint64_t last0 = __shfl_sync(FULL, e0, 31);
      if (lane == 0) p1 = last0;
      const bool k0 = e0 != KEY_EMPTY && (lane == 0 || e0 != p0);
      const bool k1 = e1 != KEY_EMPTY && e1 != p1;
      const unsigned m0 = __ballot_sync(FULL, k0), m1 = __ballot_sync(FULL, k1);
      const int pos0 = __popc(m0 & lanemask_lt()), pos1 = __popc(m0) + __popc(m1 & lanemask_lt());
      stage[w][lane] = KEY_EMPTY;
      __syncwarp();
      if (k0 && pos0 < 32) stage[w][pos0] = e0;
      if (k1 && pos1 < 32) stage[w][pos1] = e1;
      __syncwarp();
      cur = lane < K ? stage[w][lane] : KEY_EMPTY;
      __syncwarp();
    }
    // flags against the round-start list (ascending, empty places last)
    const uint64_t pk =
        lane < K ? key_at(start_ids, start_dists, (size_t)v * K + lane) : KEY_EMPTY;
    const uint8_t pf = lane < K ? start_flags[(size_t)v * K + lane] : FLAG_NEW;
    int at = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint64_t probe = __shfl_sync(FULL, pk, at + step - 1);
      if (probe <= cur) at += step;
    }
    const uint64_t lastk = __shfl_sync(FULL, pk, 31);
    if (at == 31 && lastk <= cur) at = 32;
    const int idx = at > 0 ? at - 1 : 0;
    const uint64_t o = __shfl_sync(FULL, pk, idx);
    const uint8_t of = (uint8_t)__shfl_sync(FULL, (int)pf, idx);
    const bool found = cur != KEY_EMPTY && at > 0 && idx < K && o == cur;
    if (lane < K) {
      out_ids[(size_t)v * K + lane] = cur == KEY_EMPTY ? -1 : key_id(cur);
      out_dists[(size_t)v * K + lane] = cur == KEY_EMPTY ? __int_as_float(0x7f800000) : key_dist(cur);
      out_flags[(size_t)v * K + lane] = found ? of : FLAG_NEW;
    }
    cnt += __popc(__ballot_sync(FULL, lane < K && cur != KEY_EMPTY && !found));
  }
  block_add(&ctr->updates, cnt, red);
}

// ---------------------------------------------------------------------------
// Merge and Sort with the rear lists (final step)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(BLOCK) k_final(int64_t N, int K, const uint64_t* keys, int Kr,
                                                 const uint64_t* rear, int32_t* out_ids,
                                                 float* out_dists, int sorted) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t v = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); v < N;
       v += nwarps) {
    uint64_t e0 = lane < K ? keys[(size_t)v * K + lane] : KEY_EMPTY;
    uint64_t e1 = lane < Kr ? rear[(size_t)v * Kr + lane] : KEY_EMPTY;
    if (sorted && K + Kr <= 32) {
      // both ascending (the list, and the rear keys as init wrote them): one
      // bitonic merge keeps all K + Kr keys in order
      e0 = warp_merge_lo32(e0, e1);
      e1 = KEY_EMPTY;
    } else {
      warp_sort64(e0, e1);
    }
    uint64_t p0 = __shfl_up_sync(FULL, e0, 1);
    uint64_t p1 = __shfl_up_sync(FULL, e1, 1);
    uint64_t last0 = __shfl_sync(FULL, e0, 31);
    if (lane == 0) p1 = last0;
    const bool k0 = e0 != KEY_EMPTY && (lane == 0 || e0 != p0);
    const bool k1 = e1 != KEY_EMPTY && e1 != p1;
    const unsigned b0 = __ballot_sync(FULL, k0), b1 = __ballot_sync(FULL, k1);
    const int pos0 = __popc(b0 & lanemask_lt());
    const int pos1 = __popc(b0) + __popc(b1 & lanemask_lt());
    if (k0 && pos0 < K) {
      out_ids[(size_t)v * K + pos0] = key_id(e0);
      out_dists[(size_t)v * K + pos0] = key_dist(e0);
    }
    if (k1 && pos1 < K) {
      out_ids[(size_t)v * K + pos1] = key_id(e1);
      out_dists[(size_t)v * K + pos1] = key_dist(e1);
    }
  }
}

// Serving commit: resident rows v < n_snap become the first K distinct keys of
// (resident list, request row); request rows for the new points are written
// to base + r.  Request ids >= n_snap are remapped to base + (id - n_snap).
__global__ void __launch_bounds__(BLOCK) k_commit(int64_t n_snap, int64_t rows, int K,
                                                  int32_t* res_ids, float* res_dists,
                                                  const int32_t* out_ids, const float* out_dists,
                                                  int64_t base) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t v = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); v < n_snap + rows;
       v += nwarps) {
    uint64_t e1 = KEY_EMPTY;
    if (lane < K) {
      int32_t id = out_ids[(size_t)v * K + lane];
      if (id >= n_snap) id = (int32_t)(base + (id - n_snap));
      e1 = make_key(out_dists[(size_t)v * K + lane], id);
    }
    const int64_t dst = v < n_snap ? v : base + (v - n_snap);
    if (v >= n_snap) {
      if (lane < K) {
        res_ids[(size_t)dst * K + lane] = key_id(e1);
        res_dists[(size_t)dst * K + lane] = key_dist(e1);
      }
      continue;
    }
    uint64_t e0 = lane < K ? make_key(res_dists[(size_t)v * K + lane], res_ids[(size_t)v * K + lane])
                           : KEY_EMPTY;
    warp_sort64(e0, e1);
    uint64_t p0 = __shfl_up_sync(FULL, e0, 1);
    uint64_t p1 = __shfl_up_sync(FULL, e1, 1);
    const uint64_t last0 = __shfl_sync(FULL, e0, 31);
    if (lane == 0) p1 = last0;
    const bool k0 = e0 != KEY_EMPTY && (lane == 0 || e0 != p0);
    const bool k1 = e1 != KEY_EMPTY && e1 != p1;
    const unsigned b0 = __ballot_sync(FULL, k0), b1 = __ballot_sync(FULL, k1);
    const int pos0 = __popc(b0 & lanemask_lt());
    const int pos1 = __popc(b0) + __popc(b1 & lanemask_lt());
    if (k0 && pos0 < K) {
      res_ids[(size_t)v * K + pos0] = key_id(e0);
      res_dists[(size_t)v * K + pos0] = key_dist(e0);
    }
    if (k1 && pos1 < K) {
      res_ids[(size_t)v * K + pos1] = key_id(e1);
      res_dists[(size_t)v * K + pos1] = key_dist(e1);
    }
  }
}

// H-Merge visiting order (Sec. 3.3: each block joined in is drawn at random
// from the whole set): position r holds row perm[r], perm a 4-round Feistel
// bijection on 2*half bits (round function H(seed, round, 7, right, 0) masked
// to half bits), cycle-walked back into [0, n).
__device__ __forceinline__ uint64_t feistel4(uint64_t x, int half, uint64_t seed) {
  const uint64_t mask = (1ull << half) - 1ull;
  uint64_t L = x >> half, R = x & mask;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t t = R;
    R = L ^ (mix_step(hash_prefix(seed, (uint64_t)r, 7, R) ^ 0ull) & mask);
    L = t;
  }
  return (L << half) | R;
}

__global__ void k_permute(int64_t n, int half, uint64_t seed, int32_t* perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t y = feistel4((uint64_t)i, half, seed);
  // the cycle through i returns to [0, n) within 2^(2*half) steps
  for (uint64_t guard = 0; y >= (uint64_t)n && guard < (1ull << (2 * half)); ++guard)
    y = feistel4(y, half, seed);
  perm[i] = (int32_t)y;
}

// Xp[r] = X[perm[r]], one warp per row.
__global__ void k_gather_rows(const float* X, const int32_t* perm, int64_t n, int d, float* Xp) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t r = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); r < n;
       r += nwarps) {
    const float* src = X + (size_t)perm[r] * d;
    float* dst = Xp + (size_t)r * d;
    for (int t = lane; t < d; t += 32) dst[t] = src[t];
  }
}

__global__ void k_set_int(int* p, int v) { *p = v; }
__global__ void k_bump_int(int* p) { *p += 1; }

__global__ void k_pack(int64_t count, const int32_t* ids, const float* dists, uint64_t* keys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) keys[i] = ids[i] < 0 ? KEY_EMPTY : make_key(dists[i], ids[i]);
}

__global__ void k_unpack(int64_t count, const uint64_t* keys, int32_t* ids, float* dists) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    uint64_t k = keys[i];
    ids[i] = k == KEY_EMPTY ? -1 : key_id(k);
    dists[i] = k == KEY_EMPTY ? __int_as_float(0x7f800000) : key_dist(k);
  }
}

// BF16 shadow copy; aux = {|b|^2, |b - x| (upper bound), |b| (upper bound),
// canonical |x|}.  rmax = max |x_t| when every x_t is an integer of magnitude
// <= 256 (BF16 holds it exactly), else -1.
template <bool HALF>
__global__ void k_bf16_prep(Rows R, int64_t N, __nv_bfloat16* Xb, float4* aux, float* rmax,
                            unsigned long long* inexact) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float* x = R.row(i);
  __nv_bfloat16* o = Xb + (size_t)i * R.d;
  float nb2 = 0.f, e2 = 0.f, nx2 = 0.f, mx = 0.f;
  bool exact = true, overflow = false;
  for (int t = 0; t < R.d; ++t) {
    float v = __ldg(x + t);
    float bf;
    if (HALF) {
      // saturated; a row beyond FP16 range gets an infinite error bound
      const float vs = fminf(fmaxf(v, -65504.0f), 65504.0f);
      overflow = overflow || vs != v;
      const __half h = __float2half_rn(vs);
      bf = __half2float(h);
      reinterpret_cast<__half*>(o)[t] = h;
    } else {
      __nv_bfloat16 b = __float2bfloat16_rn(v);
      bf = __bfloat162float(b);
      o[t] = b;
    }
    nb2 = __fmaf_rn(bf, bf, nb2);
    float e = __fsub_rn(bf, v);  // exact: bf and v are within a factor of two
    e2 = __fmaf_rn(e, e, e2);
    nx2 = __fmaf_rn(v, v, nx2);
    exact = exact && v == rintf(v) && fabsf(v) <= (HALF ? 2048.0f : 256.0f);
    mx = fmaxf(mx, fabsf(v));
  }
  // sums of d non-negative terms carry at most d+1 relative roundings
  const float grow = 1.0f + (float)(R.d + 2) * 1.2e-7f;
  aux[i] = make_float4(nb2,
                       overflow ? __int_as_float(0x7f800000)
                                : __fsqrt_ru(e2 * grow) * 1.000001f,
                       __fsqrt_ru(nb2 * grow) * 1.000001f, __fsqrt_rn(nx2));
  rmax[i] = exact ? mx : -1.0f;
  if (!exact && inexact) atomicAdd(inexact, 1ull);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <int METRIC, int SRC>
cudaError_t launch_init_m(const InitArgs& a, int grid, cudaStream_t st) {
  const size_t smem = a.vec4 ? (size_t)WARPS_PER_BLOCK * INIT_ROWS * INIT_STRIDE * 4 : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_init<METRIC, SRC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_init<METRIC, SRC><<<grid, BLOCK, smem, st>>>(a);
  return cudaGetLastError();
}

template <int METRIC>
cudaError_t launch_init_src(const InitArgs& a, int grid, cudaStream_t st) {
  // 16-bit rows only for aligned rows (vec4) of a tensor-core metric, d % 8 == 0
  if (a.Xe && a.vec4 && a.rows.d % 8 == 0)
    return a.half ? launch_init_m<METRIC, 2>(a, grid, st) : launch_init_m<METRIC, 1>(a, grid, st);
  return launch_init_m<METRIC, 0>(a, grid, st);
}

cudaError_t launch_init(const InitArgs& a, cudaStream_t st) {
  int grid = grid_for_warps(a.N);
  switch (a.metric) {
    case L2: return launch_init_src<L2>(a, grid, st);
    case IP: return launch_init_src<IP>(a, grid, st);
    case COS: return launch_init_src<COS>(a, grid, st);
    case L1: return launch_init_m<L1, 0>(a, grid, st);
    case JACCARD: return launch_init_m<JACCARD, 0>(a, grid, st);
    default: return launch_init_m<CHI2, 0>(a, grid, st);
  }
}

cudaError_t launch_exclusive_scan(const int32_t* cnt, int64_t n, unsigned long long* tile_sum,
                                  unsigned long long* offs, unsigned long long* total,
                                  cudaStream_t st) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles == 0) return cudaMemsetAsync(offs, 0, sizeof(unsigned long long), st);
  k_scan_tiles<<<(unsigned)ntiles, 256, 0, st>>>(cnt, n, tile_sum);
  k_scan_sums<<<1, 1024, 0, st>>>(tile_sum, ntiles, total);
  k_scan_apply<<<(unsigned)ntiles, 256, 0, st>>>(cnt, n, tile_sum, offs, total);
  return cudaGetLastError();
}

// Set rows: offsets from 0, non-decreasing, within the nnz items; items
// ascending without repeats and non-negative; rows below 2^23 items (the
// Jaccard counts stay exact in FP32).  One warp per row.
__global__ void k_check_sets(const int64_t* off, const int32_t* items, int64_t nnz, int64_t n,
                             DevCounters* ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
       i += nw) {
    const int64_t a = off[i], b = off[i + 1];
    bool bad = (i == 0 && a != 0) || (i == n - 1 && b != nnz) || a < 0 || b < a || b > nnz ||
               b - a >= (1 << 23);
    if (!bad)
      for (int64_t t = a + lane; t < b; t += 32) {
        const int32_t x = items[t];
        if (x < 0 || (t > a && items[t - 1] >= x)) bad = true;
      }
    if (__any_sync(FULL, bad) && lane == 0) raise_err(ctr, DERR_BAD_ID, i);
  }
}

cudaError_t launch_check_sets(const int64_t* off, const int32_t* items, int64_t nnz, int64_t n,
                              DevCounters* ctr, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_check_sets<<<grid_for_warps(n), BLOCK, 0, st>>>(off, items, nnz, n, ctr);
  return cudaGetLastError();
}

cudaError_t launch_norms(Rows rows, int64_t N, float* norms, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_norms<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rows, N, norms);
  return cudaGetLastError();
}

cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st) {
  int grid = grid_for_warps(a.N);
  k_sample_fwd<<<grid, BLOCK, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.rcnt) {
    if (a.active_only) {
      k_sample_count_old<<<grid, BLOCK, 0, st>>>(a);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    const int64_t n2 = 2 * a.N;
    const int64_t ntiles = (n2 + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<<<(unsigned)ntiles, 256, 0, st>>>(a.rcnt, n2, a.tile_sum);
    k_scan_sums<<<1, 1024, 0, st>>>(a.tile_sum, ntiles, a.total);
    k_scan_apply<<<(unsigned)ntiles, 256, 0, st>>>(a.rcnt, n2, a.tile_sum, a.roffs, a.total);
    k_sample_scatter<<<grid, BLOCK, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_sample_rev<<<grid, BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_build_records(int64_t N, int K, const uint64_t* keys, const float* norms,
                                 int cap_new, int cap_old, const int32_t* new_ids,
                                 const int32_t* new_cnt, const int32_t* old_ids,
                                 const int32_t* old_cnt, unsigned char* rec, int rec_cap,
                                 cudaStream_t st) {
  k_build_records<<<grid_for_warps(N), BLOCK, 0, st>>>(N, K, keys, norms, cap_new, cap_old,
                                                       new_ids, new_cnt, old_ids, old_cnt, rec,
                                                       rec_cap);
  return cudaGetLastError();
}

cudaError_t launch_bucket_update(const MergeArgs& a, cudaStream_t st) {
  if (a.prefetch)
    k_merge_lists<true><<<grid_for_warps(a.N), BLOCK, 0, st>>>(a);
  else
    k_merge_lists<false><<<grid_for_warps(a.N), BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

// First two words of each node's entry fields: exactness width and norm (0
// where absent).
__global__ void k_fill_info(int64_t N, const float* wx, const float* norms, uint4* info) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  reinterpret_cast<uint2*>(info + i)[0] =
      make_uint2(__float_as_uint(wx ? wx[i] : 0.0f), __float_as_uint(norms ? norms[i] : 0.0f));
}

cudaError_t launch_fill_info(int64_t N, const float* wx, const float* norms, uint4* info,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_fill_info<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, wx, norms, info);
  return cudaGetLastError();
}

cudaError_t launch_mask_counts(int64_t N, int64_t lo, int64_t hi, const int32_t* in_new,
                               const int32_t* in_old, int32_t* out_new, int32_t* out_old,
                               cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_mask_counts<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, lo, hi, in_new, in_old, out_new,
                                                             out_old);
  return cudaGetLastError();
}

cudaError_t launch_union(int64_t n, int K, int parts, const int32_t* part_ids,
                         const float* part_dists, const int32_t* start_ids,
                         const float* start_dists, const uint8_t* start_flags, int32_t* out_ids,
                         float* out_dists, uint8_t* out_flags, DevCounters* ctr, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_union<<<grid_for_warps(n), BLOCK, 0, st>>>(n, K, parts, part_ids, part_dists, start_ids,
                                               start_dists, start_flags, out_ids, out_dists,
                                               out_flags, ctr);
  return cudaGetLastError();
}

cudaError_t launch_final(int64_t N, int K, const uint64_t* keys, int Kr, const uint64_t* rear,
                         int32_t* out_ids, float* out_dists, bool sorted, cudaStream_t st) {
  k_final<<<grid_for_warps(N), BLOCK, 0, st>>>(N, K, keys, Kr, rear, out_ids, out_dists,
                                               sorted ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_list_dists(Rows rows, int64_t n, const int32_t* G, int K, int metric,
                              const float* norms, int32_t* ids, float* dists, DevCounters* ctr,
                              cudaStream_t st) {
  const int grid = grid_for_warps(n);
  const int vec4 = (rows.d % 4 == 0 && ((uintptr_t)rows.X1 & 15u) == 0 &&
                    ((uintptr_t)rows.X2 & 15u) == 0) ? 1 : 0;
  switch (metric) {
    case L2: k_list_dists<L2><<<grid, BLOCK, 0, st>>>(rows, n, G, K, norms, vec4, ids, dists, ctr); break;
    case IP: k_list_dists<IP><<<grid, BLOCK, 0, st>>>(rows, n, G, K, norms, vec4, ids, dists, ctr); break;
    case COS: k_list_dists<COS><<<grid, BLOCK, 0, st>>>(rows, n, G, K, norms, vec4, ids, dists, ctr); break;
    case L1: k_list_dists<L1><<<grid, BLOCK, 0, st>>>(rows, n, G, K, norms, vec4, ids, dists, ctr); break;
    default: k_list_dists<CHI2><<<grid, BLOCK, 0, st>>>(rows, n, G, K, norms, vec4, ids, dists, ctr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_commit(int64_t n_snap, int64_t rows, int K, int32_t* res_ids,
                          float* res_dists, const int32_t* out_ids, const float* out_dists,
                          int64_t base, cudaStream_t st) {
  k_commit<<<grid_for_warps(n_snap + rows), BLOCK, 0, st>>>(n_snap, rows, K, res_ids, res_dists,
                                                           out_ids, out_dists, base);
  return cudaGetLastError();
}

cudaError_t launch_permute(int64_t n, uint64_t seed, int32_t* perm, cudaStream_t st) {
  int b = 2;
  while ((1ll << b) < n) b += 2;
  k_permute<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, b / 2, seed, perm);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* X, const int32_t* perm, int64_t n, int d, float* Xp,
                               cudaStream_t st) {
  k_gather_rows<<<grid_for_warps(n), BLOCK, 0, st>>>(X, perm, n, d, Xp);
  return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, cudaStream_t st) {
  k_set_int<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_bump_int(int* p, cudaStream_t st) {
  k_bump_int<<<1, 1, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pack(int64_t count, const int32_t* ids, const float* dists, uint64_t* keys,
                        cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  k_pack<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, ids, dists, keys);
  return cudaGetLastError();
}

cudaError_t launch_unpack(int64_t count, const uint64_t* keys, int32_t* ids, float* dists,
                          cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  k_unpack<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, keys, ids, dists);
  return cudaGetLastError();
}

cudaError_t launch_bf16_prep(Rows rows, int64_t N, __nv_bfloat16* Xb, float4* aux, float* rmax,
                             int half, unsigned long long* inexact, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  if (half)
    k_bf16_prep<true><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rows, N, Xb, aux, rmax, inexact);
  else
    k_bf16_prep<false><<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rows, N, Xb, aux, rmax,
                                                                    inexact);
  return cudaGetLastError();
}

}  // namespace knnm
