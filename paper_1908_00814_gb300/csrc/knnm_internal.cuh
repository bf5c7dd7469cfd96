// knnm_internal.cuh -- device helpers and kernel interfaces shared by the
// translation units of libknnm.so (never installed, never seen by callers).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

struct knnm_ctx;

namespace knnm {

// ---------------------------------------------------------------------------
// List entries are packed 64-bit keys: (orderable FP32 distance bits) << 32 |
// id.  Unsigned comparison of two keys is the (distance, id) order of the
// lists; equal keys mean the same id (distances are canonical, so one id has
// one distance).  KEY_EMPTY sorts after every real entry.
// ---------------------------------------------------------------------------
constexpr uint64_t KEY_EMPTY = ~0ull;
constexpr uint8_t FLAG_OLD = 0;
constexpr uint8_t FLAG_NEW = 1;

enum Metric { L2 = 0, IP = 1, COS = 2, L1 = 3, CHI2 = 4, JACCARD = 5 };
enum Mode { SYMMETRIC = 0, JOINT = 1 };
enum Stream { STREAM_FWD_NEW = 0, STREAM_REV_NEW = 1, STREAM_REV_OLD = 2, STREAM_INIT = 3 };

// Error bits a kernel may raise in the context's device error word.
enum DevErr : unsigned {
  DERR_BAD_ID = 1u,        // input id out of range or self
  DERR_DUP_ID = 2u,        // input row repeats an id
  DERR_CAPACITY = 4u,      // candidate list longer than its capacity
  DERR_WAIT_TIMEOUT = 8u,  // an mbarrier wait ran out of iterations
  DERR_BAD_PAIR = 16u      // a candidate index out of range
};

__host__ __device__ __forceinline__ uint32_t float_to_ordered(float f) {
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float ordered_to_float(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

__host__ __device__ __forceinline__ uint64_t make_key(float dist, int32_t id) {
  return ((uint64_t)float_to_ordered(dist) << 32) | (uint32_t)id;
}
__host__ __device__ __forceinline__ int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)k; }
__host__ __device__ __forceinline__ float key_dist(uint64_t k) {
  return ordered_to_float((uint32_t)(k >> 32));
}

// ---------------------------------------------------------------------------
// Counter-based random numbers: chained SplitMix64 steps (Steele, Lea and
// Flood, OOPSLA 2014), one step per absorbed 64-bit word.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix_step(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Hash prefix over (seed, t, stream, owner); absorb the member with mix_step.
__host__ __device__ __forceinline__ uint64_t hash_prefix(uint64_t seed, uint64_t t,
                                                         uint64_t stream, uint64_t owner) {
  return mix_step(mix_step(mix_step(mix_step(seed) ^ t) ^ stream) ^ owner);
}

// Sampling key: high half of the hash, member id in the low half.
__host__ __device__ __forceinline__ uint64_t sampling_key(uint64_t prefix, int32_t member) {
  uint64_t h = mix_step(prefix ^ (uint64_t)(int64_t)member);
  return (h & 0xFFFFFFFF00000000ull) | (uint32_t)member;
}

// ---------------------------------------------------------------------------
// Canonical FP32 distances: one accumulator, dimensions in index order,
// correctly rounded operations only (no reassociation, no contraction).
// ---------------------------------------------------------------------------
template <int METRIC>
struct Canon;

template <>
struct Canon<L2> {
  __device__ __forceinline__ static float step(float acc, float a, float b) {
    float x = __fsub_rn(a, b);
    return __fmaf_rn(x, x, acc);
  }
};
template <>
struct Canon<IP> {
  __device__ __forceinline__ static float step(float acc, float a, float b) {
    return __fmaf_rn(a, b, acc);
  }
};
template <>
struct Canon<COS> {
  __device__ __forceinline__ static float step(float acc, float a, float b) {
    return __fmaf_rn(a, b, acc);
  }
};
template <>
struct Canon<L1> {
  __device__ __forceinline__ static float step(float acc, float a, float b) {
    return __fadd_rn(acc, fabsf(__fsub_rn(a, b)));
  }
};
// Chi-square: (a - b)^2 / (a + b) per term, 0 when a + b = 0.
template <>
struct Canon<CHI2> {
  __device__ __forceinline__ static float step(float acc, float a, float b) {
    const float x = __fsub_rn(a, b), s = __fadd_rn(a, b);
    return __fadd_rn(acc, s == 0.0f ? 0.0f : __fdiv_rn(__fmul_rn(x, x), s));
  }
};

// Turns the accumulated value into the distance.  `na`, `nb` are the
// canonical norms (sqrt of the in-order fmaf sum of squares), used by COS only.
template <int METRIC>
__device__ __forceinline__ float canon_finish(float acc, float na, float nb) {
  if (METRIC == IP) return __fsub_rn(0.0f, acc);
  if (METRIC == COS) {
    float den = __fmul_rn(na, nb);
    if (den == 0.0f) return 1.0f;
    return __fsub_rn(1.0f, __fdiv_rn(acc, den));
  }
  return acc;
}

// Canonical distance of two rows read from global memory (any alignment).
template <int METRIC>
__device__ __forceinline__ float canon_dist_global(const float* __restrict__ a,
                                                   const float* __restrict__ b, int d, float na,
                                                   float nb) {
  float acc = 0.0f;
  for (int t = 0; t < d; ++t) acc = Canon<METRIC>::step(acc, __ldg(a + t), __ldg(b + t));
  return canon_finish<METRIC>(acc, na, nb);
}

// Same with 16-byte loads; a and b 16-byte aligned, d a multiple of 4.
template <int METRIC>
__device__ __forceinline__ float canon_dist_global4(const float* __restrict__ a,
                                                    const float* __restrict__ b, int d, float na,
                                                    float nb) {
  float acc = 0.0f;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll 4
  for (int t = 0; t < (d >> 2); ++t) {
    const float4 x = __ldg(a4 + t), y = __ldg(b4 + t);
    acc = Canon<METRIC>::step(acc, x.x, y.x);
    acc = Canon<METRIC>::step(acc, x.y, y.y);
    acc = Canon<METRIC>::step(acc, x.z, y.z);
    acc = Canon<METRIC>::step(acc, x.w, y.w);
  }
  return canon_finish<METRIC>(acc, na, nb);
}

__device__ __forceinline__ float canon_norm_global(const float* __restrict__ a, int d) {
  float acc = 0.0f;
  for (int t = 0; t < d; ++t) {
    float v = __ldg(a + t);
    acc = __fmaf_rn(v, v, acc);
  }
  return __fsqrt_rn(acc);
}

// Row i of the dataset split in two arrays (rows < nx1 in X1, the rest in X2).
// Sets (JACCARD) are rows of a CSR array instead: row i holds the ascending,
// repeat-free items items[off[i] .. off[i+1]).
struct Rows {
  const float* X1;
  const float* X2;
  int64_t nx1;
  int d;
  const int64_t* off = nullptr;
  const int32_t* items = nullptr;
  __host__ __device__ __forceinline__ const float* row(int64_t i) const {
    return i < nx1 ? X1 + (size_t)i * d : X2 + (size_t)(i - nx1) * d;
  }
};

// Jaccard distance 1 - |A n B| / |A u B| of sets i and j (0 for two empty
// sets): the counts are exact integers, then one division and one subtraction.
__device__ __forceinline__ float jaccard_rows(const Rows& R, int64_t i, int64_t j) {
  const int64_t ai = __ldg(R.off + i), bi = __ldg(R.off + j);
  const int na = (int)(__ldg(R.off + i + 1) - ai), nb = (int)(__ldg(R.off + j + 1) - bi);
  const int32_t* a = R.items + ai;
  const int32_t* b = R.items + bi;
  int x = 0, y = 0, inter = 0;
  while (x < na && y < nb) {
    const int32_t p = __ldg(a + x), q = __ldg(b + y);
    inter += p == q;
    x += p <= q;
    y += q <= p;
  }
  const int uni = na + nb - inter;
  return uni == 0 ? 0.0f : __fsub_rn(1.0f, __fdiv_rn((float)inter, (float)uni));
}

// ---------------------------------------------------------------------------
// Warp utilities (K <= 32 entries: one per lane).
// ---------------------------------------------------------------------------
constexpr unsigned FULL = 0xFFFFFFFFu;

// Ascending bitonic sort of one 64-bit key per lane.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      uint64_t o = __shfl_xor_sync(FULL, v, j);
      bool lower = (lane & j) == 0;
      bool asc = (lane & k) == 0;
      uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
      v = (lower == asc) ? mn : mx;
    }
  }
  return v;
}

// A bitonic sequence of 32 keys (one per lane) put in ascending order.
__device__ __forceinline__ uint64_t warp_bitonic_clean32(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const uint64_t o = __shfl_xor_sync(FULL, v, j);
    const uint64_t mn = v < o ? v : o, mx = v < o ? o : v;
    v = (lane & j) == 0 ? mn : mx;
  }
  return v;
}

// The 32 smallest of the union of two ascending 32-key sequences, ascending:
// min(a[i], b[31-i]) keeps exactly those 32 and is bitonic.
__device__ __forceinline__ uint64_t warp_merge_lo32(uint64_t a, uint64_t b) {
  const int lane = threadIdx.x & 31;
  const uint64_t br = __shfl_sync(FULL, b, 31 - lane);
  return warp_bitonic_clean32(a < br ? a : br);
}

// Ascending bitonic sort of 64 keys, element e = h*32 + lane held in v[h].
__device__ __forceinline__ void warp_sort64(uint64_t& v0, uint64_t& v1) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {
        // partners are (lane, h=0) and (lane, h=1); both ascending for k = 64
        uint64_t mn = v0 < v1 ? v0 : v1, mx = v0 < v1 ? v1 : v0;
        v0 = mn;
        v1 = mx;
      } else {
        uint64_t o0 = __shfl_xor_sync(FULL, v0, j);
        uint64_t o1 = __shfl_xor_sync(FULL, v1, j);
        bool lower = (lane & j) == 0;
        bool asc0 = ((lane) & k) == 0;
        bool asc1 = ((lane + 32) & k) == 0;
        uint64_t mn0 = v0 < o0 ? v0 : o0, mx0 = v0 < o0 ? o0 : v0;
        uint64_t mn1 = v1 < o1 ? v1 : o1, mx1 = v1 < o1 ? o1 : v1;
        v0 = (lower == asc0) ? mn0 : mx0;
        v1 = (lower == asc1) ? mn1 : mx1;
      }
    }
  }
}

// Inserts `x` into the ascending array slots[0..m) that keeps the m smallest
// distinct keys ever offered to it.  Slots only ever decrease (atomicMin), so
// the result does not depend on the order or interleaving of insertions: slot
// j ends up holding the (j+1)-th smallest distinct key offered.  A key equal
// to one already held is a duplicate and is dropped.  Reads of slots that are
// already below x skip ahead; a stale read only makes the skip shorter.
__device__ __forceinline__ void slots_insert(uint64_t* slots, int m, uint64_t x) {
  int j = 0;
  for (; j < m; ++j) {
    uint64_t cur = *((volatile uint64_t*)(slots + j));
    if (cur == x) return;
    if (cur > x) break;
  }
  for (; j < m; ++j) {
    unsigned long long old = atomicMin((unsigned long long*)(slots + j), (unsigned long long)x);
    if (old == x) return;
    if (old > x) {
      if (old == KEY_EMPTY) return;
      x = old;
    }
  }
}

// slots_insert for a key that is usually no improvement: one read of the m-th
// slot rejects it (slots only decrease, so a key not below the current m-th
// can never be among the m smallest, and an equal key is already held).
// Out of line: the rare overflow path stays out of the join kernels' hot code.
static __device__ __noinline__ void slots_insert_checked(uint64_t* slots, int m, uint64_t x) {
  if (x >= *((volatile uint64_t*)(slots + m - 1))) return;
  slots_insert(slots, m, x);
}

// Proposal sink of the join, the input of UpdateNN.  A proposal for target v
// takes the next slot of v's bucket (bcap slots, claimed by an atomic on v's
// count).  Once v's bucket is full it is inserted straight into v's live
// list.  Either way it ends in the top-K union of the round.  Each lane offers
// up to NP proposals; n_prop / n_direct count this lane's offers and direct
// inserts.
template <int NP>
__device__ __forceinline__ void emit_to_buckets(uint64_t* bucket, int32_t* bcnt, int bcap,
                                                uint64_t* live, int K, const bool (&has)[NP],
                                                const int32_t (&tgt)[NP],
                                                const uint64_t (&key)[NP],
                                                unsigned long long& n_prop,
                                                unsigned long long& n_direct) {
  int pos[NP];
#pragma unroll
  for (int x = 0; x < NP; ++x) pos[x] = has[x] ? atomicAdd(bcnt + tgt[x], 1) : 0;
#pragma unroll
  for (int x = 0; x < NP; ++x) {
    if (has[x]) {
      ++n_prop;
      if (pos[x] < bcap) {
        bucket[(size_t)tgt[x] * bcap + pos[x]] = key[x];
      } else {
        ++n_direct;
        slots_insert_checked(live + (size_t)tgt[x] * K, K, key[x]);
      }
    }
  }
}

// The same sink with the slot claims of one batch kept in flight while the
// warp computes the next batch: offer() first writes the previous batch (whose
// atomics have returned by then), then claims slots for the new one, one
// atomic per proposal.  finish() writes the last batch.
template <int NP>
struct DeferredSink {
  bool has[NP];
  int32_t tgt[NP];
  uint64_t key[NP];
  int pos[NP];
  unsigned long long nprop = 0, ndirect = 0;

  __device__ __forceinline__ DeferredSink() {
#pragma unroll
    for (int x = 0; x < NP; ++x) {
      has[x] = false;
      tgt[x] = 0;
      key[x] = 0ull;
      pos[x] = 0;
    }
  }
  __device__ __forceinline__ void finish(uint64_t* bucket, int bcap, uint64_t* live, int K) {
#pragma unroll
    for (int x = 0; x < NP; ++x) {
      if (has[x]) {
        ++nprop;
        if (pos[x] < bcap) {
          bucket[(size_t)tgt[x] * bcap + pos[x]] = key[x];
        } else {
          ++ndirect;
          slots_insert_checked(live + (size_t)tgt[x] * K, K, key[x]);
        }
        has[x] = false;
      }
    }
  }
  __device__ __forceinline__ void offer(uint64_t* bucket, int32_t* bcnt, int bcap, uint64_t* live,
                                        int K, const bool (&h)[NP], const int32_t (&t)[NP],
                                        const uint64_t (&k)[NP]) {
    finish(bucket, bcap, live, K);
#pragma unroll
    for (int x = 0; x < NP; ++x) {
      has[x] = h[x];
      tgt[x] = t[x];
      key[x] = k[x];
      pos[x] = h[x] ? atomicAdd(bcnt + t[x], 1) : 0;
    }
  }
};

// ---------------------------------------------------------------------------
// mbarrier + bulk async copy (the TMA engine's non-tensor form).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared, completion counted on `bar` in bytes.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
constexpr uint32_t WAIT_LIMIT = 1u << 22;

// ---------------------------------------------------------------------------
// Kernel launchers (defined in knnm_kernels.cu / knnm_join.cu).  All take the
// stream they run on and return cudaGetLastError() of the launch.
// ---------------------------------------------------------------------------
struct DevCounters {
  unsigned long long updates;     // c_t
  unsigned long long dist_evals;  // pairs compared
  unsigned long long proposals;   // proposals written to the buffer
  unsigned long long overflow;    // proposals inserted directly (buffer full)
  unsigned long long reranked;    // BF16 path: FP32 recomputations
  unsigned long long err;         // DevErr bits
  unsigned long long err_row;     // smallest offending row
  unsigned long long gathered;    // candidate rows staged by the join
  unsigned long long inexact;     // rows that are not small integers (16-bit copies)
};

struct InitArgs {
  int mode;
  Rows rows;
  int64_t N, n1;
  const int32_t* G1;
  const int32_t* G2;
  int K, K_keep, metric;
  uint64_t seed;
  const float* norms;  // canonical norms [N] for COS, else nullptr
  int vec4;            // rows are 16-byte aligned and d % 4 == 0
  uint64_t* keys;      // [N][K]
  uint8_t* flags;      // [N][K]
  uint64_t* rear;      // [N][Kr]
  DevCounters* ctr;
  // When every row is exact in its 16-bit copy (small non-negative integers),
  // the distances are taken from the 16-bit extended rows [N][dx] instead of
  // the FP32 rows: the same values in the same order, half the bytes.
  const __nv_bfloat16* Xe = nullptr;
  int dx = 0;
  int half = 0;  // the 16-bit rows are FP16 (else BF16)
};
cudaError_t launch_init(const InitArgs& a, cudaStream_t st);

cudaError_t launch_norms(Rows rows, int64_t N, float* norms, cudaStream_t st);

struct SampleArgs {
  int64_t N;
  int K, s;
  uint64_t seed;
  int t;
  const int* t_dev = nullptr;  // when set, the round index is read from here (graph replay)
  const uint64_t* keys;   // [N][K]
  uint8_t* flags;         // [N][K], sampled entries flipped to old
  uint64_t* prev_keys;    // [N][K] snapshot for the finalize step (may be null)
  uint64_t* rev_new;      // [N][s] slots, KEY_EMPTY-initialised
  uint64_t* rev_old;      // [N][s]
  int cap_new, cap_old;
  int32_t* new_ids;  // [N][cap_new]
  int32_t* new_cnt;  // [N]
  int32_t* old_ids;  // [N][cap_old]
  int32_t* old_cnt;  // [N]
  DevCounters* ctr;
  // optional per-node candidate records for the pipelined join (may be null)
  unsigned char* rec = nullptr;  // [N][rec_bytes]
  int rec_cap = 0;               // ids per record (multiple of 4)
  const float* norms = nullptr;  // canonical norms (COS) copied into the records, else null
  int K_list = 0;                // list length, for the k-th key of each candidate
  // [N] per node {exactness width, canonical norm, round-start k-th key}: a
  // record entry's fields from one 16-byte gather (16 MB per 1M nodes: stays
  // in L2).  The sampler writes the k-th keys; info_c picks the word that goes
  // into the records' third column (0 the width, 1 the norm, -1 none).  When
  // null, the k-th keys come from the lists and the norms from `norms`.
  uint4* info = nullptr;
  int info_c = -1;
  // Bucketed reverse sampling (used when rcnt is set; rev_new/rev_old unused):
  // Bucketed reverse sampling (used when rcnt is set; rev_new/rev_old unused):
  int32_t* rcnt = nullptr;             // [2N] in-edges per (target, stream); zero on entry and exit
  unsigned long long* roffs = nullptr;  // [2N+1] bucket offsets
  int32_t* rbucket = nullptr;          // [N*K] reverse in-edges' source ids grouped by (target, stream)
  unsigned long long* tile_sum = nullptr;  // [ceil(2N/1024)+1] scan scratch
  unsigned long long* total = nullptr;     // scan total
  // Join-only sampling (bucketed path): old(u) is built only for nodes whose
  // new(u) is not empty, the only ones the join pairs from; the others get
  // empty candidate sets.  The step entry point keeps it off (full outputs).
  int active_only = 0;
  // Only the candidate records are read after the sampler (the join of this
  // round takes its candidates from them): the reverse samples need not be in
  // key order and new_ids / old_ids keep the forward sets only.
  int records_only = 0;
};
cudaError_t launch_sample(const SampleArgs& a, cudaStream_t st);
// Context internals used by the serving loop (knnm_api.cu): grow the
// context's scratch to at least `bytes`; bytes it holds now.
int ctx_reserve(knnm_ctx* ctx, uint64_t bytes);
uint64_t ctx_scratch_bytes(const knnm_ctx* ctx);

// Canonical distances of the K listed neighbours of each row, sorted by
// (distance, id); rows with an id out of range, self or repeated raise an error.
cudaError_t launch_list_dists(Rows rows, int64_t n, const int32_t* G, int K, int metric,
                              const float* norms, int32_t* ids, float* dists, DevCounters* ctr,
                              cudaStream_t st);
// Serving commit of one request's merged rows into the resident lists.
cudaError_t launch_commit(int64_t n_snap, int64_t rows, int K, int32_t* res_ids,
                          float* res_dists, const int32_t* out_ids, const float* out_dists,
                          int64_t base, cudaStream_t st);
// H-Merge: visiting order (a Feistel bijection of [0, n)) and the rows in it.
cudaError_t launch_permute(int64_t n, uint64_t seed, int32_t* perm, cudaStream_t st);
cudaError_t launch_gather_rows(const float* X, const int32_t* perm, int64_t n, int d, float* Xp,
                               cudaStream_t st);
// *p = v (one thread); *p += 1 (one thread).
cudaError_t launch_set_int(int* p, int v, cudaStream_t st);
cudaError_t launch_bump_int(int* p, cudaStream_t st);

// Candidate record of one node, read by the pipelined join with one bulk copy:
//   int32 {nn, no, 0, 0} | cap entries of 16 bytes {int32 id, float c, uint64 kth}
// (new candidates first).  kth is the k-th key of the candidate's list at round
// start; c its exactness width (tensor-core join) or canonical norm (FP32 join,
// COS).  One 16-byte load gives all three.
__host__ __device__ __forceinline__ int rec_bytes(int cap) { return 16 + 16 * cap; }
__device__ __forceinline__ uint4 rec_entry(int32_t id, float c, uint64_t kth) {
  return make_uint4((uint32_t)id, __float_as_uint(c), (uint32_t)kth, (uint32_t)(kth >> 32));
}
__device__ __forceinline__ int32_t rec_id(uint4 e) { return (int32_t)e.x; }
__device__ __forceinline__ float rec_c(uint4 e) { return __uint_as_float(e.y); }
__device__ __forceinline__ uint64_t rec_kth(uint4 e) { return ((uint64_t)e.w << 32) | e.z; }
__host__ __device__ __forceinline__ int round_up4(int x) { return (x + 3) & ~3; }

// Fills the width and norm words of every node's entry fields (SampleArgs::info).
cudaError_t launch_fill_info(int64_t N, const float* wx, const float* norms, uint4* info,
                             cudaStream_t st);

// Builds records from public candidate lists (the step-API path).
cudaError_t launch_build_records(int64_t N, int K, const uint64_t* keys, const float* norms,
                                 int cap_new, int cap_old, const int32_t* new_ids,
                                 const int32_t* new_cnt, const int32_t* old_ids,
                                 const int32_t* old_cnt, unsigned char* rec, int rec_cap,
                                 cudaStream_t st);

struct JoinArgs {
  int mode;
  Rows rows;
  int64_t N, n1;
  int K, metric;
  const float* norms;  // COS
  const uint64_t* keys;  // round-start lists [N][K] (read for the k-th key)
  int cap_new, cap_old;
  const int32_t* new_ids;
  const int32_t* new_cnt;
  const int32_t* old_ids;
  const int32_t* old_cnt;
  uint64_t* bucket;     // [N][bcap] proposal keys per target (UpdateNN input)
  int32_t* bcnt;        // [N] proposals offered per target this round (zero on entry)
  int bcap;             // bucket slots per target
  uint64_t* live_keys;  // lists receiving direct inserts once a bucket is full
  DevCounters* ctr;
  // BF16 path
  const __nv_bfloat16* Xb;  // [N][d] bf16 copy
  const float4* aux;        // per-row {bf16 squared norm, bf16 rounding-error norm, bf16 norm, canonical norm}
  const float* rmax;        // per-row max |x| of exact-integer rows, -1 otherwise
  int use_bulk;             // rows may be fetched with bulk async copies
  uint32_t wait_polls = WAIT_LIMIT;  // polls before an mbarrier wait gives up
};
// Ring join (knnm_join_pipe.cu): per-node candidate records and rows are
// staged by bulk copies into each warp's own shared-memory ring.
struct PipeArgs {
  const unsigned char* rec;  // [N][rec_bytes(cap)] candidate records
  int cap;                   // ids per record
  const __nv_bfloat16* Xe;   // BF16 rows with a 32-byte error-data tail [N][dx]
  int dx;                    // bf16 elements per extended row
  int nstages;               // unused by the ring kernel
  int cw;                    // warps per block
  int ring_rows;             // rows in each warp's ring
  int warp_bytes;            // shared memory per warp
  int row_bytes;             // bytes staged per candidate row
  int row_stride;            // bytes between staged rows
  int stage_bytes;           // record + rows of one stage
  int pair_cap;              // cap_new * (cap_new + cap_old)
  int gstr;                  // floats per row of the staged Gram block
};
// Fills the layout fields of P (not rec / Xe), the dynamic shared memory and
// the persistent grid; fails when the shapes do not fit the pipeline.
cudaError_t plan_pipe(int precision, int metric, int cap_new, int cap_old, int d, PipeArgs* P,
                      size_t* smem, int* grid);
cudaError_t launch_pipe(int precision, const JoinArgs& a, const PipeArgs& P, size_t smem,
                        int grid, cudaStream_t st);
// Tensor-core estimates, error bounds (0 for exact integer rows) and canonical
// distances of the pairs (pi[r], pj[r]), computed as the tensor-core join does.
cudaError_t launch_tc_estimate(int precision, int metric, const __nv_bfloat16* Xe, int dx,
                               Rows rows, const int32_t* pi, const int32_t* pj, int64_t P,
                               float* est, float* bound, float* canon, cudaStream_t st);
// 16-bit rows (BF16, or FP16 when half != 0; stored through __nv_bfloat16
// pointers as raw 16-bit elements) with their error-data tails; wx (optional)
// receives each row's exactness width, the tail's fifth float.
cudaError_t launch_bf16_ext(Rows rows, int64_t N, int dx, __nv_bfloat16* Xe, float* wx, int half,
                            unsigned long long* inexact, cudaStream_t st);

// Persistent join kernels: `grid` blocks loop over the nodes.
struct JoinPlan {
  int grid;       // blocks (= proposal regions)
  size_t smem;    // dynamic shared memory per block
  int chunk;      // dimensions staged per pass (FP32 kernel)
};
cudaError_t plan_join(int precision, int metric, int cap_new, int cap_old, int d, JoinPlan* out);
cudaError_t launch_join(int precision, const JoinArgs& a, const JoinPlan& plan, cudaStream_t st);

struct MergeArgs {
  int64_t N;
  int K;
  uint64_t* keys;             // [N][K] lists, merged in place
  const uint64_t* prev_keys;  // [N][K] round-start snapshot (flags / c_t)
  uint8_t* flags;             // [N][K] round-start flags in, merged flags out
  int32_t* cnt;               // [N] proposals offered per target; consumed back to zero
  int bcap;                   // bucket slots per target
  const uint64_t* bucket;     // [N][bcap] proposal keys per target
  DevCounters* ctr;
  int prefetch = 0;           // load each node's data one node ahead (rounds of
                              // few proposals: latency-bound, not issue-bound)
};
// The per-node merge of list and bucket (UpdateNN of the whole round) with
// flags and c_t.
cudaError_t launch_bucket_update(const MergeArgs& a, cudaStream_t st);

// sorted: every list and every rear list is ascending (the merge driver's own
// arrays), so the two are merged rather than sorted together.
cudaError_t launch_final(int64_t N, int K, const uint64_t* keys, int Kr, const uint64_t* rear,
                         int32_t* out_ids, float* out_dists, bool sorted, cudaStream_t st);

// Candidate counts with every node outside [lo, hi) set to 0.
cudaError_t launch_mask_counts(int64_t N, int64_t lo, int64_t hi, const int32_t* in_new,
                               const int32_t* in_old, int32_t* out_new, int32_t* out_old,
                               cudaStream_t st);
// Per row: the first K distinct keys of `parts` lists [parts][n][K], flags
// against the start lists, c_t added to ctr->updates.
cudaError_t launch_union(int64_t n, int K, int parts, const int32_t* part_ids,
                         const float* part_dists, const int32_t* start_ids,
                         const float* start_dists, const uint8_t* start_flags, int32_t* out_ids,
                         float* out_dists, uint8_t* out_flags, DevCounters* ctr, cudaStream_t st);

// Conversions between the packed working lists and the (ids, dists) arrays.
cudaError_t launch_pack(int64_t count, const int32_t* ids, const float* dists, uint64_t* keys,
                        cudaStream_t st);
cudaError_t launch_unpack(int64_t count, const uint64_t* keys, int32_t* ids, float* dists,
                          cudaStream_t st);

// BF16 shadow copy and per-row error data for the tensor-core path.
// rmax[i] = max |x| of row i when BF16 holds the row exactly as integers, else -1.
cudaError_t launch_bf16_prep(Rows rows, int64_t N, __nv_bfloat16* Xb, float4* aux, float* rmax,
                             int half, unsigned long long* inexact, cudaStream_t st);

// Validates set rows (CSR): errors land in ctr (err, err_row).
cudaError_t launch_check_sets(const int64_t* off, const int32_t* items, int64_t nnz, int64_t n,
                              DevCounters* ctr, cudaStream_t st);

// Exclusive scan of cnt[0..n) into offs[0..n] (offs[n] = total); tile_sum
// needs ceil(n / 1024) entries.
cudaError_t launch_exclusive_scan(const int32_t* cnt, int64_t n, unsigned long long* tile_sum,
                                  unsigned long long* offs, unsigned long long* total,
                                  cudaStream_t st);

// ---------------------------------------------------------------------------
// Graph diversification (Alg. 3) and the top-down search (Sec. 3.4):
// knnm_gd.cu.
// ---------------------------------------------------------------------------
struct GdCounters {
  unsigned long long dist_evals;  // distances computed
  unsigned long long edges;       // sum of output degrees
  unsigned long long full_rows;   // rows whose degree reached the cap
  unsigned long long max_in;      // largest in-degree of the input graph
  unsigned long long overflow;    // search: queries whose visited table ran out of room
  unsigned long long err;         // DevErr bits
  unsigned long long err_row;     // smallest offending row
};

struct GdArgs {
  const float* X;      // [n][d]
  int64_t n;
  int d;
  int vec4;            // rows 16-byte aligned and d % 4 == 0
  const float* norms;  // canonical norms [n] (COS), else nullptr
  const int32_t* G;    // [n][K] input graph
  int K;
  int M;               // output degree cap
  int stage;           // rows staged in shared memory (set by plan_diversify)
  int stride;          // floats between staged rows
  int32_t* indeg;      // [n] in-degrees (zeroed by the launcher)
  int32_t* rev_fill;   // [n] reverse-bucket cursors (zeroed by the launcher)
  unsigned long long* rev_off;  // [n+1]
  unsigned long long* tile_sum;
  unsigned long long* total;
  uint64_t* rev;       // [n*K] reverse entries (distance, source)
  uint64_t* fwd;       // [n][K] forward kept entries
  int32_t* fwd_cnt;    // [n]
  int32_t* out_ids;    // [n][M]
  float* out_dists;    // [n][M]
  int32_t* out_deg;    // [n]
  GdCounters* ctr;
};
// Fills the staging fields of a (vec4, d, K, M set); false when the layout
// would leave a shared-memory region misaligned.
bool plan_diversify(GdArgs* a);
cudaError_t launch_diversify(const GdArgs& a, int metric, cudaStream_t st);
cudaError_t launch_gather_checked(const float* X, int64_t n_src, const int32_t* perm, int64_t n,
                                  int d, float* out, GdCounters* ctr, cudaStream_t st);

constexpr int SEARCH_MAX_LAYERS = 32;
struct SearchArgs {
  const float* X;  // [n][d], layer l covers rows [0, rows[l])
  int64_t n;
  int d;
  int vec4;
  const float* aux;  // [n][2] per row: max |x| of an integer row (else -1), canonical norm
  int n_layers;
  int64_t rows[SEARCH_MAX_LAYERS];
  int width[SEARCH_MAX_LAYERS];
  const int32_t* g[SEARCH_MAX_LAYERS];  // [rows[l]][width[l]], ids < 0 are padding
  const float* Q;  // [nq][d]
  int64_t nq;
  int ef, k_out;
  uint64_t seed;
  int hbits;       // visited table of 2^hbits ids per query
  int warps;       // warps per block
  int warp_bytes;  // shared memory per warp
  int32_t* out_ids;
  float* out_dists;
  uint32_t* out_evals;  // [nq] or nullptr
  GdCounters* ctr;
};
// Fills hbits / warps / warp_bytes and the launch shape.
cudaError_t plan_search(SearchArgs* a, size_t* smem, int* grid);
cudaError_t launch_search(const SearchArgs& a, int metric, size_t smem, int grid, cudaStream_t st);
// Per-row search data aux [n][2]: {max |x| when the row is all integers of
// magnitude <= 2^24, else -1; canonical norm}.
cudaError_t launch_row_aux(const float* X, int64_t n, int d, float* aux, cudaStream_t st);

}  // namespace knnm
