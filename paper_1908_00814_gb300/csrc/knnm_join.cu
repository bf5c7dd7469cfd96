// knnm_join.cu -- the local join of one round (Alg. 1 / Alg. 2 inner loops):
// for every node u, every allowed pair of its candidate set new(u) u old(u) is
// compared and offered to UpdateNN of both endpoints.
//
// Two persistent kernels, one block of 128 threads per node at a time:
//   * k_join_fp32: the candidate rows are staged in shared memory with 1-D
//     bulk async copies (TMA engine, mbarrier completion), one thread computes
//     one pair's canonical FP32 distance.  Long rows are processed in chunks
//     of dimensions with per-pair accumulators kept in shared memory, which
//     keeps the in-order accumulation.
//   * k_join_bf16: the BF16 copies of the candidate rows are staged the same
//     way; the Gram block of new x all candidates is computed with
//     mma.sync m16n8k16 (BF16 in, FP32 accumulate).  A pair whose estimated
//     distance minus a proven error bound could still reach the k-th distance
//     of an endpoint is recomputed canonically in FP32 from global memory;
//     all others are skipped, so the proposals are exactly the FP32 kernel's.
//
// A proposal (p <- q, d) is written only when its key (d, q) is below p's
// k-th key (read when the block starts node u): no other proposal can enter
// the top-k union.  Proposals go to their target's bucket; once a bucket is
// full they are inserted into the target's live list at once.
#include "knnm_internal.cuh"

namespace knnm {

namespace {

constexpr int JT = 128;  // threads per join block

__device__ __forceinline__ bool pair_allowed(int mode, int64_t n1, int32_t p, int32_t q) {
  const bool p1 = p < n1, q1 = q < n1;
  return mode == SYMMETRIC ? (p1 != q1) : !(p1 && q1);
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct JoinShared {
  int32_t* cid;      // [cap_rows] candidate ids, new first
  uint64_t* kth;     // [cap_rows] k-th key of each candidate's list
  float* cnorm;      // [cap_rows] canonical norms (COS)
  uint16_t* pairs;   // [pair_cap] (i << 8) | j
  uint64_t* bar;     // mbarrier
  int* scal;         // [0] npairs, [1] proposals offered, [2] re-rank count, [3] direct inserts
};

// Loads the candidate list of node u (ids, k-th keys, norms); returns nn, M.
__device__ __forceinline__ void load_candidates(const JoinArgs& a, int64_t u, JoinShared& S,
                                                int& nn, int& M) {
  nn = a.new_cnt[u];
  int no = a.old_cnt[u];
  if (nn > a.cap_new || no > a.cap_old || nn < 0 || no < 0) {
    if (threadIdx.x == 0) {
      atomicOr(&a.ctr->err, (unsigned long long)DERR_CAPACITY);
      atomicMin(&a.ctr->err_row, (unsigned long long)u);
    }
    nn = min(max(nn, 0), a.cap_new);
    no = min(max(no, 0), a.cap_old);
  }
  M = nn + no;
  for (int r = threadIdx.x; r < M; r += JT) {
    int32_t id = r < nn ? a.new_ids[(size_t)u * a.cap_new + r]
                        : a.old_ids[(size_t)u * a.cap_old + (r - nn)];
    if (id < 0 || id >= a.N) {
      atomicOr(&a.ctr->err, (unsigned long long)DERR_BAD_PAIR);
      atomicMin(&a.ctr->err_row, (unsigned long long)u);
      id = 0;
    }
    S.cid[r] = id;
    S.kth[r] = a.keys[(size_t)id * a.K + (a.K - 1)];
    if (a.metric == COS) S.cnorm[r] = a.norms[id];
  }
}

// Compacts the allowed pairs (i < nn, i < j < M, set mask) into S.pairs.
__device__ __forceinline__ int build_pairs(const JoinArgs& a, int nn, int M, JoinShared& S) {
  if (threadIdx.x == 0) S.scal[0] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int total = nn * M;
  for (int f0 = 0; f0 < total; f0 += JT) {
    int f = f0 + threadIdx.x;
    bool ok = false;
    int i = 0, j = 0;
    if (f < total) {
      i = f / M;
      j = f - i * M;
      ok = j > i && pair_allowed(a.mode, a.n1, S.cid[i], S.cid[j]);
    }
    unsigned b = __ballot_sync(FULL, ok);
    int base = 0;
    if (lane == 0 && b) base = atomicAdd(&S.scal[0], __popc(b));
    base = __shfl_sync(FULL, base, 0);
    if (ok) {
      unsigned lt = b & ((1u << lane) - 1u);
      S.pairs[base + __popc(lt)] = (uint16_t)((i << 8) | j);
    }
  }
  __syncthreads();
  return S.scal[0];
}

// Offers this warp's proposals (up to two per lane) to UpdateNN; the block
// counts offers in S.scal[1] and direct inserts in S.scal[3].
__device__ __forceinline__ void emit(const JoinArgs& a, JoinShared& S, bool hp, int32_t tp,
                                     uint64_t kp, bool hq, int32_t tq, uint64_t kq) {
  const bool has[2] = {hp, hq};
  const int32_t tgt[2] = {tp, tq};
  const uint64_t key[2] = {kp, kq};
  unsigned long long np_ = 0, nd_ = 0;
  emit_to_buckets<2>(a.bucket, a.bcnt, a.bcap, a.live_keys, a.K, has, tgt, key, np_, nd_);
  const unsigned n = __reduce_add_sync(FULL, (unsigned)np_);
  const unsigned nd = __reduce_add_sync(FULL, (unsigned)nd_);
  if ((threadIdx.x & 31) == 0 && n) {
    atomicAdd(&S.scal[1], (int)n);
    if (nd) atomicAdd(&S.scal[3], (int)nd);
  }
}

// Bulk-copies elements [off, off + elems) of each candidate row into
// consecutive shared rows of `stride_bytes` (TMA engine, completion counted on
// the block's mbarrier).  Row r's source is row_ptr(cid[r]) + off.  Returns
// false if the bounded wait ran out; the copies in flight are then given a
// second bounded wait so that they land before the buffer is reused.
template <typename T, typename RowPtr>
__device__ __forceinline__ bool stage_rows(const JoinArgs& a, JoinShared& S, int M, RowPtr row_ptr,
                                           int off, int elems, unsigned char* dst,
                                           int stride_bytes, uint32_t& phase) {
  if (M == 0) return true;
  if (threadIdx.x == 0) {
    fence_proxy_async();
    mbar_arrive_expect_tx(S.bar, (uint32_t)(M * elems * sizeof(T)));
    for (int r = 0; r < M; ++r)
      bulk_g2s(dst + (size_t)r * stride_bytes, row_ptr(S.cid[r]) + off,
               (uint32_t)(elems * sizeof(T)), S.bar);
  }
  bool ok = mbar_wait_bounded(S.bar, phase, a.wait_polls);
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(&a.ctr->err, (unsigned long long)DERR_WAIT_TIMEOUT);
    mbar_wait_bounded(S.bar, phase, WAIT_LIMIT);
  }
  phase ^= 1u;
  return ok;
}

struct Fp32Row {
  Rows R;
  __device__ __forceinline__ const float* operator()(int32_t id) const { return R.row(id); }
};
struct Bf16Row {
  const __nv_bfloat16* Xb;
  int d;
  __device__ __forceinline__ const __nv_bfloat16* operator()(int32_t id) const {
    return Xb + (size_t)id * d;
  }
};

// Same with plain loads (rows of any alignment or split across two arrays).
__device__ __forceinline__ void load_rows_plain(const JoinArgs& a, JoinShared& S, int M, int off,
                                                int elems, float* dst, int stride) {
  for (int idx = threadIdx.x; idx < M * elems; idx += JT) {
    int r = idx / elems, t = idx - r * elems;
    dst[(size_t)r * stride + t] = __ldg(a.rows.row(S.cid[r]) + off + t);
  }
}

// ---------------------------------------------------------------------------
// FP32 canonical join
// ---------------------------------------------------------------------------

template <int METRIC>
__global__ void __launch_bounds__(JT) k_join_fp32(JoinArgs a, int chunk, int pair_cap) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int cap_rows = a.cap_new + a.cap_old;
  const int stride = chunk + 4;  // floats; 16-byte rows offset by 16 bytes
  const int d = a.rows.d;
  const bool chunked = chunk < d;
  float* srows = (float*)smem;
  unsigned char* p = smem + (size_t)cap_rows * stride * sizeof(float);
  JoinShared S;
  S.kth = (uint64_t*)p;
  p += (size_t)cap_rows * 8;
  S.bar = (uint64_t*)p;
  p += 16;
  S.cid = (int32_t*)p;
  p += (size_t)cap_rows * 4;
  S.cnorm = (float*)p;
  p += (size_t)cap_rows * 4;
  S.scal = (int*)p;
  p += 16;
  float* sacc = (float*)p;
  if (chunked) p += (size_t)pair_cap * 4;
  S.pairs = (uint16_t*)p;

  if (threadIdx.x == 0) {
    mbar_init(S.bar, 1);
    fence_mbar_init();
    S.scal[1] = 0;
    S.scal[3] = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  unsigned long long evals = 0, gathered = 0;
  const bool bulk = a.use_bulk != 0;

  for (int64_t u = blockIdx.x; u < a.N; u += gridDim.x) {
    int nn, M;
    load_candidates(a, u, S, nn, M);
    __syncthreads();
    const int np = build_pairs(a, nn, M, S);
    evals += (threadIdx.x == 0) ? (unsigned long long)np : 0ull;
    gathered += (threadIdx.x == 0 && np > 0) ? (unsigned long long)M : 0ull;
    for (int c0 = 0; c0 < d; c0 += chunk) {
      const int cw = min(chunk, d - c0);
      if (np > 0) {
        if (bulk)
          stage_rows<float>(a, S, M, Fp32Row{a.rows}, c0, cw, (unsigned char*)srows,
                            stride * (int)sizeof(float), phase);
        else
          load_rows_plain(a, S, M, c0, cw, srows, stride);
      }
      __syncthreads();
      const bool last = c0 + cw >= d;
      for (int q0 = 0; q0 < np; q0 += JT) {
        const int q = q0 + threadIdx.x;
        bool hp = false, hq = false;
        int32_t tp = 0, tq = 0;
        uint64_t kp = 0, kq = 0;
        if (q < np) {
          const uint16_t pr = S.pairs[q];
          const int i = pr >> 8, j = pr & 0xFF;
          const float* ra = srows + (size_t)i * stride;
          const float* rb = srows + (size_t)j * stride;
          float acc = (chunked && c0 > 0) ? sacc[q] : 0.0f;
          int t = 0;
          for (; t + 4 <= cw; t += 4) {
            const float4 x = *reinterpret_cast<const float4*>(ra + t);
            const float4 y = *reinterpret_cast<const float4*>(rb + t);
            acc = Canon<METRIC>::step(acc, x.x, y.x);
            acc = Canon<METRIC>::step(acc, x.y, y.y);
            acc = Canon<METRIC>::step(acc, x.z, y.z);
            acc = Canon<METRIC>::step(acc, x.w, y.w);
          }
          for (; t < cw; ++t) acc = Canon<METRIC>::step(acc, ra[t], rb[t]);
          if (!last) {
            sacc[q] = acc;
          } else {
            const float dist = canon_finish<METRIC>(acc, METRIC == COS ? S.cnorm[i] : 0.f,
                                                    METRIC == COS ? S.cnorm[j] : 0.f);
            const int32_t pi = S.cid[i], pj = S.cid[j];
            kp = make_key(dist, pj);
            kq = make_key(dist, pi);
            hp = kp < S.kth[i];
            hq = kq < S.kth[j];
            tp = pi;
            tq = pj;
          }
        }
        if (last) emit(a, S, hp, tp, kp, hq, tq, kq);
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.ctr->proposals, (unsigned long long)S.scal[1]);
    atomicAdd(&a.ctr->overflow, (unsigned long long)S.scal[3]);
    atomicAdd(&a.ctr->dist_evals, evals);
    atomicAdd(&a.ctr->gathered, gathered);
  }
}

// ---------------------------------------------------------------------------
// Jaccard join on sets (CSR rows): one thread per pair intersects the two
// sorted item lists from global memory; no rows are staged.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(JT) k_join_jaccard(JoinArgs a, int pair_cap) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int cap_rows = a.cap_new + a.cap_old;
  unsigned char* p = smem;
  JoinShared S;
  S.kth = (uint64_t*)p;
  p += (size_t)cap_rows * 8;
  S.bar = (uint64_t*)p;
  p += 16;
  S.cid = (int32_t*)p;
  p += (size_t)cap_rows * 4;
  S.cnorm = (float*)p;
  p += (size_t)cap_rows * 4;
  S.scal = (int*)p;
  p += 16;
  S.pairs = (uint16_t*)p;
  (void)pair_cap;
  if (threadIdx.x == 0) S.scal[1] = S.scal[3] = 0;
  __syncthreads();
  unsigned long long evals = 0, gathered = 0;
  for (int64_t u = blockIdx.x; u < a.N; u += gridDim.x) {
    int nn, M;
    load_candidates(a, u, S, nn, M);
    __syncthreads();
    const int np = build_pairs(a, nn, M, S);
    evals += (threadIdx.x == 0) ? (unsigned long long)np : 0ull;
    gathered += (threadIdx.x == 0 && np > 0) ? (unsigned long long)M : 0ull;
    for (int q0 = 0; q0 < np; q0 += JT) {
      const int q = q0 + threadIdx.x;
      bool hp = false, hq = false;
      int32_t tp = 0, tq = 0;
      uint64_t kp = 0, kq = 0;
      if (q < np) {
        const uint16_t pr = S.pairs[q];
        const int i = pr >> 8, j = pr & 0xFF;
        const int32_t pi = S.cid[i], pj = S.cid[j];
        const float dist = jaccard_rows(a.rows, pi, pj);
        kp = make_key(dist, pj);
        kq = make_key(dist, pi);
        hp = kp < S.kth[i];
        hq = kq < S.kth[j];
        tp = pi;
        tq = pj;
      }
      emit(a, S, hp, tp, kp, hq, tq, kq);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&a.ctr->proposals, (unsigned long long)S.scal[1]);
    atomicAdd(&a.ctr->overflow, (unsigned long long)S.scal[3]);
    atomicAdd(&a.ctr->dist_evals, evals);
    atomicAdd(&a.ctr->gathered, gathered);
  }
}

// ---------------------------------------------------------------------------
// BF16 tensor-core join with FP32 re-rank
// ---------------------------------------------------------------------------

constexpr int TC_ROWS = 64;  // candidate rows per block (new + old, padded)
constexpr int TC_NEW = 32;   // new rows (two m16 tiles)

__device__ __forceinline__ void ldmatrix_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                            uint32_t& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldmatrix_x2(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_u32(p)));
}
// 16-bit inputs (both BF16, or both FP16), FP32 accumulation.
template <bool HALF>
__device__ __forceinline__ void mma_bf16(float* c, uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  if (HALF)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Upper bound on |estimate - canonical distance| for one pair.
//   g      FP32 (tensor-core) dot product of the BF16 rows
//   ai/aj  aux rows {|b|^2, |b - x|, |b|, canonical |x|}
// The estimate is returned in *est.
template <int METRIC>
__device__ __forceinline__ float tc_bound(float g, float4 ai, float4 aj, int d, float* est) {
  const float u = 5.9604645e-8f;                     // 2^-24
  const float g_mma = (float)(d + 32) * 9.5367432e-7f;  // (d+32) * 2^-20 per |a||b|
  const float g_can = (float)(d + 4) * u * 1.01f;       // in-order FP32 sum, relative
  const float si = ai.z, sj = aj.z;                     // |b_i|, |b_j| (rounded up)
  const float ei = ai.y, ej = aj.y;                     // |b_i - x_i|, |b_j - x_j|
  if (METRIC == L2) {
    const float dt = (ai.x + aj.x) - 2.0f * g;
    *est = dt;
    // tensor-core and norm arithmetic, absolute
    const float A = g_mma * (si + sj) * (si + sj) + 4.0f * u * (ai.x + aj.x + 2.0f * fabsf(g));
    // BF16 rounding of the inputs: | |x_i-x_j| - |b_i-b_j| | <= ei + ej
    const float e = ei + ej;
    const float up = fmaxf(dt + A, 0.0f);
    const float B = 2.0f * e * sqrtf(up) + e * e;
    // canonical FP32 evaluation of the exact distance
    const float C = g_can * (up + B);
    return (A + B + C) * 1.001f + 1e-30f;
  } else {
    // |x_i.x_j - b_i.b_j| <= |b_i| ej + |x_j| ei,  |x_j| <= |b_j| + ej
    const float dot_err = g_mma * si * sj + si * ej + (sj + ej) * ei +
                          g_can * (si + ei) * (sj + ej);
    if (METRIC == IP) {
      *est = -g;
      return dot_err * 1.001f + 1e-30f;
    }
    const float den = ai.w * aj.w;  // canonical norms
    if (den == 0.0f) {
      *est = 1.0f;
      return 0.0f;
    }
    *est = 1.0f - g / den;
    return (dot_err / den) * 1.001f + 8.0f * u + 1e-30f;
  }
}

// Rows whose every value is a non-negative integer <= 256 are held exactly by
// BF16 (rmax = their max, else -1).  If d * (max_i^2 + max_j^2) < 2^24 every
// product and every partial sum of the dot product, the norms, their sum and
// the canonical in-order sum of (x_i - x_j)^2 are integers below 2^24, so the
// tensor-core accumulation and the canonical FP32 evaluation are both exact
// and agree bit for bit.
__device__ __forceinline__ bool exact_pair(float ri, float rj, int d) {
  if (ri < 0.f || rj < 0.f) return false;
  const long long mi = (long long)ri, mj = (long long)rj;
  return (long long)d * (mi * mi + mj * mj) < (1ll << 24);
}

// The canonical distance from an exact dot product g, finished with the same
// correctly rounded operations as the canonical evaluation.
template <int METRIC>
__device__ __forceinline__ float exact_estimate(float g, float4 ai, float4 aj) {
  if (METRIC == L2) return __fsub_rn(__fadd_rn(ai.x, aj.x), __fmul_rn(2.0f, g));
  return canon_finish<METRIC>(g, ai.w, aj.w);
}

template <int METRIC, bool HALF>
__global__ void __launch_bounds__(JT) k_join_bf16(JoinArgs a, int pair_cap) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int d = a.rows.d;
  const int bstride = d * 2 + 16;  // bytes per staged BF16 row
  unsigned char* srows = smem;
  unsigned char* p = smem + (size_t)TC_ROWS * bstride;
  JoinShared S;
  S.kth = (uint64_t*)p;
  p += TC_ROWS * 8;
  S.bar = (uint64_t*)p;
  p += 16;
  S.cid = (int32_t*)p;
  p += TC_ROWS * 4;
  S.cnorm = (float*)p;
  p += TC_ROWS * 4;
  S.scal = (int*)p;
  p += 16;
  float4* saux = (float4*)p;
  p += TC_ROWS * sizeof(float4);
  float* srmax = (float*)p;
  p += TC_ROWS * 4;
  uint16_t* cand = (uint16_t*)p;  // pairs to re-rank
  p += (size_t)pair_cap * 2;
  S.pairs = (uint16_t*)p;  // unused by this kernel except as scratch
  int* s_rr = S.scal + 2;  // re-rank count

  if (threadIdx.x == 0) {
    mbar_init(S.bar, 1);
    fence_mbar_init();
    S.scal[1] = 0;
    S.scal[3] = 0;
  }
  // zero the padding rows once: rows >= M of a node are never read as pairs but
  // feed the MMA tiles
  for (int idx = threadIdx.x; idx < TC_ROWS * bstride / 4; idx += JT) ((uint32_t*)srows)[idx] = 0u;
  __syncthreads();
  uint32_t phase = 0;
  unsigned long long evals = 0, reranked = 0, gathered = 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int64_t u = blockIdx.x; u < a.N; u += gridDim.x) {
    int nn, M;
    load_candidates(a, u, S, nn, M);
    if (threadIdx.x == 0) s_rr[0] = 0;
    for (int r = threadIdx.x; r < M; r += JT) {
      saux[r] = a.aux[S.cid[r]];
      srmax[r] = a.rmax[S.cid[r]];
    }
    __syncthreads();
    if (nn > 0 && M > 1) {
      gathered += (threadIdx.x == 0) ? (unsigned long long)M : 0ull;
      stage_rows<__nv_bfloat16>(a, S, M, Bf16Row{a.Xb, d}, 0, d, srows, bstride, phase);
      __syncthreads();
      // Gram tile: warp w takes m-tile (w & 1) (rows 16*(w&1) ..) and n-tiles
      // (w >> 1) * 4 .. +4 (columns 32*(w>>1) ..).  Rows/cols past M are zero.
      const int mt = warp & 1, ng = warp >> 1;
      float c[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x) c[x][0] = c[x][1] = c[x][2] = c[x][3] = 0.f;
      const bool active = mt * 16 < nn && ng * 32 < M;
      if (active) {
        for (int k0 = 0; k0 < d; k0 += 16) {
          uint32_t a0, a1, a2, a3;
          // A fragment: rows mt*16 + (lane & 15), cols k0 + (lane >> 4) * 8
          const unsigned char* pa =
              srows + (size_t)(mt * 16 + (lane & 15)) * bstride + (k0 + (lane >> 4) * 8) * 2;
          ldmatrix_x4(a0, a1, a2, a3, pa);
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            uint32_t b0, b1;
            // B fragment (col-major K x 8): candidate rows n0 + (lane & 7),
            // cols k0 + ((lane >> 3) & 1) * 8
            const int n0 = ng * 32 + x * 8;
            const unsigned char* pb =
                srows + (size_t)(n0 + (lane & 7)) * bstride + (k0 + ((lane >> 3) & 1) * 8) * 2;
            ldmatrix_x2(b0, b1, pb);
            mma_bf16<HALF>(c[x], a0, a1, a2, a3, b0, b1);
          }
        }
        // C fragment: c[x][0..1] at row lane/4, cols 2*(lane%4)+{0,1};
        // c[x][2..3] at row lane/4 + 8.
#pragma unroll
        for (int x = 0; x < 4; ++x) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int i = mt * 16 + (lane >> 2) + ((h & 2) ? 8 : 0);
            const int j = ng * 32 + x * 8 + 2 * (lane & 3) + (h & 1);
            bool ok = i < nn && j < M && j > i &&
                      pair_allowed(a.mode, a.n1, S.cid[i], S.cid[j]);
            bool hp = false, hq = false;
            int32_t tp = 0, tq = 0;
            uint64_t kp = 0, kq = 0;
            if (ok) {
              float est;
              if (exact_pair(srmax[i], srmax[j], d)) {
                // both rows are small non-negative integers: the tensor-core sum
                // and the canonical FP32 sum are the same exact integers
                est = exact_estimate<METRIC>(c[x][h], saux[i], saux[j]);
                tp = S.cid[i];
                tq = S.cid[j];
                kp = make_key(est, tq);
                kq = make_key(est, tp);
                hp = kp < S.kth[i];
                hq = kq < S.kth[j];
              } else {
                const float E = tc_bound<METRIC>(c[x][h], saux[i], saux[j], d, &est);
                const float thr = fmaxf(key_dist(S.kth[i]), key_dist(S.kth[j]));
                // a pair whose lower bound exceeds both k-th distances is dropped
                if (est - E <= thr) {
                  int pos = atomicAdd(s_rr, 1);
                  cand[pos] = (uint16_t)((i << 8) | j);
                }
              }
            }
            emit(a, S, hp, tp, kp, hq, tq, kq);
            evals += ok ? 1ull : 0ull;
          }
        }
      }
    }
    __syncthreads();
    const int nr = s_rr[0];
    reranked += (threadIdx.x == 0) ? (unsigned long long)nr : 0ull;
    for (int q0 = 0; q0 < nr; q0 += JT) {
      const int q = q0 + threadIdx.x;
      bool hp = false, hq = false;
      int32_t tp = 0, tq = 0;
      uint64_t kp = 0, kq = 0;
      if (q < nr) {
        const uint16_t pr = cand[q];
        const int i = pr >> 8, j = pr & 0xFF;
        const int32_t pi = S.cid[i], pj = S.cid[j];
        const float dist =
            a.use_bulk ? canon_dist_global4<METRIC>(a.rows.row(pi), a.rows.row(pj), d,
                                                     saux[i].w, saux[j].w)
                       : canon_dist_global<METRIC>(a.rows.row(pi), a.rows.row(pj), d,
                                                     saux[i].w, saux[j].w);
        kp = make_key(dist, pj);
        kq = make_key(dist, pi);
        hp = kp < S.kth[i];
        hq = kq < S.kth[j];
        tp = pi;
        tq = pj;
      }
      emit(a, S, hp, tp, kp, hq, tq, kq);
    }
    __syncthreads();
  }
  // block totals
  __shared__ unsigned long long red[JT / 32];
  unsigned long long e = evals;
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
  if (lane == 0) red[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < JT / 32; ++w) tot += red[w];
    atomicAdd(&a.ctr->proposals, (unsigned long long)S.scal[1]);
    atomicAdd(&a.ctr->overflow, (unsigned long long)S.scal[3]);
    atomicAdd(&a.ctr->dist_evals, tot);
    atomicAdd(&a.ctr->reranked, reranked);
    atomicAdd(&a.ctr->gathered, gathered);
  }
}

size_t fp32_smem_bytes(int cap_rows, int chunk, int pair_cap, bool chunked) {
  size_t b = (size_t)cap_rows * (chunk + 4) * 4;  // rows
  b += (size_t)cap_rows * 8 + 16 + (size_t)cap_rows * 4 * 2 + 16;
  if (chunked) b += (size_t)pair_cap * 4;
  b += (size_t)pair_cap * 2;
  return (b + 127) & ~(size_t)127;
}

size_t bf16_smem_bytes(int d, int pair_cap) {
  size_t b = (size_t)TC_ROWS * (d * 2 + 16);
  b += TC_ROWS * 8 + 16 + TC_ROWS * 4 * 2 + 16 + TC_ROWS * sizeof(float4) + TC_ROWS * 4;
  b += (size_t)pair_cap * 2 * 2;
  return (b + 127) & ~(size_t)127;
}

template <typename KernelT>
cudaError_t occupancy_grid(KernelT kernel, size_t smem, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, JT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = sms * per_sm;
  return cudaSuccess;
}

template <int METRIC>
cudaError_t plan_metric(int precision, int cap_new, int cap_old, int d, JoinPlan* out) {
  const int cap_rows = cap_new + cap_old;
  const int pair_cap = cap_new * cap_rows;
  if (precision != 0 && METRIC != L1 && METRIC != CHI2) {
    out->chunk = d;
    out->smem = bf16_smem_bytes(d, pair_cap);
    return precision == 2 ? occupancy_grid(k_join_bf16<METRIC, true>, out->smem, &out->grid)
                          : occupancy_grid(k_join_bf16<METRIC, false>, out->smem, &out->grid);
  }
  // FP32: stage whole rows when they fit in ~56 KB, else chunks of dimensions
  const size_t budget = 56 * 1024;
  int d4 = (d + 3) & ~3;
  int chunk = d4;
  if (fp32_smem_bytes(cap_rows, chunk, pair_cap, false) > budget) {
    size_t fixed = fp32_smem_bytes(cap_rows, 0, pair_cap, true);
    long per = (long)cap_rows * 4;
    long c = budget > fixed ? (long)((budget - fixed) / per) - 4 : 32;
    c = c < 32 ? 32 : c;
    chunk = (int)(c & ~3L);
    if (chunk >= d4) chunk = d4;
  }
  out->chunk = chunk;
  out->smem = fp32_smem_bytes(cap_rows, chunk, pair_cap, chunk < d);
  return occupancy_grid(k_join_fp32<METRIC>, out->smem, &out->grid);
}

}  // namespace

cudaError_t plan_join(int precision, int metric, int cap_new, int cap_old, int d, JoinPlan* out) {
  if (cap_new + cap_old > 255) return cudaErrorInvalidValue;
  if (metric == JACCARD) {
    const int cap_rows = cap_new + cap_old;
    out->chunk = 0;
    out->smem = ((size_t)cap_rows * 16 + 32 + (size_t)cap_new * cap_rows * 2 + 127) & ~(size_t)127;
    return occupancy_grid(k_join_jaccard, out->smem, &out->grid);
  }
  if (precision != 0 && metric != L1 && metric != CHI2 &&
      (cap_new > TC_NEW || cap_new + cap_old > TC_ROWS))
    return cudaErrorInvalidValue;
  switch (metric) {
    case L2: return plan_metric<L2>(precision, cap_new, cap_old, d, out);
    case IP: return plan_metric<IP>(precision, cap_new, cap_old, d, out);
    case COS: return plan_metric<COS>(precision, cap_new, cap_old, d, out);
    case L1: return plan_metric<L1>(precision, cap_new, cap_old, d, out);
    default: return plan_metric<CHI2>(precision, cap_new, cap_old, d, out);
  }
}

cudaError_t launch_join(int precision, const JoinArgs& a, const JoinPlan& plan, cudaStream_t st) {
  const int pair_cap = a.cap_new * (a.cap_new + a.cap_old);
  if (a.metric == JACCARD) {
    k_join_jaccard<<<plan.grid, JT, plan.smem, st>>>(a, pair_cap);
  } else if (precision == 2 && a.metric != L1 && a.metric != CHI2) {
    switch (a.metric) {
      case L2: k_join_bf16<L2, true><<<plan.grid, JT, plan.smem, st>>>(a, pair_cap); break;
      case IP: k_join_bf16<IP, true><<<plan.grid, JT, plan.smem, st>>>(a, pair_cap); break;
      default: k_join_bf16<COS, true><<<plan.grid, JT, plan.smem, st>>>(a, pair_cap); break;
    }
  } else if (precision == 1 && a.metric != L1 && a.metric != CHI2) {
    switch (a.metric) {
      case L2: k_join_bf16<L2, false><<<plan.grid, JT, plan.smem, st>>>(a, pair_cap); break;
      case IP: k_join_bf16<IP, false><<<plan.grid, JT, plan.smem, st>>>(a, pair_cap); break;
      default: k_join_bf16<COS, false><<<plan.grid, JT, plan.smem, st>>>(a, pair_cap); break;
    }
  } else {
    switch (a.metric) {
      case L2: k_join_fp32<L2><<<plan.grid, JT, plan.smem, st>>>(a, plan.chunk, pair_cap); break;
      case IP: k_join_fp32<IP><<<plan.grid, JT, plan.smem, st>>>(a, plan.chunk, pair_cap); break;
      case COS: k_join_fp32<COS><<<plan.grid, JT, plan.smem, st>>>(a, plan.chunk, pair_cap); break;
      case L1: k_join_fp32<L1><<<plan.grid, JT, plan.smem, st>>>(a, plan.chunk, pair_cap); break;
      default: k_join_fp32<CHI2><<<plan.grid, JT, plan.smem, st>>>(a, plan.chunk, pair_cap); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace knnm
