// knnm_join_pipe.cu -- the local join (Alg. 1 / Alg. 2 inner loops) as a
// warp-specialized, multi-stage bulk-copy pipeline.
//
// One block per SM; its nodes u = blockIdx.x + k * gridDim.x are processed by
// CW consumer warps, warp w taking k = w, w + CW, ...  Each warp owns two
// shared-memory stages (node k uses stage k % 2CW), so the rows of its next
// node are in flight while it computes the current one.  A stage holds one
// node's candidate record (ids, round-start k-th keys, norms) and its rows.
//   * warp 0 (producer) polls the stages: as soon as a stage is free it
//     issues the bulk copy of the next record into it; as soon as a record has
//     landed it issues one bulk copy per candidate row (TMA engine, completion
//     counted on the stage's mbarriers).  It never blocks on one stage while
//     another could make progress.
//   * each consumer warp works alone on its node (warp-level sync only):
//     FP32 compacts the allowed pairs (set masks of Alg. 1 / Alg. 2) and
//     computes four pairs per lane at a time, canonical in-order FP32 from the
//     staged rows; BF16 computes the Gram block new x all candidates on the
//     tensor cores (mma.sync m16n8k16, FP32 accumulate) one column tile at a
//     time and evaluates each tile's pairs straight from the accumulators.  A
//     BF16 pair is exact when both rows are small integers, otherwise it is
//     re-ranked in canonical FP32 whenever the proven bound cannot rule it out.
// Both precisions emit exactly the proposals of the single-stage kernels.
#include "knnm_internal.cuh"

namespace knnm {

namespace {

constexpr int GSTR = 68;  // floats per row of the staged Gram block

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
// Named barrier among the consumer warps that also ORs a predicate across them.
__device__ __forceinline__ bool consumer_sync_or(int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void fence_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool allowed(int mode, int64_t n1, int32_t p, int32_t q) {
  const bool p1 = p < n1, q1 = q < n1;
  return mode == SYMMETRIC ? (p1 != q1) : !(p1 && q1);
}

__device__ __forceinline__ void ldm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                       const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldm_x2(uint32_t& r0, uint32_t& r1, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float* c, uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Error bound of a tensor-core estimate (see knnm_join.cu for the derivation):
// ai/aj = {|b|^2, |b - x|, |b|, canonical |x|}.
template <int METRIC>
__device__ __forceinline__ float bound_tc(float g, float4 ai, float4 aj, int d, float* est) {
  const float u = 5.9604645e-8f;
  const float g_mma = (float)(d + 32) * 9.5367432e-7f;
  const float g_can = (float)(d + 4) * u * 1.01f;
  const float si = ai.z, sj = aj.z, ei = ai.y, ej = aj.y;
  if (METRIC == L2) {
    const float dt = (ai.x + aj.x) - 2.0f * g;
    *est = dt;
    const float A = g_mma * (si + sj) * (si + sj) + 4.0f * u * (ai.x + aj.x + 2.0f * fabsf(g));
    const float e = ei + ej;
    const float up = fmaxf(dt + A, 0.0f);
    const float B = 2.0f * e * sqrtf(up) + e * e;
    const float C = g_can * (up + B);
    return (A + B + C) * 1.001f + 1e-30f;
  } else {
    // symmetric in (i, j): |x_i.x_j - b_i.b_j| <= |b_i| e_j + |b_j| e_i + e_i e_j
    const float dot_err = g_mma * si * sj + si * ej + sj * ei + ei * ej +
                          g_can * (si + ei) * (sj + ej);
    if (METRIC == IP) {
      *est = -g;
      return dot_err * 1.001f + 1e-30f;
    }
    const float den = ai.w * aj.w;
    if (den == 0.0f) {
      *est = 1.0f;
      return 0.0f;
    }
    *est = 1.0f - g / den;
    return (dot_err / den) * 1.001f + 8.0f * u + 1e-30f;
  }
}

__device__ __forceinline__ bool exact_rows(float ri, float rj, int d) {
  if (ri < 0.f || rj < 0.f) return false;
  const long long mi = (long long)ri, mj = (long long)rj;
  return (long long)d * (mi * mi + mj * mj) < (1ll << 24);
}

template <int METRIC>
__device__ __forceinline__ float exact_value(float g, float4 ai, float4 aj) {
  if (METRIC == L2) return __fsub_rn(__fadd_rn(ai.x, aj.x), __fmul_rn(2.0f, g));
  return canon_finish<METRIC>(g, ai.w, aj.w);
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Proposals of one warp (up to two per lane) into the block's region.
__device__ __forceinline__ void emit_props(const JoinArgs& a, int* fill, bool hp, int32_t tp,
                                           uint64_t kp, bool hq, int32_t tq, uint64_t kq) {
  const int lane = threadIdx.x & 31;
  const unsigned bp = __ballot_sync(FULL, hp), bq = __ballot_sync(FULL, hq);
  const int n = __popc(bp) + __popc(bq);
  if (n == 0) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(fill, n);
  base = __shfl_sync(FULL, base, 0);
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t region = (uint64_t)blockIdx.x * a.region_cap;
  if (hp) {
    const uint64_t pos = (uint64_t)base + __popc(bp & lt);
    if (pos < a.region_cap) {
      a.prop_tgt[region + pos] = tp;
      a.prop_key[region + pos] = kp;
      atomicAdd(&a.prop_cnt[tp], 1);
    } else {
      slots_insert(a.live_keys + (size_t)tp * a.K, a.K, kp);
    }
  }
  if (hq) {
    const uint64_t pos = (uint64_t)base + __popc(bp) + __popc(bq & lt);
    if (pos < a.region_cap) {
      a.prop_tgt[region + pos] = tq;
      a.prop_key[region + pos] = kq;
      atomicAdd(&a.prop_cnt[tq], 1);
    } else {
      slots_insert(a.live_keys + (size_t)tq * a.K, a.K, kq);
    }
  }
}

struct Stage {
  const int32_t* hdr;
  const int32_t* cid;
  const uint64_t* kth;
  const float* cn;
  const unsigned char* rows;
};

// Allowed partners of candidate i among the M candidates, as a bit mask over
// j: j > i, j < M and the set test of Alg. 1 (S-Merge: the other set) or
// Alg. 2 (J-Merge: not both in S1).  s1 = bit mask of candidates in S1.
__device__ __forceinline__ uint64_t partner_mask(int mode, int i, int M, uint64_t s1) {
  const uint64_t live = M >= 64 ? ~0ull : ((1ull << M) - 1ull);
  const uint64_t above = i >= 63 ? 0ull : ~((2ull << i) - 1ull);
  const bool in1 = (s1 >> i) & 1ull;
  const uint64_t set = mode == SYMMETRIC ? (in1 ? ~s1 : s1) : (in1 ? ~s1 : ~0ull);
  return live & above & set;
}

__device__ __forceinline__ uint64_t s1_mask(const Stage& st, int M, int64_t n1) {
  const int lane = threadIdx.x & 31;
  const bool lo = lane < M && st.cid[lane] < n1;
  const bool hi = lane + 32 < M && st.cid[lane + 32] < n1;
  return (uint64_t)__ballot_sync(FULL, lo) | ((uint64_t)__ballot_sync(FULL, hi) << 32);
}

// Writes the warp's proposals: each lane holds up to NP (target, key) slots
// flagged in `has`; one shared atomic reserves the warp's span of the region.
template <int NP>
__device__ __forceinline__ void emit_many(const JoinArgs& a, int* fill, const bool (&has)[NP],
                                          const int32_t (&tgt)[NP], const uint64_t (&key)[NP]) {
  const int lane = threadIdx.x & 31;
  int c = 0;
#pragma unroll
  for (int x = 0; x < NP; ++x) c += has[x] ? 1 : 0;
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(FULL, incl, 31);
  if (total == 0) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(fill, total);
  base = __shfl_sync(FULL, base, 0) + incl - c;
  const uint64_t region = (uint64_t)blockIdx.x * a.region_cap;
#pragma unroll
  for (int x = 0; x < NP; ++x) {
    if (has[x]) {
      const uint64_t pos = (uint64_t)base;
      if (pos < a.region_cap) {
        a.prop_tgt[region + pos] = tgt[x];
        a.prop_key[region + pos] = key[x];
        atomicAdd(&a.prop_cnt[tgt[x]], 1);
      } else {
        slots_insert(a.live_keys + (size_t)tgt[x] * a.K, a.K, key[x]);
      }
      ++base;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 consumer: one warp, one node.
// ---------------------------------------------------------------------------
template <int METRIC>
__device__ __forceinline__ void consume_fp32(const JoinArgs& a, const PipeArgs& P, const Stage& st,
                                             int nn, int M, uint16_t* pairs, int* fill,
                                             unsigned long long& evals) {
  const int lane = threadIdx.x & 31;
  // pair list: lane i (< nn) writes the partners of candidate i
  const uint64_t s1 = s1_mask(st, M, a.n1);
  uint64_t pm = lane < nn ? partner_mask(a.mode, lane, M, s1) : 0ull;
  const int cnt = __popcll(pm);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int np = __shfl_sync(FULL, incl, 31);
  int pos = incl - cnt;
  while (pm) {
    const int j = __ffsll((long long)pm) - 1;
    pm &= pm - 1ull;
    pairs[pos++] = (uint16_t)((lane << 8) | j);
  }
  __syncwarp();
  if (lane == 0) evals += (unsigned long long)np;
  const int d = a.rows.d;
  const int sf = P.row_stride / 4;
  const float* rows = (const float*)st.rows;
  for (int q0 = 0; q0 < np;) {
    // two pairs per lane while at least 33 remain, else one
    const int pl = (np - q0 > 32) ? 2 : 1;
    const float* ra[2];
    const float* rb[2];
    float acc[2] = {0.0f, 0.0f};
    int pi[2], pj[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int q = q0 + t * 32 + lane;
      const uint16_t pr = (t < pl && q < np) ? pairs[q] : pairs[q0];
      pi[t] = pr >> 8;
      pj[t] = pr & 0xFF;
      ra[t] = rows + (size_t)pi[t] * sf;
      rb[t] = rows + (size_t)pj[t] * sf;
    }
    if (pl == 2) {
      for (int x = 0; x < d; x += 4) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const float4 u = *reinterpret_cast<const float4*>(ra[t] + x);
          const float4 v = *reinterpret_cast<const float4*>(rb[t] + x);
          acc[t] = Canon<METRIC>::step(acc[t], u.x, v.x);
          acc[t] = Canon<METRIC>::step(acc[t], u.y, v.y);
          acc[t] = Canon<METRIC>::step(acc[t], u.z, v.z);
          acc[t] = Canon<METRIC>::step(acc[t], u.w, v.w);
        }
      }
    } else {
      for (int x = 0; x < d; x += 4) {
        const float4 u = *reinterpret_cast<const float4*>(ra[0] + x);
        const float4 v = *reinterpret_cast<const float4*>(rb[0] + x);
        acc[0] = Canon<METRIC>::step(acc[0], u.x, v.x);
        acc[0] = Canon<METRIC>::step(acc[0], u.y, v.y);
        acc[0] = Canon<METRIC>::step(acc[0], u.z, v.z);
        acc[0] = Canon<METRIC>::step(acc[0], u.w, v.w);
      }
    }
    bool has[4];
    int32_t tgt[4];
    uint64_t key[4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int q = q0 + t * 32 + lane;
      const bool live = t < pl && q < np;
      const int i = pi[t], j = pj[t];
      const float dist = canon_finish<METRIC>(acc[t], METRIC == COS ? st.cn[i] : 0.f,
                                              METRIC == COS ? st.cn[j] : 0.f);
      const int32_t ci = st.cid[i], cj = st.cid[j];
      key[2 * t] = make_key(dist, cj);
      key[2 * t + 1] = make_key(dist, ci);
      tgt[2 * t] = ci;
      tgt[2 * t + 1] = cj;
      has[2 * t] = live && key[2 * t] < st.kth[i];
      has[2 * t + 1] = live && key[2 * t + 1] < st.kth[j];
    }
    emit_many<4>(a, fill, has, tgt, key);
    q0 += 32 * pl;
  }
}

// ---------------------------------------------------------------------------
// BF16 consumer: one warp, one node.  Column tile nt (8 candidates) at a time
// over both 16-row tiles of new candidates; the C fragment gives each lane
// rows i_r = lane/4 + 8r (r = 0..3) and columns 2*(lane%4) + {0,1}.  Row-side
// data of the lane's four rows are read once per node.
// ---------------------------------------------------------------------------
template <int METRIC>
__device__ __forceinline__ void consume_tc(const JoinArgs& a, const PipeArgs& P, const Stage& st,
                                           int nn, int M, uint16_t* rr, int* fill,
                                           unsigned long long& evals,
                                           unsigned long long& reranked) {
  const int lane = threadIdx.x & 31;
  const int d = a.rows.d;
  const int dpad = (d + 15) & ~15;
  const int stride = P.row_stride;
  const unsigned char* rows = st.rows;
  const uint64_t s1 = s1_mask(st, M, a.n1);
  uint64_t pmask[4];
  int32_t ci[4];
  uint64_t ki[4];
  float4 ai[4];
  float ri[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = (lane >> 2) + 8 * r;
    pmask[r] = i < nn ? partner_mask(a.mode, i, M, s1) : 0ull;
    const int ii = i < M ? i : 0;
    ci[r] = st.cid[ii];
    ki[r] = st.kth[ii];
    ai[r] = *(const float4*)(rows + (size_t)ii * stride + dpad * 2);
    ri[r] = *(const float*)(rows + (size_t)ii * stride + dpad * 2 + 16);
  }
  const bool two = nn > 16;
  const int ntiles = (M + 7) >> 3;
  int nr = 0;
  unsigned long long ev = 0;
  const unsigned char* pa0 = rows + (size_t)(lane & 15) * stride + (lane >> 4) * 16;
  const unsigned char* pa1 = pa0 + (size_t)16 * stride;
  for (int nt = 0; nt < ntiles; ++nt) {
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    const unsigned char* pb =
        rows + (size_t)(nt * 8 + (lane & 7)) * stride + ((lane >> 3) & 1) * 16;
#pragma unroll 8
    for (int k0 = 0; k0 < dpad; k0 += 16) {
      uint32_t x0, x1, x2, x3, y0, y1;
      ldm_x2(y0, y1, pb + k0 * 2);
      ldm_x4(x0, x1, x2, x3, pa0 + k0 * 2);
      mma16816(c0, x0, x1, x2, x3, y0, y1);
      if (two) {
        ldm_x4(x0, x1, x2, x3, pa1 + k0 * 2);
        mma16816(c1, x0, x1, x2, x3, y0, y1);
      }
    }
    bool mark[8];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = nt * 8 + 2 * (lane & 3) + e;
      bool any = false;
#pragma unroll
      for (int r = 0; r < 4; ++r) any |= ((pmask[r] >> j) & 1ull) != 0ull;
      int32_t cj = 0;
      uint64_t kj = 0;
      float4 aj = make_float4(0.f, 0.f, 0.f, 0.f);
      float rj = -1.f;
      if (any) {
        cj = st.cid[j];
        kj = st.kth[j];
        aj = *(const float4*)(rows + (size_t)j * stride + dpad * 2);
        rj = *(const float*)(rows + (size_t)j * stride + dpad * 2 + 16);
      }
      bool has[8];
      int32_t tgt[8];
      uint64_t key[8];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int x = e * 4 + r;
        const float g = (r < 2) ? c0[(r & 1) * 2 + e] : c1[(r & 1) * 2 + e];
        const bool ok = ((pmask[r] >> j) & 1ull) != 0ull;
        has[2 * r] = has[2 * r + 1] = false;
        mark[x] = false;
        tgt[2 * r] = ci[r];
        tgt[2 * r + 1] = cj;
        key[2 * r] = key[2 * r + 1] = 0ull;
        if (ok) {
          ++ev;
          if (exact_rows(ri[r], rj, d)) {
            const float dist = exact_value<METRIC>(g, ai[r], aj);
            key[2 * r] = make_key(dist, cj);
            key[2 * r + 1] = make_key(dist, ci[r]);
            has[2 * r] = key[2 * r] < ki[r];
            has[2 * r + 1] = key[2 * r + 1] < kj;
          } else {
            float est;
            const float E = bound_tc<METRIC>(g, ai[r], aj, d, &est);
            mark[x] = est - E <= fmaxf(key_dist(ki[r]), key_dist(kj));
          }
        }
      }
      emit_many<8>(a, fill, has, tgt, key);
    }
    // pairs the bound cannot settle go to the warp's re-rank list
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const unsigned b = __ballot_sync(FULL, mark[x]);
      if (b) {
        const int i = (lane >> 2) + 8 * (x & 3);
        const int j = nt * 8 + 2 * (lane & 3) + (x >> 2);
        if (mark[x]) rr[nr + __popc(b & ((1u << lane) - 1u))] = (uint16_t)((i << 8) | j);
        nr += __popc(b);
      }
    }
  }
  __syncwarp();
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(FULL, ev, o);
  evals += (lane == 0) ? ev : 0ull;
  reranked += (lane == 0) ? (unsigned long long)nr : 0ull;
  for (int q0 = 0; q0 < nr; q0 += 32) {
    const int q = q0 + lane;
    bool hp = false, hq = false;
    int32_t tp = 0, tq = 0;
    uint64_t kp = 0, kq = 0;
    if (q < nr) {
      const uint16_t pr = rr[q];
      const int i = pr >> 8, j = pr & 0xFF;
      tp = st.cid[i];
      tq = st.cid[j];
      const float4 a_i = *(const float4*)(rows + (size_t)i * stride + dpad * 2);
      const float4 a_j = *(const float4*)(rows + (size_t)j * stride + dpad * 2);
      const float dist =
          canon_dist_global<METRIC>(a.rows.row(tp), a.rows.row(tq), d, a_i.w, a_j.w);
      kp = make_key(dist, tq);
      kq = make_key(dist, tp);
      hp = kp < st.kth[i];
      hq = kq < st.kth[j];
    }
    emit_props(a, fill, hp, tp, kp, hq, tq, kq);
  }
}

template <int METRIC, bool TC>
__global__ void __launch_bounds__(32 * 9, 1) k_join_pipe(JoinArgs a, PipeArgs P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int CW = P.cw;
  const int NS = 2 * CW;
  const int RB = rec_bytes(P.cap);
  uint64_t* full = (uint64_t*)(smem + (size_t)NS * P.stage_bytes);
  uint64_t* empty = full + NS;
  uint64_t* recb = empty + NS;
  int* scal = (int*)(recb + NS);  // [0] region fill, [1] bail
  unsigned char* lists = (unsigned char*)(scal + 16);
  const size_t list_bytes = ((size_t)P.pair_cap * 2 + 15) & ~(size_t)15;
  unsigned long long* red = (unsigned long long*)(lists + (size_t)CW * list_bytes);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
      mbar_init(recb + s, 1);
    }
    scal[0] = scal[1] = 0;
    fence_mbar_init();
  }
  if (threadIdx.x < 3 * 9) red[threadIdx.x] = 0ull;
  __syncthreads();

  const int64_t nk = a.N > (int64_t)blockIdx.x ? (a.N - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto node_of = [&](int64_t k) { return (int64_t)blockIdx.x + k * (int64_t)gridDim.x; };

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    int64_t kr = 0, kw = 0;
    uint32_t idle = 0;
    while (kw < nk) {
      bool progressed = false;
      // next record, once its stage is free
      if (kr < nk && kr < kw + NS) {
        const int s = (int)(kr % NS);
        bool free_ = true;
        if (kr >= NS) {
          bool t = false;
          if (lane == 0) t = mbar_test(empty + s, (uint32_t)(((kr / NS) - 1) & 1));
          free_ = __shfl_sync(FULL, t, 0);
        }
        if (free_) {
          if (lane == 0) {
            fence_async();
            mbar_arrive_expect_tx(recb + s, (uint32_t)RB);
            bulk_g2s(smem + (size_t)s * P.stage_bytes, P.rec + (size_t)node_of(kr) * RB,
                     (uint32_t)RB, recb + s);
          }
          ++kr;
          progressed = true;
        }
      }
      // rows of the oldest node whose record has landed
      if (kw < kr) {
        const int s = (int)(kw % NS);
        bool t = false;
        if (lane == 0) t = mbar_test(recb + s, (uint32_t)((kw / NS) & 1));
        if (__shfl_sync(FULL, t, 0)) {
          const unsigned char* R = smem + (size_t)s * P.stage_bytes;
          const int32_t* h = (const int32_t*)R;
          const int nn = min(max(h[0], 0), a.cap_new), no = min(max(h[1], 0), a.cap_old);
          const int M = nn + no;
          const bool need = nn > 0 && M > 1;
          if (lane == 0) {
            if (need)
              mbar_arrive_expect_tx(full + s, (uint32_t)(M * P.row_bytes));
            else
              mbar_arrive(full + s);
          }
          __syncwarp();
          if (need) {
            const int32_t* cid = (const int32_t*)(R + 16);
            unsigned char* dst = smem + (size_t)s * P.stage_bytes + RB;
            for (int r = lane; r < M; r += 32) {
              int32_t id = cid[r];
              if (id < 0 || id >= a.N) id = 0;
              const void* src = TC ? (const void*)(P.Xe + (size_t)id * P.dx)
                                   : (const void*)a.rows.row(id);
              bulk_g2s(dst + (size_t)r * P.row_stride, src, (uint32_t)P.row_bytes, full + s);
            }
          }
          ++kw;
          progressed = true;
        }
      }
      if (progressed) {
        idle = 0;
      } else if (++idle > (WAIT_LIMIT << 1)) {
        if (lane == 0) {
          atomicOr(&a.ctr->err, (unsigned long long)DERR_WAIT_TIMEOUT);
          atomicExch(&scal[1], 1);
        }
        break;
      } else {
        __nanosleep(32);
      }
    }
    return;
  }

  // ------------------------------------------------------------------ consumers
  const int cw = warp - 1;
  uint16_t* mylist = (uint16_t*)(lists + (size_t)cw * list_bytes);
  unsigned long long evals = 0, gathered = 0, reranked = 0;
  int64_t k = cw;
  bool bailed = false;
  for (; k < nk; k += CW) {
    const int s = (int)(k % NS);
    const uint32_t par = (uint32_t)((k / NS) & 1);
    bool ok = mbar_wait_bounded(recb + s, par, WAIT_LIMIT) &&
              mbar_wait_bounded(full + s, par, WAIT_LIMIT);
    ok = __all_sync(FULL, ok);
    if (!ok) {
      if (lane == 0) atomicOr(&a.ctr->err, (unsigned long long)DERR_WAIT_TIMEOUT);
      bailed = true;
      break;
    }
    const unsigned char* R = smem + (size_t)s * P.stage_bytes;
    Stage st;
    st.hdr = (const int32_t*)R;
    st.cid = (const int32_t*)(R + 16);
    st.kth = (const uint64_t*)(R + 16 + 4 * P.cap);
    st.cn = (const float*)(R + 16 + 12 * P.cap);
    st.rows = R + RB;
    const int nn = min(max(st.hdr[0], 0), a.cap_new);
    const int no = min(max(st.hdr[1], 0), a.cap_old);
    const int M = nn + no;
    if (nn > 0 && M > 1) {
      if (lane == 0) gathered += (unsigned long long)M;
      if (TC)
        consume_tc<METRIC>(a, P, st, nn, M, mylist, &scal[0], evals, reranked);
      else
        consume_fp32<METRIC>(a, P, st, nn, M, mylist, &scal[0], evals);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
  }
  if (bailed && lane == 0) {
    // wait (bounded) for the copies still owed to this warp's two stages
    for (int x = 0; x < 2; ++x) {
      const int64_t kk = k + (int64_t)x * CW;
      if (kk < nk) mbar_wait_bounded(full + (kk % NS), (uint32_t)((kk / NS) & 1), WAIT_LIMIT);
    }
  }
  // block totals
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(FULL, evals, o);
    gathered += __shfl_xor_sync(FULL, gathered, o);
    reranked += __shfl_xor_sync(FULL, reranked, o);
  }
  if (lane == 0) {
    atomicAdd(&red[0], evals);
    atomicAdd(&red[1], gathered);
    atomicAdd(&red[2], reranked);
  }
  asm volatile("bar.sync 1, %0;" ::"r"(CW * 32) : "memory");
  if (threadIdx.x == 32) {
    const int fill = scal[0];
    a.region_cnt[blockIdx.x] = (unsigned long long)min((uint64_t)fill, a.region_cap);
    atomicAdd(&a.ctr->proposals, (unsigned long long)fill);
    if ((uint64_t)fill > a.region_cap)
      atomicAdd(&a.ctr->overflow, (unsigned long long)((uint64_t)fill - a.region_cap));
    atomicAdd(&a.ctr->dist_evals, red[0]);
    atomicAdd(&a.ctr->gathered, red[1]);
    atomicAdd(&a.ctr->reranked, red[2]);
  }
}

// BF16 rows with their error data in a 32-byte tail:
//   bf16 x[0..d), zeros up to dpad = round_up(d, 16), then floats
//   {|b|^2, |b - x| (upper), |b| (upper), canonical |x|, rmax, 0, 0, 0}.
__global__ void k_bf16_ext(Rows R, int64_t N, int dx, __nv_bfloat16* Xe) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int d = R.d, dpad = (d + 15) & ~15;
  const float* x = R.row(i);
  __nv_bfloat16* o = Xe + (size_t)i * dx;
  float nb2 = 0.f, e2 = 0.f, nx2 = 0.f, mx = 0.f;
  bool exact = true;
  for (int t = 0; t < d; ++t) {
    const float v = __ldg(x + t);
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    const float bf = __bfloat162float(b);
    o[t] = b;
    nb2 = __fmaf_rn(bf, bf, nb2);
    const float e = __fsub_rn(bf, v);
    e2 = __fmaf_rn(e, e, e2);
    nx2 = __fmaf_rn(v, v, nx2);
    exact = exact && v == rintf(v) && v >= 0.0f && v <= 256.0f;
    mx = fmaxf(mx, fabsf(v));
  }
  for (int t = d; t < dpad; ++t) o[t] = __float2bfloat16_rn(0.0f);
  const float grow = 1.0f + (float)(d + 2) * 1.2e-7f;
  float* tail = (float*)(o + dpad);
  tail[0] = nb2;
  tail[1] = __fsqrt_ru(e2 * grow) * 1.000001f;
  tail[2] = __fsqrt_ru(nb2 * grow) * 1.000001f;
  tail[3] = __fsqrt_rn(nx2);
  tail[4] = exact ? mx : -1.0f;
  tail[5] = tail[6] = tail[7] = 0.0f;
}

template <int METRIC, bool TC>
cudaError_t setup_pipe(size_t smem, int threads) {
  return cudaFuncSetAttribute(k_join_pipe<METRIC, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

}  // namespace

cudaError_t plan_pipe(int precision, int metric, int cap_new, int cap_old, int d, PipeArgs* P,
                      size_t* smem, int* grid) {
  const bool tc = precision == 1 && metric != L1;
  const int cap = round_up4(cap_new + cap_old);
  if (cap_new + cap_old > 255 || cap > 64) return cudaErrorInvalidValue;
  if (tc && (cap_new > 32 || d % 8 != 0)) return cudaErrorInvalidValue;
  if (!tc && d % 4 != 0) return cudaErrorInvalidValue;
  P->cap = cap;
  const int RB = rec_bytes(cap);
  int rows_alloc;
  if (tc) {
    const int dpad = (d + 15) & ~15;
    P->dx = dpad + 16;
    P->row_bytes = P->dx * 2;
    P->row_stride = P->row_bytes + 16;
    rows_alloc = ((cap + 7) & ~7) < 32 ? 32 : ((cap + 7) & ~7);
  } else {
    P->dx = 0;
    P->row_bytes = d * 4;
    P->row_stride = d * 4 + 16;
    rows_alloc = cap;
  }
  P->stage_bytes = (RB + rows_alloc * P->row_stride + 127) & ~127;
  P->pair_cap = cap_new * (cap_new + cap_old);
  const size_t list_bytes = ((size_t)P->pair_cap * 2 + 15) & ~(size_t)15;
  // one block per SM: 2 stages + one list per consumer warp, up to 8 warps
  const size_t budget = 200 * 1024;
  int cw = 8;
  auto need = [&](int c) {
    return (size_t)2 * c * P->stage_bytes + (size_t)3 * 8 * 2 * c + 64 + (size_t)c * list_bytes +
           3 * 9 * 8;
  };
  while (cw > 1 && need(cw) > budget) --cw;
  if (need(cw) > budget) return cudaErrorInvalidValue;
  P->cw = cw;
  P->nstages = 2 * cw;
  *smem = need(cw);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *grid = sms;
  switch (metric) {
    case L2: return tc ? setup_pipe<L2, true>(*smem, 0) : setup_pipe<L2, false>(*smem, 0);
    case IP: return tc ? setup_pipe<IP, true>(*smem, 0) : setup_pipe<IP, false>(*smem, 0);
    case COS: return tc ? setup_pipe<COS, true>(*smem, 0) : setup_pipe<COS, false>(*smem, 0);
    default: return setup_pipe<L1, false>(*smem, 0);
  }
}

cudaError_t launch_pipe(int precision, const JoinArgs& a, const PipeArgs& P, size_t smem,
                        int grid, cudaStream_t st) {
  const bool tc = precision == 1 && a.metric != L1;
  const int threads = 32 * (P.cw + 1);
  if (tc) {
    switch (a.metric) {
      case L2: k_join_pipe<L2, true><<<grid, threads, smem, st>>>(a, P); break;
      case IP: k_join_pipe<IP, true><<<grid, threads, smem, st>>>(a, P); break;
      default: k_join_pipe<COS, true><<<grid, threads, smem, st>>>(a, P); break;
    }
  } else {
    switch (a.metric) {
      case L2: k_join_pipe<L2, false><<<grid, threads, smem, st>>>(a, P); break;
      case IP: k_join_pipe<IP, false><<<grid, threads, smem, st>>>(a, P); break;
      case COS: k_join_pipe<COS, false><<<grid, threads, smem, st>>>(a, P); break;
      default: k_join_pipe<L1, false><<<grid, threads, smem, st>>>(a, P); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_bf16_ext(Rows rows, int64_t N, int dx, __nv_bfloat16* Xe, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_bf16_ext<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rows, N, dx, Xe);
  return cudaGetLastError();
}

}  // namespace knnm
