// knnm_join_pipe.cu -- the local join (Alg. 1 / Alg. 2 inner loops) with each
// warp streaming its own nodes through a shared-memory row ring.
//
// Warp g of the grid takes nodes u = g, g + G, ... (G warps in all).  Its
// shared memory holds a ring of candidate rows, three candidate-record slots
// (ids, round-start k-th keys, norms; written by the sampler) and a pair list.
// While it computes node j it already has the rows of node j+1 and the record
// of node j+2 in flight: 1-D bulk copies on the TMA engine (cp.async.bulk, one
// per row, issued by one lane per row, completion counted in bytes on the
// slot's mbarrier), so staging a node's rows costs one or two warp
// instructions.  Node j+1's rows go right after node j's in the ring when both
// fit, else after node j is done.
//   * FP32: the allowed pairs (set masks of Alg. 1 / Alg. 2, from 64-bit
//     candidate masks) are listed, then each lane computes one or two pairs at
//     a time, canonical in-order FP32 from the ring.
//   * BF16: the Gram block new x all candidates is computed on the tensor cores
//     (mma.sync m16n8k16, FP32 accumulate) into a per-warp buffer, then each
//     listed pair is finished from it: exact when both rows are small
//     integers, otherwise re-ranked in canonical FP32 whenever the proven
//     bound cannot rule it out.
// Both precisions emit exactly the proposals of the single-stage kernels.
#include "knnm_internal.cuh"

namespace knnm {

namespace {



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
// D += A * B with 16-bit inputs (both BF16, or both FP16) and FP32 accumulation.
template <bool HALF>
__device__ __forceinline__ void mma16816(float* c, uint32_t a0, uint32_t a1, uint32_t a2,
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

// Both rows are small non-negative integers and d * (max_i^2 + max_j^2) < 2^24:
// every partial sum of the canonical accumulation is then an exact integer, and
// so is the tensor-core Gram value.  w = d * max^2 rounded up, or -1 (tail[4]).
__device__ __forceinline__ bool exact_rows(float wi, float wj) {
  return wi >= 0.0f && wj >= 0.0f && __fadd_ru(wi, wj) < 16777216.0f;
}

template <int METRIC>
__device__ __forceinline__ float exact_value(float g, float4 ai, float4 aj) {
  if (METRIC == L2) return __fsub_rn(__fadd_rn(ai.x, aj.x), __fmul_rn(2.0f, g));
  return canon_finish<METRIC>(g, ai.w, aj.w);
}

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

// Offers the warp's proposals (up to 4 per lane) to UpdateNN; their bucket
// slots are claimed now and written at the warp's next offer.
using Sink = DeferredSink<4>;
__device__ __forceinline__ void emit_many(const JoinArgs& a, Sink& sink, const bool (&has)[4],
                                          const int32_t (&tgt)[4], const uint64_t (&key)[4]) {
  sink.offer(a.bucket, a.bcnt, a.bcap, a.live_keys, a.K, has, tgt, key);
}



// Bounded wait of the whole warp: true only when every lane saw the phase
// complete, so that a timeout sends all lanes down the same path.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  return __all_sync(FULL, mbar_wait_bounded(bar, parity, limit));
}

struct Rec {
  const uint4* e;  // per candidate {id, width or norm, k-th key}: one 16-byte load
  int nn, M;
  __device__ __forceinline__ int32_t id(int r) const { return rec_id(e[r]); }
};

__device__ __forceinline__ Rec read_rec(const JoinArgs& a, const unsigned char* R) {
  Rec r;
  const int32_t* h = (const int32_t*)R;
  r.nn = min(max(h[0], 0), a.cap_new);
  r.M = r.nn + min(max(h[1], 0), a.cap_old);
  r.e = (const uint4*)(R + 16);
  return r;
}

// Lists the allowed pairs (i < nn, i < j < M, set test) into `pairs`, sorted by
// first index, then second.  *np0 receives the number of pairs whose first
// index is below 16.  Two ways to the same list: with many new candidates each
// lane walks half a row's partner mask (the cost follows the longest half-row),
// with few the warp expands one row at a time (the cost follows the rows).
constexpr int LIST_LANES_FROM = 8;
__device__ __forceinline__ int list_pairs(const JoinArgs& a, const Rec& rc, uint16_t* pairs,
                                          int* np0) {
  const int lane = threadIdx.x & 31;
  const bool lo = lane < rc.M && rc.id(lane) < a.n1;
  const bool hi = lane + 32 < rc.M && rc.id(lane + 32) < a.n1;
  const uint64_t s1 = (uint64_t)__ballot_sync(FULL, lo) | ((uint64_t)__ballot_sync(FULL, hi) << 32);
  const uint64_t pm = lane < rc.nn ? partner_mask(a.mode, lane, rc.M, s1) : 0ull;
  const int cnt = __popcll(pm);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int np = __shfl_sync(FULL, incl, 31);
  *np0 = __shfl_sync(FULL, incl, 15);
  const int excl = incl - cnt;
  if (rc.nn >= LIST_LANES_FROM) {
    // Sixteen rows a pass: lane r < 16 writes the pairs of row rb + r with
    // partners below 32, lane r + 16 those with partners from 32 on, each in
    // ascending order from the row's offset; the loop runs as long as the
    // largest half-row.
    for (int rb = 0; rb < rc.nn; rb += 16) {
      const int row = rb + (lane & 15);
      const uint32_t m0 = (uint32_t)__shfl_sync(FULL, (unsigned)pm, row);
      const uint32_t m1 = (uint32_t)__shfl_sync(FULL, (unsigned)(pm >> 32), row);
      const int b = __shfl_sync(FULL, excl, row);
      uint32_t m = row < rc.nn ? (lane < 16 ? m0 : m1) : 0u;
      int pos = lane < 16 ? b : b + __popc(m0);
      const int tag = (row << 8) | (lane < 16 ? 0 : 32);
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1u;
        pairs[pos++] = (uint16_t)(tag | j);
      }
    }
  } else {
    // few rows: the warp writes one row at a time, lane j its partner j and
    // j + 32 (ranks within the row from the mask)
    const unsigned lt = (1u << lane) - 1u;
    for (int i = 0; i < rc.nn; ++i) {
      const uint32_t m0 = (uint32_t)__shfl_sync(FULL, (unsigned)pm, i);
      const uint32_t m1 = (uint32_t)__shfl_sync(FULL, (unsigned)(pm >> 32), i);
      const int b = __shfl_sync(FULL, excl, i);
      if ((m0 >> lane) & 1u) pairs[b + __popc(m0 & lt)] = (uint16_t)((i << 8) | lane);
      if ((m1 >> lane) & 1u)
        pairs[b + __popc(m0) + __popc(m1 & lt)] = (uint16_t)((i << 8) | (lane + 32));
    }
  }
  __syncwarp();
  return np;
}

// ---------------------------------------------------------------------------
// One node's distances and proposals, rows read through row_ptr(r).
// ---------------------------------------------------------------------------
template <int METRIC, typename RowPtr>
__device__ __forceinline__ void node_fp32(const JoinArgs& a, const Rec& rc, int np,
                                          const uint16_t* pairs, RowPtr row_ptr, Sink& sink) {
  const int lane = threadIdx.x & 31;
  const int d = a.rows.d;
  for (int q0 = 0; q0 < np;) {
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
      ra[t] = (const float*)row_ptr(pi[t]);
      rb[t] = (const float*)row_ptr(pj[t]);
    }
    if (pl == 2) {
      for (int x = 0; x < d; x += 4) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const float4 p4 = *reinterpret_cast<const float4*>(ra[t] + x);
          const float4 q4 = *reinterpret_cast<const float4*>(rb[t] + x);
          acc[t] = Canon<METRIC>::step(acc[t], p4.x, q4.x);
          acc[t] = Canon<METRIC>::step(acc[t], p4.y, q4.y);
          acc[t] = Canon<METRIC>::step(acc[t], p4.z, q4.z);
          acc[t] = Canon<METRIC>::step(acc[t], p4.w, q4.w);
        }
      }
    } else {
      for (int x = 0; x < d; x += 4) {
        const float4 p4 = *reinterpret_cast<const float4*>(ra[0] + x);
        const float4 q4 = *reinterpret_cast<const float4*>(rb[0] + x);
        acc[0] = Canon<METRIC>::step(acc[0], p4.x, q4.x);
        acc[0] = Canon<METRIC>::step(acc[0], p4.y, q4.y);
        acc[0] = Canon<METRIC>::step(acc[0], p4.z, q4.z);
        acc[0] = Canon<METRIC>::step(acc[0], p4.w, q4.w);
      }
    }
    bool has[4];
    int32_t tgt[4];
    uint64_t key[4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int q = q0 + t * 32 + lane;
      const bool live = t < pl && q < np;
      const int i = pi[t], jj = pj[t];
      const uint4 ei = rc.e[i], ej = rc.e[jj];
      const float dist = canon_finish<METRIC>(acc[t], METRIC == COS ? rec_c(ei) : 0.f,
                                              METRIC == COS ? rec_c(ej) : 0.f);
      const int32_t ci = rec_id(ei), cj = rec_id(ej);
      key[2 * t] = make_key(dist, cj);
      key[2 * t + 1] = make_key(dist, ci);
      tgt[2 * t] = ci;
      tgt[2 * t + 1] = cj;
      has[2 * t] = live && key[2 * t] < rec_kth(ei);
      has[2 * t + 1] = live && key[2 * t + 1] < rec_kth(ej);
    }
    emit_many(a, sink, has, tgt, key);
    q0 += 32 * pl;
  }
}

// BF16: the Gram block is computed one 16-row tile of new candidates at a time
// into a 16 x gstr buffer (gstr >= every candidate count; columns beyond it are
// not stored); pairs come sorted by their first index, so tile mt serves the
// pairs [split(mt), split(mt + 1)).  Each record's third column holds the
// rows' exactness widths (the fifth float of the extended row's tail, which
// the ring does not stage).
template <int METRIC, bool HALF, typename RowPtr>
__device__ __forceinline__ void node_tc(const JoinArgs& a, const Rec& rc, int np,
                                        uint16_t* pairs, int np0, RowPtr row_ptr, float* G,
                                        const int gstr, Sink& sink,
                                        unsigned long long& reranked) {
  const int lane = threadIdx.x & 31;
  const int d = a.rows.d;
  const int dpad = (d + 15) & ~15;
  const int mtiles = (rc.nn + 15) >> 4, ntiles = (rc.M + 7) >> 3;
  int nr = 0;  // re-rank pairs, compacted to the front of the pair list
  for (int mt = 0; mt < mtiles; ++mt) {
    const unsigned char* pa = row_ptr(mt * 16 + (lane & 15)) + (lane >> 4) * 16;
    // columns j > i only: the first 8-column tile that can hold one is 2 * mt;
    // four independent accumulator tiles per pass
    for (int nt = 2 * mt; nt < ntiles; nt += 4) {
      float c[4][4];
      const unsigned char* pb[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        c[t][0] = c[t][1] = c[t][2] = c[t][3] = 0.f;
        const int tile = nt + t < ntiles ? nt + t : ntiles - 1;
        // rows past the last candidate (padding of the last 8-column tile)
        // read the last candidate instead: every read stays inside the ring,
        // and those columns are never used
        pb[t] = row_ptr(min(tile * 8 + (lane & 7), rc.M - 1)) + ((lane >> 3) & 1) * 16;
      }
#pragma unroll 4
      for (int k0 = 0; k0 < dpad; k0 += 16) {
        uint32_t x0, x1, x2, x3;
        ldm_x4(x0, x1, x2, x3, pa + k0 * 2);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          uint32_t y0, y1;
          ldm_x2(y0, y1, pb[t] + k0 * 2);
          mma16816<HALF>(c[t], x0, x1, x2, x3, y0, y1);
        }
      }
      const int r0 = lane >> 2;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int col = (nt + t) * 8 + 2 * (lane & 3);
        if (nt + t < ntiles && col < gstr) {  // gstr % 4 == 0: col + 1 < gstr too
          G[r0 * gstr + col] = c[t][0];
          G[r0 * gstr + col + 1] = c[t][1];
          G[(r0 + 8) * gstr + col] = c[t][2];
          G[(r0 + 8) * gstr + col + 1] = c[t][3];
        }
      }
    }
    __syncwarp();
    const int q_lo = mt == 0 ? 0 : np0, q_hi = mt == 0 ? np0 : np;
    // two pairs per lane per pass: independent chains for the schedulers
    for (int q0 = q_lo; q0 < q_hi; q0 += 64) {
      bool has[4] = {false, false, false, false};
      int32_t tgt[4] = {0, 0, 0, 0};
      uint64_t key[4] = {0ull, 0ull, 0ull, 0ull};
      bool mark[2] = {false, false};
      uint16_t pr[2] = {0, 0};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = q0 + 32 * u + lane;
        if (q < q_hi) {
          pr[u] = pairs[q];
          const int i = pr[u] >> 8, jj = pr[u] & 0xFF;
          const float g = G[(i & 15) * gstr + jj];
          const float4 ai = *(const float4*)(row_ptr(i) + dpad * 2);
          const float4 aj = *(const float4*)(row_ptr(jj) + dpad * 2);
          const uint4 ei = rc.e[i], ej = rc.e[jj];
          tgt[2 * u] = rec_id(ei);
          tgt[2 * u + 1] = rec_id(ej);
          if (exact_rows(rec_c(ei), rec_c(ej))) {
            const float dist = exact_value<METRIC>(g, ai, aj);
            key[2 * u] = make_key(dist, tgt[2 * u + 1]);
            key[2 * u + 1] = make_key(dist, tgt[2 * u]);
            has[2 * u] = key[2 * u] < rec_kth(ei);
            has[2 * u + 1] = key[2 * u + 1] < rec_kth(ej);
          } else {
            float est;
            const float E = bound_tc<METRIC>(g, ai, aj, d, &est);
            mark[u] = est - E <= fmaxf(key_dist(rec_kth(ei)), key_dist(rec_kth(ej)));
          }
        }
      }
      emit_many(a, sink, has, tgt, key);
      // entries up to q0 + 63 are consumed, so the front of the list is free
      const unsigned lt = (1u << lane) - 1u;
      const unsigned b0 = __ballot_sync(FULL, mark[0]), b1 = __ballot_sync(FULL, mark[1]);
      __syncwarp();
      if (mark[0]) pairs[nr + __popc(b0 & lt)] = pr[0];
      if (mark[1]) pairs[nr + __popc(b0) + __popc(b1 & lt)] = pr[1];
      nr += __popc(b0) + __popc(b1);
      __syncwarp();
    }
    __syncwarp();
  }
  if (lane == 0) reranked += (unsigned long long)nr;
  for (int q0 = 0; q0 < nr; q0 += 32) {
    const int q = q0 + lane;
    bool has[4] = {false, false, false, false};
    int32_t tgt[4] = {0, 0, 0, 0};
    uint64_t key[4] = {0ull, 0ull, 0ull, 0ull};
    if (q < nr) {
      const uint16_t pr = pairs[q];
      const int i = pr >> 8, jj = pr & 0xFF;
      const uint4 ei = rc.e[i], ej = rc.e[jj];
      const int32_t tp = rec_id(ei), tq = rec_id(ej);
      const float4 ai = *(const float4*)(row_ptr(i) + dpad * 2);
      const float4 aj = *(const float4*)(row_ptr(jj) + dpad * 2);
      const float dist =
          a.use_bulk ? canon_dist_global4<METRIC>(a.rows.row(tp), a.rows.row(tq), d, ai.w, aj.w)
                     : canon_dist_global<METRIC>(a.rows.row(tp), a.rows.row(tq), d, ai.w, aj.w);
      tgt[0] = tp;
      tgt[1] = tq;
      key[0] = make_key(dist, tq);
      key[1] = make_key(dist, tp);
      has[0] = key[0] < rec_kth(ei);
      has[1] = key[1] < rec_kth(ej);
    }
    emit_many(a, sink, has, tgt, key);
  }
}

// ---------------------------------------------------------------------------
// The kernel.  Per warp: NREC record slots, each with two mbarriers (record
// landed, rows landed) armed by lane 0 with the bytes to expect and completed
// by the bulk copies; a FIFO ring of R rows.  Rows of up to AHEAD nodes beyond the current one are in flight
// whenever the ring has room.
// ---------------------------------------------------------------------------
constexpr int NREC = 3;
constexpr int AHEAD = 1;
constexpr int MAX_WARPS = 12;  // warps per block (one block per SM)
constexpr int MIN_WARPS = 4;

template <int METRIC, bool TC, bool HALF>
__global__ void __launch_bounds__(MAX_WARPS * 32, 1) k_join_ring(JoinArgs a, PipeArgs P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RB = rec_bytes(P.cap);
  const int R = P.ring_rows;
  const int stride = P.row_stride;
  unsigned char* my = smem + (size_t)warp * P.warp_bytes;
  unsigned char* ring = my;
  unsigned char* recs = ring + (size_t)R * stride;
  uint64_t* recbar = (uint64_t*)(recs + (size_t)NREC * RB);
  uint64_t* rowbar = recbar + NREC;
  uint16_t* pairs = (uint16_t*)(rowbar + NREC);
  float* G = (float*)((unsigned char*)pairs + (((size_t)P.pair_cap * 2 + 15) & ~(size_t)15));
  unsigned long long* red = (unsigned long long*)(smem + (size_t)W * P.warp_bytes);
  if (lane == 0) {
    for (int x = 0; x < NREC; ++x) {
      mbar_init(recbar + x, 1);
      mbar_init(rowbar + x, 1);
    }
    fence_mbar_init();
  }
  if (threadIdx.x < 8) red[threadIdx.x] = 0ull;
  __syncthreads();

  const int64_t GW = (int64_t)gridDim.x * W;
  const int64_t g0 = (int64_t)blockIdx.x * W + warp;
  const int64_t count = a.N > g0 ? (a.N - 1 - g0) / GW + 1 : 0;  // nodes of this warp
  unsigned long long evals = 0, gathered = 0, reranked = 0;
  Sink sink;
  bool failed = false;

  auto slot_of = [&](int64_t j) { return (int)(j % NREC); };
  auto par_of = [&](int64_t j) { return (uint32_t)((j / NREC) & 1); };
  auto rec_at = [&](int64_t j) { return recs + (size_t)slot_of(j) * RB; };
  // Phases armed but not yet waited for, per slot (bit x) with their parity:
  // after a timeout they are waited out before the warp leaves, so that no
  // copy or arrival is still in flight into the block's shared memory.
  unsigned rec_pend = 0, rec_parb = 0, row_pend = 0, row_parb = 0;
  auto arm = [&](unsigned& pend, unsigned& parb, int64_t j) {
    const int x = slot_of(j);
    pend |= 1u << x;
    parb = (parb & ~(1u << x)) | (par_of(j) << x);
  };
  auto fetch_rec = [&](int64_t j) {
    const unsigned char* src = P.rec + (size_t)(g0 + j * GW) * RB;
    unsigned char* dst = rec_at(j);
    if (lane == 0) {
      mbar_arrive_expect_tx(recbar + slot_of(j), (uint32_t)RB);
      bulk_g2s(dst, src, (uint32_t)RB, recbar + slot_of(j));
    }
    arm(rec_pend, rec_parb, j);
  };
  auto fetch_rows = [&](int64_t j, int base, int M, bool staged) {
    if (lane == 0) mbar_arrive_expect_tx(rowbar + slot_of(j), staged ? (uint32_t)(M * P.row_bytes) : 0u);
    __syncwarp();
    if (staged) {
      const uint4* ent = (const uint4*)(rec_at(j) + 16);
      for (int r = lane; r < M; r += 32) {
        int32_t id = rec_id(ent[r]);
        if (id < 0 || id >= a.N) id = 0;
        const unsigned char* src = TC ? (const unsigned char*)(P.Xe + (size_t)id * P.dx)
                                      : (const unsigned char*)a.rows.row(id);
        int slot = base + r;
        if (slot >= R) slot -= R;
        bulk_g2s(ring + (size_t)slot * stride, src, (uint32_t)P.row_bytes, rowbar + slot_of(j));
      }
    }
    arm(row_pend, row_parb, j);
  };

  // prologue: records of the first NREC - 1 nodes
  for (int64_t j = 0; j < count && j < NREC - 1; ++j) fetch_rec(j);
  int64_t next_rows = 0;     // next node whose rows are to be fetched
  int64_t ring_head = 0, ring_tail = 0;  // rows of finished / fetched nodes
  int base_of[NREC];         // ring base of each slot's node
  int used_of[NREC];         // rows each slot's node occupies in the ring
#pragma unroll
  for (int x = 0; x < NREC; ++x) base_of[x] = used_of[x] = 0;

  for (int64_t j = 0; j < count; ++j) {
    // fetch rows of nodes j .. j + AHEAD while their records are in and the ring has room
    while (next_rows < count && next_rows <= j + AHEAD) {
      const int sl = slot_of(next_rows);
      if (!warp_wait(recbar + sl, par_of(next_rows), a.wait_polls)) {
        failed = true;
        break;
      }
      rec_pend &= ~(1u << sl);
      __syncwarp();
      const Rec rn = read_rec(a, rec_at(next_rows));
      const bool st = rn.nn > 0 && rn.M > 1;
      const int need = st ? rn.M : 0;
      if (next_rows > j && ring_tail - ring_head + need > R) break;  // no room yet
      const int base = (int)(ring_tail % R);
      fetch_rows(next_rows, base, rn.M, st);
#pragma unroll
      for (int x = 0; x < NREC; ++x)
        if (x == sl) {
          base_of[x] = base;
          used_of[x] = need;
        }
      ring_tail += need;
      ++next_rows;
    }
    if (failed) break;
    const int sl = slot_of(j);
    if (!warp_wait(rowbar + sl, par_of(j), a.wait_polls)) {
      failed = true;
      break;
    }
    row_pend &= ~(1u << sl);
    __syncwarp();
    // the record slot of node j - 1 is free: fetch the record of node j + NREC - 1
    if (j + NREC - 1 < count) fetch_rec(j + NREC - 1);
    const Rec rc = read_rec(a, rec_at(j));
    int base = 0, used = 0;
#pragma unroll
    for (int x = 0; x < NREC; ++x)
      if (x == sl) {
        base = base_of[x];
        used = used_of[x];
      }
    if (rc.nn > 0 && rc.M > 1) {
      if (lane == 0) gathered += (unsigned long long)rc.M;
      auto row_ptr = [&](int r) {
        int slot = base + r;
        if (slot >= R) slot -= R;
        return (const unsigned char*)(ring + (size_t)slot * stride);
      };
      int np0 = 0;  // pairs with first index < 16 come first
      const int np = list_pairs(a, rc, pairs, &np0);
      if (lane == 0) evals += (unsigned long long)np;
      if (TC) {
        node_tc<METRIC, HALF>(a, rc, np, pairs, np0, row_ptr, G, P.gstr, sink, reranked);
      } else {
        node_fp32<METRIC>(a, rc, np, pairs, row_ptr, sink);
      }
    }
    __syncwarp();
    ring_head += used;
  }
  sink.finish(a.bucket, a.bcap, a.live_keys, a.K);
  unsigned long long nprop = sink.nprop, ndirect = sink.ndirect;
  if (failed) {
    if (lane == 0) atomicOr(&a.ctr->err, (unsigned long long)DERR_WAIT_TIMEOUT);
    // let the copies of every armed phase land before the warp leaves
    // (bounded as well)
#pragma unroll
    for (int x = 0; x < NREC; ++x) {
      if ((rec_pend >> x) & 1u) warp_wait(recbar + x, (rec_parb >> x) & 1u, WAIT_LIMIT);
      if ((row_pend >> x) & 1u) warp_wait(rowbar + x, (row_parb >> x) & 1u, WAIT_LIMIT);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(FULL, evals, o);
    gathered += __shfl_xor_sync(FULL, gathered, o);
    reranked += __shfl_xor_sync(FULL, reranked, o);
    nprop += __shfl_xor_sync(FULL, nprop, o);
    ndirect += __shfl_xor_sync(FULL, ndirect, o);
  }
  if (lane == 0) {
    atomicAdd(&red[0], evals);
    atomicAdd(&red[1], gathered);
    atomicAdd(&red[2], reranked);
    atomicAdd(&red[3], nprop);
    atomicAdd(&red[4], ndirect);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&a.ctr->dist_evals, red[0]);
    atomicAdd(&a.ctr->gathered, red[1]);
    atomicAdd(&a.ctr->reranked, red[2]);
    atomicAdd(&a.ctr->proposals, red[3]);
    atomicAdd(&a.ctr->overflow, red[4]);
  }
}

// BF16 rows with their error data in a 32-byte tail:
//   bf16 x[0..d), zeros up to dpad = round_up(d, 16), then floats
//   {|b|^2, |b - x| (upper), |b| (upper), canonical |x|, rmax, 0, 0, 0}.
// One warp per 32 rows.  Each 32-row x 32-dimension chunk is read coalesced
// into shared memory; then every lane walks its own row through the chunk in
// index order (the canonical norm needs the in-order sum) and writes its 16-bit
// elements eight at a time.
constexpr int EXT_WARPS = 8;

template <bool HALF>
__global__ void __launch_bounds__(EXT_WARPS * 32) k_bf16_ext(Rows R, int64_t N, int dx,
                                                            __nv_bfloat16* Xe, float* wx,
                                                            unsigned long long* inexact) {
  __shared__ float tile[EXT_WARPS][32][33];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * EXT_WARPS + w) * 32;
  if (row0 >= N) return;  // whole warp
  const int d = R.d, dpad = (d + 15) & ~15;
  const int64_t i = row0 + lane;
  const bool live = i < N;
  __nv_bfloat16* o = Xe + (size_t)(live ? i : row0) * dx;
  float nb2 = 0.f, e2 = 0.f, nx2 = 0.f, mx = 0.f;
  bool exact = true, overflow = false;
  for (int t0 = 0; t0 < d; t0 += 32) {
    for (int r = 0; r < 32; ++r) {
      const int64_t rr = row0 + r;
      tile[w][r][lane] = (rr < N && t0 + lane < d) ? __ldg(R.row(rr) + t0 + lane) : 0.0f;
    }
    __syncwarp();
    const int tn = min(32, d - t0);
    for (int q0 = 0; q0 < tn; q0 += 8) {
      uint32_t packed[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q0 + q < tn) {
          const float v = tile[w][lane][q0 + q];
          float bf;
          uint32_t bits;
          if (HALF) {
            // saturated: a row with a value beyond FP16 range gets an infinite
            // error bound below, so every pair with it is re-ranked
            const float vs = fminf(fmaxf(v, -65504.0f), 65504.0f);
            overflow = overflow || vs != v;
            const __half h = __float2half_rn(vs);
            bf = __half2float(h);
            bits = __half_as_ushort(h);
          } else {
            const __nv_bfloat16 b = __float2bfloat16_rn(v);
            bf = __bfloat162float(b);
            bits = __bfloat16_as_ushort(b);
          }
          packed[q >> 1] |= bits << ((q & 1) * 16);
          nb2 = __fmaf_rn(bf, bf, nb2);
          const float e = __fsub_rn(bf, v);  // exact: bf and v are within a factor of two
          e2 = __fmaf_rn(e, e, e2);
          nx2 = __fmaf_rn(v, v, nx2);
          exact = exact && v == rintf(v) && v >= 0.0f && v <= (HALF ? 2048.0f : 256.0f);
          mx = fmaxf(mx, fabsf(v));
        }
      }
      // elements past d stay +0 (the same bits in both formats); d % 8 == 0 on
      // the tensor-core paths, so q0 + 8 <= dpad
      if (live)
        *reinterpret_cast<uint4*>(o + t0 + q0) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
    __syncwarp();
  }
  if (!live) return;
  for (int t = (d + 7) & ~7; t < dpad; t += 8)
    *reinterpret_cast<uint4*>(o + t) = make_uint4(0u, 0u, 0u, 0u);
  const float grow = 1.0f + (float)(d + 2) * 1.2e-7f;
  float* tail = (float*)(o + dpad);
  tail[0] = nb2;
  tail[1] = overflow ? __int_as_float(0x7f800000) : __fsqrt_ru(e2 * grow) * 1.000001f;
  tail[2] = __fsqrt_ru(nb2 * grow) * 1.000001f;
  tail[3] = __fsqrt_rn(nx2);
  tail[4] = exact ? __double2float_ru((double)d * (double)mx * (double)mx) : -1.0f;
  if (wx) wx[i] = tail[4];
  if (!exact && inexact) atomicAdd(inexact, 1ull);
  tail[5] = tail[6] = tail[7] = 0.0f;
}

template <int METRIC, bool TC, bool HALF>
cudaError_t setup_ring(size_t smem, int threads, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_join_ring<METRIC, TC, HALF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_join_ring<METRIC, TC, HALF>, threads,
                                                       smem);
}

// Tensor-core estimates of given pairs exactly as node_tc computes them: the
// 16-bit extended rows are staged with the ring's row stride, the Gram value of
// pair r comes from the same mma16816 chain over k0 = 0, 16, ... (A row r of a
// 16-row tile against B row r), and is finished by exact_value / bound_tc.
// One warp per 16 pairs; the canonical FP32 distance is computed beside it.
template <int METRIC, bool HALF>
__global__ void __launch_bounds__(32) k_tc_estimate(const __nv_bfloat16* Xe, int dx, Rows rows,
                                                    const int32_t* pi, const int32_t* pj,
                                                    int64_t P, float* est, float* bound,
                                                    float* canon) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int lane = threadIdx.x;
  const int d = rows.d, dpad = (d + 15) & ~15;
  const int row_bytes = dx * 2, stride = row_bytes + 16, cpr = row_bytes >> 4;
  unsigned char* A = sm;
  unsigned char* B = sm + (size_t)16 * stride;
  float* G = (float*)(sm + (size_t)32 * stride);  // 16 x 17
  for (int64_t g = blockIdx.x; g * 16 < P; g += gridDim.x) {
    const int64_t base = g * 16;
    for (int c = lane; c < 32 * cpr; c += 32) {
      const int r = c / cpr, o = c - r * cpr;
      const int64_t q = base + (r & 15) < P ? base + (r & 15) : base;
      const int32_t id = r < 16 ? pi[q] : pj[q];
      const uint4 v = *reinterpret_cast<const uint4*>(
          reinterpret_cast<const unsigned char*>(Xe + (size_t)id * dx) + o * 16);
      *reinterpret_cast<uint4*>((r < 16 ? A + (size_t)r * stride : B + (size_t)(r - 16) * stride) +
                                o * 16) = v;
    }
    __syncwarp();
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    const unsigned char* pa = A + (size_t)(lane & 15) * stride + (lane >> 4) * 16;
    const unsigned char* pb0 = B + (size_t)(lane & 7) * stride + ((lane >> 3) & 1) * 16;
    const unsigned char* pb1 = B + (size_t)(8 + (lane & 7)) * stride + ((lane >> 3) & 1) * 16;
    for (int k0 = 0; k0 < dpad; k0 += 16) {
      uint32_t x0, x1, x2, x3, y0, y1;
      ldm_x4(x0, x1, x2, x3, pa + k0 * 2);
      ldm_x2(y0, y1, pb0 + k0 * 2);
      mma16816<HALF>(c0, x0, x1, x2, x3, y0, y1);
      ldm_x2(y0, y1, pb1 + k0 * 2);
      mma16816<HALF>(c1, x0, x1, x2, x3, y0, y1);
    }
    const int r0 = lane >> 2, col = 2 * (lane & 3);
    G[r0 * 17 + col] = c0[0];
    G[r0 * 17 + col + 1] = c0[1];
    G[(r0 + 8) * 17 + col] = c0[2];
    G[(r0 + 8) * 17 + col + 1] = c0[3];
    G[r0 * 17 + 8 + col] = c1[0];
    G[r0 * 17 + 8 + col + 1] = c1[1];
    G[(r0 + 8) * 17 + 8 + col] = c1[2];
    G[(r0 + 8) * 17 + 8 + col + 1] = c1[3];
    __syncwarp();
    if (lane < 16 && base + lane < P) {
      const float gv = G[lane * 17 + lane];
      const unsigned char* ti = A + (size_t)lane * stride + dpad * 2;
      const unsigned char* tj = B + (size_t)lane * stride + dpad * 2;
      const float4 ai = *(const float4*)ti, aj = *(const float4*)tj;
      const float ri = *(const float*)(ti + 16), rj = *(const float*)(tj + 16);
      float e, b = 0.0f;
      if (exact_rows(ri, rj))
        e = exact_value<METRIC>(gv, ai, aj);
      else
        b = bound_tc<METRIC>(gv, ai, aj, d, &e);
      est[base + lane] = e;
      bound[base + lane] = b;
      canon[base + lane] =
          canon_dist_global<METRIC>(rows.row(pi[base + lane]), rows.row(pj[base + lane]), d, ai.w, aj.w);
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t plan_pipe(int precision, int metric, int cap_new, int cap_old, int d, PipeArgs* P,
                      size_t* smem, int* grid) {
  const bool tc = precision != 0 && metric != L1 && metric != CHI2;
  const bool hf = precision == 2;
  const int cap = round_up4(cap_new + cap_old);
  if (cap_new + cap_old > 255 || cap > 64) return cudaErrorInvalidValue;
  if (tc && (cap_new > 32 || d % 8 != 0)) return cudaErrorInvalidValue;
  if (!tc && d % 4 != 0) return cudaErrorInvalidValue;
  P->cap = cap;
  const int RB = rec_bytes(cap);
  // Ring rows: the largest candidate set (the rows of the next node come in
  // when both fit).  Every byte per warp counts: the kernel is latency-bound
  // and the warps per SM are set by the shared memory each one holds.
  int ring = (cap_new + cap_old + 1) & ~1;
  P->gstr = (cap_new + cap_old + 3) & ~3;
  if (tc) {
    const int dpad = (d + 15) & ~15;
    P->dx = dpad + 16;
    // staged: the 16-bit elements and the tail's first four floats (the fifth,
    // the exactness width, travels in the record); a stride of 16 mod 32
    // bytes keeps the 8-row ldmatrix reads free of bank conflicts
    P->row_bytes = dpad * 2 + 16;
    P->row_stride = P->row_bytes;
    if (ring < 32) ring = 32;  // the 16-row A tiles reach row 31
  } else {
    P->dx = 0;
    P->row_bytes = d * 4;
    P->row_stride = d * 4 + 16;
  }
  P->ring_rows = ring;
  // pairs (i, j) with i < nn <= cap_new, i < j < M <= cap_new + cap_old
  P->pair_cap = cap_new * (cap_new + cap_old) - cap_new * (cap_new + 1) / 2;
  size_t wb = (size_t)ring * P->row_stride + (size_t)NREC * RB + 2 * NREC * 8 +
              (((size_t)P->pair_cap * 2 + 15) & ~(size_t)15);
  if (tc) wb += (size_t)16 * P->gstr * 4;
  wb = (wb + 127) & ~(size_t)127;
  P->warp_bytes = (int)wb;
  // warps per block: as many as fit the 227 KB a block may hold (at most
  // MAX_WARPS), one block per SM
  int w = MAX_WARPS;
  while (w > 1 && (size_t)w * wb + 64 > 227 * 1024) --w;
  // long rows leave too few warps per SM to hide the gathers: the caller takes
  // the single-stage kernel instead
  if (w < MIN_WARPS || (size_t)w * wb + 64 > 227 * 1024) return cudaErrorInvalidValue;
  P->cw = w;
  P->nstages = 0;
  P->stage_bytes = 0;
  *smem = (size_t)w * wb + 64;
  int per = 0;
  cudaError_t e;
  switch (metric) {
    case L2:
      e = !tc ? setup_ring<L2, false, false>(*smem, 32 * w, &per)
              : hf ? setup_ring<L2, true, true>(*smem, 32 * w, &per)
                   : setup_ring<L2, true, false>(*smem, 32 * w, &per);
      break;
    case IP:
      e = !tc ? setup_ring<IP, false, false>(*smem, 32 * w, &per)
              : hf ? setup_ring<IP, true, true>(*smem, 32 * w, &per)
                   : setup_ring<IP, true, false>(*smem, 32 * w, &per);
      break;
    case COS:
      e = !tc ? setup_ring<COS, false, false>(*smem, 32 * w, &per)
              : hf ? setup_ring<COS, true, true>(*smem, 32 * w, &per)
                   : setup_ring<COS, true, false>(*smem, 32 * w, &per);
      break;
    case L1: e = setup_ring<L1, false, false>(*smem, 32 * w, &per); break;
    default: e = setup_ring<CHI2, false, false>(*smem, 32 * w, &per); break;
  }
  if (e != cudaSuccess) return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *grid = sms * per;
  return cudaSuccess;
}

cudaError_t launch_pipe(int precision, const JoinArgs& a, const PipeArgs& P, size_t smem,
                        int grid, cudaStream_t st) {
  const bool tc = precision != 0 && a.metric != L1 && a.metric != CHI2;
  const int threads = 32 * P.cw;
  if (tc && precision == 2) {
    switch (a.metric) {
      case L2: k_join_ring<L2, true, true><<<grid, threads, smem, st>>>(a, P); break;
      case IP: k_join_ring<IP, true, true><<<grid, threads, smem, st>>>(a, P); break;
      default: k_join_ring<COS, true, true><<<grid, threads, smem, st>>>(a, P); break;
    }
  } else if (tc) {
    switch (a.metric) {
      case L2: k_join_ring<L2, true, false><<<grid, threads, smem, st>>>(a, P); break;
      case IP: k_join_ring<IP, true, false><<<grid, threads, smem, st>>>(a, P); break;
      default: k_join_ring<COS, true, false><<<grid, threads, smem, st>>>(a, P); break;
    }
  } else {
    switch (a.metric) {
      case L2: k_join_ring<L2, false, false><<<grid, threads, smem, st>>>(a, P); break;
      case IP: k_join_ring<IP, false, false><<<grid, threads, smem, st>>>(a, P); break;
      case COS: k_join_ring<COS, false, false><<<grid, threads, smem, st>>>(a, P); break;
      case L1: k_join_ring<L1, false, false><<<grid, threads, smem, st>>>(a, P); break;
      default: k_join_ring<CHI2, false, false><<<grid, threads, smem, st>>>(a, P); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_bf16_ext(Rows rows, int64_t N, int dx, __nv_bfloat16* Xe, float* wx, int half,
                            unsigned long long* inexact, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((N + EXT_WARPS * 32 - 1) / (EXT_WARPS * 32));
  if (half)
    k_bf16_ext<true><<<blocks, EXT_WARPS * 32, 0, st>>>(rows, N, dx, Xe, wx, inexact);
  else
    k_bf16_ext<false><<<blocks, EXT_WARPS * 32, 0, st>>>(rows, N, dx, Xe, wx, inexact);
  return cudaGetLastError();
}

cudaError_t launch_tc_estimate(int precision, int metric, const __nv_bfloat16* Xe, int dx,
                               Rows rows, const int32_t* pi, const int32_t* pj, int64_t P,
                               float* est, float* bound, float* canon, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  const size_t smem = (size_t)32 * (dx * 2 + 16) + 16 * 17 * 4;
  const int64_t groups = (P + 15) / 16;
  const unsigned grid = (unsigned)(groups < 65535 ? groups : 65535);
  cudaError_t e = cudaSuccess;
#define KNNM_EST(M, H)                                                                      \
  do {                                                                                      \
    e = cudaFuncSetAttribute(k_tc_estimate<M, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                    \
    if (e != cudaSuccess) return e;                                                         \
    k_tc_estimate<M, H><<<grid, 32, smem, st>>>(Xe, dx, rows, pi, pj, P, est, bound, canon); \
  } while (0)
  const bool h = precision == 2;
  switch (metric) {
    case L2: if (h) KNNM_EST(L2, true); else KNNM_EST(L2, false); break;
    case IP: if (h) KNNM_EST(IP, true); else KNNM_EST(IP, false); break;
    default: if (h) KNNM_EST(COS, true); else KNNM_EST(COS, false); break;
  }
#undef KNNM_EST
  return cudaGetLastError();
}

}  // namespace knnm
