// Graph diversification (Alg. 3) of a finished k-NN graph, and the top-down
// search on the H-Merge hierarchy (Sec. 3.4).
//
// Diversification runs in three passes: in-degree count + scan (reverse-list
// offsets); one warp per row for the forward list (canonical distances, sort,
// all intra-list pairs at once, then Alg. 3's sequential keep/drop decision
// replayed on the occlusion bitmasks, and the reverse entries scattered into
// their targets' buckets); one warp per row for the reverse list (batches of
// the 32 nearest unprocessed entries, tested against the entries kept so far,
// then against each other) and the union with the forward result.
//
// Search: one warp per query, the query staged in shared memory.  Greedy moves
// on the layers above the bottom; best-first at the bottom over a rank list of
// ef entries in shared memory, with a per-query visited table (open
// addressing).  When the table is crowded a row may be compared again; a row
// that was dropped from the full rank list can never re-enter it (its key is
// above the list's last entry, which only decreases), and repeats of listed
// rows are dropped, so the result is that of the exact visited set.
#include "knnm_internal.cuh"

namespace knnm {
namespace {

constexpr int GD_WARPS = 8;
constexpr int VISIT_PROBES = 32;

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

template <int METRIC>
__device__ __forceinline__ float dist_rows(const float* __restrict__ X, int d, int vec4,
                                           const float* __restrict__ norms, int32_t i,
                                           int32_t j) {
  const float* a = X + (size_t)i * d;
  const float* b = X + (size_t)j * d;
  const float na = METRIC == COS ? __ldg(norms + i) : 0.0f;
  const float nb = METRIC == COS ? __ldg(norms + j) : 0.0f;
  return vec4 ? canon_dist_global4<METRIC>(a, b, d, na, nb)
              : canon_dist_global<METRIC>(a, b, d, na, nb);
}

// Canonical distance of the staged query (shared memory, 16-byte aligned) and
// a row in global memory, query first.
template <int METRIC>
__device__ __forceinline__ float dist_query(const float* qs, const float* __restrict__ r, int d,
                                            int vec4, float nq, float nr) {
  float acc = 0.0f;
  if (vec4) {
    const float4* q4 = reinterpret_cast<const float4*>(qs);
    const float4* r4 = reinterpret_cast<const float4*>(r);
#pragma unroll 4
    for (int t = 0; t < (d >> 2); ++t) {
      const float4 x = q4[t], y = __ldg(r4 + t);
      acc = Canon<METRIC>::step(acc, x.x, y.x);
      acc = Canon<METRIC>::step(acc, x.y, y.y);
      acc = Canon<METRIC>::step(acc, x.z, y.z);
      acc = Canon<METRIC>::step(acc, x.w, y.w);
    }
  } else {
    for (int t = 0; t < d; ++t) acc = Canon<METRIC>::step(acc, qs[t], __ldg(r + t));
  }
  return canon_finish<METRIC>(acc, nq, nr);
}

// Pair p of the strict lower triangle, row-major: p = i (i - 1) / 2 + c, c < i.
__device__ __forceinline__ void tri_decode(int p, int& i, int& c) {
  int r = (int)((1.0f + sqrtf(8.0f * (float)p + 1.0f)) * 0.5f);
  while (r * (r - 1) / 2 > p) --r;
  while ((r + 1) * r / 2 <= p) ++r;
  i = r;
  c = p - r * (r - 1) / 2;
}

// Number of entries of the ascending array a[0..n) below x.
__device__ __forceinline__ int count_below(const uint64_t* a, int n, uint64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = __shfl_xor_sync(FULL, v, o);
    v = y < v ? y : v;
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ void record_error(GdCounters* c, unsigned bit, int64_t row) {
  atomicOr(&c->err, (unsigned long long)bit);
  atomicMin(&c->err_row, (unsigned long long)row);
}

__host__ __device__ __forceinline__ int gd_warp_bytes(int M) { return 8 * M + 8 * 32 + 4 * 32; }

// ---------------------------------------------------------------------------
// Diversification
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_gd_count(const GdArgs a) {
  const int64_t total = a.n * a.K;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = a.G[i];
    const int64_t u = i / a.K;
    if (v < 0 || v >= a.n || v == u) {
      record_error(a.ctr, DERR_BAD_ID, u);
      continue;
    }
    atomicAdd(&a.indeg[v], 1);
  }
}

// Forward list of row u: Alg. 3 decided on all intra-list pairs at once.
// Entry i (in (distance, id) order) is occluded by an earlier entry c when
// m(s_i, s_c) < m(s_i, u); Alg. 3 keeps entry i iff none of its occluders is
// kept, which the sequential pass over the bitmasks replays exactly.
template <int METRIC>
__global__ void __launch_bounds__(GD_WARPS * 32) k_gd_forward(const GdArgs a) {
  __shared__ uint32_t occl_s[GD_WARPS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* occl = occl_s[w];
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long evals = 0;
  for (int64_t u = (int64_t)blockIdx.x * GD_WARPS + w; u < a.n;
       u += (int64_t)gridDim.x * GD_WARPS) {
    uint64_t key = KEY_EMPTY;
    if (lane < a.K) {
      const int32_t v = a.G[u * a.K + lane];
      if (v >= 0 && v < a.n && v != u)
        key = make_key(dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, (int32_t)u, v), v);
    }
    key = warp_sort32(key);
    const int nv = __popc(__ballot_sync(FULL, key != KEY_EMPTY));
    const uint64_t prev = __shfl_up_sync(FULL, key, 1);
    if (lane > 0 && key != KEY_EMPTY && prev == key) record_error(a.ctr, DERR_DUP_ID, u);
    const int32_t id = key_id(key);
    const float dl = key_dist(key);
    if (key != KEY_EMPTY) {  // reverse entry (distance, u) into the bucket of id
      const int slot = atomicAdd(&a.rev_fill[id], 1);
      a.rev[a.rev_off[id] + (unsigned long long)slot] = make_key(dl, (int32_t)u);
    }
    occl[lane] = 0u;
    __syncwarp();
    const int P = nv * (nv - 1) / 2;
    for (int base = 0; base < P; base += 32) {
      const int p = base + lane;
      int i = 1, c = 0;
      if (p < P) tri_decode(p, i, c);
      const int32_t si = __shfl_sync(FULL, id, i), sc = __shfl_sync(FULL, id, c);
      const float di = __shfl_sync(FULL, dl, i);
      if (p < P && dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, si, sc) < di)
        atomicOr(&occl[i], 1u << c);
    }
    evals += (unsigned long long)P;
    __syncwarp();
    uint32_t kept = nv > 0 ? 1u : 0u;
    for (int i = 1; i < nv; ++i)
      if ((occl[i] & kept) == 0u) kept |= 1u << i;
    if ((kept >> lane) & 1u) a.fwd[u * a.K + __popc(kept & lt)] = key;
    if (lane == 0) a.fwd_cnt[u] = __popc(kept);
    __syncwarp();
  }
  if (lane == 0 && evals) atomicAdd(&a.ctr->dist_evals, evals);
}

// Reverse list of row u (Alg. 3 on it, independently of the forward list),
// then the union with the forward result, cut to M entries.  Once M reverse
// entries are kept no later one can reach the first M of the union.
template <int METRIC>
__global__ void __launch_bounds__(GD_WARPS * 32) k_gd_reverse(const GdArgs a) {
  extern __shared__ __align__(16) unsigned char gd_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int M = a.M;
  uint64_t* kept = reinterpret_cast<uint64_t*>(gd_sm + (size_t)w * gd_warp_bytes(M));
  uint64_t* fk = kept + M;
  uint32_t* occl = reinterpret_cast<uint32_t*>(fk + 32);
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long evals = 0, edges = 0, full = 0, max_in = 0;
  for (int64_t u = (int64_t)blockIdx.x * GD_WARPS + w; u < a.n;
       u += (int64_t)gridDim.x * GD_WARPS) {
    const unsigned long long r0 = a.rev_off[u];
    const int m = (int)(a.rev_off[u + 1] - r0);
    max_in = max(max_in, (unsigned long long)m);
    const uint64_t* R = a.rev + r0;
    int nk = 0;
    uint64_t last = 0;
    bool have_last = false;
    while (nk < M) {
      // the 32 nearest entries after the last one processed, ascending
      uint64_t best = KEY_EMPTY;
      for (int c0 = 0; c0 < m; c0 += 32) {
        uint64_t v = c0 + lane < m ? R[c0 + lane] : KEY_EMPTY;
        if (have_last && v <= last) v = KEY_EMPTY;
        v = warp_sort32(v);
        best = c0 == 0 ? v : warp_merge_lo32(best, v);
      }
      const int nb = __popc(__ballot_sync(FULL, best != KEY_EMPTY));
      if (nb == 0) break;
      const int32_t s = key_id(best);
      const float ds = key_dist(best);
      bool surv = lane < nb;
      for (int j = 0; surv && j < nk; ++j) {
        ++evals;
        if (dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, s, key_id(kept[j])) < ds) surv = false;
      }
      const unsigned sm = __ballot_sync(FULL, surv);
      occl[lane] = 0u;
      __syncwarp();
      const int P = nb * (nb - 1) / 2;
      for (int base = 0; base < P; base += 32) {
        const int p = base + lane;
        int i = 1, c = 0;
        if (p < P) tri_decode(p, i, c);
        const int32_t si = __shfl_sync(FULL, s, i), sc = __shfl_sync(FULL, s, c);
        const float di = __shfl_sync(FULL, ds, i);
        if (p < P && ((sm >> i) & 1u) && ((sm >> c) & 1u)) {
          ++evals;
          if (dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, si, sc) < di)
            atomicOr(&occl[i], 1u << c);
        }
      }
      __syncwarp();
      uint32_t kb = 0u;
      int room = M - nk;
      for (int i = 0; i < nb && room > 0; ++i)
        if (((sm >> i) & 1u) && (occl[i] & kb) == 0u) {
          kb |= 1u << i;
          --room;
        }
      if ((kb >> lane) & 1u) kept[nk + __popc(kb & lt)] = best;
      nk += __popc(kb);
      __syncwarp();
      if (nb < 32) break;
      last = __shfl_sync(FULL, best, 31);
      have_last = true;
    }
    // union with the forward result; a repeated id has one distance, so a
    // repeat is an equal key
    const int fc = a.fwd_cnt[u];
    fk[lane] = lane < fc ? a.fwd[u * a.K + lane] : KEY_EMPTY;
    __syncwarp();
    int nr = 0;
    for (int c0 = 0; c0 < nk; c0 += 32) {
      const uint64_t r = c0 + lane < nk ? kept[c0 + lane] : KEY_EMPTY;
      bool keep = r != KEY_EMPTY;
      for (int j = 0; keep && j < fc; ++j) keep = fk[j] != r;
      const unsigned b = __ballot_sync(FULL, keep);
      if (keep) kept[nr + __popc(b & lt)] = r;
      nr += __popc(b);
      __syncwarp();
    }
    int32_t* oi = a.out_ids + (size_t)u * M;
    float* od = a.out_dists + (size_t)u * M;
    if (lane < fc) {
      const uint64_t f = fk[lane];
      const int pos = lane + count_below(kept, nr, f);
      if (pos < M) {
        oi[pos] = key_id(f);
        od[pos] = key_dist(f);
      }
    }
    for (int j = lane; j < nr; j += 32) {
      const uint64_t r = kept[j];
      const int pos = j + count_below(fk, fc, r);
      if (pos < M) {
        oi[pos] = key_id(r);
        od[pos] = key_dist(r);
      }
    }
    const int deg = min(M, fc + nr);
    for (int j = deg + lane; j < M; j += 32) {
      oi[j] = -1;
      od[j] = f_inf();
    }
    if (lane == 0) {
      a.out_deg[u] = deg;
      edges += (unsigned long long)deg;
      full += deg == M ? 1ull : 0ull;
    }
    __syncwarp();
  }
  evals = warp_sum64(evals);
  if (lane == 0) {
    if (evals) atomicAdd(&a.ctr->dist_evals, evals);
    if (edges) atomicAdd(&a.ctr->edges, edges);
    if (full) atomicAdd(&a.ctr->full_rows, full);
    atomicMax(&a.ctr->max_in, max_in);
  }
}

// ---------------------------------------------------------------------------
// Search
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ int round16(int x) { return (x + 15) & ~15; }
__host__ __device__ __forceinline__ int search_qbytes(int d) { return round16(4 * d); }
__host__ __device__ __forceinline__ int search_warp_bytes(int d, int ef, int hbits) {
  return search_qbytes(d) + 16 * ef + 2 * round16(ef) + 8 * 32 + (4 << hbits);
}

// Marks id v as seen: 1 when newly recorded, 0 when recorded before, 2 when
// the table had no free slot within the probe limit (v counts as unseen).
__device__ __forceinline__ int visit(int32_t* H, int hbits, int32_t v) {
  const uint32_t mask = (1u << hbits) - 1u;
  uint32_t h = ((uint32_t)v * 0x9E3779B1u) >> (32 - hbits);
  for (int probe = 0; probe < VISIT_PROBES; ++probe) {
    const int32_t old = atomicCAS(&H[h], -1, v);
    if (old == -1) return 1;
    if (old == v) return 0;
    h = (h + 1u) & mask;
  }
  return 2;
}

template <int METRIC>
__global__ void __launch_bounds__(256) k_search(const SearchArgs a) {
  extern __shared__ __align__(16) unsigned char s_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned char* base = s_sm + (size_t)w * a.warp_bytes;
  float* qs = reinterpret_cast<float*>(base);
  uint64_t* LA = reinterpret_cast<uint64_t*>(base + search_qbytes(a.d));
  uint64_t* LB = LA + a.ef;
  uint8_t* FA = reinterpret_cast<uint8_t*>(LB + a.ef);
  uint8_t* FB = FA + round16(a.ef);
  uint64_t* cand = reinterpret_cast<uint64_t*>(FB + round16(a.ef));
  int32_t* H = reinterpret_cast<int32_t*>(cand + 32);
  const int hsize = 1 << a.hbits;
  const int L = a.n_layers;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long evals_all = 0, overflow = 0;
  for (int64_t q = (int64_t)blockIdx.x * a.warps + w; q < a.nq;
       q += (int64_t)gridDim.x * a.warps) {
    const float* qg = a.Q + (size_t)q * a.d;
    for (int t = lane; t < a.d; t += 32) qs[t] = qg[t];
    __syncwarp();
    float qn = 0.0f;
    if (METRIC == COS) {
      if (lane == 0) {
        float acc = 0.0f;
        for (int t = 0; t < a.d; ++t) acc = __fmaf_rn(qs[t], qs[t], acc);
        qn = __fsqrt_rn(acc);
      }
      qn = __shfl_sync(FULL, qn, 0);
    }
    auto dist_q = [&](int32_t v) {
      const float nr = METRIC == COS ? __ldg(a.norms + v) : 0.0f;
      return dist_query<METRIC>(qs, a.X + (size_t)v * a.d, a.d, a.vec4, qn, nr);
    };
    uint32_t ev = 1;
    const int32_t start =
        (int32_t)(mix_step(hash_prefix(a.seed, 0, 9, (uint64_t)q) ^ 0ull) % (uint64_t)a.rows[0]);
    float d0 = 0.0f;
    if (lane == 0) d0 = dist_q(start);
    uint64_t ck = make_key(__shfl_sync(FULL, d0, 0), start);
    // greedy descent through the layers above the bottom
    for (int l = 0; l + 1 < L; ++l) {
      const int wl = a.width[l];
      for (;;) {  // the current key strictly decreases, so this ends
        uint64_t best = ck;
        const int32_t* nb = a.g[l] + (size_t)key_id(ck) * wl;
        for (int c0 = 0; c0 < wl; c0 += 32) {
          int32_t v = c0 + lane < wl ? nb[c0 + lane] : -1;
          if (v >= a.rows[l]) {
            record_error(a.ctr, DERR_BAD_ID, key_id(ck));
            v = -1;
          }
          uint64_t k = KEY_EMPTY;
          if (v >= 0) k = make_key(dist_q(v), v);
          ev += __popc(__ballot_sync(FULL, v >= 0));
          const uint64_t m = warp_min64(k);
          best = m < best ? m : best;
        }
        if (best == ck) break;
        ck = best;
      }
    }
    // best-first search at the bottom
    for (int i = lane; i < hsize; i += 32) H[i] = -1;
    __syncwarp();
    if (lane == 0) {
      visit(H, a.hbits, key_id(ck));
      LA[0] = ck;
      FA[0] = 0;
    }
    __syncwarp();
    int cnt = 1;
    bool crowded = false;
    const int wb = a.width[L - 1];
    const int32_t* gb = a.g[L - 1];
    for (;;) {
      int e = -1;
      for (int c0 = 0; c0 < cnt; c0 += 32) {
        const unsigned b = __ballot_sync(FULL, c0 + lane < cnt && FA[c0 + lane] == 0);
        if (b) {
          e = c0 + __ffs(b) - 1;
          break;
        }
      }
      if (e < 0) break;
      const int32_t ue = key_id(LA[e]);
      __syncwarp();
      if (lane == 0) FA[e] = 1;
      __syncwarp();
      const int32_t* nb = gb + (size_t)ue * wb;
      for (int c0 = 0; c0 < wb; c0 += 32) {
        int32_t v = c0 + lane < wb ? nb[c0 + lane] : -1;
        if (v >= a.n) {
          record_error(a.ctr, DERR_BAD_ID, ue);
          v = -1;
        }
        bool fresh = false;
        if (v >= 0) {
          const int r = visit(H, a.hbits, v);
          fresh = r != 0;
          crowded = crowded || r == 2;
        }
        uint64_t k = KEY_EMPTY;
        if (fresh) k = make_key(dist_q(v), v);
        ev += __popc(__ballot_sync(FULL, fresh));
        const uint64_t thr = cnt == a.ef ? LA[cnt - 1] : KEY_EMPTY;
        if (k >= thr) k = KEY_EMPTY;
        if (!__any_sync(FULL, k != KEY_EMPTY)) continue;
        k = warp_sort32(k);
        const uint64_t pk = __shfl_up_sync(FULL, k, 1);
        bool keep = k != KEY_EMPTY && !(lane > 0 && pk == k);
        if (keep) {
          const int pos = count_below(LA, cnt, k);
          keep = !(pos < cnt && LA[pos] == k);
        }
        const unsigned kb = __ballot_sync(FULL, keep);
        if (keep) cand[__popc(kb & lt)] = k;
        const int nc = __popc(kb);
        __syncwarp();
        for (int i = lane; i < cnt; i += 32) {
          const uint64_t x = LA[i];
          const int pos = i + count_below(cand, nc, x);
          if (pos < a.ef) {
            LB[pos] = x;
            FB[pos] = FA[i];
          }
        }
        if (lane < nc) {
          const uint64_t x = cand[lane];
          const int pos = lane + count_below(LA, cnt, x);
          if (pos < a.ef) {
            LB[pos] = x;
            FB[pos] = 0;
          }
        }
        cnt = min(a.ef, cnt + nc);
        uint64_t* tl = LA;
        LA = LB;
        LB = tl;
        uint8_t* tf = FA;
        FA = FB;
        FB = tf;
        __syncwarp();
      }
    }
    int32_t* oi = a.out_ids + (size_t)q * a.k_out;
    float* od = a.out_dists + (size_t)q * a.k_out;
    for (int j = lane; j < a.k_out; j += 32) {
      if (j < cnt) {
        oi[j] = key_id(LA[j]);
        od[j] = key_dist(LA[j]);
      } else {
        oi[j] = -1;
        od[j] = f_inf();
      }
    }
    if (lane == 0 && a.out_evals) a.out_evals[q] = ev;
    evals_all += ev;
    overflow += __any_sync(FULL, crowded) ? 1ull : 0ull;
    // the two rank buffers swap an odd or even number of times per query:
    // start the next query from the region layout again
    LA = reinterpret_cast<uint64_t*>(base + search_qbytes(a.d));
    LB = LA + a.ef;
    FA = reinterpret_cast<uint8_t*>(LB + a.ef);
    FB = FA + round16(a.ef);
    __syncwarp();
  }
  if (lane == 0) {
    if (evals_all) atomicAdd(&a.ctr->dist_evals, evals_all);
    if (overflow) atomicAdd(&a.ctr->overflow, overflow);
  }
}

// out[r] = X[perm[r]], one warp per row; an index outside [0, n_src) is
// reported and its row left unwritten.
__global__ void k_gather_checked(const float* X, int64_t n_src, const int32_t* perm, int64_t n,
                                 int d, float* out, GdCounters* ctr) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += nw) {
    const int32_t p = perm[r];
    if (p < 0 || p >= n_src) {
      if (lane == 0) record_error(ctr, DERR_BAD_ID, r);
      continue;
    }
    const float* src = X + (size_t)p * d;
    float* dst = out + (size_t)r * d;
    for (int t = lane; t < d; t += 32) dst[t] = src[t];
  }
}

template <typename F>
cudaError_t set_smem(F* kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int gd_grid(int64_t n) {
  const int64_t want = (n + GD_WARPS - 1) / GD_WARPS;
  return (int)std::min<int64_t>(std::max<int64_t>(want, 1), 152 * 32);
}

}  // namespace

cudaError_t launch_gather_checked(const float* X, int64_t n_src, const int32_t* perm, int64_t n,
                                  int d, float* out, GdCounters* ctr, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_gather_checked<<<gd_grid(n), GD_WARPS * 32, 0, st>>>(X, n_src, perm, n, d, out, ctr);
  return cudaGetLastError();
}

size_t gd_reverse_smem(int M) { return (size_t)GD_WARPS * gd_warp_bytes(M); }

cudaError_t launch_diversify(const GdArgs& a, int metric, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.indeg, 0, (size_t)a.n * 4, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.rev_fill, 0, (size_t)a.n * 4, st)) != cudaSuccess) return e;
  const int64_t total = a.n * a.K;
  const int cg = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_gd_count<<<cg, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_exclusive_scan(a.indeg, a.n, a.tile_sum, a.rev_off, a.total, st)) !=
      cudaSuccess)
    return e;
  const int grid = gd_grid(a.n);
  const size_t smem = gd_reverse_smem(a.M);
  switch (metric) {
#define KNNM_GD_CASE(M_)                                                     \
  case M_:                                                                   \
    k_gd_forward<M_><<<grid, GD_WARPS * 32, 0, st>>>(a);                     \
    if ((e = cudaGetLastError()) != cudaSuccess) return e;                   \
    if (smem > 48 * 1024 && (e = set_smem(k_gd_reverse<M_>, smem)) != cudaSuccess) return e; \
    k_gd_reverse<M_><<<grid, GD_WARPS * 32, smem, st>>>(a);                  \
    break;
    KNNM_GD_CASE(L2)
    KNNM_GD_CASE(IP)
    KNNM_GD_CASE(COS)
    KNNM_GD_CASE(L1)
#undef KNNM_GD_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t plan_search(SearchArgs* a, size_t* smem, int* grid) {
  int hbits = 11;
  while (hbits < 14 && (1 << hbits) < 32 * a->ef) ++hbits;
  a->hbits = hbits;
  a->warp_bytes = search_warp_bytes(a->d, a->ef, hbits);
  const int cap = 227 * 1024;
  if (a->warp_bytes > cap) return cudaErrorInvalidValue;
  int warps = 4;
  while (warps > 1 && warps * a->warp_bytes > cap) --warps;
  a->warps = warps;
  *smem = (size_t)warps * a->warp_bytes;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int per_sm = std::max(1, (int)((228 * 1024) / (*smem + 1024)));
  const int64_t want = (a->nq + warps - 1) / warps;
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
  return cudaSuccess;
}

cudaError_t launch_search(const SearchArgs& a, int metric, size_t smem, int grid,
                          cudaStream_t st) {
  cudaError_t e;
  switch (metric) {
#define KNNM_SEARCH_CASE(M_)                                                  \
  case M_:                                                                    \
    if ((e = set_smem(k_search<M_>, smem)) != cudaSuccess) return e;          \
    k_search<M_><<<grid, a.warps * 32, smem, st>>>(a);                        \
    break;
    KNNM_SEARCH_CASE(L2)
    KNNM_SEARCH_CASE(IP)
    KNNM_SEARCH_CASE(COS)
    KNNM_SEARCH_CASE(L1)
#undef KNNM_SEARCH_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace knnm
