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
// addressing).  Rows are compared four at a time, eight lanes each, by a
// reordered sum; that estimate is the canonical distance when both rows are
// small integers (every partial sum exact), settles a row that provably
// cannot enter the list otherwise, and leaves the rest to the in-order sum.  When the table is crowded a row may be compared again; a row
// that was dropped from the full rank list can never re-enter it (its key is
// above the list's last entry, which only decreases), and repeats of listed
// rows are dropped, so the result is that of the exact visited set.
#include "knnm_internal.cuh"

namespace knnm {
namespace {

constexpr int GD_WARPS = 8;   // forward pass and helpers
constexpr int REV_WARPS = 4;  // reverse pass (its staged batch takes ~17 KB per warp at d = 128)
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

// Canonical distance of two rows staged in shared memory (16-byte aligned,
// d % 4 == 0), a first.
template <int METRIC>
__device__ __forceinline__ float dist_staged(const float* ra, const float* rb, int d, float na,
                                             float nb) {
  float acc = 0.0f;
  const float4* a4 = reinterpret_cast<const float4*>(ra);
  const float4* b4 = reinterpret_cast<const float4*>(rb);
#pragma unroll 4
  for (int t = 0; t < (d >> 2); ++t) {
    const float4 x = a4[t], y = b4[t];
    acc = Canon<METRIC>::step(acc, x.x, y.x);
    acc = Canon<METRIC>::step(acc, x.y, y.y);
    acc = Canon<METRIC>::step(acc, x.z, y.z);
    acc = Canon<METRIC>::step(acc, x.w, y.w);
  }
  return canon_finish<METRIC>(acc, na, nb);
}

// Same with the second row in global memory (16-byte aligned).
template <int METRIC>
__device__ __forceinline__ float dist_staged_global(const float* ra, const float* __restrict__ rb,
                                                    int d, float na, float nb) {
  float acc = 0.0f;
  const float4* a4 = reinterpret_cast<const float4*>(ra);
  const float4* b4 = reinterpret_cast<const float4*>(rb);
#pragma unroll 4
  for (int t = 0; t < (d >> 2); ++t) {
    const float4 x = a4[t], y = __ldg(b4 + t);
    acc = Canon<METRIC>::step(acc, x.x, y.x);
    acc = Canon<METRIC>::step(acc, x.y, y.y);
    acc = Canon<METRIC>::step(acc, x.z, y.z);
    acc = Canon<METRIC>::step(acc, x.w, y.w);
  }
  return canon_finish<METRIC>(acc, na, nb);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// The warp copies rows ids[0..count) of X into dst (stride floats apart);
// every lane takes 16-byte pieces; completion is awaited by the caller.
__device__ __forceinline__ void stage_rows(float* dst, int stride, const float* X, int d,
                                           const int32_t* ids, int count, int lane) {
  const int n4 = d >> 2;
  for (int r = 0; r < count; ++r) {
    const float* src = X + (size_t)ids[r] * d;
    float* to = dst + (size_t)r * stride;
    for (int t = lane; t < n4; t += 32) cp_async16(to + 4 * t, src + 4 * t);
  }
}

// Pair p of the strict lower triangle, row-major: p = i (i - 1) / 2 + c, c < i.
__device__ __forceinline__ void tri_decode(int p, int& i, int& c) {
  int r = (int)((1.0f + sqrtf(8.0f * (float)p + 1.0f)) * 0.5f);
  while (r * (r - 1) / 2 > p) --r;
  while ((r + 1) * r / 2 <= p) ++r;
  i = r;
  c = p - r * (r - 1) / 2;
}

// occl[i] |= bit for every lane, where the lanes' rows i are non-decreasing
// (consecutive pairs of the triangle): the bits of a run of equal i are OR-ed
// by shuffles and its first lane alone writes, instead of one shared-memory
// atomic per lane on the same word.
__device__ __forceinline__ void or_by_row(uint32_t* occl, uint32_t bit, int i, bool valid,
                                          int lane) {
  if (!valid) i = -1 - lane;  // a run of its own
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t b2 = __shfl_down_sync(FULL, bit, o);
    const int i2 = __shfl_down_sync(FULL, i, o);
    if (lane + o < 32 && i2 == i) bit |= b2;
  }
  const int up = __shfl_up_sync(FULL, i, 1);
  if (valid && bit != 0u && (lane == 0 || up != i)) atomicOr(&occl[i], bit);
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

// Reverse pass, per warp: the batch's rows (32 x stride floats when staging),
// kept keys [M], forward keys [32], occlusion masks [32], batch ids [32].
__host__ __device__ __forceinline__ int gd_rows_bytes(int stage, int stride) {
  return stage ? 32 * stride * 4 : 0;
}
__host__ __device__ __forceinline__ int gd_kept_bytes(int M) { return (8 * M + 15) & ~15; }
__host__ __device__ __forceinline__ int gd_warp_bytes(int M, int stage, int stride) {
  return gd_rows_bytes(stage, stride) + gd_kept_bytes(M) + 8 * 32 + 4 * 32 + 4 * 32;
}

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
  __shared__ int32_t ids_s[GD_WARPS][33];
  extern __shared__ __align__(16) unsigned char fwd_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* occl = occl_s[w];
  int32_t* sid = ids_s[w];  // staged rows: slot 0 = the row itself, slot 1 + j = its entry j
  float* rows = reinterpret_cast<float*>(fwd_sm) + (size_t)w * (a.K + 1) * a.stride;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long evals = 0;
  for (int64_t u = (int64_t)blockIdx.x * GD_WARPS + w; u < a.n;
       u += (int64_t)gridDim.x * GD_WARPS) {
    int32_t v = -1;
    if (lane < a.K) {
      v = a.G[u * a.K + lane];
      if (v < 0 || v >= a.n || v == u) v = -1;  // reported by the count pass
    }
    uint64_t key = KEY_EMPTY;
    if (a.stage) {  // the row and its entries, in list order, into shared memory
      if (lane == 0) sid[0] = (int32_t)u;
      if (lane < a.K) sid[1 + lane] = v >= 0 ? v : (int32_t)u;
      __syncwarp();
      stage_rows(rows, a.stride, a.X, a.d, sid, a.K + 1, lane);
      cp_async_wait_all();
      __syncwarp();
      if (v >= 0) {
        const float nu = METRIC == COS ? __ldg(a.norms + u) : 0.0f;
        const float nv_ = METRIC == COS ? __ldg(a.norms + v) : 0.0f;
        key = make_key(dist_staged<METRIC>(rows, rows + (size_t)(1 + lane) * a.stride, a.d, nu,
                                           nv_), v);
      }
    } else if (v >= 0) {
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
    int my_slot = 0;  // staged slot of this lane's (sorted) entry
    if (a.stage && key != KEY_EMPTY)
      for (int j = 0; j < a.K; ++j)
        if (sid[1 + j] == id) {
          my_slot = 1 + j;
          break;
        }
    occl[lane] = 0u;
    __syncwarp();
    const int P = nv * (nv - 1) / 2;
    for (int base = 0; base < P; base += 32) {
      const int p = base + lane;
      int i = 1, c = 0;
      if (p < P) tri_decode(p, i, c);
      const int32_t si = __shfl_sync(FULL, id, i), sc = __shfl_sync(FULL, id, c);
      const int ti = __shfl_sync(FULL, my_slot, i), tc = __shfl_sync(FULL, my_slot, c);
      const float di = __shfl_sync(FULL, dl, i);
      uint32_t bit = 0u;
      if (p < P) {
        float dic;
        if (a.stage) {
          const float ni = METRIC == COS ? __ldg(a.norms + si) : 0.0f;
          const float nc = METRIC == COS ? __ldg(a.norms + sc) : 0.0f;
          dic = dist_staged<METRIC>(rows + (size_t)ti * a.stride, rows + (size_t)tc * a.stride,
                                    a.d, ni, nc);
        } else {
          dic = dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, si, sc);
        }
        bit = dic < di ? 1u << c : 0u;
      }
      or_by_row(occl, bit, i, p < P, lane);
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
__global__ void __launch_bounds__(REV_WARPS * 32) k_gd_reverse(const GdArgs a) {
  extern __shared__ __align__(16) unsigned char gd_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int M = a.M;
  unsigned char* wbase = gd_sm + (size_t)w * gd_warp_bytes(M, a.stage, a.stride);
  float* rows = reinterpret_cast<float*>(wbase);  // the batch's rows when staging
  uint64_t* kept = reinterpret_cast<uint64_t*>(wbase + gd_rows_bytes(a.stage, a.stride));
  uint64_t* fk = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(kept) +
                                             gd_kept_bytes(M));
  uint32_t* occl = reinterpret_cast<uint32_t*>(fk + 32);
  int32_t* sid = reinterpret_cast<int32_t*>(occl + 32);
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long evals = 0, edges = 0, full = 0, max_in = 0;
  for (int64_t u = (int64_t)blockIdx.x * REV_WARPS + w; u < a.n;
       u += (int64_t)gridDim.x * REV_WARPS) {
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
      if (a.stage) {
        sid[lane] = s;
        __syncwarp();
        stage_rows(rows, a.stride, a.X, a.d, sid, nb, lane);
        cp_async_wait_all();
        __syncwarp();
      }
      bool surv = lane < nb;
      for (int j = 0; surv && j < nk; ++j) {
        ++evals;
        const int32_t kj = key_id(kept[j]);
        float dk;
        if (a.stage) {
          const float ns = METRIC == COS ? __ldg(a.norms + s) : 0.0f;
          const float nk2 = METRIC == COS ? __ldg(a.norms + kj) : 0.0f;
          dk = dist_staged_global<METRIC>(rows + (size_t)lane * a.stride, a.X + (size_t)kj * a.d,
                                          a.d, ns, nk2);
        } else {
          dk = dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, s, kj);
        }
        if (dk < ds) surv = false;
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
        uint32_t bit = 0u;
        if (p < P && ((sm >> i) & 1u) && ((sm >> c) & 1u)) {
          ++evals;
          float dic;
          if (a.stage) {
            const float ni = METRIC == COS ? __ldg(a.norms + si) : 0.0f;
            const float nc = METRIC == COS ? __ldg(a.norms + sc) : 0.0f;
            dic = dist_staged<METRIC>(rows + (size_t)i * a.stride, rows + (size_t)c * a.stride,
                                      a.d, ni, nc);
          } else {
            dic = dist_rows<METRIC>(a.X, a.d, a.vec4, a.norms, si, sc);
          }
          bit = dic < di ? 1u << c : 0u;
        }
        or_by_row(occl, bit, i, p < P, lane);
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
      if (keep) {
        const int pos = count_below(fk, fc, r);
        keep = !(pos < fc && fk[pos] == r);
      }
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
// Per-warp shared memory: query, the rank list with its expanded flags, 32
// candidate keys (also the ids of the rows being compared), the visited table.
__host__ __device__ __forceinline__ int search_warp_bytes(int d, int ef, int hbits) {
  return search_qbytes(d) + round16(8 * ef) + round16(ef) + 8 * 32 + (4 << hbits);
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

// Per-row search data: {max |x| when every coordinate is an integer of
// magnitude <= 2^24, else -1; canonical norm}.  One warp per row: the row is
// read coalesced into shared memory, checked by all lanes, and its norm summed
// in index order by lane 0.
constexpr int AUX_WARPS = 8;
constexpr int AUX_CHUNK = 1024;  // floats staged per pass
__global__ void __launch_bounds__(AUX_WARPS * 32) k_row_aux(const float* X, int64_t n, int d,
                                                            float2* aux) {
  __shared__ float stage[AUX_WARPS][AUX_CHUNK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* sx = stage[w];
  for (int64_t i = (int64_t)blockIdx.x * AUX_WARPS + w; i < n;
       i += (int64_t)gridDim.x * AUX_WARPS) {
    const float* r = X + (size_t)i * d;
    float acc = 0.0f, mx = 0.0f;
    bool integral = true;
    for (int t0 = 0; t0 < d; t0 += AUX_CHUNK) {
      const int len = min(AUX_CHUNK, d - t0);
      for (int t = lane; t < len; t += 32) {
        const float x = __ldg(r + t0 + t);
        sx[t] = x;
        mx = fmaxf(mx, fabsf(x));
        integral = integral && x == rintf(x);
      }
      __syncwarp();
      if (lane == 0)
        for (int t = 0; t < len; ++t) acc = __fmaf_rn(sx[t], sx[t], acc);
      __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    integral = __all_sync(FULL, integral);
    if (lane == 0) aux[i] = make_float2(integral && mx <= 16777216.0f ? mx : -1.0f, __fsqrt_rn(acc));
  }
}

// True when every partial sum of the pair's canonical accumulation is an
// integer below 2^24 in magnitude: then any summation order gives the
// canonical bits.  qm, rm: max |coordinate| of two integer rows.
template <int METRIC>
__device__ __forceinline__ bool exact_pair(float qm, float rm, int d) {
  if (qm < 0.0f || rm < 0.0f) return false;
  const unsigned long long q = (unsigned long long)qm, r = (unsigned long long)rm;
  const unsigned long long lim = 1ull << 24;
  if (METRIC == L2) return (unsigned long long)d * (q + r) * (q + r) < lim;
  if (METRIC == L1) return (unsigned long long)d * (q + r) < lim;
  if (METRIC == CHI2) return false;  // a quotient per term: not exact in general
  return (unsigned long long)d * q * r < lim;  // IP, COS: the dot product
}

// Upper bound on |estimate - canonical| for one pair, where both are sums of
// the same exactly known terms in different orders (each within
// gamma_d * sum|terms| of the exact sum, gamma_m = m u / (1 - m u)).
template <int METRIC>
__device__ __forceinline__ float pair_bound(float est, float g, float nq, float nr, float den) {
  if (METRIC == L2 || METRIC == L1)  // non-negative terms
    return 2.0f * g * est / (1.0f - g) * 1.0001f;
  if (METRIC == CHI2) return __int_as_float(0x7f800000);  // terms of either sign: no skip
  const float dot = 2.2f * g * nq * nr;  // sum |a_i b_i| <= |a||b| (norms within gamma)
  if (METRIC == IP) return dot * 1.0001f + 1e-37f;
  if (den == 0.0f) return 0.0f;  // both read 1
  return (dot / den) * 1.0001f + 8.0f * 5.9604645e-8f;  // COS: division and 1 - x
}

template <int METRIC>
__global__ void __launch_bounds__(128) k_search(const SearchArgs a) {
  extern __shared__ __align__(16) unsigned char s_sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned char* base = s_sm + (size_t)w * a.warp_bytes;
  float* qs = reinterpret_cast<float*>(base);
  unsigned char* lists = base + search_qbytes(a.d);
  uint64_t* LA = reinterpret_cast<uint64_t*>(lists);
  uint8_t* FA = lists + round16(8 * a.ef);
  uint64_t* cand = reinterpret_cast<uint64_t*>(FA + round16(a.ef));
  int32_t* vid = reinterpret_cast<int32_t*>(cand);  // row ids under comparison (before a merge)
  int32_t* H = reinterpret_cast<int32_t*>(cand + 32);
  const int hsize = 1 << a.hbits;
  const int L = a.n_layers;
  const unsigned lt = (1u << lane) - 1u;
  const int grp = lane >> 3, part = lane & 7;  // 4 rows per pass, 8 lanes per row
  // gamma_{d+2} for the estimate bounds
  const float g = (float)(a.d + 2) * 5.9604645e-8f / (1.0f - (float)(a.d + 2) * 5.9604645e-8f);
  unsigned long long evals_all = 0, overflow = 0;
  for (int64_t q = (int64_t)blockIdx.x * a.warps + w; q < a.nq;
       q += (int64_t)gridDim.x * a.warps) {
    const float* qg = a.Q + (size_t)q * a.d;
    bool qint = true;
    float qmax = 0.0f;
    for (int t = lane; t < a.d; t += 32) {
      const float x = qg[t];
      qs[t] = x;
      qmax = fmaxf(qmax, fabsf(x));
      qint = qint && x == rintf(x);
    }
    for (int o = 16; o > 0; o >>= 1) qmax = fmaxf(qmax, __shfl_xor_sync(FULL, qmax, o));
    qmax = (__all_sync(FULL, qint) && qmax <= 16777216.0f) ? qmax : -1.0f;
    __syncwarp();
    float qn = 0.0f;
    if (METRIC == COS || METRIC == IP) {
      if (lane == 0) {
        float acc = 0.0f;
        for (int t = 0; t < a.d; ++t) acc = __fmaf_rn(qs[t], qs[t], acc);
        qn = __fsqrt_rn(acc);
      }
      qn = __shfl_sync(FULL, qn, 0);
    }
    // Keys of the rows v of the lanes with `want`.  A row is first estimated
    // by 8 lanes (a reordered sum of the canonical terms); the estimate is the
    // canonical value when exact_pair holds; otherwise, when `filter` is set
    // and the estimate proves the row's distance above thr, the row cannot
    // enter and comes back as KEY_EMPTY; every other row gets its canonical
    // distance from its own lane (in-order sum).
    auto eval = [&](int32_t v, bool want, bool filter, float thr) {
      const unsigned m = __ballot_sync(FULL, want);
      const int cnt_f = __popc(m), rank = __popc(m & lt);
      float2 ax = make_float2(-1.0f, 0.0f);
      if (want) {
        vid[rank] = v;
        ax = __ldg(reinterpret_cast<const float2*>(a.aux) + v);  // consumed after the rows
      }
      __syncwarp();
      float est_acc = 0.0f;
      const int n4 = a.d >> 2;
      // 8 rows per batch, two per 8-lane group; every load of a batch is issued
      // before any of its sums starts
      for (int p0 = 0; p0 < cnt_f; p0 += 8) {
        const int ra = p0 + grp, rb = p0 + 4 + grp;
        const bool va = ra < cnt_f, vb = rb < cnt_f;
        const float* rowa = a.X + (size_t)(va ? vid[ra] : 0) * a.d;
        const float* rowb = a.X + (size_t)(vb ? vid[rb] : 0) * a.d;
        float acca = 0.0f, accb = 0.0f;
        if (a.vec4) {
          const float4* q4 = reinterpret_cast<const float4*>(qs);
          const float4* a4 = reinterpret_cast<const float4*>(rowa);
          const float4* b4 = reinterpret_cast<const float4*>(rowb);
          for (int c0 = part; c0 < n4; c0 += 32) {
            float4 ya[4], yb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = c0 + 8 * u;
              const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
              ya[u] = (va && c < n4) ? __ldg(a4 + c) : z;
              yb[u] = (vb && c < n4) ? __ldg(b4 + c) : z;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = c0 + 8 * u;
              if (c < n4) {
                const float4 x = q4[c];
                acca = Canon<METRIC>::step(acca, x.x, ya[u].x);
                acca = Canon<METRIC>::step(acca, x.y, ya[u].y);
                acca = Canon<METRIC>::step(acca, x.z, ya[u].z);
                acca = Canon<METRIC>::step(acca, x.w, ya[u].w);
                accb = Canon<METRIC>::step(accb, x.x, yb[u].x);
                accb = Canon<METRIC>::step(accb, x.y, yb[u].y);
                accb = Canon<METRIC>::step(accb, x.z, yb[u].z);
                accb = Canon<METRIC>::step(accb, x.w, yb[u].w);
              }
            }
          }
        } else {
          for (int t = part; t < a.d; t += 8) {
            const float ya = va ? __ldg(rowa + t) : 0.0f, yb = vb ? __ldg(rowb + t) : 0.0f;
            acca = Canon<METRIC>::step(acca, qs[t], ya);
            accb = Canon<METRIC>::step(accb, qs[t], yb);
          }
        }
        acca = __fadd_rn(acca, __shfl_xor_sync(FULL, acca, 1));
        acca = __fadd_rn(acca, __shfl_xor_sync(FULL, acca, 2));
        acca = __fadd_rn(acca, __shfl_xor_sync(FULL, acca, 4));
        accb = __fadd_rn(accb, __shfl_xor_sync(FULL, accb, 1));
        accb = __fadd_rn(accb, __shfl_xor_sync(FULL, accb, 2));
        accb = __fadd_rn(accb, __shfl_xor_sync(FULL, accb, 4));
        const int src = ((rank - p0) & 3) << 3;
        const float ea = __shfl_sync(FULL, acca, src), eb = __shfl_sync(FULL, accb, src);
        if (want && rank >= p0 && rank < p0 + 4) est_acc = ea;
        if (want && rank >= p0 + 4 && rank < p0 + 8) est_acc = eb;
      }
      __syncwarp();
      uint64_t k = KEY_EMPTY;
      bool need = false;
      if (want) {
        const float nr = ax.y;
        const float est = canon_finish<METRIC>(est_acc, qn, nr);
        if (exact_pair<METRIC>(qmax, ax.x, a.d)) {
          k = make_key(est, v);
        } else {
          const float den = __fmul_rn(qn, nr);
          need = !(filter && est - pair_bound<METRIC>(est, g, qn, nr, den) > thr);
        }
      }
      if (__any_sync(FULL, need) && need)
        k = make_key(dist_query<METRIC>(qs, a.X + (size_t)v * a.d, a.d, a.vec4, qn, ax.y), v);
      return k;
    };
    uint32_t ev = 1;
    const int32_t start =
        (int32_t)(mix_step(hash_prefix(a.seed, 0, 9, (uint64_t)q) ^ 0ull) % (uint64_t)a.rows[0]);
    uint64_t ck = eval(start, lane == 0, false, 0.0f);
    ck = __shfl_sync(FULL, ck, 0);
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
          const uint64_t k = eval(v, v >= 0, true, key_dist(best));
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
    int cnt = 1, hint = 0;  // entries before `hint` are expanded
    bool crowded = false;
    const int wb = a.width[L - 1];
    const int32_t* gb = a.g[L - 1];
    for (;;) {
      int e = -1;
      for (int c0 = hint & ~31; c0 < cnt; c0 += 32) {
        const int i = c0 + lane;
        const unsigned b = __ballot_sync(FULL, i >= hint && i < cnt && FA[i] == 0);
        if (b) {
          e = c0 + __ffs(b) - 1;
          break;
        }
      }
      if (e < 0) break;
      hint = e + 1;
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
        const bool full = cnt == a.ef;
        const uint64_t thr = full ? LA[cnt - 1] : KEY_EMPTY;
        uint64_t k = eval(v, fresh, full, full ? key_dist(thr) : 0.0f);
        ev += __popc(__ballot_sync(FULL, fresh));
        if (k >= thr) k = KEY_EMPTY;
        const unsigned cm = __ballot_sync(FULL, k != KEY_EMPTY);
        if (cm == 0u) continue;
        if (cm & (cm - 1u)) {
          k = warp_sort32(k);  // two or more: ascending in lanes 0..
        } else {
          const uint64_t one = __shfl_sync(FULL, k, __ffs(cm) - 1);
          k = lane == 0 ? one : KEY_EMPTY;
        }
        const uint64_t pk = __shfl_up_sync(FULL, k, 1);
        bool keep = k != KEY_EMPTY && !(lane > 0 && pk == k);
        int below = 0;  // entries of the current list below this candidate
        if (keep) {
          below = count_below(LA, cnt, k);
          keep = !(below < cnt && LA[below] == k);
        }
        const unsigned kb = __ballot_sync(FULL, keep);
        if (kb == 0u) continue;
        const int nc = __popc(kb), rank = __popc(kb & lt);
        if (keep) cand[rank] = k;
        const int pmin = __shfl_sync(FULL, below, __ffs(kb) - 1);
        __syncwarp();
        // In place: entries from pmin on move right past the candidates below
        // them (chunks from the end; targets strictly increase, so no write
        // lands on an entry not yet read); those pushed beyond ef drop out.
        for (int c0 = (cnt - 1) & ~31; c0 >= (pmin & ~31); c0 -= 32) {
          const int i = c0 + lane;
          const bool mv = i >= pmin && i < cnt;
          uint64_t x = 0;
          uint8_t f = 0;
          int np = 0;
          if (mv) {
            x = LA[i];
            f = FA[i];
            np = i + count_below(cand, nc, x);
          }
          __syncwarp();
          if (mv && np < a.ef) {
            LA[np] = x;
            FA[np] = f;
          }
          __syncwarp();
        }
        if (keep && rank + below < a.ef) {
          LA[rank + below] = k;
          FA[rank + below] = 0;
        }
        cnt = min(a.ef, cnt + nc);
        hint = min(hint, pmin);
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

size_t gd_reverse_smem(int M, int stage, int stride) {
  return (size_t)REV_WARPS * gd_warp_bytes(M, stage, stride);
}

bool plan_diversify(GdArgs* a) {
  // stage rows in shared memory when 32 rows per warp fit a 227 KB block
  a->stride = a->d + 4;
  a->stage = (a->vec4 && (size_t)GD_WARPS * 33 * a->stride * 4 <= 227 * 1024 &&
               gd_reverse_smem(a->M, 1, a->stride) <= 227 * 1024)
                 ? 1
                 : 0;
  // every warp's region must start 16-byte aligned (staged rows, 64-bit keys)
  return gd_warp_bytes(a->M, a->stage, a->stride) % 16 == 0 &&
         (!a->stage || ((size_t)(a->K + 1) * a->stride * 4) % 16 == 0);
}

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
  const size_t smem = gd_reverse_smem(a.M, a.stage, a.stride);
  const size_t fsmem = a.stage ? (size_t)GD_WARPS * (a.K + 1) * a.stride * 4 : 0;
  const int rgrid = (int)std::min<int64_t>((a.n + REV_WARPS - 1) / REV_WARPS, 152 * 64);
  switch (metric) {
#define KNNM_GD_CASE(M_)                                                             \
  case M_:                                                                           \
    if ((e = set_smem(k_gd_forward<M_>, fsmem)) != cudaSuccess) return e;            \
    k_gd_forward<M_><<<grid, GD_WARPS * 32, fsmem, st>>>(a);                         \
    if ((e = cudaGetLastError()) != cudaSuccess) return e;                           \
    if ((e = set_smem(k_gd_reverse<M_>, smem)) != cudaSuccess) return e;             \
    k_gd_reverse<M_><<<rgrid, REV_WARPS * 32, smem, st>>>(a);                        \
    break;
    KNNM_GD_CASE(L2)
    KNNM_GD_CASE(IP)
    KNNM_GD_CASE(COS)
    KNNM_GD_CASE(L1)
    KNNM_GD_CASE(CHI2)
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
  if (a->warp_bytes % 16 != 0) return cudaErrorInvalidValue;  // every region 16-byte aligned
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

cudaError_t launch_row_aux(const float* X, int64_t n, int d, float* aux, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + AUX_WARPS - 1) / AUX_WARPS, 152 * 8);
  k_row_aux<<<grid, AUX_WARPS * 32, 0, st>>>(X, n, d, reinterpret_cast<float2*>(aux));
  return cudaGetLastError();
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
    KNNM_SEARCH_CASE(CHI2)
#undef KNNM_SEARCH_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace knnm
