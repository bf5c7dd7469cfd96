// knnm_kernels.cu -- list kernels of the merge: init (Divide / Append /
// Initialize of Alg. 1 and Alg. 2), the sampler of each round (Reverse(G) and
// the new/old candidate sets), the top-k insert (UpdateNN), the flag/counter
// pass, the final Merge and Sort, and small conversion kernels.
//
// Lists are packed 64-bit keys (distance order bits << 32 | id), K <= 32, so a
// whole list fits one warp with one entry per lane.
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
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
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
__device__ __forceinline__ float dist_rows(const Rows& R, int64_t i, int64_t j, const float* norms) {
  float na = 0.f, nb = 0.f;
  if (METRIC == COS) {
    na = norms[i];
    nb = norms[j];
  }
  return canon_dist_global<METRIC>(R.row(i), R.row(j), R.d, na, nb);
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
  for (int c0 = 0; c0 < limit && got < want; c0 += 32) {
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

template <int METRIC>
__global__ void __launch_bounds__(BLOCK) k_init(InitArgs a) {
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
      uint64_t key = KEY_EMPTY;
      if (lane < K && !bad) {
        int64_t g = own_base + loc;
        key = make_key(dist_rows<METRIC>(a.rows, i, g, a.norms), (int32_t)g);
      }
      key = warp_sort32(key);
      if (lane >= Kk && lane < K) a.rear[(size_t)i * Kr + (lane - Kk)] = key;
      kept = lane < Kk ? key : KEY_EMPTY;
      want = Kr;
      base = i < a.n1 ? a.n1 : 0;
      n_src = i < a.n1 ? a.N - a.n1 : a.n1;
    } else {
      // Initialize (Alg. 2): K random members of S1 u S2.
      want = K;
      base = 0;
      n_src = a.N;
      if (Kr > 0 && lane < Kr) a.rear[(size_t)i * Kr + lane] = KEY_EMPTY;
    }
    int32_t drawn = draw_random(a.seed, i, base, n_src, want, K);
    uint64_t dkey = KEY_EMPTY;
    if (lane < want) dkey = make_key(dist_rows<METRIC>(a.rows, i, drawn, a.norms), drawn);
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

__global__ void k_norms(Rows R, int64_t N, float* norms) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) norms[i] = canon_norm_global(R.row(i), R.d);
}

// ---------------------------------------------------------------------------
// Sampler (round step 1)
// ---------------------------------------------------------------------------

// Forward sets of each node u and the pushes into the reverse slot arrays.
__global__ void __launch_bounds__(BLOCK) k_sample_fwd(SampleArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int K = a.K, s = a.s;
  for (int64_t u = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); u < a.N;
       u += nwarps) {
    uint64_t key = lane < K ? a.keys[(size_t)u * K + lane] : KEY_EMPTY;
    uint8_t f = lane < K ? a.flags[(size_t)u * K + lane] : FLAG_OLD;
    if (a.prev_keys && lane < K) a.prev_keys[(size_t)u * K + lane] = key;
    const int32_t v = key_id(key);
    const bool isnew = lane < K && f == FLAG_NEW;
    const bool isold = lane < K && f != FLAG_NEW;
    const uint64_t pre = hash_prefix(a.seed, (uint64_t)a.t, STREAM_FWD_NEW, (uint64_t)u);
    const uint64_t sk = isnew ? sampling_key(pre, v) : KEY_EMPTY;
    int rank = 0;
    for (int m = 0; m < K; ++m) rank += (__shfl_sync(FULL, sk, m) < sk) ? 1 : 0;
    const bool sel = isnew && rank < s;
    if (sel) a.flags[(size_t)u * K + lane] = FLAG_OLD;
    const unsigned bs = __ballot_sync(FULL, sel), bo = __ballot_sync(FULL, isold);
    if (sel) a.new_ids[(size_t)u * a.cap_new + __popc(bs & lanemask_lt())] = v;
    if (isold) a.old_ids[(size_t)u * a.cap_old + __popc(bo & lanemask_lt())] = v;
    if (lane == 0) {
      a.new_cnt[u] = __popc(bs);
      a.old_cnt[u] = __popc(bo);
    }
    if (sel)
      slots_insert(a.rev_new + (size_t)v * s, s,
                   sampling_key(hash_prefix(a.seed, (uint64_t)a.t, STREAM_REV_NEW, (uint64_t)v),
                                (int32_t)u));
    if (isold)
      slots_insert(a.rev_old + (size_t)v * s, s,
                   sampling_key(hash_prefix(a.seed, (uint64_t)a.t, STREAM_REV_OLD, (uint64_t)v),
                                (int32_t)u));
  }
}

// new(u) = fwd_new u rev_new;  old(u) = (fwd_old u rev_old) \ new(u).
__global__ void __launch_bounds__(BLOCK) k_sample_rev(SampleArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int s = a.s;
  for (int64_t u = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); u < a.N;
       u += nwarps) {
    const int nf = a.new_cnt[u], of = a.old_cnt[u];
    const int32_t fn = lane < nf ? a.new_ids[(size_t)u * a.cap_new + lane] : -1;
    const int32_t fo = lane < of ? a.old_ids[(size_t)u * a.cap_old + lane] : -2;
    const uint64_t rk = lane < s ? a.rev_new[(size_t)u * s + lane] : KEY_EMPTY;
    const uint64_t ok = lane < s ? a.rev_old[(size_t)u * s + lane] : KEY_EMPTY;
    const int32_t rn = rk != KEY_EMPTY ? key_id(rk) : -3;
    const int32_t ro = ok != KEY_EMPTY ? key_id(ok) : -4;
    bool rn_dup = false, fo_in_rn = false, ro_drop = false;
    for (int m = 0; m < nf; ++m) {
      int32_t x = __shfl_sync(FULL, fn, m);
      rn_dup |= (rn == x);
      ro_drop |= (ro == x);
    }
    for (int m = 0; m < s; ++m) {
      int32_t x = __shfl_sync(FULL, rn, m);
      fo_in_rn |= (fo == x);
      ro_drop |= (ro == x);
    }
    for (int m = 0; m < of; ++m) ro_drop |= (ro == __shfl_sync(FULL, fo, m));
    const bool add_rn = rn >= 0 && !rn_dup;
    const bool keep_fo = fo >= 0 && !fo_in_rn;
    const bool keep_ro = ro >= 0 && !ro_drop;
    const unsigned b1 = __ballot_sync(FULL, add_rn), b2 = __ballot_sync(FULL, keep_fo),
                   b3 = __ballot_sync(FULL, keep_ro);
    const int nn = nf + __popc(b1), no = __popc(b2) + __popc(b3);
    __syncwarp();
    if (add_rn) a.new_ids[(size_t)u * a.cap_new + nf + __popc(b1 & lanemask_lt())] = rn;
    if (keep_fo) a.old_ids[(size_t)u * a.cap_old + __popc(b2 & lanemask_lt())] = fo;
    if (keep_ro) a.old_ids[(size_t)u * a.cap_old + __popc(b2) + __popc(b3 & lanemask_lt())] = ro;
    if (lane == 0) {
      a.new_cnt[u] = nn;
      a.old_cnt[u] = no;
    }
  }
}

// ---------------------------------------------------------------------------
// Top-k insert (UpdateNN) and the flag / counter pass
// ---------------------------------------------------------------------------

// One thread per proposal; region b of the buffer was filled by join block b.
__global__ void k_update(UpdateArgs a, const unsigned long long* region_cnt, uint64_t region_cap) {
  const uint64_t cnt = region_cnt[blockIdx.x];
  const uint64_t base = (uint64_t)blockIdx.x * region_cap;
  for (uint64_t o = threadIdx.x; o < cnt; o += blockDim.x) {
    int32_t tgt = a.prop_tgt[base + o];
    uint64_t key = a.prop_key[base + o];
    slots_insert(a.keys + (size_t)tgt * a.K, a.K, key);
  }
}

__global__ void __launch_bounds__(BLOCK) k_finalize(FinalizeArgs a) {
  __shared__ unsigned long long red[WARPS_PER_BLOCK];
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  const int K = a.K;
  unsigned long long cnt = 0;
  const int64_t nodes_per_pass = nwarps;
  // every warp runs the same number of passes so the block reduction is safe
  const int64_t passes = (a.N + nodes_per_pass - 1) / nodes_per_pass;
  const int64_t w0 = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
  for (int64_t p = 0; p < passes; ++p) {
    int64_t v = w0 + p * nodes_per_pass;
    if (v >= a.N) continue;
    uint64_t nk = lane < K ? a.keys[(size_t)v * K + lane] : KEY_EMPTY;
    uint64_t pk = lane < K ? a.prev_keys[(size_t)v * K + lane] : KEY_EMPTY - 1;
    uint8_t pf = lane < K ? a.flags[(size_t)v * K + lane] : FLAG_NEW;
    bool found = false;
    uint8_t fl = FLAG_NEW;
    for (int m = 0; m < K; ++m) {
      uint64_t o = __shfl_sync(FULL, pk, m);
      uint8_t of = (uint8_t)__shfl_sync(FULL, (int)pf, m);
      if (o == nk) {
        found = true;
        fl = of;
      }
    }
    __syncwarp();
    if (lane < K) a.flags[(size_t)v * K + lane] = found ? fl : FLAG_NEW;
    cnt += __popc(__ballot_sync(FULL, lane < K && !found));
  }
  block_add(&a.ctr->updates, cnt, red);
}

// ---------------------------------------------------------------------------
// Merge and Sort with the rear lists (final step)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(BLOCK) k_final(int64_t N, int K, const uint64_t* keys, int Kr,
                                                 const uint64_t* rear, int32_t* out_ids,
                                                 float* out_dists) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WARPS_PER_BLOCK;
  for (int64_t v = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5); v < N;
       v += nwarps) {
    uint64_t e0 = lane < K ? keys[(size_t)v * K + lane] : KEY_EMPTY;
    uint64_t e1 = lane < Kr ? rear[(size_t)v * Kr + lane] : KEY_EMPTY;
    warp_sort64(e0, e1);
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

// BF16 shadow copy; aux = {|b|^2, |b - x| (upper bound), |b| (upper bound), canonical |x|}.
__global__ void k_bf16_prep(Rows R, int64_t N, __nv_bfloat16* Xb, float4* aux) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float* x = R.row(i);
  __nv_bfloat16* o = Xb + (size_t)i * R.d;
  float nb2 = 0.f, e2 = 0.f, nx2 = 0.f;
  for (int t = 0; t < R.d; ++t) {
    float v = __ldg(x + t);
    __nv_bfloat16 b = __float2bfloat16_rn(v);
    float bf = __bfloat162float(b);
    o[t] = b;
    nb2 = __fmaf_rn(bf, bf, nb2);
    float e = __fsub_rn(bf, v);  // exact: bf and v are within a factor of two
    e2 = __fmaf_rn(e, e, e2);
    nx2 = __fmaf_rn(v, v, nx2);
  }
  // sums of d non-negative terms carry at most d+1 relative roundings
  const float grow = 1.0f + (float)(R.d + 2) * 1.2e-7f;
  aux[i] = make_float4(nb2, __fsqrt_ru(e2 * grow) * 1.000001f, __fsqrt_ru(nb2 * grow) * 1.000001f,
                       __fsqrt_rn(nx2));
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

cudaError_t launch_init(const InitArgs& a, cudaStream_t st) {
  int grid = grid_for_warps(a.N);
  switch (a.metric) {
    case L2: k_init<L2><<<grid, BLOCK, 0, st>>>(a); break;
    case IP: k_init<IP><<<grid, BLOCK, 0, st>>>(a); break;
    case COS: k_init<COS><<<grid, BLOCK, 0, st>>>(a); break;
    default: k_init<L1><<<grid, BLOCK, 0, st>>>(a); break;
  }
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
  k_sample_rev<<<grid, BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_update_regions(const UpdateArgs& a, const unsigned long long* region_cnt,
                                  uint64_t region_cap, int regions, cudaStream_t st) {
  k_update<<<regions, 256, 0, st>>>(a, region_cnt, region_cap);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t st) {
  k_finalize<<<grid_for_warps(a.N), BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_final(int64_t N, int K, const uint64_t* keys, int Kr, const uint64_t* rear,
                         int32_t* out_ids, float* out_dists, cudaStream_t st) {
  k_final<<<grid_for_warps(N), BLOCK, 0, st>>>(N, K, keys, Kr, rear, out_ids, out_dists);
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

cudaError_t launch_bf16_prep(Rows rows, int64_t N, __nv_bfloat16* Xb, float4* aux,
                             cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  k_bf16_prep<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(rows, N, Xb, aux);
  return cudaGetLastError();
}

}  // namespace knnm
