/*
 * knnm_oracle.c -- CPU oracle for the k-NN graph merge of Zhao, Wang, Lin and
 * Ngo, "On the Merge of k-NN Graph": Symmetric Merge (S-Merge, Alg. 1), Joint
 * Merge (J-Merge, Alg. 2) and the NN-Descent build that J-Merge reduces to when
 * the existing graph is empty; the H-Merge visiting order (Sec. 3.3); graph
 * diversification (Alg. 3) and the top-down search on the hierarchy (Sec. 3.4).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded
 * restatement of the method, written to check the CUDA library against.  It
 * shares no code, header, table or helper with the CUDA library; only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Readings taken where the paper is silent (each one is pinned by a test in
 * tests/test_oracle_*.py unless marked otherwise):
 *   - Distance (Alg. 1, l <- m(s_i, s_j)): one FP32 accumulator, dimensions in
 *     index order, fmaf per term.  L2 is the squared Euclidean distance (same
 *     ranking as l2), IP is 0 - dot, COS is 1 - dot/(|a||b|) (1 when a norm is
 *     zero), L1 adds |a_t - b_t| in order, CHI2 adds (a_t - b_t)^2 / (a_t + b_t)
 *     in order (a term with a_t + b_t = 0 adds 0; meant for non-negative rows),
 *     JACCARD is 1 - |A n B| / |A u B| of two sets given as 0/1 rows (the counts
 *     as sums of min and max; 0 for two empty sets).
 *   - List order: ascending (distance, id); ids unique per list, no self.
 *   - Random numbers: H(seed, t, stream, owner, member) = five chained
 *     SplitMix64 steps (Steele, Lea and Flood, OOPSLA 2014), each absorbing one
 *     word by xor.  A sampling key is (high 32 bits of H) << 32 | member.
 *   - Init (Alg. 1 "Divide"/"Append", Alg. 2 "Initialize"): the input list is
 *     re-sorted by recomputed distance; the first K_keep = floor(r*K) entries
 *     stay, the rest is the rear list G^v.  Random members are drawn as
 *     base + H(seed, 0, 3, i, c) mod n_src for c = 0, 1, ..., skipping self and
 *     repeats; after 32*K draws the row is completed with the smallest unused ids.
 *   - Round t (the NN-Descent iteration the paper cites for Alg. 1): each node
 *     samples s = max(1, floor(rho*K)) of its entries flagged new (smallest
 *     sampling key, stream 0) and flips them to old; all entries flagged old at
 *     round start form its old forward set.  Reverse lists are cut to the s
 *     smallest keys (stream 1 for new, 2 for old).  new(u) = forward-new union
 *     reverse-new; old(u) = (forward-old union reverse-old) minus new(u).
 *   - Local join: unordered pairs with at least one member in new(u); S-Merge
 *     keeps only pairs across S1/S2 (Alg. 1), J-Merge drops pairs inside S1
 *     (Alg. 2).  Each pair updates both endpoints (UpdateNN).
 *   - UpdateNN: insert into the sorted K-list if it ranks within the first K and
 *     the id is not listed yet; an inserted entry is flagged new.
 *   - c_t = number of (node, id) entries present after round t that were not
 *     present before it; stop when c_t <= delta*N*K or t = max_iters.
 *   - Final merge (Alg. 1 "Merge and Sort", Alg. 2 likewise): first K distinct
 *     ids of the working list merged with the rear list.
 *   - Literal mode (tests only): every entry counts as new every round and the
 *     reverse lists are not cut, which is Alg. 1 / Alg. 2 as printed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_L2 = 0, ORC_IP = 1, ORC_COS = 2, ORC_L1 = 3, ORC_CHI2 = 4, ORC_JACCARD = 5 };
enum { ORC_SYMMETRIC = 0, ORC_JOINT = 1 };
enum { STREAM_FWD_NEW = 0, STREAM_REV_NEW = 1, STREAM_REV_OLD = 2, STREAM_INIT = 3 };
enum { FLAG_OLD = 0, FLAG_NEW = 1 };
enum { ORC_OK = 0, ORC_ERR_INVALID = -1, ORC_ERR_NOMEM = -2, ORC_ERR_CAPACITY = -3 };

/* ------------------------------------------------------------------ */
/* Distance m(.,.) of Alg. 1 / Alg. 2                                    */
/* ------------------------------------------------------------------ */

static float canonical_norm(const float* a, int d) {
  float acc = 0.0f;
  for (int t = 0; t < d; ++t) acc = fmaf(a[t], a[t], acc);
  return sqrtf(acc);
}

float orc_distance(int metric, const float* a, const float* b, int d) {
  float acc = 0.0f;
  if (metric == ORC_L2) {
    for (int t = 0; t < d; ++t) {
      float x = a[t] - b[t];
      acc = fmaf(x, x, acc);
    }
    return acc;
  }
  if (metric == ORC_IP) {
    for (int t = 0; t < d; ++t) acc = fmaf(a[t], b[t], acc);
    return 0.0f - acc;
  }
  if (metric == ORC_COS) {
    for (int t = 0; t < d; ++t) acc = fmaf(a[t], b[t], acc);
    float den = canonical_norm(a, d) * canonical_norm(b, d);
    if (den == 0.0f) return 1.0f;
    return 1.0f - acc / den;
  }
  if (metric == ORC_L1) {
    for (int t = 0; t < d; ++t) acc = acc + fabsf(a[t] - b[t]);
    return acc;
  }
  if (metric == ORC_CHI2) {  /* the chi-square distance of the NUSWide experiments (Sec. 5) */
    for (int t = 0; t < d; ++t) {
      const float x = a[t] - b[t];
      const float s = a[t] + b[t];
      const float q = x * x;
      acc = acc + (s == 0.0f ? 0.0f : q / s);
    }
    return acc;
  }
  if (metric == ORC_JACCARD) {  /* the Kosarak metric of Sec. 5: sets as 0/1 rows */
    float inter = 0.0f, uni = 0.0f;
    for (int t = 0; t < d; ++t) {
      inter = inter + fminf(a[t], b[t]);
      uni = uni + fmaxf(a[t], b[t]);
    }
    return uni == 0.0f ? 0.0f : 1.0f - inter / uni;
  }
  return NAN;
}

/* ------------------------------------------------------------------ */
/* Counter-based random numbers                                          */
/* ------------------------------------------------------------------ */

/* One SplitMix64 step: advance the state by the golden gamma and mix it. */
static uint64_t splitmix_step(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* The SplitMix64 generator itself, exported so tests can check the step
 * against the generator's published output sequence. */
uint64_t orc_splitmix64_next(uint64_t* state) {
  uint64_t out = splitmix_step(*state);
  *state += 0x9E3779B97F4A7C15ull;
  return out;
}

uint64_t orc_hash(uint64_t seed, uint64_t t, uint64_t stream, uint64_t owner, uint64_t member) {
  uint64_t h = splitmix_step(seed);
  h = splitmix_step(h ^ t);
  h = splitmix_step(h ^ stream);
  h = splitmix_step(h ^ owner);
  return splitmix_step(h ^ member);
}

static uint64_t sample_key(uint64_t seed, int t, int stream, int64_t owner, int32_t member) {
  uint64_t h = orc_hash(seed, (uint64_t)t, (uint64_t)stream, (uint64_t)owner, (uint64_t)member);
  return (h & 0xFFFFFFFF00000000ull) | (uint64_t)(uint32_t)member;
}

/* ------------------------------------------------------------------ */
/* Sorted neighbour lists                                                */
/* ------------------------------------------------------------------ */

/* Entry order: smaller distance first, then smaller id. */
static int entry_less(float da, int32_t ia, float db, int32_t ib) {
  return da < db || (da == db && ia < ib);
}

/* UpdateNN(G[p], q, l) of Alg. 1: put <q, l> into the sorted K-list of p when it
 * ranks within the first K and q is not listed yet.  Returns 1 when inserted. */
static int update_nn(int32_t* ids, float* dists, uint8_t* flags, int K, int32_t q, float l) {
  for (int j = 0; j < K; ++j)
    if (ids[j] == q) return 0;
  if (!entry_less(l, q, dists[K - 1], ids[K - 1])) return 0;
  int pos = K - 1;
  while (pos > 0 && entry_less(l, q, dists[pos - 1], ids[pos - 1])) {
    ids[pos] = ids[pos - 1];
    dists[pos] = dists[pos - 1];
    if (flags) flags[pos] = flags[pos - 1];
    --pos;
  }
  ids[pos] = q;
  dists[pos] = l;
  if (flags) flags[pos] = FLAG_NEW;
  return 1;
}

/* Insertion sort of m (id, distance) pairs into entry order. */
static void sort_entries(int32_t* ids, float* dists, int m) {
  for (int a = 1; a < m; ++a) {
    int32_t id = ids[a];
    float dv = dists[a];
    int b = a;
    while (b > 0 && entry_less(dv, id, dists[b - 1], ids[b - 1])) {
      ids[b] = ids[b - 1];
      dists[b] = dists[b - 1];
      --b;
    }
    ids[b] = id;
    dists[b] = dv;
  }
}

static const float* row(const float* X, int64_t i, int d) { return X + (size_t)i * (size_t)d; }

/* ------------------------------------------------------------------ */
/* Init: Divide / Append (Alg. 1), Divide / Append / Initialize (Alg. 2)  */
/* ------------------------------------------------------------------ */

/* Draws `want` distinct ids from [base, base + n_src) \ {self} for node i. */
static void draw_random(uint64_t seed, int64_t i, int64_t base, int64_t n_src, int want,
                        int K, int32_t* out) {
  int got = 0;
  for (int c = 0; c < 32 * K && got < want; ++c) {
    int64_t j = base + (int64_t)(orc_hash(seed, 0, STREAM_INIT, (uint64_t)i, (uint64_t)c) %
                                 (uint64_t)n_src);
    if (j == i) continue;
    int seen = 0;
    for (int a = 0; a < got; ++a)
      if (out[a] == (int32_t)j) seen = 1;
    if (!seen) out[got++] = (int32_t)j;
  }
  for (int64_t j = base; j < base + n_src && got < want; ++j) {
    if (j == i) continue;
    int seen = 0;
    for (int a = 0; a < got; ++a)
      if (out[a] == (int32_t)j) seen = 1;
    if (!seen) out[got++] = (int32_t)j;
  }
}

/* mode ORC_SYMMETRIC: rows [0, n1) take G1 (ids local to S1), rows [n1, n) take
 * G2 (ids local to S2).  mode ORC_JOINT: rows [0, n1) take G1, rows [n1, n) are
 * raw.  Global ids put S1 first.  Outputs are [n][K] working lists and
 * [n][K - K_keep] rear lists (id -1, distance +inf where a row has none). */
int orc_init(int mode, const float* X, int64_t n, int64_t n1, int d, int metric,
             const int32_t* G1, const int32_t* G2, int K, int K_keep, uint64_t seed,
             int32_t* ids, float* dists, uint8_t* flags, int32_t* rear_ids, float* rear_dists) {
  const int Kr = K - K_keep;
  const int64_t n2 = n - n1;
  if (K < 1 || K_keep < 0 || K_keep > K || n1 < 0 || n2 < 0) return ORC_ERR_INVALID;
  if (mode == ORC_SYMMETRIC && (n1 < K + 1 || n2 < K + 1 || n1 < Kr || n2 < Kr))
    return ORC_ERR_INVALID;
  if (mode == ORC_JOINT && (n < K + 1 || (n1 > 0 && (n1 < K + 1 || n2 < Kr))))
    return ORC_ERR_INVALID;
  int32_t* tmp_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  float* tmp_d = (float*)malloc(sizeof(float) * (size_t)K);
  int32_t* drawn = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  if (!tmp_ids || !tmp_d || !drawn) {
    free(tmp_ids); free(tmp_d); free(drawn);
    return ORC_ERR_NOMEM;
  }
  int rc = ORC_OK;
  for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
    int32_t* L = ids + (size_t)i * K;
    float* D = dists + (size_t)i * K;
    int32_t* R = Kr > 0 ? rear_ids + (size_t)i * Kr : NULL;
    float* RD = Kr > 0 ? rear_dists + (size_t)i * Kr : NULL;
    for (int j = 0; j < K; ++j) flags[(size_t)i * K + j] = FLAG_NEW;
    for (int j = 0; j < Kr; ++j) { R[j] = -1; RD[j] = INFINITY; }
    const int32_t* in = NULL;
    int64_t own_base = 0, own_n = 0;
    if (i < n1) { in = G1 + (size_t)i * K; own_base = 0; own_n = n1; }
    else if (mode == ORC_SYMMETRIC) { in = G2 + (size_t)(i - n1) * K; own_base = n1; own_n = n2; }
    if (in) {
      /* Divide: recompute distances, sort, keep the top K_keep, rear the rest. */
      for (int j = 0; j < K; ++j) {
        int32_t loc = in[j];
        if (loc < 0 || loc >= own_n || own_base + loc == i) { rc = ORC_ERR_INVALID; break; }
        for (int a = 0; a < j; ++a)
          if (in[a] == loc) rc = ORC_ERR_INVALID;
        tmp_ids[j] = (int32_t)(own_base + loc);
        tmp_d[j] = orc_distance(metric, row(X, i, d), row(X, own_base + loc, d), d);
      }
      if (rc != ORC_OK) break;
      sort_entries(tmp_ids, tmp_d, K);
      for (int j = 0; j < K_keep; ++j) { L[j] = tmp_ids[j]; D[j] = tmp_d[j]; }
      for (int j = 0; j < Kr; ++j) { R[j] = tmp_ids[K_keep + j]; RD[j] = tmp_d[K_keep + j]; }
      /* Append: K - K_keep random members of the other set. */
      int64_t base = (i < n1) ? n1 : 0;
      int64_t n_src = (i < n1) ? n2 : n1;
      draw_random(seed, i, base, n_src, Kr, K, drawn);
      for (int j = 0; j < Kr; ++j) {
        L[K_keep + j] = drawn[j];
        D[K_keep + j] = orc_distance(metric, row(X, i, d), row(X, drawn[j], d), d);
      }
    } else {
      /* Initialize (Alg. 2): K random members of S1 u S2. */
      draw_random(seed, i, 0, n, K, K, drawn);
      for (int j = 0; j < K; ++j) {
        L[j] = drawn[j];
        D[j] = orc_distance(metric, row(X, i, d), row(X, drawn[j], d), d);
      }
    }
    sort_entries(L, D, K);
  }
  free(tmp_ids); free(tmp_d); free(drawn);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Round step 1: Reverse(G) and the sampled new/old sets of each node      */
/* ------------------------------------------------------------------ */

typedef struct { uint64_t key; int32_t id; } keyed_t;

static int cmp_keyed(const void* a, const void* b) {
  uint64_t x = ((const keyed_t*)a)->key, y = ((const keyed_t*)b)->key;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static int contains(const int32_t* a, int m, int32_t v) {
  for (int j = 0; j < m; ++j)
    if (a[j] == v) return 1;
  return 0;
}

/* Fills new_ids[n][cap_new] / old_ids[n][cap_old] with counts; flips the flags
 * of the sampled forward-new entries to old (not in literal mode). */
int orc_sample(int64_t n, int K, const int32_t* ids, uint8_t* flags, uint64_t seed, int t, int s,
               int literal, int cap_new, int cap_old, int32_t* new_ids, int32_t* new_cnt,
               int32_t* old_ids, int32_t* old_cnt) {
  int rc = ORC_OK;
  /* Forward sets. fwd_kind: 0 not used, 1 forward-new, 2 forward-old. */
  uint8_t* fwd_kind = (uint8_t*)calloc((size_t)n * K, 1);
  keyed_t* cand = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)K);
  int64_t* rn_cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* ro_cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!fwd_kind || !cand || !rn_cnt || !ro_cnt) { rc = ORC_ERR_NOMEM; goto out_early; }
  for (int64_t u = 0; u < n; ++u) {
    const int32_t* L = ids + (size_t)u * K;
    uint8_t* F = flags + (size_t)u * K;
    uint8_t* kind = fwd_kind + (size_t)u * K;
    if (literal) {
      for (int j = 0; j < K; ++j) kind[j] = 1;
      continue;
    }
    int m = 0;
    for (int j = 0; j < K; ++j) {
      if (F[j] == FLAG_NEW) { cand[m].key = sample_key(seed, t, STREAM_FWD_NEW, u, L[j]); cand[m].id = j; ++m; }
      else kind[j] = 2;
    }
    qsort(cand, (size_t)m, sizeof(keyed_t), cmp_keyed);
    for (int a = 0; a < m && a < s; ++a) { kind[cand[a].id] = 1; F[cand[a].id] = FLAG_OLD; }
  }
  /* Reverse(G): count, then fill the in-lists. */
  for (int64_t u = 0; u < n; ++u)
    for (int j = 0; j < K; ++j) {
      int32_t v = ids[(size_t)u * K + j];
      if (fwd_kind[(size_t)u * K + j] == 1) rn_cnt[v + 1]++;
      if (fwd_kind[(size_t)u * K + j] == 2) ro_cnt[v + 1]++;
    }
  for (int64_t v = 0; v < n; ++v) { rn_cnt[v + 1] += rn_cnt[v]; ro_cnt[v + 1] += ro_cnt[v]; }
  {
    keyed_t* rn = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(rn_cnt[n] + 1));
    keyed_t* ro = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)(ro_cnt[n] + 1));
    int64_t* rn_fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* ro_fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!rn || !ro || !rn_fill || !ro_fill) {
      free(rn); free(ro); free(rn_fill); free(ro_fill);
      rc = ORC_ERR_NOMEM;
      goto out_early;
    }
    memcpy(rn_fill, rn_cnt, sizeof(int64_t) * (size_t)(n + 1));
    memcpy(ro_fill, ro_cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t u = 0; u < n; ++u)
      for (int j = 0; j < K; ++j) {
        int32_t v = ids[(size_t)u * K + j];
        uint8_t kind = fwd_kind[(size_t)u * K + j];
        if (kind == 1) {
          keyed_t* e = &rn[rn_fill[v]++];
          e->id = (int32_t)u;
          e->key = sample_key(seed, t, STREAM_REV_NEW, v, (int32_t)u);
        } else if (kind == 2) {
          keyed_t* e = &ro[ro_fill[v]++];
          e->id = (int32_t)u;
          e->key = sample_key(seed, t, STREAM_REV_OLD, v, (int32_t)u);
        }
      }
    /* Per node: forward part, then the s smallest reverse keys, deduplicated. */
    for (int64_t u = 0; u < n && rc == ORC_OK; ++u) {
      const int32_t* L = ids + (size_t)u * K;
      const uint8_t* kind = fwd_kind + (size_t)u * K;
      int32_t* NW = new_ids + (size_t)u * cap_new;
      int32_t* OL = old_ids + (size_t)u * cap_old;
      int nn = 0, no = 0;
      for (int j = 0; j < K; ++j)
        if (kind[j] == 1) {
          if (nn >= cap_new) { rc = ORC_ERR_CAPACITY; break; }
          NW[nn++] = L[j];
        }
      int64_t b = rn_cnt[u], e = rn_cnt[u + 1];
      qsort(rn + b, (size_t)(e - b), sizeof(keyed_t), cmp_keyed);
      int64_t take = literal ? (e - b) : (e - b < s ? e - b : s);
      for (int64_t a = 0; a < take && rc == ORC_OK; ++a) {
        int32_t v = rn[b + a].id;
        if (contains(NW, nn, v)) continue;
        if (nn >= cap_new) { rc = ORC_ERR_CAPACITY; break; }
        NW[nn++] = v;
      }
      for (int j = 0; j < K && rc == ORC_OK; ++j)
        if (kind[j] == 2 && !contains(NW, nn, L[j]) && !contains(OL, no, L[j])) {
          if (no >= cap_old) { rc = ORC_ERR_CAPACITY; break; }
          OL[no++] = L[j];
        }
      b = ro_cnt[u]; e = ro_cnt[u + 1];
      qsort(ro + b, (size_t)(e - b), sizeof(keyed_t), cmp_keyed);
      take = e - b < s ? e - b : s;
      for (int64_t a = 0; a < take && rc == ORC_OK; ++a) {
        int32_t v = ro[b + a].id;
        if (contains(NW, nn, v) || contains(OL, no, v)) continue;
        if (no >= cap_old) { rc = ORC_ERR_CAPACITY; break; }
        OL[no++] = v;
      }
      new_cnt[u] = nn;
      old_cnt[u] = no;
    }
    free(rn); free(ro); free(rn_fill); free(ro_fill);
  }
out_early:
  free(fwd_kind); free(cand); free(rn_cnt); free(ro_cnt);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Round step 2: local join and UpdateNN (Alg. 1 / Alg. 2 inner loops)     */
/* ------------------------------------------------------------------ */

static int pair_allowed(int mode, int64_t n1, int32_t p, int32_t q) {
  int p1 = p < n1, q1 = q < n1;
  if (mode == ORC_SYMMETRIC) return p1 != q1;
  return !(p1 && q1);
}

static void evaluate_pair(const float* X, int d, int metric, int K, int32_t* ids, float* dists,
                          uint8_t* flags, int32_t p, int32_t q) {
  float l = orc_distance(metric, row(X, p, d), row(X, q, d), d);
  update_nn(ids + (size_t)p * K, dists + (size_t)p * K, flags + (size_t)p * K, K, q, l);
  update_nn(ids + (size_t)q * K, dists + (size_t)q * K, flags + (size_t)q * K, K, p, l);
}

int orc_join(int mode, const float* X, int64_t n, int64_t n1, int d, int metric, int K,
             int32_t* ids, float* dists, uint8_t* flags, int cap_new, int cap_old,
             const int32_t* new_ids, const int32_t* new_cnt, const int32_t* old_ids,
             const int32_t* old_cnt, int64_t* c_out, int64_t* evals_out) {
  int32_t* start = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * K);
  if (!start) return ORC_ERR_NOMEM;
  memcpy(start, ids, sizeof(int32_t) * (size_t)n * K);
  int64_t evals = 0;
  for (int64_t u = 0; u < n; ++u) {
    const int32_t* NW = new_ids + (size_t)u * cap_new;
    const int32_t* OL = old_ids + (size_t)u * cap_old;
    for (int i = 0; i < new_cnt[u]; ++i) {
      int32_t p = NW[i];
      for (int j = i + 1; j < new_cnt[u]; ++j) {
        int32_t q = NW[j];
        if (!pair_allowed(mode, n1, p, q)) continue;
        ++evals;
        evaluate_pair(X, d, metric, K, ids, dists, flags, p, q);
      }
      for (int j = 0; j < old_cnt[u]; ++j) {
        int32_t q = OL[j];
        if (p == q || !pair_allowed(mode, n1, p, q)) continue;
        ++evals;
        evaluate_pair(X, d, metric, K, ids, dists, flags, p, q);
      }
    }
  }
  int64_t c = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int j = 0; j < K; ++j)
      if (!contains(start + (size_t)v * K, K, ids[(size_t)v * K + j])) ++c;
  free(start);
  *c_out = c;
  *evals_out = evals;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Final step: Merge and Sort with the rear lists                          */
/* ------------------------------------------------------------------ */

int orc_final(int64_t n, int K, const int32_t* ids, const float* dists, int Kr,
              const int32_t* rear_ids, const float* rear_dists, int32_t* out_ids, float* out_dists) {
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(K + Kr + 1));
  float* cd = (float*)malloc(sizeof(float) * (size_t)(K + Kr + 1));
  if (!ci || !cd) { free(ci); free(cd); return ORC_ERR_NOMEM; }
  for (int64_t v = 0; v < n; ++v) {
    int m = 0;
    for (int j = 0; j < K; ++j) { ci[m] = ids[(size_t)v * K + j]; cd[m] = dists[(size_t)v * K + j]; ++m; }
    for (int j = 0; j < Kr; ++j) {
      int32_t id = rear_ids[(size_t)v * Kr + j];
      if (id < 0) continue;
      ci[m] = id; cd[m] = rear_dists[(size_t)v * Kr + j]; ++m;
    }
    sort_entries(ci, cd, m);
    int w = 0;
    for (int a = 0; a < m && w < K; ++a) {
      if (contains(out_ids + (size_t)v * K, w, ci[a])) continue;
      out_ids[(size_t)v * K + w] = ci[a];
      out_dists[(size_t)v * K + w] = cd[a];
      ++w;
    }
  }
  free(ci); free(cd);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Whole merges: Alg. 1 (mode ORC_SYMMETRIC), Alg. 2 (ORC_JOINT), build   */
/* (ORC_JOINT with n1 = 0, which is NN-Descent).                           */
/* ------------------------------------------------------------------ */

int orc_merge(int mode, const float* X, int64_t n, int64_t n1, int d, int metric,
              const int32_t* G1, const int32_t* G2, int K, float keep_ratio, float sample_rate,
              int max_iters, float delta, uint64_t seed, int literal, int32_t* out_ids,
              float* out_dists, int64_t* c_hist, int64_t* evals_hist, int* rounds_out) {
  int K_keep = (int)((double)keep_ratio * (double)K);
  if (mode == ORC_JOINT && n1 == 0) K_keep = K;
  int Kr = K - K_keep;
  int s = (int)((double)sample_rate * (double)K);
  if (s < 1) s = 1;
  int cap_new = literal ? (int)(n < 2147483647 ? n : 2147483647) : 2 * s;
  int cap_old = literal ? 1 : K + s;
  size_t nk = (size_t)n * K;
  int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * nk);
  float* dists = (float*)malloc(sizeof(float) * nk);
  uint8_t* flags = (uint8_t*)malloc(nk);
  int32_t* rear_ids = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n * Kr + 1));
  float* rear_dists = (float*)malloc(sizeof(float) * ((size_t)n * Kr + 1));
  int32_t* new_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * cap_new);
  int32_t* old_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * cap_old);
  int32_t* new_cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* old_cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int rc = ORC_OK;
  int rounds = 0;
  if (!ids || !dists || !flags || !rear_ids || !rear_dists || !new_ids || !old_ids || !new_cnt ||
      !old_cnt) {
    rc = ORC_ERR_NOMEM;
    goto done;
  }
  rc = orc_init(mode, X, n, n1, d, metric, G1, G2, K, K_keep, seed, ids, dists, flags, rear_ids,
                rear_dists);
  if (rc != ORC_OK) goto done;
  for (int t = 1; t <= max_iters; ++t) {
    rc = orc_sample(n, K, ids, flags, seed, t, s, literal, cap_new, cap_old, new_ids, new_cnt,
                    old_ids, old_cnt);
    if (rc != ORC_OK) goto done;
    int64_t c = 0, evals = 0;
    rc = orc_join(mode, X, n, n1, d, metric, K, ids, dists, flags, cap_new, cap_old, new_ids,
                  new_cnt, old_ids, old_cnt, &c, &evals);
    if (rc != ORC_OK) goto done;
    if (c_hist) c_hist[t - 1] = c;
    if (evals_hist) evals_hist[t - 1] = evals;
    rounds = t;
    if ((double)c <= (double)delta * (double)n * (double)K) break;
  }
  rc = orc_final(n, K, ids, dists, Kr, rear_ids, rear_dists, out_ids, out_dists);
done:
  if (rounds_out) *rounds_out = rounds;
  free(ids); free(dists); free(flags); free(rear_ids); free(rear_dists);
  free(new_ids); free(old_ids); free(new_cnt); free(old_cnt);
  return rc;
}

/* ------------------------------------------------------------------ */
/* H-Merge sampling order (Sec. 3.3: each joined block is drawn at random   */
/* from the whole set).  Reading: position r holds row perm[r], perm a      */
/* bijection of [0, n) made by a 4-round Feistel network on b bits (b even, */
/* 2^b >= n, b >= 2) whose round function is H(seed, round, 7, right half,  */
/* 0) masked to b/2 bits, cycle-walked back into [0, n).                    */
/* ------------------------------------------------------------------ */

static uint64_t feistel(uint64_t x, int half, uint64_t seed) {
  const uint64_t mask = (1ull << half) - 1ull;
  uint64_t L = x >> half, R = x & mask;
  for (int r = 0; r < 4; ++r) {
    const uint64_t t = R;
    R = L ^ (orc_hash(seed, (uint64_t)r, 7, R, 0) & mask);
    L = t;
  }
  return (L << half) | R;
}

int orc_permute(int64_t n, uint64_t seed, int32_t* perm) {
  if (n < 1) return ORC_ERR_INVALID;
  int b = 2;
  while ((1ll << b) < n) b += 2;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t y = feistel((uint64_t)i, b / 2, seed);
    while (y >= (uint64_t)n) y = feistel(y, b / 2, seed);
    perm[i] = (int32_t)y;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Brute force: exact k-NN graph and the brute-force merge of Sec. 1       */
/* ------------------------------------------------------------------ */

/* Exact k-NN lists in entry order, from every pair's canonical distance. */
int orc_bruteforce_knn(const float* X, int64_t n, int d, int metric, int K, int32_t* ids,
                       float* dists) {
  for (int64_t i = 0; i < n; ++i) {
    int32_t* L = ids + (size_t)i * K;
    float* D = dists + (size_t)i * K;
    for (int j = 0; j < K; ++j) { L[j] = -1; D[j] = INFINITY; }
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      update_nn(L, D, NULL, K, (int32_t)j, orc_distance(metric, row(X, i, d), row(X, j, d), d));
    }
  }
  return ORC_OK;
}

/* Sec. 1: cross-compare every x_i in S1 with every y_j in S2 and insert the
 * edge into G1[i] and G2[j] when it ranks in the top k.  G1/G2 ids are local;
 * the output uses global ids (S1 first). */
int orc_bruteforce_merge(const float* X, int64_t n, int64_t n1, int d, int metric,
                         const int32_t* G1, const int32_t* G2, int K, int32_t* out_ids,
                         float* out_dists) {
  for (int64_t i = 0; i < n; ++i) {
    int32_t* L = out_ids + (size_t)i * K;
    float* D = out_dists + (size_t)i * K;
    for (int j = 0; j < K; ++j) {
      int32_t g = i < n1 ? G1[(size_t)i * K + j] : (int32_t)(n1 + G2[(size_t)(i - n1) * K + j]);
      L[j] = g;
      D[j] = orc_distance(metric, row(X, i, d), row(X, g, d), d);
    }
    sort_entries(L, D, K);
  }
  for (int64_t i = 0; i < n1; ++i)
    for (int64_t j = n1; j < n; ++j) {
      float l = orc_distance(metric, row(X, i, d), row(X, j, d), d);
      update_nn(out_ids + (size_t)i * K, out_dists + (size_t)i * K, NULL, K, (int32_t)j, l);
      update_nn(out_ids + (size_t)j * K, out_dists + (size_t)j * K, NULL, K, (int32_t)i, l);
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Graph diversification (Alg. 3, Sec. 3.4), run on a finished k-NN graph. */
/* Readings:                                                               */
/*   - A list is examined in (distance, id) order.  Its first entry is     */
/*     kept; a later entry s is dropped as soon as one kept entry c has    */
/*     m(s, c) < m(s, owner), else kept (Alg. 3: a strict "<" occludes).   */
/*   - The reverse list of a is {b : a in G[b]} with distance m(a, b), in  */
/*     (distance, id) order, taken from the input graph; it is            */
/*     diversified by the same rule on its own.                           */
/*   - "Merged": the union of both kept sets without repeats, in           */
/*     (distance, id) order, cut to the first max_degree entries and       */
/*     padded with id -1 / distance +inf.                                  */
/* ------------------------------------------------------------------ */

/* Alg. 3 on one list in entry order; the kept entries are moved to the front
 * (in order) and their count is returned.  Stops once max_keep are kept: no
 * later entry could reach the first max_keep of the union. */
static int diversify_list(const float* X, int d, int metric, int32_t* ids, float* dists, int m,
                          int max_keep, uint64_t* evals) {
  int kept = 0;
  for (int i = 0; i < m && kept < max_keep; ++i) {
    int occluded = 0;
    for (int c = 0; c < kept && !occluded; ++c) {
      ++*evals;
      occluded = orc_distance(metric, row(X, ids[i], d), row(X, ids[c], d), d) < dists[i];
    }
    if (!occluded) {
      ids[kept] = ids[i];
      dists[kept] = dists[i];
      ++kept;
    }
  }
  return kept;
}

/* Diversified lists of the rows listed in `rows` (all rows when rows is NULL,
 * n_rows = n).  G [n][K] is a k-NN graph (ids in [0, n), no self, no repeats
 * per row).  out_ids/out_dists [n_rows][max_degree], out_deg [n_rows];
 * evals (may be NULL) receives the distance evaluations of Alg. 3's loops. */
int orc_diversify(const float* X, int64_t n, int d, int metric, const int32_t* G, int K,
                  int max_degree, const int64_t* rows, int64_t n_rows, int32_t* out_ids,
                  float* out_dists, int32_t* out_deg, uint64_t* evals) {
  if (n < 1 || K < 1 || max_degree < 1) return ORC_ERR_INVALID;
  /* reverse lists of the whole graph (counting sort by target) */
  int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* src = (int32_t*)malloc((size_t)n * K * sizeof(int32_t));
  int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t max_in = 0;
  if (!start || !src || !fill) {
    free(start); free(src); free(fill);
    return ORC_ERR_NOMEM;
  }
  for (int64_t i = 0; i < (int64_t)n * K; ++i) {
    if (G[i] < 0 || G[i] >= n) { free(start); free(src); free(fill); return ORC_ERR_INVALID; }
    start[G[i] + 1]++;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (start[i + 1] > max_in) max_in = start[i + 1];
    start[i + 1] += start[i];
  }
  for (int64_t i = 0; i < n; ++i) fill[i] = start[i];
  for (int64_t b = 0; b < n; ++b)
    for (int j = 0; j < K; ++j) src[fill[G[(size_t)b * K + j]]++] = (int32_t)b;
  const int cap = (int)(max_in > K ? max_in : K);
  int32_t* fi = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  float* fd = (float*)malloc(sizeof(float) * (size_t)K);
  int32_t* ri = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  float* rd = (float*)malloc(sizeof(float) * (size_t)cap);
  uint64_t ev = 0;
  int rc = ORC_OK;
  if (!fi || !fd || !ri || !rd) rc = ORC_ERR_NOMEM;
  const int64_t count = rows ? n_rows : n;
  for (int64_t r = 0; r < count && rc == ORC_OK; ++r) {
    const int64_t a = rows ? rows[r] : r;
    if (a < 0 || a >= n) { rc = ORC_ERR_INVALID; break; }
    for (int j = 0; j < K; ++j) {
      fi[j] = G[(size_t)a * K + j];
      fd[j] = orc_distance(metric, row(X, a, d), row(X, fi[j], d), d);
      if (fi[j] == a) rc = ORC_ERR_INVALID;
      for (int c = 0; c < j; ++c)
        if (fi[c] == fi[j]) rc = ORC_ERR_INVALID;
    }
    if (rc != ORC_OK) break;
    sort_entries(fi, fd, K);
    const int nf = diversify_list(X, d, metric, fi, fd, K, K, &ev);
    const int m = (int)(start[a + 1] - start[a]);
    for (int j = 0; j < m; ++j) {
      ri[j] = src[start[a] + j];
      rd[j] = orc_distance(metric, row(X, a, d), row(X, ri[j], d), d);
    }
    sort_entries(ri, rd, m);
    const int nr = diversify_list(X, d, metric, ri, rd, m, max_degree, &ev);
    /* union of two entry-ordered lists; one id has one distance, so a repeat
     * is an equal entry */
    int32_t* oi = out_ids + (size_t)r * max_degree;
    float* od = out_dists + (size_t)r * max_degree;
    int x = 0, y = 0, k = 0;
    while (k < max_degree && (x < nf || y < nr)) {
      int take_f;
      if (x < nf && y < nr) {
        if (fi[x] == ri[y]) { ++y; continue; }
        take_f = entry_less(fd[x], fi[x], rd[y], ri[y]);
      } else {
        take_f = x < nf;
      }
      if (take_f) { oi[k] = fi[x]; od[k] = fd[x]; ++x; }
      else { oi[k] = ri[y]; od[k] = rd[y]; ++y; }
      ++k;
    }
    out_deg[r] = k;
    for (; k < max_degree; ++k) { oi[k] = -1; od[k] = INFINITY; }
  }
  if (evals) *evals = ev;
  free(start); free(src); free(fill); free(fi); free(fd); free(ri); free(rd);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Top-down search on the hierarchy (Sec. 3.4).  Readings:                */
/*   - Layers run from the top (fewest rows) to the bottom; layer l holds   */
/*     the first layer_rows[l] rows of X and a graph of layer_width[l]      */
/*     entries per row (ids < 0 are padding and skipped).                  */
/*   - Query q starts at row H(seed, 0, 9, q, 0) mod layer_rows[0] (q its  */
/*     index in the batch; qidx, when given, supplies it per query).       */
/*   - Above the bottom: greedy.  All neighbours of the current row are    */
/*     compared with the query; the current row moves to the nearest of   */
/*     them while that one ranks before it in (distance, id) order.        */
/*   - Bottom: best-first over a rank list of at most ef entries in        */
/*     (distance, id) order, seeded with the row the upper layers reached. */
/*     The first unexpanded entry is expanded: each neighbour not seen     */
/*     before is compared and enters the list when the list has room or    */
/*     it ranks before the last entry (which then leaves).  The search     */
/*     stops when every entry of the list is expanded; the first k_out     */
/*     entries are the result (-1 / +inf padding when fewer).              */
/* ------------------------------------------------------------------ */

int orc_search(const float* X, int64_t n, int d, int metric, int n_layers,
               const int64_t* layer_rows, const int32_t* layer_width, const int32_t* graphs,
               const float* Q, int64_t nq, const int64_t* qidx, int ef, int k_out,
               uint64_t seed, int32_t* out_ids, float* out_dists, uint64_t* out_evals) {
  if (n < 1 || n_layers < 1 || ef < 1 || k_out < 1 || k_out > ef) return ORC_ERR_INVALID;
  if (layer_rows[n_layers - 1] != n) return ORC_ERR_INVALID;
  const int32_t** G = (const int32_t**)malloc(sizeof(int32_t*) * (size_t)n_layers);
  uint8_t* seen = (uint8_t*)malloc((size_t)n);
  int32_t* li = (int32_t*)malloc(sizeof(int32_t) * ((size_t)ef + 1));
  float* ld = (float*)malloc(sizeof(float) * ((size_t)ef + 1));
  uint8_t* done = (uint8_t*)malloc((size_t)ef + 1);
  if (!G || !seen || !li || !ld || !done) {
    free(G); free(seen); free(li); free(ld); free(done);
    return ORC_ERR_NOMEM;
  }
  const int32_t* g = graphs;
  for (int l = 0; l < n_layers; ++l) {
    G[l] = g;
    g += (size_t)layer_rows[l] * layer_width[l];
  }
  for (int64_t q = 0; q < nq; ++q) {
    const float* x = row(Q, q, d);
    uint64_t ev = 1;
    const uint64_t qi = (uint64_t)(qidx ? qidx[q] : q);
    int32_t cur = (int32_t)(orc_hash(seed, 0, 9, qi, 0) % (uint64_t)layer_rows[0]);
    float dcur = orc_distance(metric, x, row(X, cur, d), d);
    for (int l = 0; l + 1 < n_layers; ++l) {
      const int w = layer_width[l];
      for (;;) {
        int32_t best = cur;
        float db = dcur;
        for (int j = 0; j < w; ++j) {
          const int32_t v = G[l][(size_t)cur * w + j];
          if (v < 0) continue;
          const float dv = orc_distance(metric, x, row(X, v, d), d);
          ++ev;
          if (entry_less(dv, v, db, best)) { best = v; db = dv; }
        }
        if (best == cur) break;
        cur = best;
        dcur = db;
      }
    }
    const int w = layer_width[n_layers - 1];
    const int32_t* Gb = G[n_layers - 1];
    memset(seen, 0, (size_t)n);
    seen[cur] = 1;
    int m = 1;
    li[0] = cur; ld[0] = dcur; done[0] = 0;
    for (;;) {
      int e = 0;
      while (e < m && done[e]) ++e;
      if (e == m) break;
      done[e] = 1;
      const int32_t u = li[e];
      for (int j = 0; j < w; ++j) {
        const int32_t v = Gb[(size_t)u * w + j];
        if (v < 0 || seen[v]) continue;
        seen[v] = 1;
        const float dv = orc_distance(metric, x, row(X, v, d), d);
        ++ev;
        if (m == ef && !entry_less(dv, v, ld[m - 1], li[m - 1])) continue;
        int p = m < ef ? m++ : ef - 1;
        while (p > 0 && entry_less(dv, v, ld[p - 1], li[p - 1])) {
          li[p] = li[p - 1]; ld[p] = ld[p - 1]; done[p] = done[p - 1];
          --p;
        }
        li[p] = v; ld[p] = dv; done[p] = 0;
      }
    }
    for (int j = 0; j < k_out; ++j) {
      out_ids[(size_t)q * k_out + j] = j < m ? li[j] : -1;
      out_dists[(size_t)q * k_out + j] = j < m ? ld[j] : INFINITY;
    }
    if (out_evals) out_evals[q] = ev;
  }
  free(G); free(seen); free(li); free(ld); free(done);
  return ORC_OK;
}
