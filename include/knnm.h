/*
 * knnm.h -- C ABI of the GB300 k-NN graph merge library (libknnm.so).
 *
 * The library merges approximate k-NN graphs as in Zhao, Wang, Lin and Ngo,
 * "On the Merge of k-NN Graph":
 *   - knnm_merge_symmetric: Symmetric Merge (S-Merge, Alg. 1, Sec. 3.1): two
 *     graphs G1 on S1 and G2 on S2 become one graph on S1 u S2.
 *   - knnm_merge_joint: Joint Merge (J-Merge, Alg. 2, Sec. 3.2): a graph G1 on
 *     S1 is expanded with a raw set S2.
 *   - knnm_build: J-Merge with an empty existing graph, i.e. NN-Descent, used
 *     to make input graphs.
 *   - knnm_*_sets: the same three merges on itemsets under the Jaccard
 *     distance (the paper's Kosarak experiments), rows as CSR arrays.
 *   - knnm_merge_tree: a graph over many parts by levels of pairwise S-Merges;
 *     knnm_hmerge: the H-Merge hierarchy (Sec. 3.3).
 *   - knnm_diversify, knnm_search(_prepare): graph diversification (Alg. 3)
 *     and the top-down search on the hierarchy (Sec. 3.4).
 *   - knnm_server_*: J-Merge applied to a stream of raw batches against a
 *     resident graph.
 * plus one entry point per step of a merge round (knnm_step_*) so that each
 * step can be checked on its own.
 *
 * Conventions shared by every call
 *   - Return value: KNNM_OK (0) or a negative KNNM_ERR_* code.  No C++
 *     exception crosses the ABI.  The message of the last failure of a context
 *     is returned by knnm_last_error().
 *   - Vectors are row-major float32 [n][d].  Graph ids are int32 [n][k]; input
 *     graphs hold ids local to their own set (0..n_set-1), outputs hold global
 *     ids with S1 rows first, then S2 rows.
 *   - Output lists are sorted by (distance, id) ascending, ids unique, no self.
 *     Distances are the library's canonical FP32 distances: one accumulator,
 *     dimensions in index order, fused multiply-add per term.  KNNM_L2 is the
 *     squared Euclidean distance (same ranking as l2), KNNM_IP is 0 - a.b,
 *     KNNM_COS is 1 - a.b/(|a||b|) (1 when a norm is zero), KNNM_L1 is the sum of
 *     |a_t - b_t| in index order, KNNM_CHI2 the sum of (a_t - b_t)^2 / (a_t + b_t)
 *     in index order (0 for a term with a_t + b_t = 0; the chi-square distance of
 *     the paper's NUSWide experiments, meant for non-negative rows).  Inputs
 *     must be finite.
 *   - knnm_merge_* and knnm_build accept host or device pointers for every
 *     array argument (the library asks the CUDA runtime which one each is).
 *     Host inputs are copied to the device and host outputs copied back inside
 *     the call.  The step entry points take device pointers only.
 *   - The caller owns every array it passes.  The library owns only its
 *     scratch, which the context keeps and reuses between calls.
 *   - Every call runs on the context's stream and has finished when it
 *     returns.  Calls on one context must not overlap.
 */
#ifndef KNNM_H
#define KNNM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  KNNM_OK = 0,
  KNNM_ERR_INVALID = -1,   /* bad argument or malformed input graph */
  KNNM_ERR_NOMEM = -2,     /* device or host allocation failed */
  KNNM_ERR_CUDA = -3,      /* a CUDA runtime call failed */
  KNNM_ERR_TIMEOUT = -4,   /* a bounded device or host wait ran out */
  KNNM_ERR_NOT_READY = -5, /* serving: the request has not completed yet */
  KNNM_ERR_DEVICE = -6     /* a kernel reported an internal error */
};

typedef enum {
  KNNM_L2 = 0,
  KNNM_IP = 1,
  KNNM_COS = 2,
  KNNM_L1 = 3,
  KNNM_CHI2 = 4,
  KNNM_JACCARD = 5 /* sets only: the knnm_*_sets entry points */
} knnm_metric;

/* KNNM_FP32: every distance is the canonical FP32 distance, one thread per pair
 * on the CUDA cores.  KNNM_BF16_RERANK: distances are first estimated from
 * BF16 copies of the vectors on the tensor cores (FP32 accumulation); a pair is
 * re-computed canonically in FP32 whenever a proven error bound cannot rule it
 * out, so the merged graph is identical to the KNNM_FP32 one.
 * KNNM_FP16_RERANK: the same with FP16 copies: 3 more mantissa bits, so the
 * bound is about 8x tighter and far fewer pairs need the re-rank on data of
 * moderate range (a row with a value beyond +-65504 re-ranks every pair).  Rows
 * of small non-negative integers (<= 256 in BF16, <= 2048 in FP16) are exact
 * on the tensor cores and never re-ranked.  L1 and CHI2 have no tensor-core
 * form and always run as KNNM_FP32. */
typedef enum { KNNM_FP32 = 0, KNNM_BF16_RERANK = 1, KNNM_FP16_RERANK = 2 } knnm_precision;

typedef struct {
  int k;             /* list length K, 1..32 (Alg. 1 Data line: k-NN graphs) */
  int metric;        /* knnm_metric */
  int precision;     /* knnm_precision */
  int max_iters;     /* cap on local-join rounds, 1..KNNM_MAX_ROUNDS */
  float sample_rate; /* rho: each round samples s = max(1, floor(rho*K)) new entries */
  float keep_ratio;  /* r of Sec. 5.2.1: K_keep = floor(r*K) entries survive Divide */
  float delta;       /* stop once a round changes <= delta*N*K list entries */
  uint64_t seed;     /* seed of every random draw (init and sampling) */
} knnm_params;

#define KNNM_MAX_ROUNDS 64

typedef struct {
  int rounds;                             /* rounds run */
  int kernel_launches;                    /* kernels the call launched */
  int64_t updates[KNNM_MAX_ROUNDS];       /* c_t: entries new to the lists after round t */
  int64_t dist_evals[KNNM_MAX_ROUNDS];    /* pairs compared in round t (scanning rate C) */
  int64_t proposals[KNNM_MAX_ROUNDS];     /* edges offered to UpdateNN after the k-th filter */
  int64_t reranked[KNNM_MAX_ROUNDS];      /* BF16 path: pairs re-computed in FP32 */
  int64_t gathered[KNNM_MAX_ROUNDS];      /* candidate rows staged by the join (sum of |new|+|old|) */
  float ms_sample[KNNM_MAX_ROUNDS];       /* device time of the sampler kernels in round t */
  float ms_join[KNNM_MAX_ROUNDS];         /* device time of the join kernel in round t */
  float ms_update[KNNM_MAX_ROUNDS];       /* device time of the top-k insert + flag pass */
  float ms_init, ms_rounds, ms_final;     /* device time of init, all rounds, final merge */
  float ms_total;                         /* wall time of the call */
  uint64_t tc_rounds;                     /* bit t-1 set: round t ran the tensor-core join */
  int64_t spilled[KNNM_MAX_ROUNDS];       /* proposals inserted straight into the lists
                                             because the join block's buffer was full */
} knnm_stats;

typedef struct knnm_ctx knnm_ctx;

/* Creates a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL means the legacy default stream). */
int knnm_create(knnm_ctx** out, int device, void* cuda_stream);
/* Frees the context and its scratch. */
int knnm_destroy(knnm_ctx* ctx);
/* Rebinds the context to another stream of the same device. */
int knnm_set_stream(knnm_ctx* ctx, void* cuda_stream);
/* Context options (knnm_set_option; KNNM_ERR_INVALID for an unknown option or
 * a value out of range):
 *   KNNM_OPT_GRAPHS (default 0): when 1, each local-join round of a whole-merge
 *     call (sampler, join, top-k update) is captured once into a CUDA graph
 *     and replayed, one graph launch per round.  Results are identical;
 *     knnm_stats then times each round as a whole (in ms_join; ms_sample and
 *     ms_update stay 0).
 *   KNNM_OPT_BUCKET_CAP (default 0, 0..4096): slots per target for the
 *     proposals a join round offers to UpdateNN; a proposal arriving at a full
 *     bucket is inserted straight into its target's live list by ordered slot
 *     insertion (the same top-K union, without the bucket).  0 takes 12*K
 *     rounded up to 32, within 64..512.  Results do not depend on it; small
 *     values force the direct-insert path.
 *   KNNM_OPT_WAIT_POLLS (default -1, >= -1): polls before a device-side wait of
 *     the join for its staged rows gives up (-1: 2^22).  A wait that gives up
 *     makes the call return KNNM_ERR_DEVICE with error bit 0x8 in its message;
 *     the kernel first lets its copies in flight land, so the context stays
 *     usable.  0 makes every such wait give up at once (tests of that path).
 *   KNNM_OPT_FAIL_ALLOC (default 0, >= 0): the next `value` scratch
 *     reservations of the context fail with KNNM_ERR_NOMEM as if the device
 *     were out of memory (host-side fault injection for tests); the context
 *     and its existing scratch stay usable.
 *   KNNM_OPT_TC_JOIN (default 0, 0..2): with a tensor-core precision, which
 *     join each round runs: 0 chooses per round (the tensor-core join while
 *     its re-rank share stays low, else the FP32 join), 1 always the
 *     tensor-core join, 2 always the FP32 join.  Results do not depend on it. */
enum {
  KNNM_OPT_GRAPHS = 1,
  KNNM_OPT_BUCKET_CAP = 2,
  KNNM_OPT_WAIT_POLLS = 3,
  KNNM_OPT_FAIL_ALLOC = 4,
  KNNM_OPT_TC_JOIN = 5
};
int knnm_set_option(knnm_ctx* ctx, int option, int value);
/* Message of the context's last failure ("" if none).  Owned by the context. */
const char* knnm_last_error(const knnm_ctx* ctx);
/* Static name of an error code. */
const char* knnm_strerror(int code);

/* The library's counter-based hash H(seed, t, stream, owner, member): five
 * chained SplitMix64 steps (Steele, Lea and Flood, OOPSLA 2014), each
 * absorbing one word by xor.  Every random choice of the library is a value
 * of H; e.g. merge j of level l of a merge tree runs with seed
 * H(seed, l, 6, j, 0).  Host function, no context. */
uint64_t knnm_hash64(uint64_t seed, uint64_t t, uint64_t stream, uint64_t owner,
                     uint64_t member);
/* Fills `p` with the defaults: K=20, L2, FP32, 10 rounds, rho=0.5, r=0.5,
 * delta=0.001, seed=0. */
void knnm_default_params(knnm_params* p);

/* S-Merge (Alg. 1).  S1 [n1][d], G1 [n1][K] (ids in 0..n1-1), S2 [n2][d],
 * G2 [n2][K] (ids in 0..n2-1).  out_ids/out_dists [n1+n2][K].  Each input row
 * must hold K distinct ids other than its own; n1, n2 >= K+1 and
 * >= K - floor(r*K).  `stats` may be NULL.  Malformed graphs give
 * KNNM_ERR_INVALID. */
int knnm_merge_symmetric(knnm_ctx* ctx, const float* S1, int64_t n1, const int32_t* G1,
                         const float* S2, int64_t n2, const int32_t* G2, int d,
                         const knnm_params* params, int32_t* out_ids, float* out_dists,
                         knnm_stats* stats);

/* J-Merge (Alg. 2).  S1 [n1][d] with graph G1 [n1][K]; raw rows S_new [n2][d].
 * Output rows: S1 first, then S_new.  n1 >= K+1 (or n1 == 0, which is
 * knnm_build), n1+n2 >= K+1, n2 >= K - floor(r*K) when n1 > 0. */
int knnm_merge_joint(knnm_ctx* ctx, const float* S1, int64_t n1, const int32_t* G1,
                     const float* S_new, int64_t n2, int d, const knnm_params* params,
                     int32_t* out_ids, float* out_dists, knnm_stats* stats);

/* NN-Descent build of S [n][d] (J-Merge with an empty graph); n >= K+1. */
int knnm_build(knnm_ctx* ctx, const float* S, int64_t n, int d, const knnm_params* params,
               int32_t* out_ids, float* out_dists, knnm_stats* stats);

/* The same three merges on sets (the Kosarak itemsets of Sec. 5) under the
 * Jaccard distance 1 - |A n B| / |A u B| (0 for two empty sets), params->metric
 * = KNNM_JACCARD, FP32 only.  All n1 + n2 rows are one CSR array on the device:
 * row i holds items[offsets[i] .. offsets[i+1]), ascending, no repeats,
 * non-negative, fewer than 2^23 per row; offsets [n1 + n2 + 1] starts at 0 and
 * ends at nnz, the length of items.  S1 is rows [0, n1), S2 (or the raw rows)
 * the rest; G1, G2 and the outputs as in the dense calls (host or device).
 * Malformed rows are KNNM_ERR_INVALID. */
int knnm_merge_symmetric_sets(knnm_ctx* ctx, const int64_t* offsets, const int32_t* items,
                              int64_t nnz, int64_t n1, int64_t n2, const int32_t* G1,
                              const int32_t* G2, const knnm_params* params, int32_t* out_ids,
                              float* out_dists, knnm_stats* stats);
int knnm_merge_joint_sets(knnm_ctx* ctx, const int64_t* offsets, const int32_t* items,
                          int64_t nnz, int64_t n1, int64_t n2, const int32_t* G1,
                          const knnm_params* params, int32_t* out_ids, float* out_dists,
                          knnm_stats* stats);
int knnm_build_sets(knnm_ctx* ctx, const int64_t* offsets, const int32_t* items, int64_t nnz,
                    int64_t n, const knnm_params* params, int32_t* out_ids, float* out_dists,
                    knnm_stats* stats);

/* Merge tree (Sec. 1 and Sec. 3: a graph over a large set made from graphs
 * built independently on its parts, by repeated two-graph merges).  S [n][d]
 * is cut into `parts` consecutive parts of part_rows[p] rows each (every part
 * >= K+1 rows); G [n][K] holds each part's graph with ids local to its part.
 * Level by level, neighbouring blocks (0,1), (2,3), ... are joined by S-Merge
 * (Alg. 1) into one block each; an odd last block waits for the next level.
 * Merge j of level l runs with seed H(params->seed, l, 6, j, 0) (the library's
 * counter-based hash).  out_ids/out_dists [n][K] hold global ids.  In `stats`,
 * rounds is the number of levels and entry l of each per-round array sums the
 * merges of level l; ms_* sum over all merges.  parts == 1 returns G with its
 * canonical distances, sorted. */
int knnm_merge_tree(knnm_ctx* ctx, const float* S, int64_t n, int d, int parts,
                    const int64_t* part_rows, const int32_t* G, const knnm_params* params,
                    int32_t* out_ids, float* out_dists, knnm_stats* stats);

/* H-Merge (Sec. 3.3): a hierarchy of graphs on growing random samples of S,
 * built by repeated J-Merge.  The rows are visited in a random order
 * (perm_out[r] = the row of S at position r: a Feistel bijection keyed by
 * params->seed); an NN-Descent graph is built on the first `first_rows`
 * positions, then each step J-Merges the next raw block of as many positions
 * as the graph already has (the whole rest when fewer than k + 1 positions
 * would remain after it), so the graph doubles.  The
 * growing graph keeps k entries per list (J-Merge never compares two rows of
 * the existing graph, so shorter lists could not be refilled); each upper
 * layer is kept as the first k/2 entries of its lists, the bottom one whole.
 * Merge l of the sequence (the build is l = 0) runs with seed
 * H(params->seed, l, 8, 0, 0).
 *   S [n][d] (host or device); first_rows >= k + 1.
 *   perm_out [n]; out_ids/out_dists [n][k]: the bottom graph, rows and ids as
 *   positions (row r is S[perm_out[r]]).
 *   layer_rows[0..n_layers): sizes of upper layers to return (each one of
 *   first_rows * 2^i below n); layer_ids: their lists one after the other,
 *   [layer_rows[i]][k/2] each, ids as positions.
 * stats: rounds = merges run; per-round arrays hold per-merge sums. */
int knnm_hmerge(knnm_ctx* ctx, const float* S, int64_t n, int d, int64_t first_rows,
                const knnm_params* params, int32_t* perm_out, int32_t* out_ids,
                float* out_dists, int n_layers, const int64_t* layer_rows, int32_t* layer_ids,
                knnm_stats* stats);

/* Rows of S in a given order: out[r] = S[perm[r]] for r < n (device pointers;
 * S [n_src][d] with every perm[r] in [0, n_src), out [n][d]).  Used to lay out
 * the H-Merge hierarchy's rows, which the graphs above address by position. */
int knnm_gather_rows(knnm_ctx* ctx, const float* S, int64_t n_src, int d, const int32_t* perm,
                     int64_t n, float* out);

/* ---------------------------------------------------------------------------
 * Graph diversification and the top-down search on the hierarchy (Sec. 3.4).
 * Device pointers only.
 * ------------------------------------------------------------------------- */

typedef struct {
  uint64_t dist_evals;   /* distances computed by the diversification kernels */
  uint64_t edges;        /* sum of the output degrees */
  int64_t full_rows;     /* rows whose degree reached max_degree */
  int64_t max_in_degree; /* largest in-degree of the input graph */
  float ms;              /* device time of the call */
} knnm_gd_stats;

/* Graph diversification (Alg. 3) of the k-NN graph G [n][k] on S [n][d]
 * (ids in [0, n), no self, no repeats in a row; k <= 32), as a post-process.
 * For each row a: its list, in (distance, id) order of the canonical distance
 * of `metric`, keeps its first entry; every later entry s is dropped when an
 * entry already kept is strictly closer to s than a is (m(s, c) < m(s, a)),
 * else kept.  The reverse list {b : a in G[b]}, in the same order, is
 * diversified by the same rule on its own.  The row's output is the union of
 * both kept sets without repeats, in (distance, id) order, cut to max_degree
 * (1..256) entries: out_ids/out_dists [n][max_degree], padded with -1 / +inf
 * after out_degree[a] entries.  A malformed G is KNNM_ERR_INVALID. */
int knnm_diversify(knnm_ctx* ctx, const float* S, int64_t n, int d, const int32_t* G, int k,
                   int metric, int max_degree, int32_t* out_ids, float* out_dists,
                   int32_t* out_degree, knnm_gd_stats* stats);

typedef struct {
  uint64_t dist_evals;     /* query-row distances computed */
  int64_t crowded_queries; /* queries whose visited table filled: some rows were
                              compared again (the results do not change) */
  float ms;                /* device time of the call */
} knnm_search_stats;

/* Per-row data the search reads, row_aux [n][2] floats: {max |x| when every
 * coordinate of the row is an integer of magnitude <= 2^24, else -1; the
 * row's canonical norm}.  Compute it once per row set and pass it to every
 * knnm_search over that set (device pointers). */
int knnm_search_prepare(knnm_ctx* ctx, const float* S, int64_t n, int d, float* row_aux);

/* Top-down k-NN search of the queries Q [nq][d] on a hierarchy of graphs
 * over S [n][d] (Sec. 3.4).  row_aux: knnm_search_prepare's output for S, or
 * NULL to compute it inside the call.  Layer l (0 = top, n_layers - 1 = bottom; at most
 * 32 layers) covers the first layer_rows[l] rows of S (non-decreasing, the
 * bottom one n) with the graph layer_ids[l] [layer_rows[l]][layer_width[l]]
 * (layer_width <= 1024; ids < 0 are padding; other ids must be below
 * layer_rows[l], else KNNM_ERR_INVALID after the call).  layer_ids is a host
 * array of device pointers.  Each query starts at row
 * H(seed, 0, 9, q, 0) mod layer_rows[0] (the library's counter-based hash).
 * Above the bottom it moves greedily: to the nearest neighbour of the current
 * row while that one ranks before it in (distance, id) order.  At the bottom
 * it runs best-first over a rank list of ef entries (k_out <= ef <= 1024):
 * the first unexpanded entry is expanded, each neighbour not compared before
 * enters when the list has room or it ranks before the last entry; it stops
 * when every listed entry is expanded.  out_ids/out_dists [nq][k_out] hold
 * the first k_out entries (-1 / +inf when fewer); out_evals [nq] (may be
 * NULL) the distances each query computed.  Every distance is the canonical
 * one: a row is first compared by a reordered sum, which is used as is only
 * when both rows are small integers (every partial sum exact) and otherwise
 * only to skip rows that provably cannot enter the rank list. */
int knnm_search(knnm_ctx* ctx, const float* S, int64_t n, int d, const float* row_aux,
                int metric, int n_layers,
                const int64_t* layer_rows, const int32_t* layer_width,
                const int32_t* const* layer_ids, const float* Q, int64_t nq, int ef, int k_out,
                uint64_t seed, int32_t* out_ids, float* out_dists, uint32_t* out_evals,
                knnm_search_stats* stats);

/* Device scratch, in bytes, that one whole-merge call of these sizes takes
 * from its context (all arrays on the device).  mode: 0 = S-Merge, 1 = J-Merge
 * (n1 = 0 is the build).  Needs a context because the join configuration
 * depends on the device. */
int knnm_merge_scratch_bytes(knnm_ctx* ctx, int mode, int64_t n1, int64_t n2, int d,
                             const knnm_params* params, uint64_t* bytes);

/* ---------------------------------------------------------------------------
 * Serving: J-Merge (Alg. 2, Sec. 3.2) applied to a stream of raw batches
 * against a graph kept resident on one device.
 *
 * The server owns the resident vectors [capacity][d] and lists [capacity][K]
 * (ids int32, canonical distances float32, sorted by (distance, id)).
 * knnm_server_submit queues a batch and returns at once; worker slots, each
 * with its own stream and scratch, take queued batches in submission order
 * whenever a slot is idle and the memory the batch needs is free (the idle
 * slot's own scratch plus the device's free memory, less hbm_reserve_bytes), so
 * batches that arrive while others are on the device run concurrently with
 * them.  Each batch r is one J-Merge:
 *   - its snapshot is the resident state when it is admitted: rows
 *     0..snapshot_rows-1 with their lists at that moment;
 *   - it runs J-Merge(snapshot, batch) on private working lists with seed
 *     H(seed, 0, 4, req_id, 0) (the library's counter-based hash), so its
 *     result does not depend on what else is running;
 *   - its commit appends the batch rows at rows commit_base.. (ids of the
 *     batch in the result are moved there) and replaces each snapshot row's
 *     list with the first K distinct entries of (current list, result list).
 *     That update is commutative and associative, so the resident graph does
 *     not depend on the order in which concurrent batches commit.
 * Edges between two batches that are in flight at the same time are not
 * searched for; later batches see both.  Each local-join round runs as one
 * captured CUDA graph when use_graphs is set.
 * ------------------------------------------------------------------------- */
typedef struct knnm_server knnm_server;

typedef struct {
  int slots;                 /* concurrent batches (worker slots), >= 1 */
  int use_graphs;            /* replay rounds as captured CUDA graphs */
  int64_t capacity_rows;     /* resident rows the server can hold in total */
  int64_t max_batch_rows;    /* largest batch submit accepts */
  uint64_t hbm_reserve_bytes;/* device memory admission leaves free */
} knnm_server_config;

typedef struct {
  uint64_t req_id;
  int status;             /* KNNM_OK or the batch's error code */
  int rounds;             /* local-join rounds of its J-Merge */
  int64_t rows;           /* batch rows */
  int64_t snapshot_rows;  /* resident rows its J-Merge saw */
  int64_t snapshot_commits;/* commits applied before its snapshot */
  int64_t commit_seq;     /* its position in the commit order (0-based) */
  int64_t commit_base;    /* resident row of its first batch row */
  int64_t dist_evals;     /* pairs compared over all rounds */
  int slot;               /* worker slot that ran it */
  double queue_ms;        /* submit -> admission */
  double run_ms;          /* admission -> commit done */
  double latency_ms;      /* submit -> commit done */
  /* where run_ms goes: the J-Merge call (host clock; it waits for the
   * snapshot copy, copies the batch in and runs init, rounds and final merge),
   * its device times of init (Divide / Append / Initialize over the snapshot
   * and batch rows), rounds and final merge, and the commit (host clock from
   * queuing the commit to its completion, including the wait for the commit
   * stream) */
  double merge_ms;
  float init_ms, rounds_ms, final_ms;
  double commit_ms;
} knnm_request_info;

typedef struct {
  int64_t submitted, completed, failed;
  int64_t resident_rows;   /* rows committed so far */
  int64_t rows_completed;  /* batch rows of completed requests */
  int64_t max_concurrent;  /* most batches in flight at one time */
  double p50_ms, p99_ms;   /* latency percentiles of completed requests */
  double busy_s;           /* first admission -> last completion, seconds */
} knnm_server_stats;

/* Creates a server on `device` from S [n][d] (host or device) and its graph G
 * [n][K] (ids in 0..n-1, host or device); the lists' distances are computed
 * canonically and sorted.  params->k, metric, precision, max_iters,
 * sample_rate, keep_ratio, delta and seed apply to every batch.  The server
 * allocates the resident arrays for cfg->capacity_rows rows up front and
 * starts cfg->slots worker threads.  n >= K+1.  It takes a device, not a
 * context: each worker slot owns a context of its own (stream, scratch), so
 * that batches run concurrently, and a caller's context could not be shared
 * by the slots (calls on one context must not overlap). */
int knnm_server_create(int device, const float* S, int64_t n, const int32_t* G, int d,
                       const knnm_params* params, const knnm_server_config* cfg,
                       knnm_server** out);
/* Queues `batch` [rows][d] (host or device) under req_id, which must be new.
 * The caller keeps the batch valid until knnm_server_wait for req_id returns.
 * KNNM_ERR_NOMEM when the batch would not fit in capacity_rows or
 * max_batch_rows; rows >= K - floor(r*K). */
int knnm_server_submit(knnm_server* srv, const float* batch, int64_t rows, uint64_t req_id);
/* Waits up to timeout_ms (< 0: no limit) for req_id.  On completion copies
 * the batch rows' merged lists (resident ids) into ids_out/dists_out [rows][K]
 * (host or device; either may be NULL), fills *info (may be NULL), forgets the
 * request and returns its status.  KNNM_ERR_TIMEOUT when it has not completed
 * in time (the request stays queued or running); KNNM_ERR_INVALID for an
 * unknown id. */
int knnm_server_wait(knnm_server* srv, uint64_t req_id, int timeout_ms, int32_t* ids_out,
                     float* dists_out, knnm_request_info* info);
/* Waits until no request is queued or running (timeout as above). */
int knnm_server_drain(knnm_server* srv, int timeout_ms);
int knnm_server_get_stats(knnm_server* srv, knnm_server_stats* out);
/* Copies the first *rows resident rows (all of them if *rows < 0 or larger;
 * *rows is set to the count copied) into vectors [rows][d], ids and dists
 * [rows][K] (host or device; any may be NULL).  Waits for pending commits;
 * call it after knnm_server_drain for a state no commit is racing. */
int knnm_server_resident(knnm_server* srv, int64_t* rows, float* vectors, int32_t* ids,
                         float* dists);
/* Message of the server's last failure ("" if none). */
const char* knnm_server_last_error(const knnm_server* srv);
/* Drains, stops the workers and frees everything. */
int knnm_server_destroy(knnm_server* srv);

/* ---------------------------------------------------------------------------
 * Round steps.  Device pointers only.  Working state of a merge of N rows is
 *   ids int32 [N][K], dists float [N][K], flags uint8 [N][K] (1 = new),
 *   rear_ids int32 [N][Kr], rear_dists float [N][Kr] (id -1 where a row has none)
 * with each list sorted by (distance, id).  Vectors are passed as X1 [nx1][d]
 * holding rows 0..nx1-1 and X2 holding rows nx1..N-1 (X2 may be NULL when
 * nx1 == N).  `set_split` is n1: rows below it are S1, the rest S2.
 * `mode` 0 = S-Merge, 1 = J-Merge (and build with set_split = 0).
 * ------------------------------------------------------------------------- */

/* Sizes a merge derives from its parameters, for sizing the step arrays:
 * K_keep = floor(keep_ratio*K) entries each input list keeps at Divide (Alg. 1;
 * K in a J-Merge with set_split == 0, i.e. a build), Kr = K - K_keep rear
 * entries (and appended random members), and the sample size
 * s = max(1, floor(sample_rate*K)) capped at K.  Any output pointer may be
 * NULL.  KNNM_ERR_INVALID for parameters a merge would reject. */
int knnm_list_widths(const knnm_params* params, int mode, int64_t set_split, int* K_keep,
                     int* Kr, int* s);

/* Divide / Append (Alg. 1) and Initialize (Alg. 2).  G1 rows cover
 * 0..set_split-1; G2 rows cover set_split..N-1 in S-Merge and must be NULL in
 * J-Merge.  K_keep = floor(keep_ratio*K) (K when set_split == 0 in J-Merge);
 * Kr = K - K_keep. */
int knnm_step_init(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1, const float* X2,
                   int64_t N, int64_t set_split, int d, const int32_t* G1, const int32_t* G2,
                   const knnm_params* params, int32_t* ids, float* dists, uint8_t* flags,
                   int32_t* rear_ids, float* rear_dists);

/* Reverse(G) and the sampled candidate sets of round t: flips the flags of the
 * sampled forward-new entries to old and writes new_ids [N][cap_new],
 * new_cnt [N], old_ids [N][cap_old], old_cnt [N] with cap_new >= 2s and
 * cap_old >= K+s, s = max(1, floor(sample_rate*K)). */
int knnm_step_sample(knnm_ctx* ctx, int64_t N, int K, const int32_t* ids, const float* dists,
                     uint8_t* flags, uint64_t seed, int t, int s, int cap_new, int cap_old,
                     int32_t* new_ids, int32_t* new_cnt, int32_t* old_ids, int32_t* old_cnt);

/* Size of the fixed scratch array used by knnm_step_sample_noalloc. */
#define KNNM_NOALLOC_SCRATCH_BYTES (8u << 20)

/* knnm_step_sample without any device allocation.  The paper has no
 * counterpart to this call; it exists for callers of this library that must
 * not allocate device memory: plug-ins whose host application owns the whole
 * device-memory budget, and serving processes that reserve all their memory at
 * start-up because cudaMalloc/cudaFree may synchronize the device and stall
 * the other streams' work on the request path.
 *
 * Same arguments, outputs and results as knnm_step_sample (device pointers),
 * except that it takes the CUDA stream directly instead of a context and runs
 * on the calling thread's current device.  Its scratch (packed list keys and
 * the two reverse-sample slot arrays) is one fixed __device__ array of
 * KNNM_NOALLOC_SCRATCH_BYTES inside the library, held by every GPU that loads
 * the library until the process exits.  Limit, with a(x) = x rounded up to a
 * multiple of 256:  a(N*K*8) + 2*a(N*s*8) + 256 <= KNNM_NOALLOC_SCRATCH_BYTES
 * (with K = 20, s = 10 that is about 26,000 rows); larger inputs, and N above
 * 2^31 - 1, return KNNM_ERR_INVALID before anything is launched.  The call
 * allocates nothing, neither device nor host memory.  Each call looks up the
 * array's device address (cudaGetSymbolAddress); the first lookup on a device
 * loads the library's device code there, so make the first call on each
 * device before any stream capture starts.  Every call ends by waiting for its
 * stream (cudaStreamSynchronize), so no call may be made while a stream
 * capture is active on that stream or, in global capture mode, anywhere in the
 * process.  Every call shares the one array: it resets what must start empty,
 * but calls whose work overlaps on the GPU (other threads, other streams) race
 * on it and must be serialized by the caller.  Returns after the stream has
 * finished the call's work. */
int knnm_step_sample_noalloc(void* cuda_stream, int64_t N, int K, const int32_t* ids,
                             const float* dists, uint8_t* flags, uint64_t seed, int t, int s,
                             int cap_new, int cap_old, int32_t* new_ids, int32_t* new_cnt,
                             int32_t* old_ids, int32_t* old_cnt);

/* Local join and UpdateNN of one round (Alg. 1 / Alg. 2 inner loops) on the
 * given candidate sets: updates ids/dists/flags in place, writes c_t to
 * *updates and the pair count to *dist_evals.  Counts must not exceed
 * cap_new/cap_old and cap_new + cap_old <= 96. */
int knnm_step_join(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1, const float* X2,
                   int64_t N, int64_t set_split, int d, const knnm_params* params, int32_t* ids,
                   float* dists, uint8_t* flags, int cap_new, int cap_old, const int32_t* new_ids,
                   const int32_t* new_cnt, const int32_t* old_ids, const int32_t* old_cnt,
                   int64_t* updates, int64_t* dist_evals);

/* The tensor-core distance estimate of the join (Alg. 1 / Alg. 2 compare step,
 * the BF16/FP16 precisions) for the pairs (pi[r], pj[r]), r < P, of rows of X
 * [n][d] (device pointers; d % 8 == 0, d <= 2048): est[r] is the estimate as
 * the tensor-core join computes it (16-bit rows, tensor-core Gram value with
 * FP32 accumulation), bound[r] the proven bound on |est - canonical| that the
 * join uses to decide whether a pair needs its canonical FP32 distance (0 when
 * both rows are small non-negative integers: the estimate is then exact), and
 * canon[r] the canonical FP32 distance.  metric: KNNM_L2, KNNM_IP or KNNM_COS;
 * precision: KNNM_BF16_RERANK or KNNM_FP16_RERANK.  Pair indices outside
 * 0..n-1 are KNNM_ERR_INVALID (checked before any launch). */
int knnm_step_tc_estimate(knnm_ctx* ctx, const float* X, int64_t n, int d, int metric,
                          int precision, const int32_t* pi, const int32_t* pj, int64_t P,
                          float* est, float* bound, float* canon);

/* knnm_step_join restricted to the nodes u in [row_lo, row_hi): only the pairs
 * of those nodes' candidate sets are compared (the local join of Alg. 1 /
 * Alg. 2 for a slice of the nodes), and their proposals update the lists of
 * every target, in or out of the range.  One rank's share of a round of the
 * sharded S-Merge (nodes partitioned by id range); the full range is
 * knnm_step_join. */
int knnm_step_join_rows(knnm_ctx* ctx, int mode, const float* X1, int64_t nx1, const float* X2,
                        int64_t N, int64_t set_split, int d, const knnm_params* params,
                        int32_t* ids, float* dists, uint8_t* flags, int cap_new, int cap_old,
                        const int32_t* new_ids, const int32_t* new_cnt, const int32_t* old_ids,
                        const int32_t* old_cnt, int64_t row_lo, int64_t row_hi,
                        int64_t* updates, int64_t* dist_evals);

/* UpdateNN of rows whose proposals were applied on several devices (Alg. 1
 * UpdateNN, synchronous reading: the new list is the top K of the round-start
 * list and all proposals).  part_ids/part_dists [parts][n][K] (device) hold
 * each part's list of the same n rows, each already the top K of the
 * round-start list and that part's proposals; the result is the first K
 * distinct (distance, id) entries of all parts, which is the top K of the
 * round-start list and every part's proposals.  start_ids/start_dists/
 * start_flags [n][K] are the round-start lists with the flags the sampler left;
 * an output entry that was in its start list keeps that flag, any other is
 * flagged new, and *updates receives how many such new entries there are (c_t
 * of these rows).  Ids < 0 in a part are empty places. */
int knnm_step_union(knnm_ctx* ctx, int64_t n, int K, int parts, const int32_t* part_ids,
                    const float* part_dists, const int32_t* start_ids, const float* start_dists,
                    const uint8_t* start_flags, int32_t* out_ids, float* out_dists,
                    uint8_t* out_flags, int64_t* updates);

/* Merge and Sort (Alg. 1 last step): first K distinct ids of each working list
 * merged with its rear list. */
int knnm_step_final(knnm_ctx* ctx, int64_t N, int K, const int32_t* ids, const float* dists,
                    int Kr, const int32_t* rear_ids, const float* rear_dists, int32_t* out_ids,
                    float* out_dists);

#ifdef __cplusplus
}
#endif

#endif /* KNNM_H */
