/* im.h -- C ABI of libim, the GB300 (sm_103a) RIS influence-maximization hot path.
 *
 * The method is GreediRIS (arXiv 2408.10982): sample random reverse-reachable
 * (RRR) sets (Def. 3, Sec. 2.1 "Sample"), turn them into covering subsets
 * S(v) = { i : v in R(i) } (Sec. 3.2), and select k seeds by max-k-cover,
 * either with the standard greedy (Sec. 3.2) or with RandGreedi over a random
 * vertex partition (Alg. 3, Alg. 4) whose local solutions are merged by the
 * streaming threshold algorithm (Alg. 5), optionally truncated (Sec. 3.3.2).
 * On one GPU the paper's m machines become m vertex partitions processed by
 * separate thread blocks, and its message passing becomes device memory.
 *
 * Conventions for every call:
 *  - Returns an im_status; IM_OK is 0, errors are negative.  No C++
 *    exception crosses this boundary.  im_last_error() gives the text of the
 *    calling thread's last failure.
 *  - Array arguments are plain pointers to either host or device memory; the
 *    library tells them apart with cudaPointerGetAttributes.  Input arrays
 *    are read during the call (and copied if kept).  Output arrays are
 *    written; when an output is in host memory the call synchronises its
 *    stream before returning, when all outputs are device memory the call
 *    only enqueues work on the stream (outputs valid once the stream reaches
 *    that point).
 *  - The caller owns every array it passes.  The library owns the opaque
 *    handles (im_graph, im_pool) and all device memory behind them; handles
 *    live on the device that was current when they were created.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Vertex ids are int32 in [0, n); edge and entry counts are int64; sample
 *    ids are uint64 below 2^32.
 *  - Randomness is Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit
 *    seed, with one counter per (sample, edge group), (sample, vertex) or
 *    (vertex) and a domain tag in counter word 3; results are therefore
 *    bit-identical for any launch shape and any split of sample ids.
 */
#ifndef IM_H
#define IM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IM_OK = 0,
    IM_ERR_INVALID_ARG = -1,   /* a size, id, pointer or option is out of range */
    IM_ERR_OOM = -2,           /* device memory could not be allocated */
    IM_ERR_CUDA = -3,          /* a CUDA runtime call failed (text in im_last_error) */
    IM_ERR_TIMEOUT = -4,       /* a bounded device wait expired (grid barrier, stream flag) */
    IM_ERR_CAPACITY = -5,      /* a pool or queue capacity was exceeded; state unchanged */
    IM_ERR_BUSY = -6,          /* the request is still running (serving poll) */
    IM_ERR_UNSUPPORTED = -7    /* a valid request the library cannot run here (e.g. no GPU) */
} im_status;

typedef enum { IM_IC = 0, IM_LT = 1 } im_model;

typedef enum { IM_GREEDY_PLAIN = 0, IM_RANDGREEDI = 1, IM_GREEDY_LAZY = 2 } im_cover_algo;

/* RandGreedi's global step (Alg. 4, line 5). */
typedef enum { IM_AGG_STREAM = 0, IM_AGG_GREEDY = 1 } im_aggregator;

/* Options of im_max_k_cover.
 *   algo            IM_GREEDY_PLAIN: standard greedy over all of V (Sec. 3.2);
 *                   the kernel that runs it is IM_TUNE_GREEDY_EVALS' choice.
 *                   IM_RANDGREEDI: Alg. 4 with Alg. 5 aggregation.
 *                   IM_GREEDY_LAZY: the lazy greedy of Alg. 2 over all of V
 *                   (re-evaluates only candidates whose stale gain bound is
 *                   on top); with ties to the smallest id its seeds, gains and
 *                   coverage equal IM_GREEDY_PLAIN's.
 *   partitions      number of random vertex parts m (RandGreedi), 1..4096.
 *   alpha_num/den   truncation alpha = num/den in (0, 1]: every partition
 *                   computes k local seeds and streams its first
 *                   max(1, ceil(alpha k)) of them (Sec. 3.3.2).
 *   delta           bucket spacing of the streaming algorithm, 0 < delta < 1/2
 *                   (Alg. 5); B = least b >= 1 with (1+delta)^b >= k buckets.
 *   partition_seed  Philox key of the vertex partition (Alg. 3).
 *   fused           RandGreedi only: 1 runs local greedy and aggregation in
 *                   one cooperative launch with the aggregator consuming seeds
 *                   as they are produced (streaming overlap, bucket bitmaps in
 *                   global memory); 0 runs them as two launches, the second
 *                   a bucket stage laid out as IM_TUNE_RG_CLUSTER says (by
 *                   default one 64-bit bucket mask per RRR set).  Results
 *                   are identical.
 *   aggregator      RandGreedi only: IM_AGG_STREAM (0) aggregates with the
 *                   streaming buckets of Alg. 5 (Sec. 3.3); IM_AGG_GREEDY (1)
 *                   is Alg. 4's global step as written: the lazy greedy of
 *                   Alg. 2 over the union of the gathered local seeds (the
 *                   first max(1, ceil(alpha k)) of every part), after all
 *                   local solutions are complete.  Its result is reported as
 *                   bucket 0 (B = 1, threshold 0) by im_randgreedi_details;
 *                   fused and delta are ignored. */
typedef struct {
    int32_t algo;
    int32_t partitions;
    int32_t alpha_num;
    int32_t alpha_den;
    double delta;
    uint64_t partition_seed;
    int32_t fused;
    int32_t aggregator;
} im_cover_opts;

typedef struct im_graph im_graph;   /* device-resident graph, library-owned */
typedef struct im_pool im_pool;     /* device-resident RRR pool, append-only */

/* Text of a status code / of this thread's last failure (never NULL). */
const char *im_status_str(im_status s);
const char *im_last_error(void);

/* Library and device facts: number of SMs, device ordinal in use. */
im_status im_device_info(int32_t *num_sms, int32_t *device);

/* Device memory of RRR pools comes from one stream-ordered memory pool per
 * device (graphs use plain cudaMalloc).  Destroying an RRR pool returns its
 * buffers to that memory pool, which keeps up to one eighth of the device's
 * memory cached for the next RRR pool instead of unmapping it (the cache
 * never holds a live buffer).  im_trim_memory waits for the current device
 * to go idle and hands every cached byte back to the driver; IM_OK also when
 * nothing is cached. */
im_status im_trim_memory(void);

/* ---- graph (Sec. 3.4 S1: the whole graph is replicated on every machine) --
 * in_off  int64[n+1]  in-CSR offsets (non-decreasing, in_off[0] = 0, in_off[n] = m)
 * in_src  int32[m]    source vertex of each in-edge; edges of a vertex in any
 *                     fixed order -- the edge id e is the CSR position
 * w       uint32[m]   edge weight as a 32-bit threshold: for IC, edge e is live
 *                     in sample s iff its Philox coin < w[e]; for LT, w[e] is
 *                     the probability (x 2^32) that the head picks this in-edge,
 *                     and a vertex's weights must sum to at most 2^32.
 * Copies the arrays to the device.  Validates offsets and ids
 * (IM_ERR_INVALID_ARG).  n >= 1, 0 <= m < 2^31. */
im_status im_graph_create(const int64_t *in_off, const int32_t *in_src, const uint32_t *w,
                          int64_t n, int64_t m, void *stream, im_graph **out);
im_status im_graph_destroy(im_graph *g);
/* n, m of a graph; lt_valid = 1 if every vertex's weights sum to <= 2^32. */
im_status im_graph_info(const im_graph *g, int64_t *n, int64_t *m, int32_t *lt_valid);

/* ---- RRR pool ---------------------------------------------------------------
 * Holds up to max_sets RRR sets with up to max_entries members in total, as
 * CSR by position (set_off int64[theta+1], members int32[T], each set
 * ascending), plus the covering-subset index built from it.  Pools are
 * append-only (samples of later IMM rounds extend earlier ones, Sec. 3.2). */
im_status im_pool_create(const im_graph *g, int64_t max_sets, int64_t max_entries,
                         im_pool **out);
im_status im_pool_destroy(im_pool *p);
/* Drop every set (theta = 0) without freeing memory. */
im_status im_pool_reset(im_pool *p);
/* theta, total entries T, and the edges examined by all sampling so far
 * (IC: every in-edge of every member, each read and given a coin; LT: the
 * in-edges a cumulative-weight scan would decide over -- up to and including
 * the picked one, or all in-edges when none is picked.  The LT sampler does
 * not read these edges: a cut-point table decides the pick with one load, so
 * for LT this count is a measure of the work a scan-based sampler does, not of
 * this one's memory traffic.  A walk of L members makes L draws, so LT walk
 * steps = T). */
im_status im_pool_info(const im_pool *p, int64_t *theta, int64_t *total, int64_t *examined);

/* ---- Sample (Alg. 1 "Sample"; Def. 3; Sec. 2.1) ------------------------------
 * Appends the RRR sets of sample ids first_sample_id .. first_sample_id +
 * num_samples - 1 to the pool, in id order.  Sample s draws its root
 * uniformly from V and runs a stochastic reverse BFS (IC) or the backward
 * random walk of the LT live-edge world (LT, requires lt_valid).
 * IM_ERR_CAPACITY if the pool would overflow (pool unchanged).
 * Synchronises the stream (the new totals are read back). */
im_status im_sample_rrr(const im_graph *g, im_model model, uint64_t seed,
                        uint64_t first_sample_id, uint64_t num_samples, im_pool *pool,
                        void *stream);

/* Copy the pool's CSR out: set_off int64[theta+1], members int32[T]. */
im_status im_pool_export(const im_pool *p, int64_t *set_off, int32_t *members, void *stream);

/* Build the covering subsets S(v) (Sec. 3.2; the all-to-all of Alg. 3 gathers
 * exactly these rows).  Done implicitly by im_max_k_cover when stale. */
im_status im_pool_index(im_pool *p, void *stream);
/* Copy S(v) out: vtx_off int64[n+1], set_ids int32[T].  The order of set ids
 * within one S(v) is unspecified (the cover does not depend on it). */
im_status im_index_export(const im_pool *p, int64_t *vtx_off, int32_t *set_ids, void *stream);

/* ---- SelectSeeds: max-k-cover over the pool (Sec. 3.2, Alg. 4, Alg. 5) -------
 * Universe: the pool's theta sets.  Greedy ties go to the smallest vertex id;
 * a greedy stops early when every remaining gain is zero, so num_seeds may be
 * < k.  Outputs: seeds int32[k], gains int64[k] (marginal gain of each seed
 * when it was taken; for a winning bucket, its gain on entering the bucket),
 * num_seeds, coverage = |union of S(seed)|.  k >= 1.
 * IM_ERR_TIMEOUT if a bounded device wait expired. */
im_status im_max_k_cover(im_pool *p, int32_t k, const im_cover_opts *opts, int32_t *seeds,
                         int64_t *gains, int32_t *num_seeds, int64_t *coverage, void *stream);

/* Details of the pool's last IM_RANDGREEDI cover, for parity checks:
 *   local_seeds int32[P*k], local_gains int64[P*k], local_n int32[P],
 *   local_cov int64[P]                       -- Alg. 4 local solutions
 *   thr int64[B], bucket_cov int64[B], bucket_n int32[B],
 *   bucket_seeds int32[B*k], bucket_gains int64[B*k]   -- Alg. 5 buckets
 *   chosen: -1 if the best bucket won, else the winning partition.
 * Any pointer may be NULL.  *P_out and *B_out receive P and B. */
im_status im_randgreedi_details(const im_pool *p, int32_t *P_out, int32_t *B_out,
                                int32_t *local_seeds, int64_t *local_gains, int32_t *local_n,
                                int64_t *local_cov, int64_t *thr, int64_t *bucket_cov,
                                int32_t *bucket_n, int32_t *bucket_seeds, int64_t *bucket_gains,
                                int32_t *chosen, void *stream);

/* Algorithmic bytes of all sampling into this pool so far -- the bytes a
 * sampler must move, by this formula (visited-set and queue traffic is
 * on-chip and not counted):
 *   IC: per member 16 (its in-CSR offset pair) + 4 (member write),
 *       per examined edge 8 (source id + weight), per set 8 (offset);
 *   LT, one walk per thread (the default): per set 8 (offset) + 4 (root
 *       write); per step 16 (the vertex record), + 16 (one cut point) when the
 *       in-degree is > 0; when the draw lies past the cut point's edge, 8 per
 *       binary-search probe actually made + 8 (the picked leaf); 4 per member
 *       added.
 *   LT, G lanes per walk: per walk step at a vertex of in-degree d: 16
 *       (offset pair) + 8 (floor(log2 d) + 1) when d > 0 (search of the
 *       cumulative weights) + 4 when an edge is picked (its source) + 4
 *       (member write), per set 8 (offset).
 * These are the bytes the kernels' own loads need, not a linear scan of the
 * in-edges the examined-edge count covers (the LT pick reads one cut point,
 * not the e + 1 edges it decides over). */
im_status im_pool_sample_bytes(const im_pool *p, int64_t *bytes);

/* ---- tuning knobs (process-wide; results never depend on them) ---------------
 *   IM_TUNE_LT_GROUP    lanes that run one LT walk: 1 (default: one walk per
 *                       thread, an exact cut-point table picks the in-edge in
 *                       O(1) expected loads, revisits are tested through a
 *                       per-walk Bloom filter), or 8, 16, 32 (a warp runs
 *                       32 / value walks in lockstep over a fanout-32 search
 *                       tree of the running sums).
 *   IM_TUNE_RG_CLUSTER  RandGreedi two-launch mode, bucket stage: 0 (default)
 *                       keeps one 64-bit bucket mask per RRR set, so one pass
 *                       over a streamed subset counts its gain for every
 *                       bucket, and spreads each group of stream slots over
 *                       the whole GPU (B <= 64; for B > 64 it picks a cluster
 *                       as below); 1..8 keeps each bucket's theta-bit bitmap
 *                       in the shared memory of a cluster of at least that
 *                       many blocks (the smallest of 1, 2, 4, 8 that holds
 *                       it); -1 keeps the bitmaps in global memory (one block
 *                       per bucket).
 *   IM_TUNE_INDEX_REPLICAS  covering-subset build: 0 (default) a stable radix
 *                       sort of the (vertex, set id) pairs by vertex, 8 bits a
 *                       pass, with 12 bytes of pool scratch per member (set ids
 *                       come out ascending inside every S(v); without the
 *                       memory, the counting build with 4 replicas runs
 *                       instead); 1, 2, 4 or 8: a counting build, histogram
 *                       and scatter through per-vertex counters and cursors
 *                       replicated that many times (a member's replica
 *                       follows its position), spreading the atomics on hub
 *                       vertices.  The order of set ids inside an S(v) is
 *                       unspecified by the interface in every case.
 *   IM_TUNE_RG_EVALS    RandGreedi local greedy: candidates re-evaluated per
 *                       round, 1, 2 (default), 4 or 8.
 *   IM_TUNE_GREEDY_EVALS  the kernel of IM_GREEDY_PLAIN: 0 (default) runs the
 *                       standard greedy that decrements the gain of every
 *                       member of every newly covered set; 1, 2, 4, 8, 16 or
 *                       32 runs the lazy greedy of Alg. 2 with that many
 *                       candidates re-evaluated at once (also the width
 *                       IM_GREEDY_LAZY uses; 0 means 16 there).
 *   IM_TUNE_LT_CACHE    one-walk-per-thread LT sampling, L2 policy of its
 *                       loads: 0 (default) plain; 1 the vertex records stay
 *                       in L2 ahead of other lines (evict_last); 2 as 1, and
 *                       the cut points leave L2 first (evict_first).
 *   IM_TUNE_GREEDY_HOT  the standard greedy's decrement kernel keeps exact
 *                       gains, and looks for the best one, only among the
 *                       vertices with |S(v)| >= tau = max_v |S(v)| >> value
 *                       (4 .. 16; default 8); the others keep |S(v)| < tau
 *                       as a stale bound until the best gain drops below
 *                       tau, when one pass makes them exact.  0 keeps every
 *                       gain exact and reads all of them at every step.
 *                       (Vertices with |S(v)| >= max |S(v)| / 64 always keep
 *                       their gain as 32 partial counts, spreading the
 *                       atomics that land on them.) */
typedef enum {
    IM_TUNE_LT_GROUP = 0,
    IM_TUNE_RG_CLUSTER = 1,
    IM_TUNE_INDEX_REPLICAS = 2,
    IM_TUNE_RG_EVALS = 3,
    IM_TUNE_GREEDY_EVALS = 4,
    IM_TUNE_LT_CACHE = 5,
    IM_TUNE_GREEDY_HOT = 6
} im_tune_knob;
im_status im_tune_set(int32_t knob, int64_t value);
im_status im_tune_get(int32_t knob, int64_t *value);

/* Autotuner (not in the paper): times every allowed value of the knobs above
 * on a probe of the caller's workload -- theta sets of graph g under model
 * and seed -- and leaves the fastest values set (process-wide).  Tried: lanes
 * per LT walk (LT only), counter replicas of the covering-subset build, and,
 * when rg_opts asks for RandGreedi, its evaluation width and (two-launch mode)
 * its bucket-stage layout, with rg_opts' partition count, alpha and delta.
 * Results never depend on these knobs, so tuning changes only speed; the
 * partition count itself is a parameter of the method and is not tuned.
 * Also tried: the L2 policy of the one-walk-per-thread LT sampler (LT with
 * one lane per walk) and the standard greedy's tau (IM_TUNE_GREEDY_HOT).
 *   out->lt_group, index_replicas, rg_evals, rg_cluster, lt_cache,
 *       greedy_hot: the chosen values (-1 where not tuned);
 *   out->ms[row][i]: the best-of-two time of the i-th value tried (rows: LT
 *       group {1, 8, 16, 32}, index build {0 (radix), 1, 2, 4, 8}, evaluation width
 *       {1, 2, 4, 8}, bucket stage {0, 1, 2, 4, 8, -1}, LT cache {0, 1, 2},
 *       greedy tau {0, 7, 8, 10}); -1 where not run.
 * Allocates a probe pool (and a small result buffer) and frees them before it
 * returns.  Synchronises the stream. */
typedef struct {
    int32_t lt_group;
    int32_t index_replicas;
    int32_t rg_evals;
    int32_t rg_cluster;
    int32_t lt_cache;
    int32_t greedy_hot;
    double ms[6][8];
} im_tune_result;
im_status im_autotune(const im_graph *g, im_model model, uint64_t seed, int64_t theta, int32_t k,
                      const im_cover_opts *rg_opts, im_tune_result *out, void *stream);

/* ---- per-kernel device timing (tracing) -------------------------------------
 * While enabled, every kernel the library launches is bracketed by a pair of
 * CUDA events on its stream.  im_profile_read waits for the recorded events
 * and returns, per kernel name, the number of launches and the total device
 * milliseconds since the last im_profile_reset:
 *   names     char[max_entries * 48], entry i at names + 48 i, NUL-terminated
 *   launches  int64[max_entries],  total_ms double[max_entries]
 *   *count    number of entries written.
 * Process-wide and thread-safe; off by default. */
im_status im_profile_enable(int32_t on);
im_status im_profile_reset(void);
im_status im_profile_read(int32_t max_entries, char *names, int64_t *launches, double *total_ms,
                          int32_t *count);

/* Diagnostics of the pool's last IM_RANDGREEDI cover: int64[(P + B) * 6].
 * Row p < P (local greedy of part p): start ns, end ns (device global timer),
 *   rounds, lazy re-evaluations, entries scanned by re-evaluations, entries
 *   covered.  Row P + b (bucket b): start ns, end ns, elements evaluated,
 *   elements accepted, entries scanned, ns spent waiting for the stream. */
im_status im_randgreedi_stats(const im_pool *p, int64_t *stats, void *stream);

/* Diagnostics of the pool's last lazy-greedy cover (IM_GREEDY_LAZY, or
 * IM_GREEDY_PLAIN with IM_TUNE_GREEDY_EVALS > 0): int64[4] = rounds, candidate
 * evaluations, covering-subset entries scanned by them, and builds of the
 * sorted bound list.  Zero if no such cover ran. */
im_status im_greedy_stats(const im_pool *p, int64_t *stats);

/* Standard greedy max-k-cover (same result as im_max_k_cover with
 * IM_GREEDY_PLAIN) for callers that cannot let the library allocate device
 * memory -- a framework whose caching allocator owns the device memory, a
 * serving loop that must not pay for cudaMalloc mid-request, a fixed memory
 * budget.  The paper has no counterpart; this is a deployment variant.
 * The caller passes the RRR sets (set_off int64[theta+1], members int32[T])
 * and the covering subsets (vtx_off int64[n+1], set_ids int32[T]) -- e.g. as
 * exported by im_pool_export / im_index_export -- and the outputs seeds
 * int32[k], gains int64[k], num_seeds int32[1], coverage int64[1]; every
 * array must be memory of the current device (or managed memory); another
 * GPU's memory gets IM_ERR_INVALID_ARG.  The arrays must form a valid
 * instance: set_off and vtx_off start at 0, never decrease and end at the
 * same total T; member ids lie in [0, n) and set ids in [0, theta).  A
 * device pass checks this before the greedy runs and returns
 * IM_ERR_INVALID_ARG (nothing written) otherwise.  The call allocates
 * nothing: its scratch is a 64 MiB static device array inside the library,
 * which every GPU that loads the library holds until the process exits.  It
 * needs 4 n + theta / 8 + 33 KB bytes of it (rounded up to 256 bytes per
 * part); larger instances get IM_ERR_CAPACITY.  Every call looks up that
 * array's device address on the current device; the first call on a device
 * also loads the library's kernels there (keep that first call outside any
 * stream capture).  All calls on a device share the one array,
 * which keeps the previous call's contents: each call clears what must start
 * at zero, but calls that overlap on the GPU (other streams or threads) race
 * and must be serialised by the caller.  Synchronises the stream. */
im_status im_max_k_cover_noalloc(const int64_t *set_off, const int32_t *members,
                                 const int64_t *vtx_off, const int32_t *set_ids, int64_t n,
                                 int64_t theta, int32_t k, int32_t *seeds, int64_t *gains,
                                 int32_t *num_seeds, int64_t *coverage, void *stream);

/* Grow a pool's capacity in place (contents kept; index rebuilt on demand). */
im_status im_pool_reserve(im_pool *p, int64_t max_sets, int64_t max_entries);

/* ---- IMM (Alg. 1) ------------------------------------------------------------
 * Estimate -> martingale rounds (Sample appending to one pool, SelectSeeds,
 * CheckGoodness) -> theta = ceil(lambda* / LB) fresh samples -> SelectSeeds.
 * The formulas the paper defers to Tang et al. (2015) / Chen (2018), natural
 * logs: l' = l (1 + ln 2 / ln n), e' = sqrt(2) e;
 * lambda' = (2 + 2e'/3)(ln C(n,k) + l' ln n + ln log2 n) n / e'^2;
 * round i = 1 .. floor(log2 n) - 1: theta_i = ceil(lambda' / (n / 2^i)), pass iff
 * n cov / theta_i >= (1 + e') n / 2^i, LB = n cov / theta_i / (1 + e');
 * lambda* = 2n ((1-1/e) sqrt(l' ln n + ln 2) + sqrt((1-1/e)(ln C(n,k) + l' ln n
 * + ln 2)))^2 / e^2.  Round samples use ids 0 .. theta_last - 1, the final
 * ones the next theta ids.  SelectSeeds follows opts (NULL: plain greedy).
 * Outputs: seeds int32[k] (host or device), num_seeds, coverage of the final
 * pool, theta; info (optional) records the rounds.  Pools are allocated and
 * grown inside; IM_ERR_OOM if the RRR sets do not fit in device memory.
 * With info->keep_pools nonzero on entry, the rounds' pool and the final pool
 * are not destroyed but handed to the caller in info->round_pool and
 * info->final_pool (the caller destroys them with im_pool_destroy); on an
 * error no pool is handed over.  Otherwise both are NULL on return. */
typedef struct {
    int32_t rounds;               /* martingale rounds run */
    int32_t keep_pools;           /* in: hand the pools to the caller */
    int64_t theta_rounds[64];     /* theta_i of each round */
    int64_t cov_rounds[64];       /* coverage of round i's seeds on its theta_i sets */
    double lb;                    /* LB (1 if no round passed) */
    int64_t theta;                /* final theta */
    int64_t round_entries;        /* members in the rounds' pool */
    int64_t final_entries;        /* members in the final pool */
    int64_t examined;             /* edges examined by the final sampling */
    im_pool *round_pool;          /* out (keep_pools): sample ids 0 .. theta_last - 1 */
    im_pool *final_pool;          /* out (keep_pools): the next theta ids */
} im_solve_info;

im_status im_solve(const im_graph *g, im_model model, int32_t k, double eps, double ell,
                   uint64_t seed, const im_cover_opts *opts, int32_t *seeds, int32_t *num_seeds,
                   int64_t *coverage, int64_t *theta, im_solve_info *info, void *stream);

/* ---- OPIM with GreediRIS seed selection (Sec. 3.3.2 and Sec. 4.4, Table 6) --
 * OPIM (Tang et al. 2018; the paper runs its RandGreedi inside it) splits each
 * round's samples into a selection half R1 (sample ids 0, 1, ...) and a
 * validation half R2 (ids 2^31, 2^31 + 1, ...).  Round i = 1 .. i_max: both
 * halves grow to theta_i = theta_0 2^(i-1) sets (appending ids); seeds are
 * selected on R1 as opts says (NULL: plain greedy; RandGreedi with its
 * truncation alpha: GreediRIS-trunc); cov1 = their coverage of R1, cov2 =
 * the sets of R2 that hold a seed, cov1u = cov1 + the k largest marginal
 * gains left on R1 (an upper bound on the optimal k-set's coverage of R1,
 * valid for any seed set); then, with a = ln(3 i_max / delta),
 *   sigma_l = ((sqrt(cov2 + 2a/9) - sqrt(a/2))^2 - a/18) n / theta_i,
 *   sigma_u = (sqrt(cov1u + a/2) + sqrt(a/2))^2 n / theta_i,
 * and the round's instance-wise guarantee is sigma_l / sigma_u; the rounds
 * stop once it reaches 1 - 1/e - eps, or after the last round.
 *   theta_max = 2n ((1-1/e) sqrt(ln(6/delta)) + sqrt((1-1/e)(ln C(n,k)
 *               + ln(6/delta))))^2 / (eps^2 k),
 *   theta_0 = ceil(theta_max eps^2 k / n), i_max = max(1, ceil(log2(
 *   theta_max / theta_0))), or, with theta_cap > 0, the last round whose
 *   theta_i <= theta_cap (the paper stops near 2^20 sets).  Natural logs.
 * Outputs: seeds int32[k] (host or device) and num_seeds of the last round;
 * info (optional) records every round.  IM_ERR_CAPACITY when a half would
 * need 2^31 or more sets (pass a cap).  Synchronises the stream. */
typedef struct {
    int32_t rounds;               /* rounds run */
    int32_t keep_pools;           /* in: hand R1 / R2 to the caller */
    int64_t theta[64];            /* sets in each half, per round */
    int64_t cov1[64];             /* coverage of the round's seeds on R1 */
    int64_t cov2[64];             /* sets of R2 that hold a seed */
    int64_t cov1_upper[64];       /* cov1 + the k largest marginal gains on R1 */
    double alpha[64];             /* sigma_l / sigma_u of each round */
    double sigma_lower, sigma_upper, guarantee;   /* of the returned seeds */
    double theta_max;
    int64_t theta0;
    int32_t max_rounds;           /* i_max */
    int32_t reserved;
    double a;                     /* ln(3 i_max / delta) */
    im_pool *r1_pool;             /* out (keep_pools): the caller destroys them */
    im_pool *r2_pool;
} im_opim_info;

im_status im_opim(const im_graph *g, im_model model, int32_t k, double eps, double delta,
                  uint64_t seed, int64_t theta_cap, const im_cover_opts *opts, int32_t *seeds,
                  int32_t *num_seeds, im_opim_info *info, void *stream);

/* ---- many queries at once (batching; not in the paper) -----------------------
 * A query: a resident graph, a model, k, theta (sample ids 0 .. theta-1) and
 * its Philox seed.  im_solve_batch solves nq queries in a fixed number of
 * launches (one sampling launch per model over all their samples, one sort,
 * one covering-subset build over all queries' vertices, one greedy launch
 * with one block per query; RandGreedi queries one after another on the
 * batch's shared index) and gives every query exactly the seeds, gains and
 * coverage that im_sample_rrr + im_max_k_cover give it alone.  seeds
 * int32[nq * kmax] and gains int64[nq * kmax] (row q: query q's seeds;
 * entries past num_seeds are unspecified; gains may be NULL), host or
 * device; res[nq] host.  An im_batch keeps its device arenas between
 * calls (grown on demand).  Synchronises the stream. */
typedef struct {
    const im_graph *graph;
    int32_t model;            /* IM_IC or IM_LT */
    int32_t k;                /* 1 <= k <= min(kmax, n) */
    int64_t theta;
    uint64_t seed;
    /* SelectSeeds of the query.  All zero: plain greedy.  algo IM_RANDGREEDI:
     * RandGreedi as im_max_k_cover runs it (two launches; fused ignored), the
     * same result as im_max_k_cover on the query's own pool.  partitions = 0
     * there lets the batch pick the partition count: every allowed count (the
     * powers of two from 16 and the SM count, parts small enough for one
     * block) is timed on the first query of that graph, model and
     * power-of-two theta, the fastest is kept for later queries of that kind,
     * and the count used is reported in im_result.partitions (it changes the
     * seeds, so a replay passes it explicitly). */
    im_cover_opts cover;
} im_query;

typedef struct {
    int32_t num_seeds;
    int32_t status;           /* im_status of the query */
    int64_t coverage;
    int64_t entries;          /* RRR set members of the query */
    int32_t partitions;       /* RandGreedi queries: the partition count used; else 0 */
    int32_t reserved;
} im_result;

typedef struct im_batch im_batch;
im_status im_batch_create(im_batch **out);
im_status im_batch_destroy(im_batch *b);
im_status im_solve_batch(im_batch *b, const im_query *q, int32_t nq, int32_t kmax, int32_t *seeds,
                         int64_t *gains, im_result *res, void *stream);

/* ---- serving (not in the paper) ------------------------------------------------
 * A request loop with continuous batching over resident graphs: workers (each
 * with its own stream and batch arena) take queued requests in arrival order,
 * admit as many as max_batch and the device-memory budget allow (footprint
 * estimated from theta and the members per set seen so far on the request's
 * graph and model; a worker with nothing in flight always admits one), run
 * them through im_solve_batch and publish the results.  Requests arriving
 * while batches run join the next batch; with workers > 1 batches overlap on
 * the device.  Every result equals the query's result alone. */
typedef struct {
    int32_t workers;          /* batches in flight at once, 1..16 */
    int32_t max_batch;        /* requests per batch, >= 1 */
    int64_t mem_budget;       /* device bytes the in-flight batches may use */
    int64_t heavy_members;    /* 0: off.  > 0 (needs workers >= 2): a request whose estimated
                                 RRR members (theta x members per set seen so far on its graph
                                 and model, 64 before any) reach this runs on worker 0 only,
                                 by itself through the single-query path (im_sample_rrr into
                                 a pool the worker keeps, then im_max_k_cover; a RandGreedi
                                 request with partitions = 0 still goes through a batch);
                                 the other workers take the remaining requests in arrival
                                 order past it (a heavy lane, so long queries do not hold up
                                 short ones) */
} im_server_opts;

typedef struct im_server im_server;
im_status im_server_create(const im_server_opts *opts, im_server **out);
/* Finishes every queued request, then stops the workers and frees their
 * batch arenas and pools. */
im_status im_server_destroy(im_server *s);
/* Queues a query (copied); *ticket identifies it.  The graph must stay alive
 * until the server is destroyed (the heavy lane keeps a pool per graph and
 * model until then). */
im_status im_server_submit(im_server *s, const im_query *q, uint64_t *ticket);
/* Result of a finished request, then forgotten: seeds int32[k] (host), number
 * of seeds, coverage, and the latency from submission to completion.
 * IM_ERR_BUSY while the request is queued or running. */
im_status im_server_poll(im_server *s, uint64_t ticket, int32_t *seeds, int32_t *num_seeds,
                         int64_t *coverage, double *latency_ms);
/* As im_server_poll, blocking up to timeout_s seconds (IM_ERR_BUSY on timeout). */
im_status im_server_wait(im_server *s, uint64_t ticket, double timeout_s, int32_t *seeds,
                         int32_t *num_seeds, int64_t *coverage, double *latency_ms);
/* Batches run, requests they held, requests still queued. */
im_status im_server_stats(im_server *s, int64_t *batches, int64_t *queries, int64_t *queued);

/* ---- spread of a seed set by forward simulation (Sec. 2; Sec. 4.1) ---------------
 * The influence spread sigma(S) is the expected number of vertices S activates.
 * Run r (r = first_run .. first_run + runs - 1) simulates the live-edge world of
 * RRR sample r -- the IC coins and LT picks im_sample_rrr uses for sample id r
 * under the same seed -- forward from S and counts the activated vertices.
 *   seeds      int32[k], host or device; duplicates allowed; ids in [0, n)
 *              (IM_ERR_INVALID_ARG otherwise)
 *   activated  int64[runs] (host or device, may be NULL): |activated set| of each run
 *   root_hit   uint8[runs] (host or device, may be NULL): 1 iff the run's root (the
 *              root of RRR sample r) is activated -- by the RIS identity, iff S
 *              meets RRR set r, so sum(root_hit) over runs 0 .. theta-1 equals the
 *              coverage of S on a pool of those samples
 *   total      host int64 (may be NULL): sum of activated; total / runs estimates
 *              sigma(S)
 * LT requires lt_valid.  Builds the graph's out-edge index on first use (kept
 * with the graph).  Device scratch is allocated stream-ordered per call.
 * Synchronises the stream. */
im_status im_spread(const im_graph *g, im_model model, const int32_t *seeds, int32_t k,
                    uint64_t seed, uint64_t first_run, uint64_t runs, int64_t *activated,
                    uint8_t *root_hit, int64_t *total, void *stream);

/* Vertex partition of Alg. 3: part[v] = (Philox(v,0,0,4).x * P) >> 32. */
im_status im_partition(int64_t n, int32_t P, uint64_t partition_seed, int32_t *part,
                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IM_H */
