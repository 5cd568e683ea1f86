/* oracle.c -- plain, slow, single-threaded CPU oracle for the RIS hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file; the product path never does.
 * It shares no code, header or table with the CUDA library: every definition
 * below is written out here from the paper (GreediRIS, arXiv 2408.10982) and,
 * for the random stream, from the Philox paper.
 *
 * Readings of the paper that this file fixes (the paper is silent on them):
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = 64-bit
 *    seed split (lo, hi); counters carry a domain tag in word 3:
 *      ROOT (s, 0, 0, 1) lane 0 ; IC coin (s, e>>2, e>>34, 2) lane e&3 ;
 *      LT draw (s, v, 0, 3) lane 0 ; partition (v, 0, 0, 4) lane 0.
 *  - uniform choice of x in [0, N) from a 32-bit draw r: (r * N) >> 32.
 *  - IC edge e is live iff its coin < w[e]; LT vertex v picks the first
 *    in-edge (CSR order) whose running weight sum exceeds its draw.
 *  - greedy ties go to the smallest vertex id; zero gain ends the greedy.
 *  - RandGreedi streams seeds in (rank j, partition p) order; bucket b has
 *    guess l*(1+delta)^b with l = max_v |S(v)|, and accepts a subset whose
 *    gain is >= ceil(guess / (2k)); B = least b >= 1 with (1+delta)^b >= k.
 * Floating point appears only in those thresholds (IEEE double, repeated
 * multiplication, no pow/log) so both sides can reproduce them exactly.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplies with   */
/* a Weyl-sequence key schedule.                                             */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;   /* multiplier M0 */
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;   /* multiplier M1 */
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;                          /* Weyl constants */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { TAG_ROOT = 1, TAG_IC = 2, TAG_LT = 3, TAG_PART = 4 };

static uint32_t draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c,
                     uint32_t tag, int lane) {
    uint32_t ctr[4] = {a, b, c, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox(ctr, key, out);
    return out[lane];
}

/* Sample s picks its source uniformly from V (Sec. 2.1, Sample step 1). */
uint32_t orc_root(uint64_t seed, uint32_t s, int64_t n) {
    uint32_t r = draw(seed, s, 0, 0, TAG_ROOT, 0);
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* The 32-bit coin of in-edge e in sample s (IC live-edge world, Def. 3). */
uint32_t orc_ic_coin(uint64_t seed, uint32_t s, int64_t e) {
    uint64_t ue = (uint64_t)e;
    return draw(seed, s, (uint32_t)(ue >> 2), (uint32_t)(ue >> 34), TAG_IC, (int)(ue & 3u));
}

/* The 32-bit draw vertex v uses to pick its live in-edge in sample s (LT). */
uint32_t orc_lt_draw(uint64_t seed, uint32_t s, uint32_t v) {
    return draw(seed, s, v, 0, TAG_LT, 0);
}

/* Uniform random vertex partition into P parts (Alg. 3, "Partition V"). */
int32_t orc_part_of(uint64_t pseed, uint32_t v, int32_t P) {
    uint32_t r = draw(pseed, v, 0, 0, TAG_PART, 0);
    return (int32_t)(((uint64_t)r * (uint64_t)P) >> 32);
}

void orc_partition(int64_t n, int32_t P, uint64_t pseed, int32_t *part) {
    for (int64_t v = 0; v < n; ++v) part[v] = orc_part_of(pseed, (uint32_t)v, P);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* One RRR set (Def. 3; Sec. 2.1 "Sample"): all vertices with a path to the */
/* root in the random live-edge subgraph, found by BFS over in-edges.  Each */
/* in-edge of each visited vertex gets its coin exactly once.  Writes the   */
/* members to out[] in discovery order, returns the count.                  */
/* visited[] (n bytes) must be all zero and is left all zero.               */
/* ------------------------------------------------------------------------ */
int64_t orc_sample_ic_one(int64_t n, const int64_t *in_off, const int32_t *in_src,
                          const uint32_t *w, uint64_t seed, uint32_t s,
                          uint8_t *visited, int32_t *out, int64_t *examined) {
    uint32_t root = orc_root(seed, s, n);
    int64_t tail = 0;
    out[tail++] = (int32_t)root;
    visited[root] = 1;
    for (int64_t head = 0; head < tail; ++head) {
        int32_t v = out[head];
        for (int64_t e = in_off[v]; e < in_off[v + 1]; ++e) {
            ++*examined;
            if (orc_ic_coin(seed, s, e) < w[e]) {
                int32_t u = in_src[e];
                if (!visited[u]) {
                    visited[u] = 1;
                    out[tail++] = u;
                }
            }
        }
    }
    for (int64_t t = 0; t < tail; ++t) visited[out[t]] = 0;
    return tail;
}

/* ------------------------------------------------------------------------ */
/* One LT RRR set.  In the LT live-edge world each vertex keeps at most one */
/* in-edge, chosen with probability equal to its weight (weights of a       */
/* vertex sum to at most 1, Sec. 2).  The reverse-reachable set of the root */
/* is then the backward chain root <- pick(root) <- ... which stops at a    */
/* vertex that picks nothing or at an already-visited vertex.  Writes the   */
/* chain in walk order, returns its length.                                 */
/* ------------------------------------------------------------------------ */
int64_t orc_sample_lt_one(int64_t n, const int64_t *in_off, const int32_t *in_src,
                          const uint32_t *w, uint64_t seed, uint32_t s,
                          uint8_t *visited, int32_t *out, int64_t *examined) {
    uint32_t cur = orc_root(seed, s, n);
    int64_t len = 0;
    out[len++] = (int32_t)cur;
    visited[cur] = 1;
    for (;;) {
        uint32_t x = orc_lt_draw(seed, s, cur);
        uint64_t run = 0;
        int64_t pick = -1;
        for (int64_t e = in_off[cur]; e < in_off[cur + 1]; ++e) {
            ++*examined;
            run += w[e];
            if ((uint64_t)x < run) { pick = e; break; }
        }
        if (pick < 0) break;
        int32_t u = in_src[pick];
        if (visited[u]) break;
        visited[u] = 1;
        out[len++] = u;
        cur = (uint32_t)u;
    }
    for (int64_t t = 0; t < len; ++t) visited[out[t]] = 0;
    return len;
}

/* ------------------------------------------------------------------------ */
/* Sample(G, count) for ids first .. first+count-1 (Alg. 1 "Sample"; each    */
/* sample keeps its id, Sec. 3.2).  Output: CSR by sample id; members sorted */
/* ascending unless keep_order != 0 (then discovery / walk order).  Arrays   */
/* are malloc'd here and released with orc_free.  model 0 = IC, 1 = LT.      */
/* Returns 0, or -1 on allocation failure.                                   */
/* ------------------------------------------------------------------------ */
int orc_sample(int model, int64_t n, const int64_t *in_off, const int32_t *in_src,
               const uint32_t *w, uint64_t seed, uint64_t first, uint64_t count,
               int keep_order, int64_t **set_off_out, int32_t **members_out,
               int64_t *total_out, int64_t *examined_out) {
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    int32_t *buf = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *set_off = (int64_t *)malloc((size_t)(count + 1) * sizeof(int64_t));
    int64_t cap = 1024, total = 0, examined = 0;
    int32_t *members = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (!visited || !buf || !set_off || !members) goto fail;
    set_off[0] = 0;
    for (uint64_t j = 0; j < count; ++j) {
        uint32_t s = (uint32_t)(first + j);
        int64_t len = model == 0
            ? orc_sample_ic_one(n, in_off, in_src, w, seed, s, visited, buf, &examined)
            : orc_sample_lt_one(n, in_off, in_src, w, seed, s, visited, buf, &examined);
        if (!keep_order) qsort(buf, (size_t)len, sizeof(int32_t), cmp_i32);
        if (total + len > cap) {
            while (total + len > cap) cap *= 2;
            int32_t *grown = (int32_t *)realloc(members, (size_t)cap * sizeof(int32_t));
            if (!grown) goto fail;
            members = grown;
        }
        memcpy(members + total, buf, (size_t)len * sizeof(int32_t));
        total += len;
        set_off[j + 1] = total;
    }
    free(visited);
    free(buf);
    *set_off_out = set_off;
    *members_out = members;
    *total_out = total;
    *examined_out = examined;
    return 0;
fail:
    free(visited); free(buf); free(set_off); free(members);
    return -1;
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Covering subsets S(v) = { i : v in R(i) } (Sec. 3.2, max-k-cover          */
/* formulation; the all-to-all of Alg. 3 gathers exactly these rows).        */
/* set_ids of each vertex come out in ascending set id.                      */
/* ------------------------------------------------------------------------ */
int orc_invert(int64_t n, int64_t theta, const int64_t *set_off, const int32_t *members,
               int64_t *vtx_off, int32_t *set_ids) {
    int64_t *cursor = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cursor) return -1;
    for (int64_t t = 0; t < set_off[theta]; ++t) cursor[members[t] + 1]++;
    vtx_off[0] = 0;
    for (int64_t v = 0; v < n; ++v) vtx_off[v + 1] = vtx_off[v] + cursor[v + 1];
    for (int64_t v = 0; v < n; ++v) cursor[v] = vtx_off[v];
    for (int64_t i = 0; i < theta; ++i)
        for (int64_t t = set_off[i]; t < set_off[i + 1]; ++t)
            set_ids[cursor[members[t]]++] = (int32_t)i;
    free(cursor);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Standard greedy max-k-cover (Sec. 3.2: repeatedly take the covering      */
/* subset of largest marginal gain).  Candidates are the ascending vertex   */
/* list cand[0..ncand) when cand is non-NULL (the local greedy of a         */
/* partition V_p, Alg. 4), else all of V; the universe is {0..theta-1}.     */
/* counts[v] is the marginal gain |S(v) \ covered|, kept exact by           */
/* decrementing the members of every newly covered set.                     */
/* Returns 0, or -1 on allocation failure.                                  */
/* ------------------------------------------------------------------------ */
int orc_greedy(int64_t n, int64_t theta, const int64_t *set_off, const int32_t *members,
               const int64_t *vtx_off, const int32_t *set_ids, int32_t k,
               const int32_t *cand, int64_t ncand, int32_t *seeds, int64_t *gains,
               int32_t *nseeds, int64_t *coverage) {
    int64_t *counts = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint8_t *covered = (uint8_t *)calloc((size_t)theta + 1, 1);
    if (!counts || !covered) { free(counts); free(covered); return -1; }
    for (int64_t v = 0; v < n; ++v) counts[v] = vtx_off[v + 1] - vtx_off[v];
    int64_t cov = 0;
    int32_t picked = 0;
    for (int32_t j = 0; j < k; ++j) {
        int64_t best = -1, best_gain = 0;
        int64_t span = cand ? ncand : n;
        for (int64_t c = 0; c < span; ++c) {
            int64_t v = cand ? cand[c] : c;
            if (counts[v] > best_gain) { best = v; best_gain = counts[v]; }
        }
        if (best < 0) break;                 /* every remaining gain is zero */
        seeds[picked] = (int32_t)best;
        gains[picked] = best_gain;
        ++picked;
        cov += best_gain;
        for (int64_t t = vtx_off[best]; t < vtx_off[best + 1]; ++t) {
            int32_t i = set_ids[t];
            if (covered[i]) continue;
            covered[i] = 1;
            for (int64_t q = set_off[i]; q < set_off[i + 1]; ++q) counts[members[q]]--;
        }
    }
    *nseeds = picked;
    *coverage = cov;
    free(counts);
    free(covered);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lazy greedy max-k-cover (Alg. 2): a max heap Q of (key, vertex) built    */
/* from |S(v)|; pop the top v, compute its marginal gain against the sets   */
/* covered so far; take v when the gain is at least the new top's key, else */
/* push v back with its gain as the key.  Keys order by (value, smaller id  */
/* first), so "at least" with equal values means v's id is the smaller one  */
/* (the tie rule of the standard greedy).  A popped gain of 0 that would be */
/* taken ends the selection (zero-gain stop).  Candidates as in orc_greedy. */
/* Returns 0, or -1 on allocation failure.                                  */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t key; int32_t v; } orc_hent;

static int orc_hent_above(orc_hent a, orc_hent b) {   /* a ranks above b */
    return a.key > b.key || (a.key == b.key && a.v < b.v);
}

static void orc_heap_push(orc_hent *h, int64_t *len, orc_hent x) {
    int64_t i = (*len)++;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (!orc_hent_above(x, h[parent])) break;
        h[i] = h[parent];
        i = parent;
    }
    h[i] = x;
}

static orc_hent orc_heap_pop(orc_hent *h, int64_t *len) {
    orc_hent top = h[0], last = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *len) break;
        if (c + 1 < *len && orc_hent_above(h[c + 1], h[c])) ++c;
        if (!orc_hent_above(h[c], last)) break;
        h[i] = h[c];
        i = c;
    }
    if (*len > 0) h[i] = last;
    return top;
}

int orc_lazy_greedy(int64_t n, int64_t theta, const int64_t *vtx_off, const int32_t *set_ids,
                    int32_t k, const int32_t *cand, int64_t ncand, int32_t *seeds,
                    int64_t *gains, int32_t *nseeds, int64_t *coverage) {
    int64_t span = cand ? ncand : n, len = 0;
    orc_hent *Q = (orc_hent *)malloc((size_t)(span > 0 ? span : 1) * sizeof(orc_hent));
    uint8_t *covered = (uint8_t *)calloc((size_t)theta + 1, 1);
    if (!Q || !covered) { free(Q); free(covered); return -1; }
    for (int64_t c = 0; c < span; ++c) {
        int32_t v = cand ? cand[c] : (int32_t)c;
        orc_hent x = { vtx_off[v + 1] - vtx_off[v], v };
        orc_heap_push(Q, &len, x);
    }
    int32_t picked = 0;
    int64_t cov = 0;
    while (picked < k && len > 0) {
        orc_hent top = orc_heap_pop(Q, &len);
        int64_t gain = 0;
        for (int64_t t = vtx_off[top.v]; t < vtx_off[top.v + 1]; ++t) gain += !covered[set_ids[t]];
        orc_hent now = { gain, top.v };
        if (len == 0 || !orc_hent_above(Q[0], now)) {
            if (gain == 0) break;              /* every remaining gain is zero */
            seeds[picked] = top.v;
            gains[picked] = gain;
            ++picked;
            cov += gain;
            for (int64_t t = vtx_off[top.v]; t < vtx_off[top.v + 1]; ++t) covered[set_ids[t]] = 1;
        } else {
            orc_heap_push(Q, &len, now);
        }
    }
    *nseeds = picked;
    *coverage = cov;
    free(Q);
    free(covered);
    return 0;
}

/* Number of buckets B = ceil(log_{1+delta}(u/l)) with u/l = k (Alg. 5;        */
/* u/l = k per the runtime analysis of Sec. 3.4), taken as the least b >= 1    */
/* with (1+delta)^b >= k, the power formed by repeated multiplication.        */
int32_t orc_num_buckets(int32_t k, double delta) {
    double x = 1.0;
    int32_t b = 0;
    while (x < (double)k) { x *= 1.0 + delta; ++b; }
    return b < 1 ? 1 : b;
}

/* Integer acceptance threshold of each bucket: ceil(l (1+delta)^b / (2k)). */
void orc_bucket_thresholds(int64_t l, int32_t k, double delta, int32_t B, int64_t *thr) {
    double guess = (double)l;
    for (int32_t b = 0; b < B; ++b) {
        thr[b] = (int64_t)ceil(guess / (2.0 * (double)k));
        guess *= 1.0 + delta;
    }
}

/* ------------------------------------------------------------------------ */
/* Streaming max-k-cover at the receiver (Alg. 5).  Elements arrive in the  */
/* order given by stream[0..nstream); each is a vertex id x carrying S(x).  */
/* Every bucket b, independently, appends x when it holds fewer than k      */
/* seeds and |S(x) \ C_b| >= thr[b].  Outputs per-bucket coverage |C_b|,    */
/* seed counts, seeds (B*k) and marginal gains (B*k).                       */
/* ------------------------------------------------------------------------ */
int orc_stream_buckets(int64_t theta, const int64_t *vtx_off, const int32_t *set_ids,
                       const int32_t *stream, int64_t nstream, int32_t k, int32_t B,
                       const int64_t *thr, int64_t *bucket_cov, int32_t *bucket_n,
                       int32_t *bucket_seeds, int64_t *bucket_gains) {
    uint8_t *cov = (uint8_t *)calloc((size_t)B * (size_t)(theta + 1), 1);
    if (!cov) return -1;
    for (int32_t b = 0; b < B; ++b) { bucket_cov[b] = 0; bucket_n[b] = 0; }
    for (int64_t q = 0; q < nstream; ++q) {
        int32_t x = stream[q];
        for (int32_t b = 0; b < B; ++b) {
            if (bucket_n[b] >= k) continue;
            uint8_t *C = cov + (size_t)b * (size_t)(theta + 1);
            int64_t gain = 0;
            for (int64_t t = vtx_off[x]; t < vtx_off[x + 1]; ++t) gain += !C[set_ids[t]];
            if (gain < thr[b]) continue;
            for (int64_t t = vtx_off[x]; t < vtx_off[x + 1]; ++t) C[set_ids[t]] = 1;
            bucket_seeds[(int64_t)b * k + bucket_n[b]] = x;
            bucket_gains[(int64_t)b * k + bucket_n[b]] = gain;
            bucket_n[b]++;
            bucket_cov[b] += gain;
        }
    }
    free(cov);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* RandGreedi max-k-cover with streaming aggregation and truncation         */
/* (Alg. 3 partition, Alg. 4 local greedy + final compare, Alg. 5 stream,   */
/* Sec. 3.3.2 truncation: each partition computes all k local seeds and     */
/* streams only its first `trunc`).  The partitions run one after another. */
/* naive != 0: Alg. 4's global step is the lazy greedy over the gathered    */
/* seeds instead of the streaming buckets (B = 1).                          */
/* Outputs:                                                                 */
/*   local_seeds/local_gains [P*k], local_n [P], local_cov [P]              */
/*   B, thr [B], bucket_cov [B], bucket_n [B], bucket_seeds [B*k],          */
/*   bucket_gains [B*k] (caller sizes them with orc_num_buckets)            */
/*   chosen: -1 when the best bucket wins, else the winning partition p     */
/*   seeds/gains [k], nseeds, coverage: the final solution                  */
/* ------------------------------------------------------------------------ */
int orc_randgreedi(int64_t n, int64_t theta, const int64_t *set_off, const int32_t *members,
                   const int64_t *vtx_off, const int32_t *set_ids, int32_t k, int32_t P,
                   uint64_t pseed, int32_t trunc, double delta, int32_t naive,
                   int32_t *local_seeds, int64_t *local_gains, int32_t *local_n,
                   int64_t *local_cov, int64_t *thr, int64_t *bucket_cov, int32_t *bucket_n,
                   int32_t *bucket_seeds, int64_t *bucket_gains, int32_t *chosen,
                   int32_t *seeds, int64_t *gains, int32_t *nseeds, int64_t *coverage) {
    int32_t *part = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *allowed = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *stream = (int32_t *)malloc((size_t)P * (size_t)k * sizeof(int32_t));
    if (!part || !allowed || !stream) { free(part); free(allowed); free(stream); return -1; }
    orc_partition(n, P, pseed, part);

    /* local greedy on every partition V_p, all k seeds */
    for (int32_t p = 0; p < P; ++p) {
        int64_t nc = 0;
        for (int64_t v = 0; v < n; ++v) if (part[v] == p) allowed[nc++] = (int32_t)v;
        if (orc_greedy(n, theta, set_off, members, vtx_off, set_ids, k, allowed, nc,
                       local_seeds + (int64_t)p * k, local_gains + (int64_t)p * k,
                       &local_n[p], &local_cov[p])) {
            free(part); free(allowed); free(stream); return -1;
        }
    }

    /* stream order: local rank j first, then partition p */
    int64_t ns = 0;
    for (int32_t j = 0; j < trunc && j < k; ++j)
        for (int32_t p = 0; p < P; ++p)
            if (j < local_n[p]) stream[ns++] = local_seeds[(int64_t)p * k + j];

    int32_t B;
    if (naive) {
        /* Alg. 4 as written: the lazy greedy (Alg. 2) over the union of the   */
        /* gathered local seeds, reported as bucket 0 with threshold 0        */
        B = 1;
        thr[0] = 0;
        if (orc_lazy_greedy(n, theta, vtx_off, set_ids, k, stream, ns, bucket_seeds,
                            bucket_gains, &bucket_n[0], &bucket_cov[0])) {
            free(part); free(allowed); free(stream); return -1;
        }
    } else {
        /* l = largest single covering subset; u = k l */
        int64_t l = 0;
        for (int64_t v = 0; v < n; ++v)
            if (vtx_off[v + 1] - vtx_off[v] > l) l = vtx_off[v + 1] - vtx_off[v];
        B = orc_num_buckets(k, delta);
        orc_bucket_thresholds(l, k, delta, B, thr);
        if (orc_stream_buckets(theta, vtx_off, set_ids, stream, ns, k, B, thr, bucket_cov,
                               bucket_n, bucket_seeds, bucket_gains)) {
            free(part); free(allowed); free(stream); return -1;
        }
    }

    /* best bucket (ties: smallest b) vs best local solution (ties: smallest p) */
    int32_t bstar = 0;
    for (int32_t b = 1; b < B; ++b) if (bucket_cov[b] > bucket_cov[bstar]) bstar = b;
    int32_t pbest = 0;
    for (int32_t p = 1; p < P; ++p) if (local_cov[p] > local_cov[pbest]) pbest = p;
    if (bucket_cov[bstar] >= local_cov[pbest]) {
        *chosen = -1;
        *nseeds = bucket_n[bstar];
        *coverage = bucket_cov[bstar];
        for (int32_t j = 0; j < bucket_n[bstar]; ++j) {
            seeds[j] = bucket_seeds[(int64_t)bstar * k + j];
            gains[j] = bucket_gains[(int64_t)bstar * k + j];
        }
    } else {
        *chosen = pbest;
        *nseeds = local_n[pbest];
        *coverage = local_cov[pbest];
        for (int32_t j = 0; j < local_n[pbest]; ++j) {
            seeds[j] = local_seeds[(int64_t)pbest * k + j];
            gains[j] = local_gains[(int64_t)pbest * k + j];
        }
    }
    free(part); free(allowed); free(stream);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Forward simulation of the diffusion from a seed set: the expected number */
/* of vertices the seeds activate, sigma(S), is what the selected seeds are */
/* judged by (Sec. 2, Def. of influence spread; Sec. 4.1 reports it).  Run */
/* r uses the live-edge world of sample id r -- the IC coins and LT picks */
/* of RRR sample r -- and activates every vertex reachable from S over live */
/* edges (BFS over out-edges).  IC: in-edge e is live iff its coin < w[e]. */
/* LT: in-edge e of v is live iff it is v's pick, found by scanning v's     */
/* in-edges with the running weight sum.                                    */
/* Outputs per run: activated[i] = |Reach(S)|, root_hit[i] = 1 if the root */
/* of sample r is activated -- by the RIS identity, exactly when S meets    */
/* RRR set r.                                                               */
/* ------------------------------------------------------------------------ */
static int64_t lt_pick(const int64_t *in_off, const uint32_t *w, uint64_t seed, uint32_t s,
                       uint32_t v) {
    uint32_t x = orc_lt_draw(seed, s, v);
    uint64_t c = 0;
    for (int64_t e = in_off[v]; e < in_off[v + 1]; ++e) {
        c += w[e];
        if ((uint64_t)x < c) return e;
    }
    return -1;
}

int orc_spread(int model, int64_t n, const int64_t *in_off, const int32_t *in_src,
               const uint32_t *w, uint64_t seed, uint64_t first, uint64_t runs,
               const int32_t *seeds, int32_t k, int64_t *activated, uint8_t *root_hit) {
    int64_t m = in_off[n];
    int32_t *dst = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int64_t *out_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *out_e = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!dst || !out_off || !out_e || !fill || !visited || !queue) {
        free(dst); free(out_off); free(out_e); free(fill); free(visited); free(queue);
        return -1;
    }
    /* head of every in-edge, and the out-edges of every vertex (in-CSR ids) */
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = in_off[v]; e < in_off[v + 1]; ++e) dst[e] = (int32_t)v;
    for (int64_t e = 0; e < m; ++e) out_off[in_src[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) out_off[v + 1] += out_off[v];
    for (int64_t v = 0; v < n; ++v) fill[v] = out_off[v];
    for (int64_t e = 0; e < m; ++e) out_e[fill[in_src[e]]++] = e;

    for (uint64_t i = 0; i < runs; ++i) {
        uint32_t s = (uint32_t)(first + i);
        int64_t tail = 0;
        for (int32_t j = 0; j < k; ++j) {
            int32_t u = seeds[j];
            if (!visited[u]) { visited[u] = 1; queue[tail++] = u; }
        }
        for (int64_t head = 0; head < tail; ++head) {
            int32_t u = queue[head];
            for (int64_t t = out_off[u]; t < out_off[u + 1]; ++t) {
                int64_t e = out_e[t];
                int32_t v = dst[e];
                if (visited[v]) continue;
                int live = model == 0 ? orc_ic_coin(seed, s, e) < w[e]
                                      : lt_pick(in_off, w, seed, s, (uint32_t)v) == e;
                if (live) { visited[v] = 1; queue[tail++] = v; }
            }
        }
        activated[i] = tail;
        if (root_hit) root_hit[i] = visited[orc_root(seed, s, n)];
        for (int64_t t = 0; t < tail; ++t) visited[queue[t]] = 0;
    }
    free(dst); free(out_off); free(out_e); free(fill); free(visited); free(queue);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* IMM sampling-effort formulas.  Alg. 1 (Sec. 2.1) names Estimate,          */
/* CheckGoodness and theta = f(LB) but defers their values to Tang et al.    */
/* (SIGMOD 2015) and Chen (2018); they are written out here from that work,  */
/* natural logs throughout:                                                  */
/*   l' = l (1 + ln 2 / ln n),  e' = sqrt(2) e,                              */
/*   lambda' = (2 + 2e'/3) (ln C(n,k) + l' ln n + ln log2 n) n / e'^2,        */
/*   alpha = sqrt(l' ln n + ln 2),                                           */
/*   beta  = sqrt((1 - 1/e) (ln C(n,k) + l' ln n + ln 2)),                   */
/*   lambda* = 2 n ((1 - 1/e) alpha + beta)^2 / e^2,                         */
/*   round i = 1 .. floor(log2 n) - 1: x_i = n / 2^i, theta_i = ceil(lambda'/x_i) */
/* out: [0] l', [1] e', [2] lambda', [3] lambda*, [4] number of rounds.     */
/* ------------------------------------------------------------------------ */
void orc_imm_constants(int64_t n, int32_t k, double eps, double ell, double out[5]) {
    const double dn = (double)n;
    const double ln_n = log(dn);
    const double lncnk = lgamma(dn + 1.0) - lgamma((double)k + 1.0) - lgamma(dn - (double)k + 1.0);
    const double l2 = ell * (1.0 + log(2.0) / ln_n);
    const double e2 = sqrt(2.0) * eps;
    const double lam1 = (2.0 + 2.0 * e2 / 3.0) * (lncnk + l2 * ln_n + log(log2(dn))) * dn / (e2 * e2);
    const double one_e = 1.0 - exp(-1.0);
    const double alpha = sqrt(l2 * ln_n + log(2.0));
    const double beta = sqrt(one_e * (lncnk + l2 * ln_n + log(2.0)));
    const double lamstar = 2.0 * dn * (one_e * alpha + beta) * (one_e * alpha + beta) / (eps * eps);
    int32_t rounds = 0;
    while (((int64_t)1 << (rounds + 2)) <= n) ++rounds;   /* floor(log2 n) - 1 */
    out[0] = l2;
    out[1] = e2;
    out[2] = lam1;
    out[3] = lamstar;
    out[4] = (double)rounds;
}

/* theta_i = ceil(lambda' / x_i), x_i = n / 2^i (Alg. 1's doubling theta-hat). */
int64_t orc_imm_round_theta(double lam1, int64_t n, int32_t i) {
    const double x = (double)n / ldexp(1.0, i);
    return (int64_t)ceil(lam1 / x);
}

/* CheckGoodness: with F = coverage / theta_i, pass iff n F >= (1 + e') x_i;  */
/* then LB = n F / (1 + e').  Returns 1 on pass.                             */
int orc_imm_check(int64_t n, int64_t coverage, int64_t theta_i, int32_t i, double e2, double *lb) {
    const double x = (double)n / ldexp(1.0, i);
    const double spread = (double)n * ((double)coverage / (double)theta_i);
    if (spread >= (1.0 + e2) * x) {
        *lb = spread / (1.0 + e2);
        return 1;
    }
    return 0;
}

/* Final sample count theta = ceil(lambda* / LB). */
int64_t orc_imm_final_theta(double lamstar, double lb) { return (int64_t)ceil(lamstar / lb); }

/* ------------------------------------------------------------------------ */
/* OPIM's instance-wise guarantee (Sec. 3.3.2 / Sec. 4.4 use OPIM of Tang   */
/* et al. 2018 in place of IMM; the paper prints none of its formulas, so   */
/* they are written out here from that work, natural logs throughout):      */
/*   theta_max = 2n ((1-1/e) sqrt(ln(6/delta))                              */
/*               + sqrt((1-1/e)(ln C(n,k) + ln(6/delta))))^2 / (eps^2 k)    */
/*   theta_0 = ceil(theta_max eps^2 k / n), theta_i = theta_0 2^(i-1)       */
/*   i_max = max(1, ceil(log2(theta_max / theta_0))), lowered to the last   */
/*   round whose theta_i stays within cap (cap > 0)                         */
/*   a = ln(3 i_max / delta)  (the failure budget of one bound in a round)  */
/* out: [0] theta_max, [1] theta_0, [2] i_max, [3] a.                       */
/* ------------------------------------------------------------------------ */
void orc_opim_constants(int64_t n, int32_t k, double eps, double delta, int64_t cap,
                        double out[4]) {
    const double dn = (double)n;
    const double lncnk = lgamma(dn + 1.0) - lgamma((double)k + 1.0) - lgamma(dn - (double)k + 1.0);
    const double one_e = 1.0 - exp(-1.0);
    const double l6 = log(6.0 / delta);
    const double s = one_e * sqrt(l6) + sqrt(one_e * (lncnk + l6));
    const double tmax = 2.0 * dn * s * s / (eps * eps * (double)k);
    const double t0 = ceil(tmax * eps * eps * (double)k / dn);
    int32_t imax = (int32_t)ceil(log2(tmax / t0));
    if (imax < 1) imax = 1;
    if (cap > 0) {
        int32_t fit = 1;
        while (fit < imax && ldexp(t0, fit) <= (double)cap) ++fit;   /* theta_{fit+1} <= cap */
        imax = fit;
    }
    out[0] = tmax;
    out[1] = t0;
    out[2] = (double)imax;
    out[3] = log(3.0 * (double)imax / delta);
}

/* Lower confidence bound on the spread of S from its coverage cov2 of the */
/* theta validation sets R2: the x solving cov2 = x + a/3 + sqrt(a^2/9 + 2ax) */
/* (upper martingale tail at budget e^-a), times n / theta.                 */
double orc_opim_lower(int64_t cov2, int64_t theta, int64_t n, double a) {
    const double r = sqrt((double)cov2 + 2.0 * a / 9.0) - sqrt(a / 2.0);
    return (r * r - a / 18.0) * (double)n / (double)theta;
}

/* Upper confidence bound on OPT from an upper bound cov1u of the optimal  */
/* k-set's coverage of the theta selection sets R1: the x solving           */
/* cov1u = x - sqrt(2ax) (lower tail), times n / theta.                     */
double orc_opim_upper(int64_t cov1u, int64_t theta, int64_t n, double a) {
    const double r = sqrt((double)cov1u + a / 2.0) + sqrt(a / 2.0);
    return r * r * (double)n / (double)theta;
}
