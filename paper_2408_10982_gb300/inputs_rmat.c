/* R-MAT edge generator for the synthetic inputs (fixture code, not the method).
 *
 * Candidates are drawn in order from a splitmix64 stream keyed by the seed
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014).  Each 64-bit output gives two 32-bit draws, one per R-MAT
 * level; a draw r picks the quadrant a (r < t1), b (r < t2), c (r < t3) or d,
 * which appends bits (0,0), (0,1), (1,0), (1,1) to (src, dst).  Candidates
 * with an endpoint >= n, self-loops and repeats are dropped; generation stops
 * after m distinct edges: the edges are the first m distinct valid
 * candidates in stream order.
 *
 * splitmix64's j-th output depends only on seed + (j + 1) * gamma, so candidate
 * c (which takes outputs c h .. c h + h - 1, h = ceil(levels / 2)) can be made
 * on its own: threads make the keys of a pass's candidates in parallel.  Then
 * threads split the key space by hash: each scans the keys in stream order
 * and keeps a hash set of the keys it owns, so a key's first occurrence is
 * found by the one thread that owns it, whatever the number of threads.  A
 * final pass writes the first m accepted candidates in order.
 * Portable C99 + POSIX threads: no intrinsics, same output on every host.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static const uint64_t kGamma = 0x9E3779B97F4A7C15ull;

static uint64_t splitmix64_at(uint64_t seed, uint64_t j) {   /* the j-th output */
    uint64_t z = seed + (j + 1) * kGamma;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t mix_key(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    return k;
}

typedef struct {
    int64_t n;
    int32_t levels;
    uint64_t seed;
    uint32_t t1, t2, t3;
} rmat_params;

/* Candidate c: returns 1 and its key s n + d when it is a valid edge. */
static int candidate(const rmat_params *p, uint64_t c, uint64_t *key) {
    const int32_t h = (p->levels + 1) / 2;
    uint64_t s = 0, d = 0, buf = 0;
    int avail = 0;
    uint64_t j = c * (uint64_t)h;
    for (int32_t l = 0; l < p->levels; ++l) {
        if (!avail) { buf = splitmix64_at(p->seed, j++); avail = 2; }
        uint32_t r = (uint32_t)(buf & 0xffffffffu);
        buf >>= 32;
        --avail;
        uint64_t sb = r >= p->t2;
        uint64_t db = (uint64_t)((r >= p->t1) ^ (r >= p->t2) ^ (r >= p->t3));
        s = (s << 1) | sb;
        d = (d << 1) | db;
    }
    if (s >= (uint64_t)p->n || d >= (uint64_t)p->n || s == d) return 0;
    *key = s * (uint64_t)p->n + d;
    return 1;
}

typedef struct {
    const rmat_params *p;
    uint64_t c0, c1;              /* candidates [c0, c1) of this pass ... */
    uint64_t *keys;               /* ... made into keys[c - base], UINT64_MAX if invalid */
    uint64_t base;
} make_job;

static void *make_run(void *arg) {
    make_job *mj = (make_job *)arg;
    for (uint64_t c = mj->c0; c < mj->c1; ++c) {
        uint64_t key;
        mj->keys[c - mj->base] = candidate(mj->p, c, &key) ? key : UINT64_MAX;
    }
    return NULL;
}

typedef struct {
    int32_t t, T;
    uint64_t *table;              /* this thread's keys (open addressing) */
    uint64_t cap;
    const uint64_t *keys;         /* the pass's candidates, in stream order */
    uint64_t count;
    uint8_t *acc;                 /* acc[i] = 1: keys[i] is a first occurrence */
    int64_t accepted;
} owner_job;

static void *owner_run(void *arg) {
    owner_job *o = (owner_job *)arg;
    int64_t got = 0;
    for (uint64_t i = 0; i < o->count; ++i) {
        const uint64_t key = o->keys[i];
        if (key == UINT64_MAX) continue;
        const uint64_t hk = mix_key(key);
        if ((int32_t)((hk >> 40) % (uint64_t)o->T) != o->t) continue;
        uint64_t h = hk & (o->cap - 1);
        int fresh = 1;
        while (o->table[h] != UINT64_MAX) {
            if (o->table[h] == key) { fresh = 0; break; }
            h = (h + 1) & (o->cap - 1);
        }
        if (!fresh) continue;
        o->table[h] = key;
        o->acc[i] = 1;
        ++got;
    }
    o->accepted = got;
    return NULL;
}

typedef struct {
    int64_t n;
    const uint64_t *keys;
    const uint8_t *acc;
    uint64_t i0, i1;
    int64_t out0, out_end;        /* first output slot, and the end of the output */
    int64_t *src, *dst;
} write_job;

static void *write_run(void *arg) {
    write_job *w = (write_job *)arg;
    int64_t at = w->out0;
    for (uint64_t i = w->i0; i < w->i1 && at < w->out_end; ++i) {
        if (!w->acc[i]) continue;
        w->src[at] = (int64_t)(w->keys[i] / (uint64_t)w->n);
        w->dst[at] = (int64_t)(w->keys[i] % (uint64_t)w->n);
        ++at;
    }
    return NULL;
}

static int32_t thread_count(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 32) c = 32;
    return (int32_t)c;
}

/* Returns the number of accepted edges (== m on success, smaller when the
 * candidate budget ran out), or -1 when memory could not be allocated. */
int64_t rmat_generate(int64_t n, int64_t m, int32_t levels, uint64_t seed,
                      uint32_t t1, uint32_t t2, uint32_t t3,
                      int64_t *src_out, int64_t *dst_out) {
    rmat_params p = {n, levels, seed, t1, t2, t3};
    const int32_t T = thread_count();
    owner_job *own = (owner_job *)calloc((size_t)T, sizeof(owner_job));
    make_job *mk = (make_job *)calloc((size_t)T, sizeof(make_job));
    write_job *wj = (write_job *)calloc((size_t)T, sizeof(write_job));
    pthread_t *th = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
    int ok = own && mk && wj && th;
    uint64_t cap = 1024;
    while (cap < (uint64_t)(m / T + 1) * 3u) cap <<= 1;
    for (int32_t t = 0; ok && t < T; ++t) {
        own[t].t = t;
        own[t].T = T;
        own[t].cap = cap;
        own[t].table = (uint64_t *)malloc(cap * sizeof(uint64_t));
        if (!own[t].table) ok = 0;
        else memset(own[t].table, 0xff, cap * sizeof(uint64_t));
    }
    const uint64_t budget = (uint64_t)m * 1000u + 1000000u;
    uint64_t done = 0;                 /* candidates examined so far */
    int64_t have = 0;
    while (ok && have < m && done < budget) {
        /* the next pass: enough candidates for the edges still missing */
        uint64_t want = (uint64_t)(m - have) + (uint64_t)(m - have) / 4u + 4096u;
        if (want > budget - done) want = budget - done;
        uint64_t *keys = (uint64_t *)malloc((size_t)want * sizeof(uint64_t));
        uint8_t *acc = (uint8_t *)calloc((size_t)want, 1);
        if (!keys || !acc) { free(keys); free(acc); ok = 0; break; }
        const uint64_t chunk = (want + (uint64_t)T - 1) / (uint64_t)T;
        for (int32_t t = 0; t < T; ++t) {
            uint64_t a = (uint64_t)t * chunk, b = a + chunk;
            if (a > want) a = want;
            if (b > want) b = want;
            mk[t].p = &p;
            mk[t].c0 = done + a;
            mk[t].c1 = done + b;
            mk[t].keys = keys;
            mk[t].base = done;
            pthread_create(&th[t], NULL, make_run, &mk[t]);
        }
        for (int32_t t = 0; t < T; ++t) pthread_join(th[t], NULL);
        for (int32_t t = 0; t < T; ++t) {
            own[t].keys = keys;
            own[t].count = want;
            own[t].acc = acc;
            pthread_create(&th[t], NULL, owner_run, &own[t]);
        }
        int64_t got = 0;
        for (int32_t t = 0; t < T; ++t) {
            pthread_join(th[t], NULL);
            got += own[t].accepted;
        }
        /* the accepted candidates of this pass, in stream order, up to m */
        int64_t at = have;
        for (int32_t t = 0; t < T; ++t) {
            uint64_t a = (uint64_t)t * chunk, b = a + chunk;
            if (a > want) a = want;
            if (b > want) b = want;
            int64_t cnt = 0;
            for (uint64_t i = a; i < b; ++i) cnt += acc[i];
            wj[t].n = n;
            wj[t].keys = keys;
            wj[t].acc = acc;
            wj[t].i0 = a;
            wj[t].i1 = b;
            wj[t].out0 = at;
            wj[t].out_end = m;
            wj[t].src = src_out;
            wj[t].dst = dst_out;
            at += cnt;
        }
        for (int32_t t = 0; t < T; ++t) pthread_create(&th[t], NULL, write_run, &wj[t]);
        for (int32_t t = 0; t < T; ++t) pthread_join(th[t], NULL);
        free(keys);
        free(acc);
        have += got;
        if (have > m) have = m;
        done += want;
    }
    for (int32_t t = 0; own && t < T; ++t) free(own[t].table);
    free(own);
    free(mk);
    free(wj);
    free(th);
    return ok ? have : -1;
}
