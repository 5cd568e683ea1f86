/* R-MAT edge generator for the synthetic inputs (fixture code, not the method).
 *
 * Candidates are drawn in order from a splitmix64 stream keyed by the seed
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014).  Each 64-bit output gives two 32-bit draws, one per R-MAT
 * level; a draw r picks the quadrant a (r < t1), b (r < t2), c (r < t3) or d,
 * which appends bits (0,0), (0,1), (1,0), (1,1) to (src, dst).  Candidates
 * with an endpoint >= n, self-loops and repeats are dropped (repeats detected
 * with an open-addressing hash set); generation stops after m distinct edges.
 * Portable C99: no intrinsics, same output on every little- or big-endian host.
 */
#include <stdint.h>
#include <stdlib.h>

static uint64_t splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
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

/* Returns the number of accepted edges (== m on success, smaller when the
 * candidate budget ran out), or -1 when memory could not be allocated. */
int64_t rmat_generate(int64_t n, int64_t m, int32_t levels, uint64_t seed,
                      uint32_t t1, uint32_t t2, uint32_t t3,
                      int64_t *src_out, int64_t *dst_out) {
    uint64_t cap = 1024;
    while (cap < (uint64_t)m * 2u) cap <<= 1;
    uint64_t *table = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!table) return -1;
    for (uint64_t i = 0; i < cap; ++i) table[i] = UINT64_MAX;
    uint64_t state = seed;
    int64_t have = 0;
    uint64_t budget = (uint64_t)m * 1000u + 1000000u;
    while (have < m && budget-- > 0) {
        uint64_t s = 0, d = 0, buf = 0;
        int avail = 0;
        for (int32_t l = 0; l < levels; ++l) {
            if (!avail) { buf = splitmix64_next(&state); avail = 2; }
            uint32_t r = (uint32_t)(buf & 0xffffffffu);
            buf >>= 32;
            --avail;
            uint64_t sb = r >= t2;
            uint64_t db = (uint64_t)((r >= t1) ^ (r >= t2) ^ (r >= t3));
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        if (s >= (uint64_t)n || d >= (uint64_t)n || s == d) continue;
        uint64_t key = s * (uint64_t)n + d;
        uint64_t h = mix_key(key) & (cap - 1);
        int fresh = 1;
        while (table[h] != UINT64_MAX) {
            if (table[h] == key) { fresh = 0; break; }
            h = (h + 1) & (cap - 1);
        }
        if (!fresh) continue;
        table[h] = key;
        src_out[have] = (int64_t)s;
        dst_out[have] = (int64_t)d;
        ++have;
    }
    free(table);
    return have;
}
