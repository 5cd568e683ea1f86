// cover.cu -- max-k-cover over the pool: standard greedy (Sec. 3.2) and
// RandGreedi with streaming aggregation and truncation (Alg. 4, Alg. 5,
// Sec. 3.3.2).
//
// Standard greedy: one cooperative persistent kernel runs all k steps.  A step
// is a grid-wide argmax over the marginal gains counts[v] (packed as
// gain << 32 | ~v so that ties go to the smallest id), a grid barrier, the
// cover of S(v*) (atomicOr on a theta-bit bitmap; every newly covered set
// decrements the gains of its members), and a second barrier.  Barriers wait
// at most kWaitLimitNs and then report IM_ERR_TIMEOUT.
//
// RandGreedi: the paper's m sender machines are m "producer" blocks, each
// running the lazy local greedy of one vertex part V_p (Alg. 2) with its
// gains in shared memory and its own theta-bit covered bitmap.  A producer
// publishes its j-th seed (j < ceil(alpha k)) in slot (j, p) of a device array
// and raises a release flag; the buckets consume the slots in (j, p) order, so
// they see the same stream order in every run.  The receiver's B bucketing
// threads become, by default, k_rg_stream_masks after the producers finish:
// one 64-bit mask per RRR set holds the buckets covering it, so one pass over
// a streamed subset counts its gain for every bucket.  Alternatives (tuning
// knob values): one "consumer" block or thread-block cluster per bucket, and
// a fused mode where producers and consumers are one cooperative launch and
// the consumers read the slots with acquire loads as they are published, the
// paper's streaming overlap.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace im {

namespace {

constexpr int kGreedyThreads = 512;
constexpr int kRGThreads = 512;
constexpr int kProdThreads = 1024;           // producer blocks of the two-launch mode
constexpr int kBatch = 256;                  // stream slots a consumer reads at once
constexpr int kUnroll = 8;                   // independent loads in flight per lane in scans
constexpr int kSpec = 32;                    // largest speculative group of stream elements
constexpr size_t kClusterSmemCap = 200 * 1024;  // bucket bitmap slice per block
constexpr int kMaskG = 64;                   // largest group of stream slots (mask stage)
constexpr int kMaskStrips = 16;              // entries per lane in one warp work item
constexpr int kMaskItem = 32 * kMaskStrips;  // entries per warp work item

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max_u64(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
        x = warp_max_u64(x);
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    const unsigned long long r = sh[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ long long block_sum_i64(long long v, long long *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum<long long>(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ll;
        x = warp_sum<long long>(x);
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    const long long r = sh[32];
    __syncthreads();
    return r;
}

// Calls f(id) for every entry of ids[off, off + len) with 16-byte vector
// loads for the aligned body (each thread keeps U of them in flight) and
// scalar loads for the unaligned head and tail; f gets -1 for padding.
// Every thread of the calling group (tid < nth, nth >= 64) must call it.
template <int U, typename F>
__device__ __forceinline__ void scan_ids(const int32_t *__restrict__ ids, int64_t off, int64_t len,
                                         int tid, int nth, F &&f) {
    const int64_t end = off + len;
    int64_t a4 = (off + 3) & ~(int64_t)3;
    if (a4 > end) a4 = end;
    const int64_t b4 = a4 + ((end - a4) & ~(int64_t)3);
    if (tid < a4 - off) f(__ldg(ids + off + tid));
    else if (tid >= 32 && tid - 32 < end - b4) f(__ldg(ids + b4 + (tid - 32)));
    const int4 *v = reinterpret_cast<const int4 *>(ids + a4);
    const int64_t n4 = (b4 - a4) >> 2;
    for (int64_t i = tid; i < n4; i += (int64_t)nth * U) {
        int4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t k = i + (int64_t)u * nth;
            w[u] = k < n4 ? __ldg(v + k) : make_int4(-1, -1, -1, -1);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            f(w[u].x);
            f(w[u].y);
            f(w[u].z);
            f(w[u].w);
        }
    }
}

// ---------------------------------------------------------------------------
// standard greedy
// ---------------------------------------------------------------------------
struct GreedyArgs {
    int64_t n, theta;
    const int64_t *set_off;
    const int32_t *members;
    const int64_t *vtx_off;
    const int32_t *set_ids;
    int32_t k;
    int32_t *counts;                    // [n], or [32 ceil(n/32)] with spread
    uint32_t *covered;                  // [ceil(theta/32)]
    unsigned long long *block_best;     // [grid]
    GridBarrier *bar;
    int32_t *seeds;
    int64_t *gains;
    int32_t *nseeds;
    int64_t *coverage;
    int *status;
    // a query inside a batch: set ids in set_ids and vertex ids in members are
    // offset by sshift and vshift (the query's first set and first vertex)
    int64_t sshift, vshift;
    // ---- optional (NULL / 0: off), used by the pool's own greedy --------------
    // counts spread over 32 ceil(n / 32) slots: vertex v at (v mod 32) L + v / 32
    int32_t spread;
    // hubs, |S(v)| >= max |S(v)| >> hub_shift (at most hub_cap): each keeps its
    // gain as kHubRep partial counts, decremented by set id mod kHubRep
    int32_t *hub_rank;                  // [n] row of a hub, or -1
    int32_t *hub_cnt;                   // [hub_cap][kHubRep]
    int32_t *hub_list;                  // [hub_cap] the vertex of each row
    int32_t *cand;                      // [n] the other vertices with |S(v)| >= tau
    int32_t *ctl;                       // [4] hub rows, candidates, max |S(v)|, 0
    int32_t hub_cap, hub_shift, cand_shift;
    unsigned long long *work;           // [2] per-step chunk counters
};

constexpr int kHubRep = 32;             // partial counts of a hub (one per set id mod 32)
// Entries of S(v*) a warp claims at a time: a chunk's newly covered sets can
// hold hundreds of members each, so small chunks spread the decrements over
// more warps (the step waits for the slowest one).
constexpr int kGreedyChunk = 16;
constexpr int kHubCap = 4096;           // hub rows at most
constexpr int kHubShift = 6;            // hubs: |S(v)| >= max |S(v)| / 64

// Standard greedy (Sec. 3.2), all k steps in one cooperative launch: a step
// takes the argmax of the gains (packed gain << 32 | ~v: ties to the smallest
// id), covers S(v*) on the theta-bit bitmap and decrements the gain of every
// member of every newly covered set; two grid barriers per step.
//
// On graphs with hubs most decrements land on a few vertices, and atomics on
// one address serialise in its L2 slice: with hub rows, a hub's gain is the
// sum of kHubRep partial counts, each taking the decrements of the sets whose
// id is that value mod kHubRep, and the spread layout puts the other
// high-degree vertices -- low ids on a degree-ordered graph -- in different
// cache lines.  The argmax reads only the hub rows and the candidate list
// (|S(v)| >= tau) while the best gain is at least tau, since every other
// gain is below |S(v)| < tau; those vertices are frozen -- not decremented,
// keeping |S(v)| as a stale bound -- which skips most decrements (low-degree
// vertices are most members).  Once the best gain falls below tau, one pass
// makes the frozen gains exact and every step reads all.
// Warps take kGreedyChunk-entry chunks of S(v*) from a per-step counter.  Every wait is
// bounded (grid_sync).
__global__ void __launch_bounds__(kGreedyThreads, 2) k_greedy(GreedyArgs a) {
    __shared__ unsigned long long shm[33];
    const uint32_t nb = gridDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)nb * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = tid >> 5, nwarps = stride >> 5;
    const int64_t words = (a.theta + 31) / 32;
    const int64_t vwords = (a.n + 31) / 32;
    const int64_t nslots = a.spread ? 32 * vwords : a.n;
    auto slot = [&](int64_t v) { return a.spread ? (v & 31) * vwords + (v >> 5) : v; };
    auto vert = [&](int64_t i) { return a.spread ? (i % vwords) * 32 + i / vwords : i; };
    unsigned long long lmax = 0;
    for (int64_t i = tid; i < nslots; i += stride) {
        const int64_t v = vert(i);
        const int32_t d = v < a.n ? (int32_t)(a.vtx_off[v + 1] - a.vtx_off[v]) : 0;
        a.counts[i] = d;
        lmax = (unsigned long long)d > lmax ? (unsigned long long)d : lmax;
    }
    for (int64_t x = tid; x < words; x += stride) a.covered[x] = 0u;
    if (a.hub_rank) {
        lmax = block_max_u64(lmax, shm);
        if (threadIdx.x == 0 && lmax) atomicMax(a.ctl + 2, (int32_t)lmax);
    }
    if (!grid_sync(a.bar, nb, a.status)) return;
    uint32_t tau = 0;                        // > 0: the argmax reads hubs + candidates
    int32_t nhub = 0, ncand = 0;
    if (a.hub_rank) {
        const uint32_t l = (uint32_t)__ldcg(a.ctl + 2);
        const uint32_t th = l >> a.hub_shift > 0 ? l >> a.hub_shift : 1;
        tau = a.cand_shift > 0 ? (l >> a.cand_shift > 0 ? l >> a.cand_shift : 1) : 0;
        for (int64_t v = tid; v < a.n; v += stride) {
            const uint32_t d = (uint32_t)(a.vtx_off[v + 1] - a.vtx_off[v]);
            int32_t r = -1;
            if (d >= th) {
                r = atomicAdd(a.ctl + 0, 1);
                if (r < a.hub_cap) {
                    a.hub_list[r] = (int32_t)v;
                    a.hub_cnt[(int64_t)r * kHubRep] = (int32_t)d;
                    for (int q = 1; q < kHubRep; ++q) a.hub_cnt[(int64_t)r * kHubRep + q] = 0;
                    a.counts[slot(v)] = 0;   // the row holds the gain
                } else {
                    r = -1;
                }
            }
            // below tau a vertex is frozen (-2): its gain stays |S(v)| < tau, a
            // stale bound, until the best gain drops below tau
            if (r < 0 && tau > 0) r = d >= tau ? -1 : -2;
            a.hub_rank[v] = r;
            if (r == -1 && tau > 0) a.cand[atomicAdd(a.ctl + 1, 1)] = (int32_t)v;
        }
        if (!grid_sync(a.bar, nb, a.status)) return;
        nhub = min(__ldcg(a.ctl + 0), a.hub_cap);
        ncand = __ldcg(a.ctl + 1);
    }
    int64_t cov = 0;
    int32_t j = 0;
    while (j < a.k) {
        unsigned long long best = 0;
        auto consider = [&](int32_t c, uint32_t v) {
            if (c > 0) {
                const unsigned long long key =
                    ((unsigned long long)(uint32_t)c << 32) | (0xffffffffu - v);
                best = key > best ? key : best;
            }
        };
        if (tau > 0) {
            for (int64_t q = tid; q < ncand; q += stride) {
                const uint32_t v = (uint32_t)__ldcg(a.cand + q);
                consider(__ldcg(a.counts + slot(v)), v);
            }
        } else {
            for (int64_t i = tid; i < nslots; i += stride)
                consider(__ldcg(a.counts + i), (uint32_t)vert(i));
        }
        for (int64_t h = gwarp; h < nhub; h += nwarps) {      // a hub's gain: its row's sum
            const int32_t c = warp_sum<int32_t>(__ldcg(a.hub_cnt + h * kHubRep + lane));
            consider(c, (uint32_t)__ldcg(a.hub_list + h));
        }
        best = block_max_u64(best, shm);
        if (threadIdx.x == 0) a.block_best[blockIdx.x] = best;
        if (!grid_sync(a.bar, nb, a.status)) return;
        unsigned long long gbest = 0;
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
            const unsigned long long x = __ldcg(a.block_best + b);
            gbest = x > gbest ? x : gbest;
        }
        gbest = block_max_u64(gbest, shm);
        if (tau > 0 && (uint32_t)(gbest >> 32) < tau) {
            // the best gain fell below tau: the frozen vertices may now win.
            // Make their gains exact against the sets covered so far, thaw
            // them, and read every gain from here on (block_best is rewritten
            // only after the barrier below, when every block has read it)
            for (int64_t v = gwarp; v < a.n; v += nwarps) {
                if (__ldcg(a.hub_rank + v) != -2) continue;
                const int64_t sb = a.vtx_off[v], se = a.vtx_off[v + 1];
                int miss = 0;
                for (int64_t t = sb + lane; t < se; t += 32) {
                    const int64_t il = __ldg(a.set_ids + t) - a.sshift;
                    miss += !((__ldcg(a.covered + (il >> 5)) >> (il & 31)) & 1u);
                }
                miss = warp_sum<int>(miss);
                if (lane == 0) {
                    a.counts[slot(v)] = miss;
                    a.hub_rank[v] = -1;
                }
            }
            tau = 0;
            if (!grid_sync(a.bar, nb, a.status)) return;
            continue;
        }
        if (gbest == 0) break;                       // every remaining gain is zero
        const int32_t vs = (int32_t)(0xffffffffu - (uint32_t)(gbest & 0xffffffffu));
        const int64_t gain = (int64_t)(gbest >> 32);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.seeds[j] = vs;
            a.gains[j] = gain;
        }
        cov += gain;
        const int64_t sb = a.vtx_off[vs], se = a.vtx_off[vs + 1];
        // chunks of S(v*) from this step's counter; the other step's counter
        // is cleared meanwhile (its last use ended at the previous step's
        // closing barrier)
        unsigned long long *work = a.work ? a.work + (j & 1) : nullptr;
        if (work && blockIdx.x == 0 && threadIdx.x == 0) a.work[(j + 1) & 1] = 0ull;
        for (int64_t base = sb + gwarp * kGreedyChunk;;) {
            if (work) {
                unsigned long long c = 0;
                if (lane == 0) c = atomicAdd(work, (unsigned long long)kGreedyChunk);
                base = sb + (int64_t)__shfl_sync(kFull, c, 0);
            }
            if (base >= se) break;
            const int64_t t = base + lane;
            int32_t i = -1;
            if (lane < kGreedyChunk && t < se) i = a.set_ids[t];
            const bool fresh = warp_bitmap_set(a.covered, i >= 0 ? i - a.sshift : -1, lane);
            if (__any_sync(kFull, fresh)) {
                // decrement the gains of every member of the lane's newly
                // covered set: the warp walks the concatenation of those
                // member lists 32 entries at a time, U loads in flight per lane
                int64_t mo = 0, ml = 0;
                if (fresh) {
                    mo = a.set_off[i];
                    ml = a.set_off[i + 1] - mo;
                }
                const int64_t incl = warp_incl_scan<int64_t>(ml, lane);
                const int64_t tot = __shfl_sync(kFull, incl, 31);
                constexpr int U = 4;
                for (int64_t p0 = 0; p0 < tot; p0 += 32 * U) {
                    int32_t mv[U], ms[U];
#pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                        const int64_t q = p0 + uu * 32 + lane;
                        int owner = 0;           // first lane whose inclusive count exceeds q
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const int64_t c = __shfl_sync(kFull, incl, owner + step - 1);
                            if (c <= q) owner += step;
                        }
                        const int64_t o_incl = __shfl_sync(kFull, incl, owner);
                        const int64_t o_ml = __shfl_sync(kFull, ml, owner);
                        const int64_t o_mo = __shfl_sync(kFull, mo, owner);
                        ms[uu] = __shfl_sync(kFull, i, owner);
                        mv[uu] = q < tot ? __ldg(a.members + o_mo + (q - (o_incl - o_ml))) : -1;
                    }
#pragma unroll
                    for (int uu = 0; uu < U; ++uu) {
                        if (mv[uu] < 0) continue;
                        const int64_t u = mv[uu] - a.vshift;
                        const int32_t hr = a.hub_rank ? __ldcg(a.hub_rank + u) : -1;
                        if (hr >= 0)
                            red_add_s32(a.hub_cnt + (int64_t)hr * kHubRep + (ms[uu] & (kHubRep - 1)),
                                        -1);
                        else if (hr == -1)
                            red_add_s32(a.counts + slot(u), -1);   // -2: frozen
                    }
                }
            }
            if (!work) base += nwarps * kGreedyChunk;
        }
        if (!grid_sync(a.bar, nb, a.status)) return;
        ++j;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.nseeds = j;
        *a.coverage = cov;
    }
}

// ---------------------------------------------------------------------------
// RandGreedi
// ---------------------------------------------------------------------------
struct RGArgs {
    int64_t n, theta, words;
    int32_t k, P, trunc, B;
    const int64_t *vtx_off;
    const int32_t *set_ids;
    const int32_t *part_off;
    const int32_t *part_vtx;
    uint32_t *covered;        // [P][words] producer bitmaps
    uint32_t *bcovered;       // [B][words] bucket bitmaps
    int32_t *local_seeds;
    int64_t *local_gains;
    int32_t *local_n;
    int64_t *local_cov;
    const int64_t *thr;
    int64_t *bucket_cov;
    int32_t *bucket_n;
    int32_t *bucket_seeds;
    int64_t *bucket_gains;
    uint32_t *flags;          // [trunc][P]: 0 empty, 1 seed ready, 2 no seed
    int32_t *elems;           // [trunc][P]
    int32_t nprod, ncons;     // block roles in this launch
    int32_t first_role;       // 0: blocks start with producers; 1: consumers only
    int32_t max_np;           // largest part: key[] and stamp[] are max_np each
    int32_t evals;            // local greedy: candidates re-evaluated per round (<= kProdW)
    long long *stats;         // [P + B][6] diagnostics (see im_randgreedi_stats)
    int *status;
    // bucket-mask stage (k_rg_stream_masks)
    unsigned long long *mask; // [theta]: bit b set once bucket b covers the set
    uint32_t *gbuf;           // [2][kMaskG][64] per-slot, per-bucket gains
    GridBarrier *bar;
    int32_t *slot_x;          // [trunc * P] element of each stream slot, -1 if none
    int64_t *slot_beg, *slot_len;   // its covering subset in set_ids
};

// Local greedy of part p (Alg. 4, one sender), run as the lazy greedy of
// Alg. 2: key[l] holds a gain of candidate l that is exact when stamp[l]
// equals the current round and an upper bound otherwise (gains only shrink,
// by submodularity).  The largest key (ties: smallest id) is taken when it is
// exact, which picks exactly the standard greedy's sequence.
//
// cmax[c] is the largest packed key (gain << 32 | ~l) of the 32 candidates of
// chunk c.  A round takes the best candidate of each of the kProdW chunks with
// the largest cmax and re-evaluates the stale ones at once (blockDim / kProdW
// threads each) against the part's covered bitmap; then, if the overall
// largest key is exact, it is taken.  Evaluating more candidates than the
// sequential rule would only replaces upper bounds by exact values, so the
// sequence of picks is unchanged while a pick takes one or two rounds instead
// of one round per stale candidate.
constexpr int kProdW = 8;

__device__ __forceinline__ unsigned long long prod_key(int32_t g, int32_t l) {
    return g > 0 ? ((unsigned long long)(uint32_t)g << 32) | (0xffffffffu - (uint32_t)l) : 0ull;
}

// cmax of chunk c, by one warp
__device__ __forceinline__ void prod_chunk_max(const int32_t *key, unsigned long long *cmax,
                                               int32_t np, int32_t c, int lane) {
    const int32_t l = c * 32 + lane;
    const unsigned long long v = warp_max_u64(l < np ? prod_key(key[l], l) : 0ull);
    if (lane == 0) cmax[c] = v;
}

__device__ void produce(const RGArgs &a, int p, int32_t *key, unsigned long long *shm,
                        long long *shs) {
    __shared__ int32_t s_cand[kProdW];
    __shared__ int32_t s_cnt[kProdW];
    __shared__ unsigned long long s_top;
    const int32_t vb = a.part_off[p], np = a.part_off[p + 1] - vb;
    const int32_t *vtx = a.part_vtx + vb;
    int32_t *stamp = key + a.max_np;
    unsigned long long *cmax = reinterpret_cast<unsigned long long *>(key + 2 * a.max_np);
    const int32_t nch = (np + 31) / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    uint32_t *cov = a.covered + (size_t)p * (size_t)a.words;
    for (int64_t x = threadIdx.x; x < a.words; x += blockDim.x) cov[x] = 0u;
    for (int32_t l = threadIdx.x; l < np; l += blockDim.x) {
        const int32_t v = vtx[l];
        key[l] = (int32_t)(a.vtx_off[v + 1] - a.vtx_off[v]);
        stamp[l] = 0;                                   // exact: nothing is covered yet
    }
    __syncthreads();
    for (int32_t c = warp; c < nch; c += nwarp) prod_chunk_max(key, cmax, np, c, lane);
    __syncthreads();
    const uint64_t t_begin = global_ns();
    long long n_rounds = 0, n_evals = 0, eval_entries = 0, cover_entries = 0;
    int64_t total = 0;
    int32_t j = 0;
    const int W = a.evals;
    const int gsz = blockDim.x / W, grp = threadIdx.x / gsz, gt = threadIdx.x % gsz;
    while (j < a.k) {
        ++n_rounds;
        // ---- the W chunks with the largest maxima (warp 0, by repeated max)
        if (warp == 0) {
            unsigned long long taken = 0ull;    // chunks already chosen, as keys
            for (int w = 0; w < W; ++w) {
                unsigned long long best = 0ull;
                for (int32_t c = lane; c < nch; c += 32) {
                    const unsigned long long v = cmax[c];
                    // skip chunks chosen earlier this round (their keys are distinct)
                    if (v > best && (w == 0 || v < taken)) best = v;
                }
                const unsigned long long m = warp_max_u64(best);
                if (lane == 0) {
                    s_cand[w] = m ? (int32_t)(0xffffffffu - (uint32_t)(m & 0xffffffffu)) : -1;
                    s_cnt[w] = 0;
                    if (w == 0) s_top = m;
                }
                taken = m;
                if (!m) {
                    for (int w2 = w + 1; w2 < W && lane == 0; ++w2) s_cand[w2] = -1;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_top == 0ull) break;                       // every gain is zero
        {
            const int32_t l0 = s_cand[0];
            if (stamp[l0] != j) {
                // ---- re-evaluate every stale candidate of the round at once
                const int32_t l = s_cand[grp];
                const bool mine = l >= 0 && stamp[l] != j;
                if (mine) {
                    const int32_t v = vtx[l];
                    const int64_t sb = a.vtx_off[v], se = a.vtx_off[v + 1];
                    int miss = 0;
                    // L1-cached probes: the bitmap is written only by this
                    // block (atomics, ordered before these loads by the block
                    // barriers), and S(v) is scanned in ascending set order
                    // when the index comes from the radix build, so
                    // neighbouring ids share cached lines
                    scan_ids<4>(a.set_ids, sb, se - sb, gt, gsz, [&](int32_t i) {
                        if (i >= 0) miss += !((__ldca(cov + (i >> 5)) >> (i & 31)) & 1u);
                    });
                    miss = warp_sum<int>(miss);
                    if (lane == 0 && miss) atomicAdd(&s_cnt[grp], miss);
                }
                __syncthreads();
                if (mine && gt == 0) {
                    key[l] = s_cnt[grp];
                    stamp[l] = j;
                    const int32_t v = vtx[l];
                    ++n_evals;
                    eval_entries += a.vtx_off[v + 1] - a.vtx_off[v];
                }
                __syncthreads();
                // refresh the maxima of the chunks that changed, then the top
                if (warp < W && s_cand[warp] >= 0)
                    prod_chunk_max(key, cmax, np, s_cand[warp] >> 5, lane);
                __syncthreads();
                if (warp == 0) {
                    unsigned long long best = 0ull;
                    for (int32_t c = lane; c < nch; c += 32) best = cmax[c] > best ? cmax[c] : best;
                    best = warp_max_u64(best);
                    if (lane == 0) s_top = best;
                }
                __syncthreads();
                if (s_top == 0ull) break;
            }
        }
        const unsigned long long top = s_top;
        const int32_t l = (int32_t)(0xffffffffu - (uint32_t)(top & 0xffffffffu));
        if (stamp[l] != j) continue;                    // the top is still an upper bound
        // ---- take it
        const int32_t v = vtx[l];
        const int64_t sb = a.vtx_off[v], se = a.vtx_off[v + 1];
        const int64_t gain = (int64_t)(top >> 32);
        if (threadIdx.x == 0) {
            a.local_seeds[(int64_t)p * a.k + j] = v;
            a.local_gains[(int64_t)p * a.k + j] = gain;
            if (j < a.trunc) {
                a.elems[(int64_t)j * a.P + p] = v;
                st_release_u32(&a.flags[(int64_t)j * a.P + p], 1u);
            }
            key[l] = 0;
        }
        total += gain;
        cover_entries += se - sb;
        scan_ids<4>(a.set_ids, sb, se - sb, threadIdx.x, blockDim.x, [&](int32_t i) {
            if (i >= 0) atomicOr(&cov[i >> 5], 1u << (i & 31));
        });
        __syncthreads();
        if (warp == 0) prod_chunk_max(key, cmax, np, l >> 5, lane);
        __syncthreads();
        ++j;
    }
    (void)shm;
    (void)shs;
    if (threadIdx.x == 0) {
        a.local_n[p] = j;
        a.local_cov[p] = total;
        for (int32_t jj = j; jj < a.trunc; ++jj) st_release_u32(&a.flags[(int64_t)jj * a.P + p], 2u);
    }
    n_evals = block_sum_i64(n_evals, shs);
    eval_entries = block_sum_i64(eval_entries, shs);
    if (threadIdx.x == 0 && a.stats) {
        long long *st = a.stats + 6 * (int64_t)p;
        st[0] = (long long)t_begin;
        st[1] = (long long)global_ns();
        st[2] = n_rounds;
        st[3] = n_evals;
        st[4] = eval_entries;
        st[5] = cover_entries;
    }
    __syncthreads();
}

// Streaming bucket b (Alg. 5): consume the stream in (j, p) order.
//
// Elements are evaluated speculatively in groups of W against the bucket as
// it stands: the first element of the group whose gain reaches the threshold
// is the next one the sequential rule accepts (every element before it saw
// the same bucket and fell short), so it is accepted and evaluation resumes
// right after it; later elements of the group are evaluated again.  W doubles
// after a group without an accept and halves after one, which bounds the
// repeated work by the number of accepts times W.
__device__ void consume(const RGArgs &a, int b, long long *shs) {
    __shared__ int32_t s_x[kBatch];
    __shared__ int64_t s_off[kBatch];
    __shared__ int64_t s_len[kBatch];
    __shared__ int s_cand[kSpec];
    __shared__ unsigned long long s_miss[kSpec];
    __shared__ int s_ncand, s_end, s_acc, s_timeout;
    uint32_t *C = a.bcovered + (size_t)b * (size_t)a.words;
    for (int64_t x = threadIdx.x; x < a.words; x += blockDim.x) C[x] = 0u;
    if (threadIdx.x == 0) s_timeout = 0;
    __syncthreads();
    const int64_t T = a.thr[b];
    const int64_t E = (int64_t)a.trunc * a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint64_t t_begin = global_ns();
    long long n_eval = 0, scanned = 0, wait_ns = 0;
    int32_t bn = 0;
    int64_t bcov = 0;
    int W = 1;
    for (int64_t base = 0; base < E && bn < a.k; base += kBatch) {
        const int cntb = (int)min((int64_t)kBatch, E - base);
        const uint64_t tw0 = global_ns();
        if (threadIdx.x < cntb) {
            const int64_t slot = base + threadIdx.x;
            uint32_t f = ld_acquire_u32(a.flags + slot);
            if (f == 0) {
                const uint64_t t0 = global_ns();
                while ((f = ld_acquire_u32(a.flags + slot)) == 0) {
                    if (global_ns() - t0 > kWaitLimitNs) {
                        raise_status(a.status, kDevTimeout);
                        s_timeout = 1;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            int32_t x = -1;
            int64_t off = 0, len = 0;
            if (f == 1) {
                x = __ldcg(a.elems + slot);
                off = a.vtx_off[x];
                len = a.vtx_off[x + 1] - off;
            }
            s_x[threadIdx.x] = x;
            s_off[threadIdx.x] = off;
            s_len[threadIdx.x] = len;
        }
        __syncthreads();
        wait_ns += (long long)(global_ns() - tw0);
        if (s_timeout) break;
        int q = 0;
        while (q < cntb && bn < a.k) {
            if (threadIdx.x == 0) {
                // next W candidates; |S(x)| < threshold rejects x without a scan
                int n = 0, r = q;
                while (r < cntb && n < W) {
                    if (s_x[r] >= 0 && s_len[r] >= T) s_cand[n++] = r;
                    ++r;
                }
                s_ncand = n;
                s_end = r;
            }
            if (threadIdx.x < kSpec) s_miss[threadIdx.x] = 0;
            __syncthreads();
            const int n = s_ncand;
            if (n == 0) {
                q = s_end;
                __syncthreads();
                continue;
            }
            // |S(x) \ C_b| for every candidate, all warps in flight at once
            for (int c = 0; c < n; ++c) {
                const int r = s_cand[c];
                const int64_t off = s_off[r], len = s_len[r];
                unsigned m = 0;
                for (int64_t c0 = (int64_t)warp * 32 * kUnroll; c0 < len;
                     c0 += (int64_t)nwarps * 32 * kUnroll) {
                    int32_t ids[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int64_t t = c0 + u * 32 + lane;
                        ids[u] = t < len ? __ldg(a.set_ids + off + t) : -1;
                    }
                    unsigned words[kUnroll];
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u)
                        words[u] = ids[u] >= 0 ? __ldcg(C + (ids[u] >> 5)) : ~0u;
#pragma unroll
                    for (int u = 0; u < kUnroll; ++u)
                        m += __popc(__ballot_sync(kFull, !((words[u] >> (ids[u] & 31)) & 1u)));
                }
                if (lane == 0 && m) atomicAdd(&s_miss[c], (unsigned long long)m);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int acc = -1;
                for (int c = 0; c < n; ++c)
                    if ((int64_t)s_miss[c] >= T) {
                        acc = c;
                        break;
                    }
                s_acc = acc;
            }
            __syncthreads();
            const int acc = s_acc;
            n_eval += acc < 0 ? n : acc + 1;
            for (int c = 0; c < n; ++c) scanned += s_len[s_cand[c]];
            if (acc < 0) {
                q = s_end;
                W = min(kSpec, 2 * W);
            } else {
                const int r = s_cand[acc];
                const int64_t off = s_off[r], len = s_len[r];
                for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
                    const int32_t i = __ldg(a.set_ids + off + t);
                    atomicOr(&C[i >> 5], 1u << (i & 31));
                }
                const int64_t gain = (int64_t)s_miss[acc];
                if (threadIdx.x == 0) {
                    a.bucket_seeds[(int64_t)b * a.k + bn] = s_x[r];
                    a.bucket_gains[(int64_t)b * a.k + bn] = gain;
                }
                ++bn;
                bcov += gain;
                q = r + 1;
                W = max(1, W / 2);
            }
            __syncthreads();
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.bucket_n[b] = bn;
        a.bucket_cov[b] = bcov;
        if (a.stats) {
            long long *st = a.stats + 6 * ((int64_t)a.P + b);
            st[0] = (long long)t_begin;
            st[1] = (long long)global_ns();
            st[2] = n_eval;
            st[3] = bn;
            st[4] = scanned;
            st[5] = wait_ns;
        }
    }
    __syncthreads();
}

// The producers alone (two-launch mode): one block of kProdThreads per part.
__global__ void __launch_bounds__(kProdThreads) k_rg_local(RGArgs a) {
    extern __shared__ int32_t key[];
    __shared__ unsigned long long shm[33];
    __shared__ long long shs[33];
    for (int p = blockIdx.x; p < a.P; p += gridDim.x) produce(a, p, key, shm, shs);
}

__global__ void __launch_bounds__(kRGThreads) k_randgreedi(RGArgs a) {
    extern __shared__ int32_t key[];
    __shared__ unsigned long long shm[33];
    __shared__ long long shs[33];
    const int r = blockIdx.x;
    if (a.first_role == 0 && r < a.nprod) {
        for (int p = r; p < a.P; p += a.nprod) produce(a, p, key, shm, shs);
    } else {
        const int c = a.first_role == 0 ? r - a.nprod : r;
        for (int b = c; b < a.B; b += a.ncons) consume(a, b, shs);
    }
}

// Streaming buckets with the bucket bitmap in shared memory (Alg. 5, run after
// the local greedy has finished).  A cluster of CS blocks serves one bucket
// at a time (buckets are taken from a global counter): block r keeps the bits
// of set ids [r * R, (r + 1) * R) in its shared memory, scans every entry of
// S(x) and tests only the ids in its own range.  The per-candidate counts of
// the CS blocks are added over distributed shared memory after a cluster
// barrier, and every block takes the same accept decision.  Candidates go in
// the same speculative groups as in consume(); partial-count arrays alternate
// between two buffers so one barrier per group suffices.
__global__ void __launch_bounds__(kRGThreads) k_rg_stream_cluster(RGArgs a, int64_t R,
                                                                  unsigned *bucket_counter) {
    extern __shared__ uint32_t bits[];               // R bits, then 2 x kSpec partial counts
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned CS = cluster.num_blocks();
    const unsigned rank = cluster.block_rank();
    const int64_t words = R / 32;
    unsigned *part = bits + words;                   // [2][kSpec]
    __shared__ int32_t w_x[kBatch];                  // stream window: element, offset, length
    __shared__ int64_t w_off[kBatch], w_len[kBatch];
    __shared__ int s_cand[kSpec];
    __shared__ unsigned long long s_tot[kSpec];
    __shared__ int s_n, s_bucket, s_end, s_acc;
    const int64_t lo = (int64_t)rank * R;
    const int lane = threadIdx.x & 31;
    const int64_t E = (int64_t)a.trunc * a.P;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_bucket = (int)atomicAdd(bucket_counter, 1u);
        cluster.sync();
        if (threadIdx.x == 0) s_bucket = *cluster.map_shared_rank(&s_bucket, 0);
        cluster.sync();
        const int b = s_bucket;
        if (b >= a.B) break;
        for (int64_t x = threadIdx.x; x < words; x += blockDim.x) bits[x] = 0u;
        const int64_t T = a.thr[b];
        const uint64_t t_begin = global_ns();
        long long n_eval = 0, scanned = 0;
        int32_t bn = 0;
        int64_t bcov = 0;
        int W = 1, phase = 0;
        cluster.sync();
        for (int64_t base = 0; base < E && bn < a.k; base += kBatch) {
            // the producers have finished: every slot is final (1 seed, 2 none)
            const int cntb = (int)min((int64_t)kBatch, E - base);
            if (threadIdx.x < cntb) {
                const int64_t slot = base + threadIdx.x;
                int32_t x = -1;
                int64_t off = 0, len = 0;
                if (ld_acquire_u32(a.flags + slot) == 1u) {
                    x = __ldcg(a.elems + slot);
                    off = a.vtx_off[x];
                    len = a.vtx_off[x + 1] - off;
                }
                w_x[threadIdx.x] = x;
                w_off[threadIdx.x] = off;
                w_len[threadIdx.x] = len;
            }
            __syncthreads();
            int qq = 0;
            while (qq < cntb && bn < a.k) {
                if (threadIdx.x == 0) {
                    // next W candidates; |S(x)| < threshold rejects x without a scan
                    int n = 0, r = qq;
                    while (r < cntb && n < W) {
                        if (w_x[r] >= 0 && w_len[r] >= T) s_cand[n++] = r;
                        ++r;
                    }
                    s_n = n;
                    s_end = r;
                }
                unsigned *mine = part + phase * kSpec;
                if (threadIdx.x < kSpec) mine[threadIdx.x] = 0u;
                __syncthreads();
                const int n = s_n;
                if (n == 0) {
                    qq = s_end;
                    __syncthreads();
                    continue;
                }
                for (int c = 0; c < n; ++c) {
                    const int r = s_cand[c];
                    unsigned m = 0;
                    scan_ids<4>(a.set_ids, w_off[r], w_len[r], threadIdx.x, blockDim.x,
                                [&](int32_t id) {
                                    const int64_t rel = (int64_t)id - lo;
                                    if (id >= 0 && rel >= 0 && rel < R)
                                        m += !((bits[rel >> 5] >> (rel & 31)) & 1u);
                                });
                    m = warp_sum<unsigned>(m);
                    if (lane == 0 && m) atomicAdd(&mine[c], m);
                }
                cluster.sync();
                // candidate c's total over the cluster, summed by thread c
                if (threadIdx.x < n) {
                    unsigned long long tot = 0;
                    for (unsigned r2 = 0; r2 < CS; ++r2)
                        tot += cluster.map_shared_rank(mine, r2)[threadIdx.x];
                    s_tot[threadIdx.x] = tot;
                }
                __syncthreads();
                if (threadIdx.x < 32) {
                    const bool ok = lane < n && (int64_t)s_tot[lane] >= T;
                    const unsigned bal = __ballot_sync(kFull, ok);
                    if (lane == 0) s_acc = bal ? __ffs(bal) - 1 : -1;
                }
                __syncthreads();
                const int acc = s_acc;
                n_eval += acc < 0 ? n : acc + 1;
                for (int c = 0; c < n; ++c) scanned += w_len[s_cand[c]];
                if (acc < 0) {
                    qq = s_end;
                    W = min(kSpec, 2 * W);
                } else {
                    const int r = s_cand[acc];
                    scan_ids<4>(a.set_ids, w_off[r], w_len[r], threadIdx.x, blockDim.x,
                                [&](int32_t id) {
                                    const int64_t rel = (int64_t)id - lo;
                                    if (id >= 0 && rel >= 0 && rel < R)
                                        atomicOr(&bits[rel >> 5], 1u << (rel & 31));
                                });
                    const int64_t gain = (int64_t)s_tot[acc];
                    if (rank == 0 && threadIdx.x == 0) {
                        a.bucket_seeds[(int64_t)b * a.k + bn] = w_x[r];
                        a.bucket_gains[(int64_t)b * a.k + bn] = gain;
                    }
                    ++bn;
                    bcov += gain;
                    qq = r + 1;
                    W = max(1, W / 2);
                }
                phase ^= 1;
                __syncthreads();
            }
            __syncthreads();
        }
        if (rank == 0 && threadIdx.x == 0) {
            a.bucket_n[b] = bn;
            a.bucket_cov[b] = bcov;
            if (a.stats) {
                long long *st = a.stats + 6 * ((int64_t)a.P + b);
                st[0] = (long long)t_begin;
                st[1] = (long long)global_ns();
                st[2] = n_eval;
                st[3] = bn;
                st[4] = scanned;
                st[5] = 0;
            }
        }
        cluster.sync();
    }
}

// Streaming buckets over per-set bucket masks (Alg. 5, run after the local
// greedy has finished; B <= 64).  mask[i] holds one bit per bucket: bit b is
// set once bucket b covers RRR set i.  A single pass over S(x) therefore
// yields the marginal gain of x for every bucket at once -- the count of
// entries whose bit b is clear -- instead of one pass per bucket.
//
// The stream is consumed in (j, p) slot order in speculative groups of up to
// kMaskG slots.  Every warp of the grid takes work items of kMaskItem entries
// of the group's subsets and adds its per-bucket counts to gbuf; after a grid
// barrier every block replays the same sequential decision for each bucket
// from those counts.  A count taken against the bucket as it stood at the
// start of the group is exact until the bucket accepts something in the
// group, and an upper bound after that (coverage only grows), so a later slot
// below the threshold is still rejected exactly; a later slot at or above it
// needs a fresh count, and the group is cut there for all buckets.  The
// accepted subsets are then or-ed into the masks and the next group starts at
// the cut.  Group sizes double after a group without a cut and halve after a
// cut.
// The slot whose work items hold item c: the largest u < gn with s_off[u] <= c.
__device__ __forceinline__ int mask_slot_of(const int64_t *s_off, int gn, int64_t c) {
    int lo = 0, hi = gn - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Exclusive prefix of the work items of slots [0, gn) (items[u] from f(u)),
// written to s_off[0..gn]; gn <= 64, run by warp 0.
template <typename F>
__device__ __forceinline__ void mask_item_prefix(int64_t *s_off, int gn, F &&f) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int u0 = 2 * lane, u1 = 2 * lane + 1;
    const int64_t a0 = u0 < gn ? f(u0) : 0, a1 = u1 < gn ? f(u1) : 0;
    const int64_t incl = warp_incl_scan<int64_t>(a0 + a1, lane);
    const int64_t excl = incl - a0 - a1;
    if (u0 < gn) s_off[u0] = excl;
    if (u1 < gn) s_off[u1] = excl + a0;
    if (lane == 31) s_off[gn] = incl;
}

__global__ void __launch_bounds__(kRGThreads) k_rg_stream_masks(RGArgs a) {
    __shared__ int32_t s_x[kMaskG];
    __shared__ int64_t s_beg[kMaskG], s_len[kMaskG];
    __shared__ uint32_t s_g[kMaskG * 64];            // the group's gains, staged once
    __shared__ unsigned long long s_pass[64];        // slots reaching each bucket's threshold
    __shared__ int64_t s_thr[64];
    __shared__ int64_t s_off[kMaskG + 1];            // work-item prefix over the group's slots
    __shared__ unsigned long long s_acc[kMaskG];     // buckets accepting each slot
    __shared__ int32_t s_n[64];
    __shared__ int64_t s_cov[64];
    __shared__ long long s_eval[64], s_scan[64];
    __shared__ int s_cut;
    const int lane = threadIdx.x & 31;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    // warps numbered block-minor, so the few work items of a small group land
    // on different SMs
    const int64_t gwarp = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int64_t nwarps = gstride >> 5;
    const int64_t nslots = (int64_t)a.trunc * a.P;
    const uint64_t t_begin = global_ns();
    for (int64_t i = gtid; i < a.theta; i += gstride) a.mask[i] = 0ull;
    for (int64_t i = gtid; i < 2 * kMaskG * 64; i += gstride) a.gbuf[i] = 0u;
    // slot table: element (or -1) and its covering-subset range, read once
    for (int64_t t = gtid; t < nslots; t += gstride) {
        const int32_t x = ld_acquire_u32(a.flags + t) == 1u ? __ldcg(a.elems + t) : -1;
        const int64_t b = x >= 0 ? a.vtx_off[x] : 0;
        a.slot_x[t] = x;
        a.slot_beg[t] = b;
        a.slot_len[t] = x >= 0 ? a.vtx_off[x + 1] - b : 0;
    }
    if (threadIdx.x < 64) {
        s_thr[threadIdx.x] = threadIdx.x < a.B ? a.thr[threadIdx.x] : 0;
        s_n[threadIdx.x] = 0;
        s_cov[threadIdx.x] = 0;
        s_eval[threadIdx.x] = 0;
        s_scan[threadIdx.x] = 0;
    }
    if (!grid_sync(a.bar, gridDim.x, a.status)) return;
    int64_t g0 = 0;
    int G = 8, buf = 0;
    while (g0 < nslots) {
        const int gn = (int)(nslots - g0 < G ? nslots - g0 : G);
        if (threadIdx.x < gn) {
            const int64_t t = g0 + threadIdx.x;
            s_x[threadIdx.x] = __ldcg(a.slot_x + t);
            s_beg[threadIdx.x] = __ldcg(a.slot_beg + t);
            s_len[threadIdx.x] = __ldcg(a.slot_len + t);
            s_acc[threadIdx.x] = 0ull;
        }
        if (threadIdx.x == 0) s_cut = gn;
        __syncthreads();
        mask_item_prefix(s_off, gn, [&](int u) { return (s_len[u] + kMaskItem - 1) / kMaskItem; });
        __syncthreads();
        uint32_t *gb = a.gbuf + (size_t)buf * kMaskG * 64;
        // ---- counts of every slot of the group against the current masks
        for (int64_t c = gwarp; c < s_off[gn]; c += nwarps) {
            const int u = mask_slot_of(s_off, gn, c);
            const int64_t e0 = (c - s_off[u]) * kMaskItem;
            const int64_t len = s_len[u];
            const int32_t *ids = a.set_ids + s_beg[u];
            // all ids first, then all masks: two memory round trips per item
            int32_t id[kMaskStrips];
#pragma unroll
            for (int st = 0; st < kMaskStrips; ++st) {
                const int64_t e = e0 + st * 32 + lane;
                id[st] = e < len ? __ldg(ids + e) : -1;
            }
            unsigned long long mk[kMaskStrips];
#pragma unroll
            for (int st = 0; st < kMaskStrips; ++st)
                mk[st] = id[st] >= 0 ? ~__ldcg(a.mask + id[st]) : 0ull;
            // 5-bit vertical counters, one bit-plane per 64-bit word
            unsigned long long c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0;
#pragma unroll
            for (int st = 0; st < kMaskStrips; ++st) {
                unsigned long long m = mk[st];
                unsigned long long t = c0 & m;
                c0 ^= m;
                m = t;
                t = c1 & m;
                c1 ^= m;
                m = t;
                t = c2 & m;
                c2 ^= m;
                m = t;
                t = c3 & m;
                c3 ^= m;
                m = t;
                c4 |= m;
            }
            // add the 32 lanes' counters bit-serially in a butterfly: after
            // round r every lane holds the sum over its 2^(r+1)-lane group
            unsigned long long pl[10] = {c0, c1, c2, c3, c4, 0, 0, 0, 0, 0};
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                unsigned long long carry = 0;
#pragma unroll
                for (int q = 0; q < 5 + r; ++q) {
                    const unsigned long long x = pl[q];
                    const unsigned long long y = __shfl_xor_sync(kFull, x, 1 << r);
                    pl[q] = x ^ y ^ carry;
                    carry = (x & y) | (carry & (x ^ y));
                }
                pl[5 + r] = carry;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = lane + 32 * h;
                uint32_t v = 0;
#pragma unroll
                for (int q = 0; q < 10; ++q) v |= (uint32_t)((pl[q] >> b) & 1ull) << q;
                if (b < a.B && v) atomicAdd(gb + u * 64 + b, v);
            }
        }
        if (!grid_sync(a.bar, gridDim.x, a.status)) return;
        // ---- the sequential rule of every bucket, replayed in every block.
        // Within a group a bucket takes at most its first passing slot: a
        // second one (while the bucket still has room) needs a fresh count,
        // so the group is cut there.
        if (threadIdx.x < 64) s_pass[threadIdx.x] = 0ull;
        __syncthreads();
        for (int i = threadIdx.x; i < gn * 64; i += blockDim.x) {
            const uint32_t g = __ldcg(gb + i);
            s_g[i] = g;
            const int u = i >> 6, b = i & 63;
            if (b < a.B && s_x[u] >= 0 && (int64_t)g >= s_thr[b]) atomicOr(&s_pass[b], 1ull << u);
        }
        __syncthreads();
        const int b = threadIdx.x;
        const bool own = b < a.B && s_n[b] < a.k;
        int first = kMaskG;
        if (own && s_pass[b]) {
            const unsigned long long pm = s_pass[b];
            first = __ffsll((long long)pm) - 1;
            const unsigned long long rest = pm & (pm - 1);
            if (rest && s_n[b] + 1 < a.k) atomicMin(&s_cut, __ffsll((long long)rest) - 1);
        }
        __syncthreads();
        const int cut = s_cut;
        if (own) {
            if (first < cut) {
                const int64_t g = (int64_t)s_g[first * 64 + b];
                atomicOr(&s_acc[first], 1ull << b);
                if (blockIdx.x == 0) {
                    a.bucket_seeds[(int64_t)b * a.k + s_n[b]] = s_x[first];
                    a.bucket_gains[(int64_t)b * a.k + s_n[b]] = g;
                }
                ++s_n[b];
                s_cov[b] += g;
            }
            // diagnostics: slots this bucket considered (up to the cut, or to
            // its accept when that filled it)
            const int last = (first < cut && s_n[b] == a.k) ? first + 1 : cut;
            for (int u = 0; u < last; ++u)
                if (s_x[u] >= 0) {
                    ++s_eval[b];
                    s_scan[b] += s_len[u];
                }
        }
        __syncthreads();
        // ---- or the accepted subsets into the masks; clear the other buffer
        mask_item_prefix(s_off, cut, [&](int u) {
            return s_acc[u] ? (s_len[u] + kMaskItem - 1) / kMaskItem : (int64_t)0;
        });
        __syncthreads();
        for (int64_t c = gwarp; c < s_off[cut]; c += nwarps) {
            const int u = mask_slot_of(s_off, cut, c);   // slots without items are skipped
            const unsigned long long acc = s_acc[u];
            const int64_t e0 = (c - s_off[u]) * kMaskItem;
            const int64_t len = s_len[u];
            const int32_t *ids = a.set_ids + s_beg[u];
            int32_t id[kMaskStrips];
#pragma unroll
            for (int st = 0; st < kMaskStrips; ++st) {
                const int64_t e = e0 + st * 32 + lane;
                id[st] = e < len ? __ldg(ids + e) : -1;
            }
#pragma unroll
            for (int st = 0; st < kMaskStrips; ++st)
                if (id[st] >= 0) atomicOr(a.mask + id[st], acc);
        }
        uint32_t *other = a.gbuf + (size_t)(buf ^ 1) * kMaskG * 64;
        for (int64_t i = gtid; i < kMaskG * 64; i += gstride) other[i] = 0u;
        if (!grid_sync(a.bar, gridDim.x, a.status)) return;
        g0 += cut;
        buf ^= 1;
        G = cut < gn ? (G > 1 ? G / 2 : 1) : (G < kMaskG ? G * 2 : kMaskG);
    }
    if (blockIdx.x == 0 && threadIdx.x < a.B) {
        const int b = threadIdx.x;
        a.bucket_n[b] = s_n[b];
        a.bucket_cov[b] = s_cov[b];
        if (a.stats) {
            long long *st = a.stats + 6 * ((int64_t)a.P + b);
            st[0] = (long long)t_begin;
            st[1] = (long long)global_ns();
            st[2] = s_eval[b];
            st[3] = s_n[b];
            st[4] = s_scan[b];
            st[5] = 0;
        }
    }
}

// Alg. 4's final compare: best bucket (ties: smallest b) against the best
// local solution (ties: smallest p); the bucket wins ties.
__global__ void k_rg_final(RGArgs a, int32_t *seeds, int64_t *gains, int32_t *nseeds,
                           int64_t *coverage, int32_t *chosen) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int bstar = 0;
    for (int b = 1; b < a.B; ++b)
        if (a.bucket_cov[b] > a.bucket_cov[bstar]) bstar = b;
    int pbest = 0;
    for (int p = 1; p < a.P; ++p)
        if (a.local_cov[p] > a.local_cov[pbest]) pbest = p;
    if (a.bucket_cov[bstar] >= a.local_cov[pbest]) {
        *chosen = -1;
        const int32_t m = a.bucket_n[bstar];
        for (int32_t j = 0; j < m; ++j) {
            seeds[j] = a.bucket_seeds[(int64_t)bstar * a.k + j];
            gains[j] = a.bucket_gains[(int64_t)bstar * a.k + j];
        }
        *nseeds = m;
        *coverage = a.bucket_cov[bstar];
    } else {
        *chosen = pbest;
        const int32_t m = a.local_n[pbest];
        for (int32_t j = 0; j < m; ++j) {
            seeds[j] = a.local_seeds[(int64_t)pbest * a.k + j];
            gains[j] = a.local_gains[(int64_t)pbest * a.k + j];
        }
        *nseeds = m;
        *coverage = a.local_cov[pbest];
    }
}

}  // namespace

int32_t num_buckets(int32_t k, double delta) {
    double x = 1.0;
    int32_t b = 0;
    while (x < (double)k) {
        x *= 1.0 + delta;
        ++b;
    }
    return b < 1 ? 1 : b;
}

im_status greedy_plain(im_pool *p, int32_t k, int32_t *d_seeds, int64_t *d_gains,
                       int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st, int *d_status) {
    const int64_t n = p->g->n, theta = p->theta;
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy, kGreedyThreads, 0));
    if (per_sm < 1) return IM_ERR_UNSUPPORTED;
    const int grid = per_sm * num_sms();
    const int64_t words = (theta + 31) / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const int32_t cand_shift = (int32_t)tune_value(IM_TUNE_GREEDY_HOT);
    const int64_t vwords = (n + 31) / 32;
    const size_t o_cnt = take((size_t)vwords * 32 * 4),
                 o_cov = take((size_t)std::max<int64_t>(words, 1) * 4),
                 o_best = take((size_t)grid * 8), o_bar = take(sizeof(GridBarrier)),
                 o_work = take(16), o_hrank = take((size_t)n * 4),
                 o_hcnt = take((size_t)kHubCap * kHubRep * 4), o_hlist = take((size_t)kHubCap * 4),
                 o_cand = take((size_t)n * 4), o_ctl = take(16);
    void *base = nullptr;
    im_status s = pool_scratch(p, off, &base);
    if (s != IM_OK) return s;
    char *B = (char *)base;
    IM_CUDA(cudaMemsetAsync(B + o_bar, 0, sizeof(GridBarrier), st));
    IM_CUDA(cudaMemsetAsync(B + o_work, 0, 16, st));
    IM_CUDA(cudaMemsetAsync(B + o_ctl, 0, 16, st));
    IM_CUDA(cudaMemsetAsync(d_nseeds, 0, sizeof(int32_t), st));
    IM_CUDA(cudaMemsetAsync(d_cov, 0, sizeof(int64_t), st));
    GreedyArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    a.theta = theta;
    a.set_off = p->set_off;
    a.members = p->members;
    a.vtx_off = p->vtx_off;
    a.set_ids = p->set_ids;
    a.k = k;
    a.counts = (int32_t *)(B + o_cnt);
    a.covered = (uint32_t *)(B + o_cov);
    a.block_best = (unsigned long long *)(B + o_best);
    a.bar = (GridBarrier *)(B + o_bar);
    a.seeds = d_seeds;
    a.gains = d_gains;
    a.nseeds = d_nseeds;
    a.coverage = d_cov;
    a.status = d_status;
    a.spread = 1;
    a.hub_rank = (int32_t *)(B + o_hrank);
    a.hub_cnt = (int32_t *)(B + o_hcnt);
    a.hub_list = (int32_t *)(B + o_hlist);
    a.cand = (int32_t *)(B + o_cand);
    a.ctl = (int32_t *)(B + o_ctl);
    a.hub_cap = kHubCap;
    a.hub_shift = kHubShift;
    a.cand_shift = cand_shift;
    a.work = (unsigned long long *)(B + o_work);
    void *args[] = {&a};
    KernelTimer kt(st, "greedy");
    IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_greedy, dim3(grid), dim3(kGreedyThreads),
                                        args, 0, st));
    return IM_OK;
}

// Launches the standard greedy kernel on caller-provided scratch (used by the
// allocation-free entry point in noalloc.cu; greedy_plain above is unchanged).
im_status greedy_launch(int64_t n, int64_t theta, const int64_t *set_off, const int32_t *members,
                        const int64_t *vtx_off, const int32_t *set_ids, int32_t k, int32_t *counts,
                        uint32_t *covered, unsigned long long *block_best, int max_grid,
                        void *barrier, int32_t *seeds, int64_t *gains, int32_t *nseeds,
                        int64_t *coverage, int *status, cudaStream_t st) {
    return greedy_launch_view(n, theta, set_off, members, vtx_off, set_ids, 0, 0, k, counts,
                              covered, block_best, max_grid, barrier, seeds, gains, nseeds,
                              coverage, status, st);
}

// The same over one query of a batch: vtx_off points at the query's first
// vertex, set_ids / members hold batch-wide set and vertex ids, offset by
// sshift and vshift from the query's own.
im_status greedy_launch_view(int64_t n, int64_t theta, const int64_t *set_off,
                             const int32_t *members, const int64_t *vtx_off,
                             const int32_t *set_ids, int64_t sshift, int64_t vshift, int32_t k,
                             int32_t *counts, uint32_t *covered, unsigned long long *block_best,
                             int max_grid, void *barrier, int32_t *seeds, int64_t *gains,
                             int32_t *nseeds, int64_t *coverage, int *status, cudaStream_t st) {
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy, kGreedyThreads, 0));
    if (per_sm < 1) return IM_ERR_UNSUPPORTED;
    const int grid = std::min(per_sm * num_sms(), max_grid);
    GreedyArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    a.theta = theta;
    a.set_off = set_off;
    a.members = members;
    a.vtx_off = vtx_off;
    a.set_ids = set_ids;
    a.k = k;
    a.counts = counts;
    a.covered = covered;
    a.block_best = block_best;
    a.bar = (GridBarrier *)barrier;
    a.seeds = seeds;
    a.gains = gains;
    a.nseeds = nseeds;
    a.coverage = coverage;
    a.status = status;
    a.sshift = sshift;
    a.vshift = vshift;
    void *args[] = {&a};
    KernelTimer kt(st, "greedy");
    IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_greedy, dim3(grid), dim3(kGreedyThreads),
                                        args, 0, st));
    return IM_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

im_status randgreedi(im_pool *p, int32_t k, const im_cover_opts *o, int32_t *d_seeds,
                     int64_t *d_gains, int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st,
                     int *d_status) {
    const int32_t P = o->partitions;
    const int64_t n = p->g->n, theta = p->theta;
    const int64_t words = std::max<int64_t>(1, (theta + 31) / 32);
    // IM_AGG_GREEDY: Alg. 4's global step as written -- a greedy (the lazy one
    // of Alg. 2) over the union of the gathered local seeds -- reported as a
    // single "bucket" 0 without a threshold
    const bool naive = o->aggregator == IM_AGG_GREEDY;
    const int32_t B = naive ? 1 : num_buckets(k, o->delta);
    int64_t tr = ((int64_t)k * o->alpha_num + o->alpha_den - 1) / o->alpha_den;
    const int32_t trunc = (int32_t)std::max<int64_t>(1, std::min<int64_t>(k, tr));

    im_status s = build_partition(p, P, o->partition_seed, st);
    if (s != IM_OK) return s;
    // the largest part sizes the producers' shared memory
    std::vector<int32_t> hoff(P + 1);
    IM_CUDA(cudaMemcpyAsync(hoff.data(), p->part_off, (P + 1) * 4, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    int32_t max_np = 0;
    for (int q = 0; q < P; ++q) max_np = std::max(max_np, hoff[q + 1] - hoff[q]);
    // key + stamp (4 bytes each per candidate) + one 8-byte maximum per 32
    const size_t prod_smem = (size_t)std::max(max_np, 1) * 8 + (size_t)((max_np + 31) / 32) * 8;
    if (prod_smem > 200 * 1024) {
        set_error("RandGreedi: a vertex part is too large for shared memory; use more partitions");
        return IM_ERR_UNSUPPORTED;
    }

    // result buffers kept in the pool for im_randgreedi_details
    const size_t need = align256((size_t)P * k * 4) + align256((size_t)P * k * 8) +
                        align256((size_t)P * 4) + align256((size_t)P * 8) +
                        align256((size_t)B * 8) * 2 + align256((size_t)B * 4) +
                        align256((size_t)B * k * 4) + align256((size_t)B * k * 8) +
                        align256((size_t)(P + B) * 6 * 8);
    if (p->rg_cap_bytes < need) {
        dev_free(p->rg_block);
        p->rg_block = nullptr;
        p->rg_cap_bytes = 0;
        IM_TRY(dev_alloc(&p->rg_block, need));
        p->rg_cap_bytes = need;
    }
    {
        char *R = (char *)p->rg_block;
        size_t at = 0;
        auto grab = [&](size_t bytes) {
            char *q = R + at;
            at += align256(bytes);
            return q;
        };
        p->rg_local_seeds = (int32_t *)grab((size_t)P * k * 4);
        p->rg_local_gains = (int64_t *)grab((size_t)P * k * 8);
        p->rg_local_n = (int32_t *)grab((size_t)P * 4);
        p->rg_local_cov = (int64_t *)grab((size_t)P * 8);
        p->rg_thr = (int64_t *)grab((size_t)B * 8);
        p->rg_bucket_cov = (int64_t *)grab((size_t)B * 8);
        p->rg_bucket_n = (int32_t *)grab((size_t)B * 4);
        p->rg_bucket_seeds = (int32_t *)grab((size_t)B * k * 4);
        p->rg_bucket_gains = (int64_t *)grab((size_t)B * k * 8);
        p->rg_stats = (long long *)grab((size_t)(P + B) * 6 * 8);
    }
    p->rg_P = P;
    p->rg_B = B;
    p->rg_k = k;

    // scratch: producer + bucket bitmaps, stream slots, flags, l
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += align256(bytes);
        return at;
    };
    const size_t o_cov = take((size_t)P * words * 4);
    const size_t o_bcov = take((size_t)B * words * 4);
    const size_t o_flags = take((size_t)trunc * P * 4);
    const size_t o_elems = take((size_t)trunc * P * 4);
    const size_t o_l = take(64);
    // bucket-mask stage (two-launch mode, automatic layout, B <= 64)
    const bool use_masks = !naive && o->fused == 0 && tune_value(IM_TUNE_RG_CLUSTER) == 0 && B <= 64;
    const size_t o_mask = use_masks ? take((size_t)std::max<int64_t>(theta, 1) * 8) : 0;
    const size_t o_gbuf = use_masks ? take((size_t)2 * kMaskG * 64 * 4) : 0;
    const size_t o_bar = use_masks ? take(sizeof(GridBarrier)) : 0;
    const size_t o_sx = use_masks ? take((size_t)trunc * P * 4) : 0;
    const size_t o_sb = use_masks ? take((size_t)trunc * P * 8) : 0;
    const size_t o_sl = use_masks ? take((size_t)trunc * P * 8) : 0;
    const size_t o_lazy = naive ? take(lazy_greedy_scratch(n, theta)) : 0;
    void *base = nullptr;
    s = pool_scratch(p, off, &base);
    if (s != IM_OK) return s;
    char *Bs = (char *)base;
    IM_CUDA(cudaMemsetAsync(Bs + o_flags, 0, (size_t)trunc * P * 4, st));
    // l = max_v |S(v)|: a lower bound on the optimum of the stream, u = k l
    int64_t l = 0;
    if (!naive) {
        s = max_segment_length(p->vtx_off, n, (int64_t *)(Bs + o_l), st);
        if (s != IM_OK) return s;
        IM_CUDA(cudaMemcpyAsync(&l, Bs + o_l, 8, cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<int64_t> thr(B, 0);
    if (!naive) {
        double guess = (double)l;
        for (int32_t b = 0; b < B; ++b) {
            thr[b] = (int64_t)std::ceil(guess / (2.0 * (double)k));
            guess *= 1.0 + o->delta;
        }
    }
    IM_CUDA(cudaMemcpyAsync(p->rg_thr, thr.data(), (size_t)B * 8, cudaMemcpyHostToDevice, st));

    RGArgs a;
    a.n = n;
    a.theta = theta;
    a.words = words;
    a.k = k;
    a.P = P;
    a.trunc = trunc;
    a.B = B;
    a.vtx_off = p->vtx_off;
    a.set_ids = p->set_ids;
    a.part_off = p->part_off;
    a.part_vtx = p->part_vtx;
    a.covered = (uint32_t *)(Bs + o_cov);
    a.bcovered = (uint32_t *)(Bs + o_bcov);
    a.local_seeds = p->rg_local_seeds;
    a.local_gains = p->rg_local_gains;
    a.local_n = p->rg_local_n;
    a.local_cov = p->rg_local_cov;
    a.thr = p->rg_thr;
    a.bucket_cov = p->rg_bucket_cov;
    a.bucket_n = p->rg_bucket_n;
    a.bucket_seeds = p->rg_bucket_seeds;
    a.bucket_gains = p->rg_bucket_gains;
    a.flags = (uint32_t *)(Bs + o_flags);
    a.elems = (int32_t *)(Bs + o_elems);
    a.status = d_status;
    a.max_np = std::max(max_np, 1);
    a.evals = (int32_t)std::min<int64_t>(kProdW, std::max<int64_t>(1, tune_value(IM_TUNE_RG_EVALS)));
    a.stats = p->rg_stats;
    a.mask = use_masks ? (unsigned long long *)(Bs + o_mask) : nullptr;
    a.gbuf = use_masks ? (uint32_t *)(Bs + o_gbuf) : nullptr;
    a.bar = use_masks ? (GridBarrier *)(Bs + o_bar) : nullptr;
    a.slot_x = use_masks ? (int32_t *)(Bs + o_sx) : nullptr;
    a.slot_beg = use_masks ? (int64_t *)(Bs + o_sb) : nullptr;
    a.slot_len = use_masks ? (int64_t *)(Bs + o_sl) : nullptr;
    if (use_masks) IM_CUDA(cudaMemsetAsync(Bs + o_bar, 0, sizeof(GridBarrier), st));

    IM_TRY(raise_dyn_smem((const void *)k_randgreedi, prod_smem));
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_randgreedi, kRGThreads,
                                                          prod_smem));
    if (per_sm < 1) return IM_ERR_UNSUPPORTED;
    const int resident = per_sm * num_sms();
    bool fused = !naive && o->fused != 0 && resident >= 2;
    if (fused) {
        a.ncons = std::min<int32_t>(B, resident / 2);
        a.nprod = std::min<int32_t>(P, resident - a.ncons);
        a.first_role = 0;
        void *args[] = {&a};
        KernelTimer kt(st, "randgreedi_fused");
        IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_randgreedi,
                                            dim3(a.nprod + a.ncons), dim3(kRGThreads), args,
                                            prod_smem, st));
    } else {
        // producers alone, then consumers alone (the stream is complete by then)
        IM_TRY(raise_dyn_smem((const void *)k_rg_local, prod_smem));
        int per_l = 0;
        IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_l, k_rg_local, kProdThreads,
                                                              prod_smem));
        if (per_l < 1) return IM_ERR_UNSUPPORTED;
        a.nprod = std::min<int32_t>(P, per_l * num_sms());
        a.ncons = 0;
        a.first_role = 0;
        {
            KernelTimer kt(st, "randgreedi_local");
            k_rg_local<<<a.nprod, kProdThreads, prod_smem, st>>>(a);
        }
        IM_CUDA(cudaGetLastError());
        const int64_t want = tune_value(IM_TUNE_RG_CLUSTER);   // 0 auto, -1 off, 1..8
        if (naive) {
            // the global greedy over the first `trunc` seeds of every part
            int32_t W = (int32_t)tune_value(IM_TUNE_GREEDY_EVALS);
            if (W <= 0) W = 16;
            IM_CUDA(cudaMemsetAsync(p->rg_bucket_n, 0, sizeof(int32_t), st));
            IM_CUDA(cudaMemsetAsync(p->rg_bucket_cov, 0, sizeof(int64_t), st));
            IM_CUDA(cudaMemsetAsync(p->rg_stats + (size_t)P * 6, 0, 6 * 8, st));
            s = greedy_lazy_launch(n, theta, p->vtx_off, p->set_ids, k, W, Bs + o_lazy,
                                   p->rg_bucket_seeds, p->rg_bucket_gains, p->rg_bucket_n,
                                   p->rg_bucket_cov, p->lz_stats, d_status, st,
                                   p->rg_local_seeds, p->rg_local_n, P, trunc, k);
            if (s != IM_OK) return s;
        } else if (use_masks) {
            // buckets: one pass over each streamed subset serves all buckets
            int per = 0;
            IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rg_stream_masks,
                                                                  kRGThreads, 0));
            if (per < 1) return IM_ERR_UNSUPPORTED;
            const int grid = std::min(per, 2) * num_sms();
            void *args[] = {&a};
            KernelTimer kt(st, "randgreedi_stream");
            IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_rg_stream_masks, dim3(grid),
                                                dim3(kRGThreads), args, 0, st));
        }
        // buckets: shared-memory bitmaps split over a cluster when theta fits
        int CS = want > 0 ? (int)want : 1;
        int64_t R = 0;
        size_t csmem = 0;
        for (; CS <= 8; CS *= 2) {
            R = (theta + (int64_t)CS * 32 - 1) / ((int64_t)CS * 32) * 32;
            csmem = (size_t)(R / 8) + 2 * kSpec * sizeof(unsigned);
            if (csmem <= kClusterSmemCap) break;
        }
        if (want < 0) CS = 16;   // global-memory bitmaps requested
        if (naive || use_masks) {
            // done above
        } else if (CS <= 8) {
            unsigned *counter = (unsigned *)(Bs + o_l) + 2;
            IM_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
            IM_TRY(raise_dyn_smem((const void *)k_rg_stream_cluster, csmem));
            const int nclusters = std::max(1, std::min<int>(B, num_sms() / CS));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(nclusters * CS);
            cfg.blockDim = dim3(kRGThreads);
            cfg.dynamicSmemBytes = csmem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = CS;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            KernelTimer kt(st, "randgreedi_stream");
            IM_CUDA(cudaLaunchKernelEx(&cfg, k_rg_stream_cluster, a, R, counter));
        } else {
            a.ncons = std::min<int32_t>(B, resident);
            a.first_role = 1;
            {
                KernelTimer kt(st, "randgreedi_stream");
                k_randgreedi<<<a.ncons, kRGThreads, prod_smem, st>>>(a);
            }
            IM_CUDA(cudaGetLastError());
        }
    }
    int32_t *d_chosen = (int32_t *)(Bs + o_l);   // l is no longer needed
    {
        KernelTimer kt(st, "randgreedi_final");
        k_rg_final<<<1, 32, 0, st>>>(a, d_seeds, d_gains, d_nseeds, d_cov, d_chosen);
    }
    IM_CUDA(cudaGetLastError());
    int32_t chosen = 0;
    IM_CUDA(cudaMemcpyAsync(&chosen, d_chosen, 4, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    p->rg_chosen = chosen;
    return IM_OK;
}

}  // namespace im
