// sample.cu -- RRR sampling (IC reverse BFS, LT backward walk), compaction into
// the pool's CSR, and the segmented sorts that put every set in ascending order.
//
// Every sampler is a persistent kernel that takes the next sample id from a
// global counter (dynamic balancing: set sizes are heavy tailed on R-MAT).
// IC (Def. 3 under the IC live-edge world): one warp per sample expands up to
// 32 queued vertices at once; their in-edge ranges are split into aligned
// groups of four edges, so each lane makes one Philox call (four coins) and
// one 16-byte load of weights and one of sources per group.  Sets longer than
// the warp's queue are re-run by k_sample_ic_big, one block per sample.  LT:
// k_sample_lt1 (default) runs one walk per thread; the picked in-edge (first
// edge whose running weight sum exceeds the draw) comes from one division when
// the vertex's in-edges weigh the same, else from a cut-point table in O(1)
// expected loads, and revisits are tested through a per-walk Bloom filter
// (flagged walks are checked exactly, two at a time).  k_sample_lt<G> runs a
// walk per group of G lanes, picking by the same division or over a fanout-32
// search tree (a tuning-knob alternative, and the second pass for walks longer
// than the thread kernel's queue).  The LT index they read (vertex records;
// running sums, tree and cut points only when some vertex's in-edges weigh
// differently) is built once per graph by build_lt_index: in-lists of up to 32
// edges get their running sums from one thread each, up to 1024 from a warp,
// longer ones from a block.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace im {

namespace {

constexpr int kSampleThreads = 256;          // 8 warps per block
constexpr int kWarps = kSampleThreads / 32;
constexpr int64_t kSmemVisBits = 1 << 16;    // visited bitmap in smem when n <= this
constexpr int kPathSmem = 256;               // LT path entries mirrored in smem (warp walks)
constexpr int kPathSmemGroup = 64;           // ... per walk when a warp runs several walks
constexpr int64_t kQueueCapIC = 1 << 14;     // per-warp queue entries (first pass)
constexpr int64_t kQueueCapLT = 1 << 11;
constexpr int kICU = 2;                      // IC edge groups per lane in flight
constexpr int kWarpSortBytes = 4096;         // per-warp smem sort buffer
constexpr int kBlockSortCap = 16384;         // ... by one block in shared memory (int32)

struct SampleArgs {
    const QueryView *qv;      // [nq] graphs and streams of the queries of this launch
    const int64_t *qstart;    // [nq + 1] first flattened sample index of each query
    int32_t nq;
    int64_t count;            // work items
    const int64_t *list;      // if non-null: work item i is sample index list[i]
    int32_t *stage;
    int64_t stage_cap;
    unsigned long long *stage_cursor;
    int64_t *stage_off;       // [count of the call]
    int32_t *sizes;           // [count of the call]; -1 marks a queue overflow
    int32_t *queues;
    int64_t qcap;
    uint32_t *gvis;
    int64_t vis_words;
    unsigned long long *examined;
    unsigned long long *alg_bytes;
    unsigned long long *work;
    int64_t *ovf_list;
    unsigned long long *ovf_count;
    int *status;
};

// The query that flattened sample index j belongs to (largest q, qstart[q] <= j).
__device__ __forceinline__ int find_query(const SampleArgs &a, int64_t j) {
    int lo = 0, hi = a.nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a.qstart + mid) <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int64_t next_item(const SampleArgs &a, int lane) {
    unsigned long long j = 0;
    if (lane == 0) j = atomicAdd(a.work, 1ull);
    j = __shfl_sync(kFull, j, 0);
    if (j >= (unsigned long long)a.count) return -1;
    return a.list ? a.list[j] : (int64_t)j;
}

// Move the finished set q[0..len) to the stage and record where it went.
__device__ __forceinline__ void emit_set(const SampleArgs &a, int64_t j, const int32_t *q,
                                         int64_t len, int lane) {
    unsigned long long pos = 0;
    if (lane == 0) pos = atomicAdd(a.stage_cursor, (unsigned long long)len);
    pos = __shfl_sync(kFull, pos, 0);
    if ((int64_t)pos + len > a.stage_cap) {
        if (lane == 0) {
            raise_status(a.status, kDevStageOverflow);
            a.sizes[j] = 0;
            a.stage_off[j] = 0;
        }
        return;
    }
    for (int64_t i = lane; i < len; i += 32) a.stage[pos + i] = q[i];
    if (lane == 0) {
        a.stage_off[j] = (int64_t)pos;
        a.sizes[j] = (int32_t)len;
    }
}

__device__ __forceinline__ void mark_overflow(const SampleArgs &a, int64_t j, int lane) {
    if (lane == 0) {
        a.sizes[j] = -1;
        a.stage_off[j] = 0;
        unsigned long long at = atomicAdd(a.ovf_count, 1ull);
        a.ovf_list[at] = j;
    }
}

// ---------------------------------------------------------------------------
// IC: stochastic reverse BFS.  Edge e of sample s is live iff lane (e & 3) of
// Philox(s, e >> 2 (low word), e >> 34, coin tag) is below w[e].
// ---------------------------------------------------------------------------
template <bool kSmemVis>
__global__ void __launch_bounds__(kSampleThreads, 4) k_sample_ic(SampleArgs a) {
    extern __shared__ uint32_t smem_vis[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wib;
    uint32_t *vis = kSmemVis ? smem_vis + (size_t)wib * a.vis_words
                             : a.gvis + (size_t)gw * (size_t)a.vis_words;
    int32_t *q = a.queues + (size_t)gw * (size_t)a.qcap;
    if (kSmemVis)
        for (int64_t i = lane; i < a.vis_words; i += 32) vis[i] = 0;
    __syncwarp();
    unsigned long long exam = 0, abytes = 0;
    for (;;) {
        const int64_t j = next_item(a, lane);
        if (j < 0) break;
        const int qi = find_query(a, j);
        const QueryView &V = a.qv[qi];
        const int64_t *in_off = V.in_off;
        const int32_t *in_src = V.in_src;
        const uint32_t *wgt = V.w;
        const uint64_t seed = V.seed;
        const uint32_t k0 = seed_lo(seed), k1 = seed_hi(seed);
        const uint32_t s = V.first + (uint32_t)(j - __ldg(a.qstart + qi));
        const uint32_t root = rrr_root(seed, s, V.n);
        if (lane == 0) {
            atomicOr(&vis[root >> 5], 1u << (root & 31));
            q[0] = (int32_t)root;
        }
        __syncwarp();
        int64_t head = 0, tail = 1;
        bool overflow = false;
        unsigned long long sexam = 0;
        while (head < tail && !overflow) {
            const int nb = (int)(tail - head < 32 ? tail - head : 32);
            int64_t eb = 0, ee = 0;
            if (lane < nb) {
                const int32_t v = q[head + lane];
                eb = __ldg(in_off + v);
                ee = __ldg(in_off + v + 1);
                sexam += (unsigned long long)(ee - eb);
            }
            head += nb;
            const int64_t g0 = eb >> 2;
            const int64_t ng = ee > eb ? ((ee - 1) >> 2) - g0 + 1 : 0;
            const int64_t incl = warp_incl_scan<int64_t>(ng, lane);
            const int64_t total = __shfl_sync(kFull, incl, 31);
            // kICU edge groups per lane per iteration: their loads and coin
            // draws are independent, so they overlap
            for (int64_t base = 0; base < total; base += 32 * kICU) {
                uint4 wv[kICU];
                int4 sv[kICU];
                int64_t gg[kICU], lo[kICU], hi[kICU];
#pragma unroll
                for (int uu = 0; uu < kICU; ++uu) {
                    const int64_t t = base + uu * 32 + lane;
                    int owner = 0;   // first lane whose inclusive group count exceeds t
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int64_t c = __shfl_sync(kFull, incl, owner + step - 1);
                        if (c <= t) owner += step;
                    }
                    const int64_t o_incl = __shfl_sync(kFull, incl, owner);
                    const int64_t o_ng = __shfl_sync(kFull, ng, owner);
                    const int64_t o_g0 = __shfl_sync(kFull, g0, owner);
                    lo[uu] = __shfl_sync(kFull, eb, owner);
                    hi[uu] = __shfl_sync(kFull, ee, owner);
                    gg[uu] = -1;
                    if (t < total) {
                        gg[uu] = o_g0 + (t - (o_incl - o_ng));
                        wv[uu] = __ldg(reinterpret_cast<const uint4 *>(wgt) + gg[uu]);
                        sv[uu] = __ldg(reinterpret_cast<const int4 *>(in_src) + gg[uu]);
                    }
                }
                unsigned fresh = 0;
                int32_t src[4 * kICU];
#pragma unroll
                for (int uu = 0; uu < kICU; ++uu) {
                    src[4 * uu + 0] = src[4 * uu + 1] = src[4 * uu + 2] = src[4 * uu + 3] = 0;
                    if (gg[uu] < 0) continue;
                    const int64_t g = gg[uu];
                    const uint4 coin = philox4x32_10(
                        make_uint4(s, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), kStreamCoin), k0,
                        k1);
                    const uint32_t cv[4] = {coin.x, coin.y, coin.z, coin.w};
                    const uint32_t wq[4] = {wv[uu].x, wv[uu].y, wv[uu].z, wv[uu].w};
                    src[4 * uu + 0] = sv[uu].x;
                    src[4 * uu + 1] = sv[uu].y;
                    src[4 * uu + 2] = sv[uu].z;
                    src[4 * uu + 3] = sv[uu].w;
                    const int64_t e0 = g << 2;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int64_t e = e0 + c;
                        if (e >= lo[uu] && e < hi[uu] && cv[c] < wq[c]) {
                            const uint32_t u = (uint32_t)src[4 * uu + c];
                            const uint32_t bit = 1u << (u & 31);
                            if (!(atomicOr(&vis[u >> 5], bit) & bit)) fresh |= 1u << (4 * uu + c);
                        }
                    }
                }
                const int nf = __popc(fresh);
                const int inclf = warp_incl_scan<int>(nf, lane);
                const int totf = __shfl_sync(kFull, inclf, 31);
                if (totf == 0) continue;
                if (tail + totf > a.qcap) {
                    // drop this sample; un-mark what was just marked
#pragma unroll
                    for (int c = 0; c < 4 * kICU; ++c)
                        if (fresh >> c & 1) {
                            const uint32_t u = (uint32_t)src[c];
                            atomicAnd(&vis[u >> 5], ~(1u << (u & 31)));
                        }
                    overflow = true;
                    break;
                }
                int64_t pos = tail + inclf - nf;
#pragma unroll
                for (int c = 0; c < 4 * kICU; ++c)
                    if (fresh >> c & 1) q[pos++] = src[c];
                tail += totf;
                __syncwarp();
            }
        }
        __syncwarp();
        if (overflow) {
            mark_overflow(a, j, lane);
        } else {
            emit_set(a, j, q, tail, lane);
            exam += sexam;
            // 16 B offsets + 4 B write per member, 8 B per examined edge, 8 B per set
            abytes += 8ull * sexam + (lane == 0 ? 20ull * (unsigned long long)tail + 8ull : 0ull);
        }
        // reset the visited bits of this sample
        if (tail > a.vis_words) {
            for (int64_t i = lane; i < a.vis_words; i += 32) vis[i] = 0;
        } else {
            for (int64_t i = lane; i < tail; i += 32) {
                const uint32_t u = (uint32_t)q[i];
                vis[u >> 5] = 0;
            }
        }
        __syncwarp();
    }
    exam = warp_sum<unsigned long long>(exam);
    abytes = warp_sum<unsigned long long>(abytes);
    if (lane == 0 && exam) atomicAdd(a.examined, exam);
    if (lane == 0 && abytes) atomicAdd(a.alg_bytes, abytes);
}

// IC, one block per sample: the second pass for the sets longer than a warp's
// queue.  The giant sets of hub-heavy graphs (hundreds of thousands of
// members, tens of millions of examined in-edges) are a level-synchronous
// BFS whose 32 warps take 32 queued vertices of the current level at a time
// and expand their in-edges four per lane (one Philox call per group of four,
// as in k_sample_ic), appending what they reach with one block-level atomic
// per warp and step.  The queue and visited bitmap (n entries / n bits per
// block) live in global memory.  The set is copied to the stage by the block.
constexpr int kICBigThreads = 1024;
constexpr int kICBigU = 2;          // edge groups per lane in flight (k_sample_ic_big)

// One group of four in-edges of sample s: coins of edge group g (edges
// 4g .. 4g+3 inside [eb, ee)) against its loaded weights wv, with sources sv;
// marks the live edges' fresh sources visited and returns their bits (the
// sources in src[]).
__device__ __forceinline__ unsigned ic_group_loaded(const uint4 wv, const int4 sv, int64_t g,
                                                    int64_t eb, int64_t ee, uint32_t s,
                                                    uint32_t k0, uint32_t k1, uint32_t *vis,
                                                    int32_t (&src)[4]) {
    const uint4 coin = philox4x32_10(
        make_uint4(s, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), kStreamCoin), k0, k1);
    const uint32_t cv[4] = {coin.x, coin.y, coin.z, coin.w};
    const uint32_t wq[4] = {wv.x, wv.y, wv.z, wv.w};
    src[0] = sv.x;
    src[1] = sv.y;
    src[2] = sv.z;
    src[3] = sv.w;
    unsigned fresh = 0;
    const int64_t e0 = g << 2;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t e = e0 + c;
        if (e >= eb && e < ee && cv[c] < wq[c]) {
            const uint32_t u = (uint32_t)src[c];
            const uint32_t bit = 1u << (u & 31);
            if (!(atomicOr(&vis[u >> 5], bit) & bit)) fresh |= 1u << c;
        }
    }
    return fresh;
}

// Appends each lane's fresh sources to the block queue (one atomic per warp).
__device__ __forceinline__ void ic_append(unsigned fresh, const int32_t (&src)[4], int lane,
                                          unsigned long long *tail, int32_t *q) {
    const int nf = __popc(fresh);
    const int inclf = warp_incl_scan<int>(nf, lane);
    const int totf = __shfl_sync(kFull, inclf, 31);
    if (totf == 0) return;
    long long at = 0;
    if (lane == 31) at = (long long)atomicAdd(tail, (unsigned long long)totf);
    at = __shfl_sync(kFull, at, 31);
    int64_t pos = at + inclf - nf;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (fresh >> c & 1) q[pos++] = src[c];
}

__global__ void __launch_bounds__(kICBigThreads) k_sample_ic_big(SampleArgs a) {
    __shared__ unsigned long long s_item, s_tail, s_cursor, s_pos;
    __shared__ unsigned long long s_red[2][kICBigThreads / 32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *q = a.queues + (size_t)blockIdx.x * (size_t)a.qcap;
    uint32_t *vis = a.gvis + (size_t)blockIdx.x * (size_t)a.vis_words;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(a.work, 1ull);
            s_tail = 0;
        }
        __syncthreads();
        const unsigned long long jw = s_item;
        if (jw >= (unsigned long long)a.count) break;
        const int64_t j = a.list ? a.list[jw] : (int64_t)jw;
        const int qi = find_query(a, j);
        const QueryView &V = a.qv[qi];
        const int64_t *in_off = V.in_off;
        const int32_t *in_src = V.in_src;
        const uint32_t *wgt = V.w;
        const uint32_t k0 = seed_lo(V.seed), k1 = seed_hi(V.seed);
        const uint32_t s = V.first + (uint32_t)(j - __ldg(a.qstart + qi));
        if (threadIdx.x == 0) {
            const uint32_t root = rrr_root(V.seed, s, V.n);
            atomicOr(&vis[root >> 5], 1u << (root & 31));
            q[0] = (int32_t)root;
            s_tail = 1;
        }
        __syncthreads();
        unsigned long long sexam = 0;
        long long head = 0;
        for (;;) {
            const long long lvl_end = (long long)s_tail;
            if (head >= lvl_end) break;
            if (threadIdx.x == 0) s_cursor = (unsigned long long)head;
            __syncthreads();
            for (;;) {
                long long base = 0;
                if (lane == 0) base = (long long)atomicAdd(&s_cursor, 32ull);
                base = __shfl_sync(kFull, base, 0);
                if (base >= lvl_end) break;
                const int nb = (int)(lvl_end - base < 32 ? lvl_end - base : 32);
                int64_t eb = 0, ee = 0;
                if (lane < nb) {
                    const int32_t v = q[base + lane];
                    eb = __ldg(in_off + v);
                    ee = __ldg(in_off + v + 1);
                    sexam += (unsigned long long)(ee - eb);
                }
                const int64_t g0 = eb >> 2;
                const int64_t ng = ee > eb ? ((ee - 1) >> 2) - g0 + 1 : 0;
                const int64_t incl = warp_incl_scan<int64_t>(ng, lane);
                const int64_t total = __shfl_sync(kFull, incl, 31);
                // kICBigU edge groups per lane in flight: their loads are issued
                // together before any coin is drawn
                for (int64_t gb = 0; gb < total; gb += 32 * kICBigU) {
                    int64_t grp[kICBigU], geb[kICBigU], gee[kICBigU];
                    uint4 wv[kICBigU];
                    int4 sv[kICBigU];
#pragma unroll
                    for (int u = 0; u < kICBigU; ++u) {
                        const int64_t t = gb + u * 32 + lane;
                        int owner = 0;   // first lane whose inclusive group count exceeds t
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const int64_t c = __shfl_sync(kFull, incl, owner + step - 1);
                            if (c <= t) owner += step;
                        }
                        const int64_t o_incl = __shfl_sync(kFull, incl, owner);
                        const int64_t o_ng = __shfl_sync(kFull, ng, owner);
                        const int64_t o_g0 = __shfl_sync(kFull, g0, owner);
                        geb[u] = __shfl_sync(kFull, eb, owner);
                        gee[u] = __shfl_sync(kFull, ee, owner);
                        grp[u] = t < total ? o_g0 + (t - (o_incl - o_ng)) : -1;
                        if (grp[u] >= 0) {
                            wv[u] = __ldg(reinterpret_cast<const uint4 *>(wgt) + grp[u]);
                            sv[u] = __ldg(reinterpret_cast<const int4 *>(in_src) + grp[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kICBigU; ++u) {
                        unsigned fresh = 0;
                        int32_t src[4] = {0, 0, 0, 0};
                        if (grp[u] >= 0)
                            fresh = ic_group_loaded(wv[u], sv[u], grp[u], geb[u], gee[u], s, k0, k1,
                                                    vis, src);
                        ic_append(fresh, src, lane, &s_tail, q);
                    }
                }
            }
            __syncthreads();
            head = lvl_end;
        }
        // emit: reserve the stage range, copy the queue, record size and offset
        const long long len = (long long)s_tail;
        unsigned long long ex = warp_sum<unsigned long long>(sexam);
        if (lane == 0) s_red[0][warp] = ex;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w2 = 0; w2 < kICBigThreads / 32; ++w2) tot += s_red[0][w2];
            s_pos = atomicAdd(a.stage_cursor, (unsigned long long)len);
            if ((long long)s_pos + len > a.stage_cap) {
                raise_status(a.status, kDevStageOverflow);
                a.sizes[j] = 0;
                a.stage_off[j] = 0;
                s_pos = ~0ull;
            } else {
                a.stage_off[j] = (int64_t)s_pos;
                a.sizes[j] = (int32_t)len;
                atomicAdd(a.examined, tot);
                // 16 B offsets + 4 B write per member, 8 B per examined edge, 8 B per set
                atomicAdd(a.alg_bytes, 8ull * tot + 20ull * (unsigned long long)len + 8ull);
            }
        }
        __syncthreads();
        if (s_pos != ~0ull)
            for (long long x = threadIdx.x; x < len; x += blockDim.x) a.stage[s_pos + x] = q[x];
        // clear this sample's visited bits
        if (len > a.vis_words) {
            for (int64_t x = threadIdx.x; x < a.vis_words; x += blockDim.x) vis[x] = 0u;
        } else {
            for (long long x = threadIdx.x; x < len; x += blockDim.x) vis[q[x] >> 5] = 0u;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// LT: backward walk of the LT live-edge world.  Vertex v picks the first
// in-edge whose running weight sum exceeds Philox(s, v, 0, pick tag).x; the
// walk stops when nothing is picked or the picked source is already on it.
//
// The pick is found in a fanout-32 search tree over v's running sums (built
// by k_lt_index): every level is read as one contiguous window of at most 32
// values, one per lane, and a ballot selects the child -- so a step costs
// ceil(log32 d) + 1 coalesced loads instead of scattered probes, and the leaf
// that matches also carries the source id.
// ---------------------------------------------------------------------------
// Group-wide helpers: a group is G consecutive lanes of a warp running one walk.
template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
    return G == 32 ? kFull : (((1u << G) - 1u) << ((lane / G) * G));
}

// One walk per group of G lanes; a warp runs 32 / G walks in lockstep.  The
// loop is warp-uniform: every iteration each group advances its own walk by
// one step (groups without a walk idle through predication, so the warp never
// splits and the Philox draw, the search and the revisit test of all its
// walks share one instruction stream); a group whose walk ended emits it and
// takes the next sample at the top of the next iteration.  Every level of the
// search tree is a window of up to 32 values; lane l of a group holds values
// [l * 32/G, (l + 1) * 32/G) of it.
template <int G>
__global__ void __launch_bounds__(kSampleThreads, G == 32 ? 8 : 5) k_sample_lt(SampleArgs a) {
    constexpr int NG = 32 / G;                       // walks per warp
    constexpr int NV = 32 / G;                       // window values per lane
    constexpr int PS = G == 32 ? kPathSmem : kPathSmemGroup;
    constexpr unsigned GBITS = G == 32 ? kFull : ((1u << G) - 1u);
    __shared__ int32_t spath[kWarps * NG][PS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G, gbase = grp * G;
    const unsigned gmask = group_mask<G>(lane);
    const int64_t slot = ((int64_t)blockIdx.x * kWarps + wib) * NG + grp;
    int32_t *q = a.queues + (size_t)slot * (size_t)a.qcap;
    int32_t *sp = spath[wib * NG + grp];
    unsigned long long exam = 0, abytes = 0;
    bool active = false, exhausted = false;
    int64_t j = 0;
    uint32_t s = 0, cur = 0, k0 = 0, k1 = 0;
    const uint4 *vrec = nullptr;
    const unsigned long long *leaf_arr = nullptr, *tree = nullptr;
    const int32_t *srcs = nullptr;
    int32_t len = 0;
    unsigned long long sexam = 0;
    uint32_t sbytes = 0;   // flushed into abytes before it can wrap
    for (;;) {
        if (!active && !exhausted) {                 // group-uniform
            unsigned long long jw = 0;
            if (gl == 0) jw = atomicAdd(a.work, 1ull);
            jw = __shfl_sync(gmask, jw, 0, G);
            if (jw < (unsigned long long)a.count) {
                j = a.list ? a.list[jw] : (int64_t)jw;
                const int qi = find_query(a, j);
                const QueryView &V = a.qv[qi];
                vrec = V.lt_vrec;
                leaf_arr = V.lt_leaf;
                tree = V.lt_tree;
                srcs = V.in_src;
                k0 = seed_lo(V.seed);
                k1 = seed_hi(V.seed);
                s = V.first + (uint32_t)(j - __ldg(a.qstart + qi));
                cur = rrr_root(V.seed, s, V.n);
                if (gl == 0) {
                    q[0] = (int32_t)cur;
                    sp[0] = (int32_t)cur;
                }
                len = 1;
                sexam = 0;
                sbytes = 8;
                active = true;
            } else {
                exhausted = true;
            }
        }
        __syncwarp();
        if (!__any_sync(kFull, active)) break;

        // ---- one step of every active walk ----
        const uint32_t x = philox4x32_10(make_uint4(s, cur, 0u, kStreamPick), k0, k1).x;
        const unsigned long long xs = (unsigned long long)x;
        const uint4 vr = active ? __ldg(vrec + cur) : make_uint4(0u, 0u, 0u, 0u);
        const int32_t d = (int32_t)vr.y;
        // in-edges of equal weight u: the pick is edge floor(x / u), no search
        // (the running sums and tree exist only when some vertex needs them)
        const bool eqw = vr.w != 0u;
        bool live = active && d > 0 && !eqw;         // group-uniform
        const uint32_t nlev = vr.z >> 28;
        const int lmax = (int)__reduce_max_sync(kFull, live ? nlev : 0u);
        const unsigned long long *lvl = tree + (vr.z & 0x0fffffffu);   // levels stored top-down
        int32_t blk = 0;
        for (int l = lmax; l >= 1; --l) {
            const bool here = live && l <= (int)nlev;
            const int32_t sz = here ? (int32_t)(((int64_t)d + (1ll << (5 * l)) - 1) >> (5 * l)) : 0;
            int lf = NV;
#pragma unroll
            for (int v = NV - 1; v >= 0; --v) {
                const int32_t idx = blk * 32 + gl * NV + v;
                if (idx < sz && xs < __ldg(lvl + idx)) lf = v;
            }
            const unsigned bal = (__ballot_sync(kFull, lf < NV) >> gbase) & GBITS;
            const int f = bal ? __ffs(bal) - 1 : 0;
            const int lfv = __shfl_sync(kFull, lf, gbase + f);
            if (here) {
                if (!bal) live = false;
                else {
                    blk = blk * 32 + f * NV + lfv;
                    lvl += sz;
                }
            }
        }
        int32_t pick = -1;
        unsigned long long leaf = 0;
        {
            int lf = NV;
            unsigned long long hit = 0;
#pragma unroll
            for (int v = NV - 1; v >= 0; --v) {
                const int32_t idx = blk * 32 + gl * NV + v;
                if (live && idx < d) {
                    const unsigned long long r = __ldg(leaf_arr + vr.x + idx);
                    if (xs < (r >> 31)) {
                        lf = v;
                        hit = r;
                    }
                }
            }
            const unsigned bal = (__ballot_sync(kFull, lf < NV) >> gbase) & GBITS;
            const int f = bal ? __ffs(bal) - 1 : 0;
            const int lfv = __shfl_sync(kFull, lf, gbase + f);
            const unsigned long long hv = __shfl_sync(kFull, hit, gbase + f);
            if (live && bal) {
                pick = blk * 32 + f * NV + lfv;
                leaf = hv;
            }
        }
        if (active && eqw) {
            const uint32_t ei = x / vr.w;
            if (ei < (uint32_t)d) {
                pick = (int32_t)ei;
                leaf = (unsigned long long)(uint32_t)__ldg(srcs + vr.x + ei);   // its source
            }
        }
        if (active && gl == 0) {
            sexam += (unsigned long long)(pick >= 0 ? pick + 1 : d);
            // vertex record, binary search of d cumulative weights (none for equal
            // weights), source, member write
            sbytes += 16u + (d > 0 && !eqw ? 8u * (uint32_t)(32 - __clz((uint32_t)d)) : 0u) +
                      (pick >= 0 ? 4u : 0u) + 4u;
            if (sbytes > (1u << 30)) {   // only long walks of the second pass get here
                abytes += sbytes;
                sbytes = 0;
            }
        }
        // revisit test of the picked source against the walk so far
        const bool picked = active && pick >= 0;
        const int32_t u = (int32_t)(leaf & 0x7fffffffull);
        const int lenmax = (int)__reduce_max_sync(kFull, picked ? (unsigned)len : 0u);
        bool seen = false;
        for (int32_t i = gl; i < lenmax; i += G)
            if (picked && i < len) seen |= (i < PS ? sp[i] : q[i]) == u;
        const bool seen_g = ((__ballot_sync(kFull, seen) >> gbase) & GBITS) != 0;
        const bool grow = picked && !seen_g && len < a.qcap;
        const bool ovf = picked && !seen_g && len >= a.qcap;
        if (grow) {
            if (gl == 0) {
                q[len] = u;
                if (len < PS) sp[len] = u;
            }
            ++len;
            cur = (uint32_t)u;
        }
        __syncwarp();
        if (active && !grow) {                       // the walk ended: emit it
            if (ovf) {
                if (gl == 0) {
                    a.sizes[j] = -1;
                    a.stage_off[j] = 0;
                    a.ovf_list[atomicAdd(a.ovf_count, 1ull)] = j;
                }
            } else {
                unsigned long long pos = 0;
                if (gl == 0) pos = atomicAdd(a.stage_cursor, (unsigned long long)len);
                pos = __shfl_sync(gmask, pos, 0, G);
                if ((int64_t)pos + len > a.stage_cap) {
                    if (gl == 0) {
                        raise_status(a.status, kDevStageOverflow);
                        a.sizes[j] = 0;
                        a.stage_off[j] = 0;
                    }
                } else {
                    for (int32_t i = gl; i < len; i += G) a.stage[pos + i] = i < PS ? sp[i] : q[i];
                    if (gl == 0) {
                        a.stage_off[j] = (int64_t)pos;
                        a.sizes[j] = len;
                    }
                }
                exam += sexam;
                if (gl == 0) abytes += sbytes;
            }
            active = false;
        }
        __syncwarp();
    }
    exam = warp_sum<unsigned long long>(exam);
    abytes = warp_sum<unsigned long long>(abytes);
    if (lane == 0 && exam) atomicAdd(a.examined, exam);
    if (lane == 0 && abytes) atomicAdd(a.alg_bytes, abytes);
}

// LT, one walk per thread.  A step is one Philox draw, the vertex record and
// one dependent load: the source of in-edge floor(x / u) when all in-edges of
// the vertex weigh u (1/in-degree weights, for one), else one guide entry (see
// k_lt_guide), with a binary search over the running sums only when the draw
// lies past the guide's edge.  The revisit test goes through a 1024-bit Bloom filter of
// the walk in shared memory (two hashes); a walk whose pick hits the filter
// waits (takes no step) until kLT1Flush walks of its warp wait, or every active
// one does, and the whole warp then checks them exactly, scanning kLT1Group of
// their paths together so that those loads are in flight at once.  Finished
// walks are copied to the stage by the whole warp as well, kLT1Group paths at
// a time, after one warp-wide reservation.
// A warp takes sample indices kLT1Chunk at a time, and all its lanes then draw
// the roots of that chunk together (one Philox call each) into a per-warp ring
// in shared memory, from which a lane starting a walk reads its root.
// Waiting changes no draw: a walk's steps are the same whenever they run.
constexpr int kLT1Threads = 256;
constexpr int kLT1Warps = kLT1Threads / 32;
constexpr int kBloomWords = 32;              // 1024 bits per walk
constexpr int64_t kQueueCapLT1 = 512;
constexpr unsigned kLT1Chunk = 32;           // sample indices a warp takes at once (one per lane)
constexpr int kLT1Flush = 2;                 // flagged walks that trigger the exact checks
constexpr int kLT1Group = 2;                 // paths scanned or copied together
// The work items of one launch stay below this count, so that the warp's chunk
// bounds fit 32 bits (a larger job takes the grouped kernel).
constexpr int64_t kLT1MaxCount = (1ll << 32) - (1ll << 28);

__device__ __forceinline__ uint32_t bloom_h1(uint32_t u) { return (u * 0x9E3779B1u) >> 22; }
__device__ __forceinline__ uint32_t bloom_h2(uint32_t u) {
    return ((u ^ (u >> 16)) * 0x85EBCA6Bu) >> 22;
}

// bl points at this thread's column: word w of its filter is bl[w * kLT1Threads]
// (a warp touching any words hits 32 distinct banks)
__device__ __forceinline__ void bloom_add(uint32_t *bl, uint32_t u) {
    const uint32_t h1 = bloom_h1(u), h2 = bloom_h2(u);
    bl[(h1 >> 5) * kLT1Threads] |= 1u << (h1 & 31);
    bl[(h2 >> 5) * kLT1Threads] |= 1u << (h2 & 31);
}

__device__ __forceinline__ bool bloom_has(const uint32_t *bl, uint32_t u) {
    const uint32_t h1 = bloom_h1(u), h2 = bloom_h2(u);
    return ((bl[(h1 >> 5) * kLT1Threads] >> (h1 & 31)) & (bl[(h2 >> 5) * kLT1Threads] >> (h2 & 31)) &
            1u) != 0;
}

// 16-byte read-only load with an L2 eviction-priority policy (createpolicy).
__device__ __forceinline__ uint4 ldg_policy(const uint4 *p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// CP (IM_TUNE_LT_CACHE): 0 plain loads; 1 the vertex records (n x 16 B, read
// at every step) are kept in L2 ahead of other lines (evict_last); 2 as 1, and
// the cut points (m x 16 B, mostly single-use) leave L2 first (evict_first).
// Launched with a.count <= kLT1MaxCount.  Four blocks per SM: the 63 registers
// the grouped scans want, with no spills (five blocks at 48 registers measured
// slower).
template <int CP>
__global__ void __launch_bounds__(kLT1Threads, 4) k_sample_lt1(SampleArgs a) {
    extern __shared__ uint32_t bloom[];          // [kBloomWords][kLT1Threads]
    // roots, sample ids and query indices of the warp's last two chunks
    __shared__ uint32_t ring_root[kLT1Warps][2 * kLT1Chunk];
    __shared__ uint32_t ring_s[kLT1Warps][2 * kLT1Chunk];
    __shared__ int32_t ring_q[kLT1Warps][2 * kLT1Chunk];
    // per warp: examined edges and algorithmic bytes of its finished walks
    __shared__ unsigned long long wsum[kLT1Warps][2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t *bl = bloom + threadIdx.x;
    int32_t *q = a.queues + ((int64_t)blockIdx.x * kLT1Threads + threadIdx.x) * a.qcap;
    if (lane == 0) {
        wsum[wib][0] = 0ull;
        wsum[wib][1] = 0ull;
    }
    // with one query in the launch, every walk has the same graph and key
    const bool one_query = a.nq == 1;
    const uint4 *vrec = one_query ? a.qv[0].lt_vrec : nullptr;
    const int32_t *srcs = one_query ? a.qv[0].in_src : nullptr;
    uint32_t k0 = one_query ? seed_lo(a.qv[0].seed) : 0u;
    uint32_t k1 = one_query ? seed_hi(a.qv[0].seed) : 0u;
    bool active = false, exhausted = false;
    bool pend = false;                           // waiting for an exact revisit check of u
    uint32_t j = 0, s = 0, cur = 0, u = 0;
    int32_t qi = 0, len = 0;
    unsigned long long sexam = 0;
    uint32_t sbytes = 0;
    // the warp's current chunk is [wend - kLT1Chunk, wend); [wnext, wend) is not
    // taken yet; the chunk's roots are in half `half` of the ring (warp-uniform)
    uint32_t wnext = 0, wend = 0;
    int half = 1;
    __syncwarp();
    for (;;) {
        // ---- lanes without a walk take the next samples of the warp's chunk
        const bool want = !active && !exhausted;
        const unsigned need = __ballot_sync(kFull, want);
        if (need) {
            const uint32_t nneed = (uint32_t)__popc(need);
            const uint32_t rank = (uint32_t)__popc(need & ((1u << lane) - 1u));
            const uint32_t avail = wend - wnext;
            uint32_t jw = wnext + rank;
            uint32_t cb = wend - kLT1Chunk;          // first index of jw's chunk
            int hw = half;                           // and the ring half holding it
            if (avail < nneed) {                     // the rest of this chunk, then a new one
                unsigned long long nb64 = 0;
                if (lane == 0) nb64 = atomicAdd(a.work, (unsigned long long)kLT1Chunk);
                const uint32_t nb = (uint32_t)__shfl_sync(kFull, nb64, 0);
                half ^= 1;
                const uint32_t jc = nb + (uint32_t)lane;
                if ((int64_t)jc < a.count) {         // lane draws the root of sample nb + lane
                    const int64_t jj = a.list ? a.list[jc] : (int64_t)jc;
                    const int qc = one_query ? 0 : find_query(a, jj);
                    const QueryView &V = a.qv[qc];
                    const uint32_t sc = V.first + (uint32_t)(jj - __ldg(a.qstart + qc));
                    ring_root[wib][half * kLT1Chunk + lane] = rrr_root(V.seed, sc, V.n);
                    ring_s[wib][half * kLT1Chunk + lane] = sc;
                    ring_q[wib][half * kLT1Chunk + lane] = qc;
                }
                __syncwarp();
                if (rank >= avail) {
                    jw = nb + (rank - avail);
                    cb = nb;
                    hw = half;
                }
                wnext = nb + (nneed - avail);
                wend = nb + kLT1Chunk;
            } else {
                wnext += nneed;
            }
            if (want) {
                if ((int64_t)jw < a.count) {
                    const int e = hw * (int)kLT1Chunk + (int)(jw - cb);
                    j = a.list ? (uint32_t)a.list[jw] : jw;
                    cur = ring_root[wib][e];
                    s = ring_s[wib][e];
                    qi = ring_q[wib][e];
                    if (!one_query) {
                        const QueryView &V = a.qv[qi];
                        vrec = V.lt_vrec;
                        srcs = V.in_src;
                        k0 = seed_lo(V.seed);
                        k1 = seed_hi(V.seed);
                    }
                    q[0] = (int32_t)cur;
#pragma unroll
                    for (int w = 0; w < kBloomWords; ++w) bl[w * kLT1Threads] = 0u;
                    bloom_add(bl, cur);
                    len = 1;
                    sexam = 0;
                    sbytes = 8u + 4u;                // set offset, root write
                    active = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(kFull, active)) break;

        // ---- one step of every active walk that is not waiting for its revisit check
        bool ending = false, accept = false;
        if (active && !pend) {
            const uint32_t x = philox4x32_10(make_uint4(s, cur, 0u, kStreamPick), k0, k1).x;
            // (the L2 policies are made where they are used: one instruction,
            // and no registers held across the loop)
            const uint4 vr =
                CP >= 1 ? ldg_policy(vrec + cur, l2_policy_evict_last()) : __ldg(vrec + cur);
            const uint32_t d = vr.y;
            int64_t e = -1;
            sbytes += 16u;                           // vertex record
            if (vr.w != 0u) {                        // equal in-weights: edge floor(x / weight)
                const uint32_t ei = x / vr.w;
                if (ei < d) {
                    e = ei;
                    u = (uint32_t)__ldg(srcs + vr.x + ei);
                    sbytes += 4u;                    // source of the pick
                }
            } else if (d > 0) {
                const QueryView &V = a.qv[qi];
                const uint4 *gp = V.lt_guide + vr.x + __umulhi(x, d);
                const uint4 gv = CP >= 2 ? ldg_policy(gp, l2_policy_evict_first()) : __ldg(gp);
                const unsigned long long cum = ((unsigned long long)gv.y << 32) | gv.x;
                sbytes += 16u;                       // cut point
                if ((unsigned long long)x < cum) {
                    e = gv.w;
                    u = gv.z;
                } else {
                    const unsigned long long *leaf = V.lt_leaf;
                    uint32_t lo = gv.w + 1, hi = d;  // first edge past the guide's with x < sum
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if ((unsigned long long)x < (__ldg(leaf + vr.x + mid) >> 31)) hi = mid;
                        else lo = mid + 1;
                        sbytes += 8u;                // search probe
                    }
                    if (lo < d) {
                        e = lo;
                        u = (uint32_t)(__ldg(leaf + vr.x + lo) & 0x7fffffffull);
                        sbytes += 8u;                // picked leaf
                    }
                }
            }
            sexam += e >= 0 ? (unsigned long long)(e + 1) : (unsigned long long)d;
            if (e < 0) ending = true;                // no in-edge picked: the walk stops
            else if (bloom_has(bl, u)) pend = true;  // maybe a revisit: check exactly
            else accept = true;
        }
        // ---- exact revisit checks of the flagged walks, once kLT1Flush of them wait
        // (or every active walk does); kLT1Group paths are scanned together
        const unsigned pm = __ballot_sync(kFull, pend);
        if (pm && (__popc(pm) >= kLT1Flush || pm == __ballot_sync(kFull, active))) {
            bool seen = false;
            unsigned rest = pm;
            do {
                int l[kLT1Group];
#pragma unroll
                for (int g = 0; g < kLT1Group; ++g) {   // lanes of the group; repeats when fewer
                    l[g] = rest ? __ffs(rest) - 1 : l[0];
                    rest &= rest - 1u;
                }
                int32_t ug[kLT1Group], lg[kLT1Group];
                int32_t lmax = 0;
#pragma unroll
                for (int g = 0; g < kLT1Group; ++g) {
                    ug[g] = __shfl_sync(kFull, (int32_t)u, l[g]);
                    lg[g] = __shfl_sync(kFull, len, l[g]);
                    lmax = max(lmax, lg[g]);
                }
                bool f[kLT1Group];
#pragma unroll
                for (int g = 0; g < kLT1Group; ++g) f[g] = false;
                for (int32_t i = lane; i < lmax; i += 32) {
                    int32_t v[kLT1Group];
#pragma unroll
                    for (int g = 0; g < kLT1Group; ++g)      // lane l[g]'s path entry i
                        v[g] = i < lg[g] ? __ldcg(q + (int64_t)(l[g] - lane) * a.qcap + i) : -1;
#pragma unroll
                    for (int g = 0; g < kLT1Group; ++g) f[g] |= v[g] == ug[g];
                }
#pragma unroll
                for (int g = 0; g < kLT1Group; ++g) {
                    const bool any = __any_sync(kFull, f[g]);
                    if (lane == l[g]) seen = any;
                }
            } while (rest);
            if (pend) {
                if (seen) ending = true;             // a revisit: the walk stops
                else accept = true;
                pend = false;
            }
        }
        bool ovf = false;
        if (accept) {
            if (len < a.qcap) {
                q[len] = (int32_t)u;
                bloom_add(bl, u);
                ++len;
                sbytes += 4u;                        // member write
                cur = u;
            } else {
                ovf = true;                          // longer than the queue: second pass
                ending = true;
                a.sizes[j] = -1;
                a.stage_off[j] = 0;
                a.ovf_list[atomicAdd(a.ovf_count, 1ull)] = (int64_t)j;
            }
        }
        // ---- finished walks go to the stage, kLT1Group paths copied together
        const bool emit = ending && !ovf;
        unsigned em = __ballot_sync(kFull, emit);
        if (em) {
            const int32_t my = emit ? len : 0;
            const int32_t incl = warp_incl_scan<int32_t>(my, lane);
            const int32_t tot = __shfl_sync(kFull, incl, 31);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.stage_cursor, (unsigned long long)tot);
            base = __shfl_sync(kFull, base, 0);
            const bool fits = (int64_t)base + tot <= a.stage_cap;
            if (emit) {
                if (fits) {
                    a.stage_off[j] = (int64_t)base + incl - my;
                    a.sizes[j] = len;
                    atomicAdd(&wsum[wib][0], sexam);
                    atomicAdd(&wsum[wib][1], (unsigned long long)sbytes);
                } else {
                    raise_status(a.status, kDevStageOverflow);
                    a.sizes[j] = 0;
                    a.stage_off[j] = 0;
                }
            }
            if (fits) {
                __syncwarp();
                do {
                    int l[kLT1Group];
#pragma unroll
                    for (int g = 0; g < kLT1Group; ++g) {
                        l[g] = em ? __ffs(em) - 1 : l[0];
                        em &= em - 1u;
                    }
                    int32_t lg[kLT1Group], og[kLT1Group];
                    int32_t lmax = 0;
#pragma unroll
                    for (int g = 0; g < kLT1Group; ++g) {
                        lg[g] = __shfl_sync(kFull, len, l[g]);
                        og[g] = __shfl_sync(kFull, incl - my, l[g]);   // offset from base
                        lmax = max(lmax, lg[g]);
                    }
                    for (int32_t i = lane; i < lmax; i += 32) {
                        int32_t v[kLT1Group];
#pragma unroll
                        for (int g = 0; g < kLT1Group; ++g)
                            v[g] = i < lg[g] ? __ldcg(q + (int64_t)(l[g] - lane) * a.qcap + i) : 0;
#pragma unroll
                        for (int g = 0; g < kLT1Group; ++g)
                            if (i < lg[g]) a.stage[(int64_t)base + og[g] + i] = v[g];
                    }
                } while (em);
            }
        }
        if (ending) active = false;
        __syncwarp();
    }
    if (lane == 0) {
        if (wsum[wib][0]) atomicAdd(a.examined, wsum[wib][0]);
        if (wsum[wib][1]) atomicAdd(a.alg_bytes, wsum[wib][1]);
    }
}

// LT search index.  vrec[v] = {eb, d, tree offset | L << 28, u} with L the
// number of upper tree levels (tree offsets stay below 2^28 since m < 2^31) and
// u the common weight of v's in-edges when they all carry the same nonzero
// weight (0 otherwise).  For such a vertex the pick needs no table: the running
// sum of edge i is (i + 1) u, so a draw x picks edge floor(x / u) when that is
// below d and nothing otherwise.
// For vertex v with in-edges [eb, eb + d):
//   leaf[e] = (sum of w over v's in-edges up to and including e) << 31 | src(e)
// (the running sum is at most 2^32 for valid LT weights -- 33 bits -- and
// source ids stay below 2^31, so the pair packs into 64 bits), and for
// d > 32 the upper levels l = L .. 1 of a fanout-32 tree, stored top-down at
// tree[tree_off(v) ..]: level l has ceil(d / 32^l) entries, entry i being the
// running sum at the last leaf of its 32^l-leaf block.
__device__ __forceinline__ int64_t lt_tree_size(int64_t d) {
    int64_t total = 0;
    while (d > 32) {
        d = (d + 31) >> 5;
        total += d;
    }
    return total;
}

// In-degree above which one block, not one warp, builds a vertex's running
// sums (a warp on R-MAT's largest in-list, ~7 x 10^4 edges, is the whole build's
// critical path).  At most m / (kLtBlockDeg + 1) vertices qualify.
constexpr int64_t kLtBlockDeg = 1024;

// Tree size of every vertex; lists the vertices of k_lt_index_block in big
// (in no particular order; nbig counts them).
__global__ void k_lt_tree_sizes(const int64_t *in_off, int64_t n, int32_t *sizes, int32_t *big,
                                int *nbig) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = in_off[v + 1] - in_off[v];
        sizes[v] = (int32_t)lt_tree_size(d);
        if (d > kLtBlockDeg) big[atomicAdd(nbig, 1)] = (int32_t)v;
    }
}

// Vertices with at most 32 in-edges (no upper tree levels): one thread each.
// The three index kernels write the vertex records and the flags always, and
// the running sums (leaf) and tree levels only when leaf is non-null.
__global__ void k_lt_index_small(const int64_t *in_off, const int32_t *in_src, const uint32_t *w,
                                 const int64_t *tree_off, unsigned long long *leaf, uint4 *vrec,
                                 int64_t n, int *invalid) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = in_off[v], e = in_off[v + 1], d = e - b;
        if (d > 32) continue;   // k_lt_index
        unsigned long long c = 0;
        const uint32_t w0 = d > 0 ? w[b] : 0u;
        bool same = true;
        for (int64_t i = b; i < e; ++i) {
            const uint32_t wi = w[i];
            same &= wi == w0;
            c += (unsigned long long)wi;
            if (leaf) leaf[i] = (c << 31) | (unsigned long long)(uint32_t)in_src[i];
        }
        if (c > (1ull << 32)) atomicExch(invalid, 1);
        if (d > 0 && !(same && w0 != 0u)) invalid[2] = 1;   // the cut points are needed
        vrec[v] = make_uint4((uint32_t)b, (uint32_t)d, (uint32_t)tree_off[v], same ? w0 : 0u);
    }
}

// Vertices with more than 32 in-edges: one warp each, running sums by warp
// scans, then the upper levels of the fanout-32 tree.
__global__ void k_lt_index(const int64_t *in_off, const int32_t *in_src, const uint32_t *w,
                           const int64_t *tree_off, unsigned long long *leaf,
                           unsigned long long *tree, uint4 *vrec, int64_t n, int *invalid) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
         v += nw) {
        const int64_t b = in_off[v], e = in_off[v + 1], d = e - b;
        if (d <= 32 || d > kLtBlockDeg) continue;   // k_lt_index_small, k_lt_index_block
        unsigned long long carry = 0;
        const uint32_t w0 = w[b];
        bool same = true;
        for (int64_t base = b; base < e; base += 32) {
            const int64_t i = base + lane;
            const uint32_t wi = i < e ? w[i] : w0;
            same &= wi == w0;
            const unsigned long long x = i < e ? (unsigned long long)wi : 0ull;
            const unsigned long long incl = warp_incl_scan<unsigned long long>(x, lane);
            if (leaf && i < e)
                leaf[i] = ((carry + incl) << 31) | (unsigned long long)(uint32_t)in_src[i];
            carry += __shfl_sync(kFull, incl, 31);
        }
        same = __all_sync(kFull, same);
        if (lane == 0 && carry > (1ull << 32)) atomicExch(invalid, 1);
        if (lane == 0 && !(same && w0 != 0u)) invalid[2] = 1;
        int L = 0;
        for (int64_t t = d; t > 32; t = (t + 31) >> 5) ++L;
        if (lane == 0)
            vrec[v] = make_uint4((uint32_t)b, (uint32_t)d,
                                 (uint32_t)tree_off[v] | ((uint32_t)L << 28), same ? w0 : 0u);
        __syncwarp();
        if (!leaf) continue;
        // upper levels, top-down
        unsigned long long *lvl = tree + tree_off[v];
        for (int l = L; l >= 1; --l) {
            const int64_t sz = (d + (1ll << (5 * l)) - 1) >> (5 * l);
            for (int64_t i = lane; i < sz; i += 32) {
                const int64_t last = min((i + 1) << (5 * l), d) - 1;
                lvl[i] = leaf[b + last] >> 31;
            }
            lvl += sz;
        }
    }
}

// Vertices with more than kLtBlockDeg in-edges: one block of 256 threads each,
// 2048 edges per pass (8 consecutive ones per thread: sequential sums, then a
// block scan of the thread totals), then the upper tree levels as above.
__global__ void __launch_bounds__(256) k_lt_index_block(
    const int64_t *in_off, const int32_t *in_src, const uint32_t *w, const int64_t *tree_off,
    const int32_t *big, int nbig, unsigned long long *leaf, unsigned long long *tree, uint4 *vrec,
    int *invalid) {
    __shared__ unsigned long long wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int j = blockIdx.x; j < nbig; j += gridDim.x) {
        const int64_t v = big[j];
        const int64_t b = in_off[v], e = in_off[v + 1], d = e - b;
        const uint32_t w0 = w[b];
        bool same = true;
        unsigned long long carry = 0;
        for (int64_t base = b; base < e; base += 2048) {
            const int64_t i0 = base + (int64_t)tid * 8;
            unsigned long long s[8], run = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t wi = i0 + q < e ? w[i0 + q] : w0;
                same &= wi == w0;
                run += i0 + q < e ? (unsigned long long)wi : 0ull;
                s[q] = run;
            }
            const unsigned long long incl = warp_incl_scan<unsigned long long>(run, lane);
            if (lane == 31) wsum[wid] = incl;
            __syncthreads();
            unsigned long long before = 0, tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const unsigned long long x = wsum[q];
                before += q < wid ? x : 0ull;
                tot += x;
            }
            const unsigned long long off = carry + before + (incl - run);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (leaf && i0 + q < e)
                    leaf[i0 + q] = ((off + s[q]) << 31) | (unsigned long long)(uint32_t)in_src[i0 + q];
            carry += tot;
            __syncthreads();   // wsum is rewritten by the next pass
        }
        same = __syncthreads_and(same) != 0;
        if (tid == 0 && carry > (1ull << 32)) atomicExch(invalid, 1);
        if (tid == 0 && !(same && w0 != 0u)) invalid[2] = 1;
        int L = 0;
        for (int64_t t = d; t > 32; t = (t + 31) >> 5) ++L;
        if (tid == 0)
            vrec[v] = make_uint4((uint32_t)b, (uint32_t)d,
                                 (uint32_t)tree_off[v] | ((uint32_t)L << 28), same ? w0 : 0u);
        __syncthreads();   // every leaf of v written by the block is visible to it
        if (!leaf) continue;   // (block-uniform)
        unsigned long long *lvl = tree + tree_off[v];
        for (int l = L; l >= 1; --l) {
            const int64_t sz = (d + (1ll << (5 * l)) - 1) >> (5 * l);
            for (int64_t i = tid; i < sz; i += blockDim.x) {
                const int64_t last = min((i + 1) << (5 * l), d) - 1;
                lvl[i] = leaf[b + last] >> 31;
            }
            lvl += sz;
        }
    }
}

// Cut points of the inverse-CDF pick, exact for any weights.  A draw x of
// vertex v (in-edges [eb, eb + d)) falls in bucket b = floor(x d / 2^32); the
// smallest draw of bucket b is lo_b = ceil(b 2^32 / d).  guide[eb + b]
// describes the first in-edge e whose running sum exceeds lo_b, or the last
// in-edge when none does: {running sum low word, high word, source, e}.
// Every edge before e has a running sum <= lo_b <= x, so x picks e exactly
// when x < running sum(e); otherwise the pick lies after e (or there is none).
__global__ void k_lt_guide(const int64_t *in_off, const unsigned long long *leaf,
                           const uint4 *vrec, int64_t n, int64_t m, uint4 *guide) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n - 1;                  // vertex owning position t
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (in_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        if (vrec[lo].w != 0u) continue;              // equal weights: no table needed
        const int64_t eb = in_off[lo], d = in_off[lo + 1] - eb, b = t - eb;
        const unsigned long long lob =
            (((unsigned long long)b << 32) + (unsigned long long)d - 1ull) / (unsigned long long)d;
        int64_t l2 = 0, h2 = d;                      // first e with lo_b < running sum(e)
        while (l2 < h2) {
            const int64_t mid = (l2 + h2) >> 1;
            if (lob < (leaf[eb + mid] >> 31)) h2 = mid;
            else l2 = mid + 1;
        }
        const int64_t e = l2 < d ? l2 : d - 1;
        const unsigned long long r = leaf[eb + e];
        const unsigned long long cum = r >> 31;
        guide[t] = make_uint4((uint32_t)cum, (uint32_t)(cum >> 32), (uint32_t)(r & 0x7fffffffull),
                              (uint32_t)e);
    }
}

// ---------------------------------------------------------------------------
// segmented sort: every segment [seg_off[i], seg_off[i+1]) ascending
// ---------------------------------------------------------------------------
template <typename Key>
__device__ __forceinline__ Key key_max();
template <>
__device__ __forceinline__ int32_t key_max<int32_t>() { return 0x7fffffff; }

template <typename Key>
__device__ __forceinline__ Key warp_bitonic32(Key v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const Key o = __shfl_xor_sync(kFull, v, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    return v;
}

// Bitonic sort of 32 E keys held by a warp in registers, element i = r 32 +
// lane in v[r] (the layout of a coalesced load).  Partners i ^ j with j < 32
// sit in other lanes (shuffle), with j >= 32 in the same lane (registers).
template <typename Key, int E>
__device__ __forceinline__ void warp_bitonic_regs(Key (&v)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j >> 5;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if (r & jr) continue;
                    const int r2 = r | jr;
                    const bool asc = (((r << 5) | lane) & k) == 0;
                    const Key x = v[r], y = v[r2];
                    const bool sw = asc ? (y < x) : (x < y);
                    v[r] = sw ? y : x;
                    v[r2] = sw ? x : y;
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const bool asc = (((r << 5) | lane) & k) == 0;
                    const Key x = v[r];
                    const Key y = __shfl_xor_sync(kFull, x, j);
                    const Key lo = y < x ? y : x, hi = y < x ? x : y;
                    v[r] = (lower == asc) ? lo : hi;
                }
            }
        }
    }
}

template <typename Key, int E>
__device__ __forceinline__ void warp_sort_copy(Key *out, const Key *src, int64_t len, int lane) {
    Key v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int64_t t = (int64_t)r * 32 + lane;
        v[r] = t < len ? src[t] : key_max<Key>();
    }
    warp_bitonic_regs<Key, E>(v, lane);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int64_t t = (int64_t)r * 32 + lane;
        if (t < len) out[t] = v[r];
    }
}

// bitonic network over buf[0..P) (P a power of two) by `nthreads` threads
template <typename Key>
__device__ __forceinline__ void bitonic_smem(Key *buf, int P, int tid, int nthreads,
                                             bool block_level) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += nthreads) {
                const int l = i ^ j;
                if (l > i) {
                    const Key x = buf[i], y = buf[l];
                    const bool asc = (i & k) == 0;
                    if ((x > y) == asc) {
                        buf[i] = y;
                        buf[l] = x;
                    }
                }
            }
            if (block_level) __syncthreads();
            else __syncwarp();
        }
    }
}

// Bitonic sort of N keys held by one thread (N a power of two, fully unrolled).
template <typename Key, int N>
__device__ __forceinline__ void thread_bitonic(Key (&v)[N]) {
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool asc = (i & k) == 0;
                    const Key x = v[i], y = v[l];
                    const bool sw = asc ? (y < x) : (x < y);
                    v[i] = sw ? y : x;
                    v[l] = sw ? x : y;
                }
            }
        }
    }
}

// One segment sorted by the whole warp (len > kLaneSort): copied from the
// stage and sorted in registers, or in the warp's shared buffer, or listed in
// `big` for k_sort_block / k_sort_giant.
template <typename Key>
__device__ __forceinline__ void warp_sort_segment(Key *out, const Key *src, int64_t len,
                                                  bool from_stage, int64_t i, Key *buf,
                                                  int64_t *big, unsigned long long *nbig,
                                                  int lane) {
    constexpr int kCapW = kWarpSortBytes / (int)sizeof(Key);
    if (len <= 32) {
        Key v = lane < len ? src[lane] : key_max<Key>();
        v = warp_bitonic32<Key>(v, lane);
        if (lane < len) out[lane] = v;
    } else if (len <= 64) {
        warp_sort_copy<Key, 2>(out, src, len, lane);
    } else if (len <= 128) {
        warp_sort_copy<Key, 4>(out, src, len, lane);
    } else if (len <= 256) {
        warp_sort_copy<Key, 8>(out, src, len, lane);
    } else if (len <= 512 && sizeof(Key) == 4) {
        warp_sort_copy<Key, 16>(out, src, len, lane);
    } else if (len <= kCapW) {
        int P = 64;
        while (P < len) P <<= 1;
        for (int t = lane; t < P; t += 32) buf[t] = t < len ? src[t] : key_max<Key>();
        __syncwarp();
        bitonic_smem<Key>(buf, P, lane, 32, false);
        for (int t = lane; t < len; t += 32) out[t] = buf[t];
    } else {
        if (from_stage)
            for (int64_t t = lane; t < len; t += 32) out[t] = src[t];
        if (lane == 0) big[atomicAdd(nbig, 1ull)] = i;
    }
    __syncwarp();
}

// Copies stage segments into place (when `stage` is non-null) and sorts the
// short ones.  A warp takes 32 consecutive segments at once (their offsets in
// one coalesced load each): segments of at most kLaneSort keys -- most RRR
// sets -- are sorted by their own lane in registers; the longer ones are
// listed in `mid` for k_sort_mid, one warp each.
constexpr int kLaneSort = 16;

template <typename Key>
__global__ void __launch_bounds__(256) k_sort_small(Key *dst, const int64_t *seg_off, int64_t nseg,
                                                    const Key *stage, const int64_t *stage_off,
                                                    int64_t *mid, unsigned long long *nmid,
                                                    bool inline_long, int64_t *big,
                                                    unsigned long long *nbig) {
    constexpr int kCapW = kWarpSortBytes / (int)sizeof(Key);
    __shared__ Key sbuf[8][kCapW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * 8;
    for (int64_t i0 = ((int64_t)blockIdx.x * 8 + wib) * 32; i0 < nseg; i0 += nw * 32) {
        const int64_t i = i0 + lane;
        int64_t o = 0, len = 0;
        const Key *src = nullptr;
        if (i < nseg) {
            o = seg_off[i];
            len = seg_off[i + 1] - o;
            src = stage ? stage + stage_off[i] : dst + o;
        }
        Key *out = dst + o;
        if (len == 1) {
            if (stage) out[0] = src[0];
        } else if (len > 1 && len <= kLaneSort) {
            Key v[kLaneSort];
#pragma unroll
            for (int r = 0; r < kLaneSort; ++r) v[r] = r < len ? src[r] : key_max<Key>();
            thread_bitonic<Key, kLaneSort>(v);
#pragma unroll
            for (int r = 0; r < kLaneSort; ++r)
                if (r < len) out[r] = v[r];
        }
        unsigned longer = __ballot_sync(kFull, len > kLaneSort);
        if (longer && inline_long) {   // many segments per warp: the warp sorts them itself
            while (longer) {
                const int l = __ffs(longer) - 1;
                longer &= longer - 1;
                const int64_t ol = __shfl_sync(kFull, o, l);
                const int64_t ll = __shfl_sync(kFull, len, l);
                const Key *sl = (const Key *)__shfl_sync(kFull, (unsigned long long)src, l);
                warp_sort_segment<Key>(dst + ol, sl, ll, stage != nullptr, i0 + l, sbuf[wib], big,
                                       nbig, lane);
            }
        } else if (longer) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(nmid, (unsigned long long)__popc(longer));
            base = __shfl_sync(kFull, base, 0);
            if (len > kLaneSort) mid[base + __popc(longer & ((1u << lane) - 1u))] = i;
        }
    }
}

// One warp per listed segment longer than kLaneSort keys (grid-stride over
// the list): sorted in registers or in the warp's shared buffer; segments
// longer than that buffer are copied into place and listed in `big`.
template <typename Key>
__global__ void __launch_bounds__(256) k_sort_mid(Key *dst, const int64_t *seg_off,
                                                  const Key *stage, const int64_t *stage_off,
                                                  const int64_t *mid,
                                                  const unsigned long long *nmid, int64_t *big,
                                                  unsigned long long *nbig) {
    constexpr int kCapW = kWarpSortBytes / (int)sizeof(Key);
    __shared__ Key sbuf[8][kCapW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * 8;
    const int64_t cnt = (int64_t)*nmid;
    for (int64_t x = (int64_t)blockIdx.x * 8 + wib; x < cnt; x += nw) {
        const int64_t i = mid[x];
        const int64_t o = seg_off[i];
        const int64_t len = seg_off[i + 1] - o;
        warp_sort_segment<Key>(dst + o, stage ? stage + stage_off[i] : dst + o, len,
                               stage != nullptr, i, sbuf[wib], big, nbig, lane);
    }
}

// One block per listed segment longer than a warp's buffer and at most kCap
// keys: bitonic sort in shared memory.
template <typename Key, int kCap>
__global__ void __launch_bounds__(1024) k_sort_block(Key *dst, const int64_t *seg_off,
                                                     const int64_t *big,
                                                     const unsigned long long *nbig,
                                                     int64_t *giant,
                                                     unsigned long long *ngiant) {
    extern __shared__ unsigned char sraw[];
    Key *buf = reinterpret_cast<Key *>(sraw);
    const int64_t nb = (int64_t)*nbig;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t i = big[b];
        const int64_t o = seg_off[i];
        const int64_t len = seg_off[i + 1] - o;
        if (len > kCap) {
            if (threadIdx.x == 0 && giant) giant[atomicAdd(ngiant, 1ull)] = i;
            continue;
        }
        int P = 64;
        while (P < len) P <<= 1;
        for (int t = threadIdx.x; t < P; t += blockDim.x)
            buf[t] = t < len ? dst[o + t] : key_max<Key>();
        __syncthreads();
        bitonic_smem<Key>(buf, P, threadIdx.x, blockDim.x, true);
        for (int t = threadIdx.x; t < len; t += blockDim.x) dst[o + t] = buf[t];
        __syncthreads();
    }
}

// Segments longer than kBlockSortCap of distinct vertex ids: mark them in an
// n-bit bitmap (one per block) and read the bitmap back in order.
__global__ void __launch_bounds__(1024) k_sort_giant(int32_t *dst, const int64_t *seg_off,
                                                     const int64_t *giant,
                                                     const unsigned long long *ngiant,
                                                     uint32_t *bitmaps, int64_t words) {
    __shared__ int64_t sh[33];
    uint32_t *bm = bitmaps + (size_t)blockIdx.x * (size_t)words;
    const int64_t ng = (int64_t)*ngiant;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b = blockIdx.x; b < ng; b += gridDim.x) {
        const int64_t i = giant[b];
        const int64_t o = seg_off[i];
        const int64_t len = seg_off[i + 1] - o;
        for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
            const uint32_t u = (uint32_t)dst[o + t];
            atomicOr(&bm[u >> 5], 1u << (u & 31));
        }
        __syncthreads();
        const int64_t per = (words + blockDim.x - 1) / blockDim.x;
        const int64_t w0 = (int64_t)threadIdx.x * per;
        const int64_t w1 = min(words, w0 + per);
        int64_t cnt = 0;
        for (int64_t x = w0; x < w1; ++x) cnt += __popc(bm[x]);
        // block exclusive scan of cnt
        int64_t incl = warp_incl_scan<int64_t>(cnt, lane);
        if (lane == 31) sh[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
            int64_t vi = warp_incl_scan<int64_t>(v, lane);
            if (lane < (int)(blockDim.x >> 5)) sh[lane] = vi - v;
        }
        __syncthreads();
        int64_t at = o + sh[warp] + incl - cnt;
        __syncthreads();
        for (int64_t x = w0; x < w1; ++x) {
            uint32_t bits = bm[x];
            while (bits) {
                const int bpos = __ffs(bits) - 1;
                bits &= bits - 1;
                dst[at++] = (int32_t)(x * 32 + bpos);
            }
        }
        __syncthreads();
        for (int64_t x = w0; x < w1; ++x) bm[x] = 0;
        __syncthreads();
    }
}

int blocks_for(const void *kernel, int threads, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * num_sms();
}

}  // namespace

template <typename Key>
im_status segmented_sort_impl(Key *keys, const int64_t *seg_off, int64_t nseg, const Key *stage,
                              const int64_t *stage_off, void *tmp, size_t tmp_bytes,
                              int64_t *ngiant_host, cudaStream_t st, const char *warp_name,
                              const char *block_name) {
    // tmp layout: [2 counters][big list nseg][giant list nseg]; the giant
    // list's space and second counter first hold the list for k_sort_mid
    if (tmp_bytes < (size_t)(2 + 2 * nseg) * 8) return IM_ERR_INVALID_ARG;
    unsigned long long *ctr = (unsigned long long *)tmp;
    int64_t *big = (int64_t *)tmp + 2;
    int64_t *giant = big + nseg;
    IM_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long), st));
    if (nseg == 0) return IM_OK;
    const int gs = blocks_for((const void *)k_sort_small<Key>, 256, 0);
    const int gm = blocks_for((const void *)k_sort_mid<Key>, 256, 0);
    // with at least four groups of 32 segments per warp the longer segments
    // spread over the warps anyway: each warp sorts its own; with fewer, they
    // are listed and k_sort_mid gives each its own warp
    const bool inline_long = nseg >= (int64_t)gs * 8 * 32 * 4;
    {
        KernelTimer kt(st, warp_name);
        k_sort_small<Key><<<gs, 256, 0, st>>>(keys, seg_off, nseg, stage, stage_off, giant,
                                               ctr + 1, inline_long, big, ctr);
        if (!inline_long)
            k_sort_mid<Key><<<gm, 256, 0, st>>>(keys, seg_off, stage, stage_off, giant, ctr + 1,
                                                 big, ctr);
    }
    IM_CUDA(cudaGetLastError());
    IM_CUDA(cudaMemsetAsync(ctr + 1, 0, sizeof(unsigned long long), st));
    constexpr int kCap = kBlockSortCap * 4 / (int)sizeof(Key);
    const size_t smem = (size_t)kCap * sizeof(Key);
    IM_TRY(raise_dyn_smem((const void *)k_sort_block<Key, kCap>, smem));
    {
        KernelTimer kt(st, block_name);
        k_sort_block<Key, kCap><<<num_sms(), 1024, smem, st>>>(keys, seg_off, big, ctr,
                                                              giant, ctr + 1);
    }
    IM_CUDA(cudaGetLastError());
    if (ngiant_host) {
        unsigned long long ng = 0;
        IM_CUDA(cudaMemcpyAsync(&ng, ctr + 1, sizeof(ng), cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        *ngiant_host = (int64_t)ng;
    }
    return IM_OK;
}

static std::mutex g_lt_index_mu;   // graphs are shared by serving workers

im_status build_lt_index(im_graph *g, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_lt_index_mu);
    if (g->lt_vrec) return IM_OK;   // set only once the whole index is built
    const int64_t n = g->n, m = g->m;
    // stream-ordered temporaries, freed on every exit
    struct Temps {
        cudaStream_t st;
        int32_t *sizes = nullptr, *big = nullptr;
        int64_t *toff = nullptr;
        int *flags = nullptr;   // [0] weights of some vertex sum above 2^32, [1] listed
                                // vertices, [2] some vertex needs the cut points
        ~Temps() {
            for (void *p : {(void *)sizes, (void *)big, (void *)toff, (void *)flags})
                if (p) cudaFreeAsync(p, st);
        }
    } t{st};
    // the index itself: handed to g once complete, freed on any failure
    struct Index {
        unsigned long long *leaf = nullptr, *tree = nullptr;
        uint4 *vrec = nullptr, *guide = nullptr;
        ~Index() {
            if (leaf || tree || vrec || guide) {
                cudaDeviceSynchronize();
                for (void *p : {(void *)leaf, (void *)tree, (void *)vrec, (void *)guide})
                    cudaFree(p);
            }
        }
    } x;
    const int64_t big_cap = m / (kLtBlockDeg + 1) + 1;
    IM_CUDA(cudaMallocAsync((void **)&t.sizes, (size_t)n * 4, st));
    IM_CUDA(cudaMallocAsync((void **)&t.big, (size_t)big_cap * 4, st));
    IM_CUDA(cudaMallocAsync((void **)&t.toff, (size_t)(n + 1) * 8 + scan_tmp_bytes(n) + 256, st));
    IM_CUDA(cudaMallocAsync((void **)&t.flags, 3 * sizeof(int), st));
    IM_CUDA(cudaMemsetAsync(t.flags, 0, 3 * sizeof(int), st));
    {
        KernelTimer kt(st, "lt_index");
        k_lt_tree_sizes<<<num_sms() * 4, 256, 0, st>>>(g->in_off, n, t.sizes, t.big, t.flags + 1);
    }
    void *scan_tmp = (char *)t.toff + (((size_t)(n + 1) * 8 + 255) & ~(size_t)255);
    IM_TRY(exclusive_scan_i32_to_i64(t.sizes, t.toff, n, nullptr, scan_tmp, scan_tmp_bytes(n), st));
    int64_t tree_total = 0;
    int nbig = 0;
    IM_CUDA(cudaMemcpyAsync(&tree_total, t.toff + n, 8, cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaMemcpyAsync(&nbig, t.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if (nbig < 0 || nbig > big_cap) {
        set_error("LT index: vertex list out of range");
        return IM_ERR_CUDA;
    }
    IM_CUDA(cudaMalloc(&x.vrec, (size_t)n * sizeof(uint4)));
    // vertex records and flags; running sums and tree when leaf is set
    auto index_pass = [&]() -> im_status {
        KernelTimer kt(st, "lt_index");
        k_lt_index_small<<<num_sms() * 8, 256, 0, st>>>(g->in_off, g->in_src, g->w, t.toff,
                                                        x.leaf, x.vrec, n, t.flags);
        k_lt_index<<<num_sms() * 8, 256, 0, st>>>(g->in_off, g->in_src, g->w, t.toff, x.leaf,
                                                  x.tree, x.vrec, n, t.flags);
        if (nbig > 0)
            k_lt_index_block<<<std::min(nbig, num_sms() * 8), 256, 0, st>>>(
                g->in_off, g->in_src, g->w, t.toff, t.big, nbig, x.leaf, x.tree, x.vrec,
                t.flags);
        IM_CUDA(cudaGetLastError());
        return IM_OK;
    };
    // first the vertex records alone: when every vertex's in-edges weigh the
    // same (1/in-degree weights, for one) the walks pick by division and need
    // neither running sums, tree nor cut points
    IM_TRY(index_pass());
    int hflags[3] = {0, 0, 0};
    IM_CUDA(cudaMemcpyAsync(hflags, t.flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    if (hflags[2] && m > 0) {
        // some vertex's in-edges weigh differently (or all zero): the full
        // index (the records are rewritten with the same values), then the cut
        // points, which serve only such vertices
        IM_CUDA(cudaMalloc(&x.leaf, (size_t)m * 8));
        IM_CUDA(cudaMalloc(&x.tree, (size_t)std::max<int64_t>(tree_total, 1) * 8));
        IM_TRY(index_pass());
        IM_CUDA(cudaMalloc(&x.guide, (size_t)m * sizeof(uint4)));
        {
            KernelTimer kt(st, "lt_index");
            k_lt_guide<<<num_sms() * 8, 256, 0, st>>>(g->in_off, x.leaf, x.vrec, n, m, x.guide);
        }
        IM_CUDA(cudaGetLastError());
        IM_CUDA(cudaStreamSynchronize(st));
    }
    g->lt_valid = hflags[0] ? 0 : 1;
    g->lt_tree = x.tree;
    g->lt_vrec = x.vrec;
    g->lt_guide = x.guide;
    g->lt_leaf = x.leaf;
    x.leaf = x.tree = nullptr;
    x.vrec = x.guide = nullptr;
    return IM_OK;
}

QueryView query_view(const im_graph *g, uint64_t seed, uint64_t first) {
    QueryView v;
    v.in_off = g->in_off;
    v.in_src = g->in_src;
    v.w = g->w;
    v.lt_vrec = g->lt_vrec;
    v.lt_leaf = g->lt_leaf;
    v.lt_tree = g->lt_tree;
    v.lt_guide = g->lt_guide;
    v.seed = seed;
    v.n = (uint32_t)g->n;
    v.first = (uint32_t)first;
    return v;
}

// ---------------------------------------------------------------------------
// One sampling launch over a table of queries (see SamplingJob).
// ---------------------------------------------------------------------------
im_status run_sampling(const SamplingJob &job, const std::function<im_status(size_t, void **)> &alloc,
                       cudaStream_t st, SamplingResult *res) {
    const im_model model = job.model;
    const int32_t nq = (int32_t)job.views.size();
    std::vector<int64_t> qstart(nq + 1, 0);
    for (int32_t q = 0; q < nq; ++q) qstart[q + 1] = qstart[q] + job.counts[q];
    const int64_t cnt = qstart[nq];
    const int64_t n = job.n_max;
    const bool smem_vis = model == IM_IC && n <= kSmemVisBits;
    const int64_t vis_words = (n + 31) / 32;

    // launch shape: persistent, occupancy-sized
    int G = model == IM_LT ? (int)tune_value(IM_TUNE_LT_GROUP) : 32;
    if (G == 1 && cnt > kLT1MaxCount) G = 32;        // chunk bounds of k_sample_lt1 are 32-bit
    const int lt_cache = (int)tune_value(IM_TUNE_LT_CACHE);
    const bool lt1 = model == IM_LT && G == 1;      // one walk per thread
    const void *kern = model == IM_LT
                           ? (G == 1    ? (lt_cache == 0   ? (const void *)k_sample_lt1<0>
                                            : lt_cache == 1 ? (const void *)k_sample_lt1<1>
                                                            : (const void *)k_sample_lt1<2>)
                              : G == 8  ? (const void *)k_sample_lt<8>
                              : G == 16 ? (const void *)k_sample_lt<16>
                                        : (const void *)k_sample_lt<32>)
                       : smem_vis ? (const void *)k_sample_ic<true>
                                  : (const void *)k_sample_ic<false>;
    const int threads = lt1 ? kLT1Threads : kSampleThreads;
    const size_t dyn_smem = smem_vis ? (size_t)kWarps * vis_words * 4
                            : lt1    ? (size_t)kBloomWords * kLT1Threads * 4
                                     : 0;
    if (dyn_smem > 48 * 1024)
        IM_TRY(raise_dyn_smem(kern, dyn_smem));
    int blocks = blocks_for(kern, threads, dyn_smem);
    // global visited bitmaps are n bits per warp: keep them within ~2 GB
    if (model == IM_IC && !smem_vis) {
        int64_t cap_blocks = std::max<int64_t>(
            num_sms(), (int64_t)(2ll << 30) / ((int64_t)kWarps * vis_words * 4));
        blocks = (int)std::min<int64_t>(blocks, cap_blocks);
    }
    const int64_t warps = (int64_t)blocks * (threads / 32);
    const int64_t slots = warps * (32 / G);           // one queue per walk in flight
    const int64_t qcap = std::min<int64_t>(
        n, lt1 ? kQueueCapLT1 : model == IM_LT ? kQueueCapLT : kQueueCapIC);

    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    const size_t o_ctr = take(8 * sizeof(unsigned long long));
    const size_t o_views = take((size_t)nq * sizeof(QueryView));
    const size_t o_qstart = take((size_t)(nq + 1) * 8);
    const size_t o_soff = take((size_t)cnt * 8);
    const size_t o_sizes = take((size_t)cnt * 4);
    const size_t o_ovf = take((size_t)cnt * 8);
    const size_t o_scan = take(scan_tmp_bytes(cnt));
    const size_t o_sort = take((size_t)(2 + 2 * cnt) * 8);
    const size_t o_q = take((size_t)slots * qcap * 4);
    const size_t o_vis = take(model == IM_IC && !smem_vis ? (size_t)warps * vis_words * 4 : 0);
    void *base = nullptr;
    im_status rs = alloc(off, &base);
    if (rs != IM_OK) return rs;
    char *B = (char *)base;
    unsigned long long *ctr = (unsigned long long *)(B + o_ctr);
    // ctr: 0 work, 1 stage cursor, 2 examined, 3 overflow count, 4 status (int),
    //      5 algorithmic bytes
    IM_CUDA(cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned long long), st));
    IM_CUDA(cudaMemcpyAsync(B + o_views, job.views.data(), (size_t)nq * sizeof(QueryView),
                            cudaMemcpyHostToDevice, st));
    IM_CUDA(cudaMemcpyAsync(B + o_qstart, qstart.data(), (size_t)(nq + 1) * 8,
                            cudaMemcpyHostToDevice, st));
    if (o_vis && model == IM_IC && !smem_vis)
        IM_CUDA(cudaMemsetAsync(B + o_vis, 0, (size_t)warps * vis_words * 4, st));

    SampleArgs a;
    a.qv = (const QueryView *)(B + o_views);
    a.qstart = (const int64_t *)(B + o_qstart);
    a.nq = nq;
    a.count = cnt;
    a.list = nullptr;
    a.stage = job.stage;
    a.stage_cap = job.stage_cap;
    a.stage_cursor = ctr + 1;
    a.stage_off = (int64_t *)(B + o_soff);
    a.sizes = (int32_t *)(B + o_sizes);
    a.queues = (int32_t *)(B + o_q);
    a.qcap = qcap;
    a.gvis = (uint32_t *)(B + o_vis);
    a.vis_words = vis_words;
    a.examined = ctr + 2;
    a.alg_bytes = ctr + 5;
    a.work = ctr;
    a.ovf_list = (int64_t *)(B + o_ovf);
    a.ovf_count = ctr + 3;
    a.status = (int *)(ctr + 4);

    auto launch = [&](int nblocks, int group) {
        KernelTimer kt(st, model == IM_LT ? "sample_lt" : "sample_ic");
        if (model == IM_LT) {
            if (group == 1) {
                if (lt_cache == 0) k_sample_lt1<0><<<nblocks, kLT1Threads, dyn_smem, st>>>(a);
                else if (lt_cache == 1) k_sample_lt1<1><<<nblocks, kLT1Threads, dyn_smem, st>>>(a);
                else k_sample_lt1<2><<<nblocks, kLT1Threads, dyn_smem, st>>>(a);
            }
            else if (group == 8) k_sample_lt<8><<<nblocks, kSampleThreads, 0, st>>>(a);
            else if (group == 16) k_sample_lt<16><<<nblocks, kSampleThreads, 0, st>>>(a);
            else k_sample_lt<32><<<nblocks, kSampleThreads, 0, st>>>(a);
        } else if (smem_vis) {
            k_sample_ic<true><<<nblocks, kSampleThreads, dyn_smem, st>>>(a);
        } else {
            k_sample_ic<false><<<nblocks, kSampleThreads, 0, st>>>(a);
        }
    };
    launch(blocks, G);
    IM_CUDA(cudaGetLastError());

    unsigned long long hc[6];
    IM_CUDA(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
    IM_CUDA(cudaStreamSynchronize(st));
    int dev_status = (int)(hc[4] & 0xffffffffu);
    if (dev_status == kDevOk && hc[3] > 0 && qcap < n) {
        // second pass for sets longer than the per-walk queue: a few warps
        // with queues of n entries re-run exactly those samples
        const int64_t novf = (int64_t)hc[3];
        const bool ic_big = model == IM_IC;
        // IC: one block per sample; LT: one walk per warp
        const int64_t per_unit = (int64_t)n * 4 + (ic_big ? vis_words * 4 : 0);
        int64_t units = ic_big ? std::min<int64_t>(novf, (int64_t)num_sms())
                               : std::min<int64_t>((novf + kWarps - 1) / kWarps, num_sms()) * kWarps;
        if (ic_big) units = std::max<int64_t>(1, std::min<int64_t>(units, (2ll << 30) / per_unit));
        const int nb2 = (int)(ic_big ? units : std::max<int64_t>(1, units / kWarps));
        const size_t need2 = (size_t)units * (size_t)per_unit;
        int32_t *q2 = nullptr;
        IM_CUDA(cudaMallocAsync((void **)&q2, need2, st));
        uint32_t *vis2 = (uint32_t *)((char *)q2 + (size_t)units * (size_t)n * 4);
        if (ic_big) IM_CUDA(cudaMemsetAsync(vis2, 0, (size_t)units * vis_words * 4, st));
        IM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st));
        SampleArgs a2 = a;
        a2.list = a.ovf_list;
        a2.count = novf;
        a2.queues = q2;
        a2.qcap = n;
        a2.gvis = vis2;
        a2.vis_words = vis_words;
        a2.ovf_list = a.ovf_list + cnt;   // never written: qcap = n cannot overflow
        a = a2;
        if (ic_big) {
            KernelTimer kt(st, "sample_ic_big");
            k_sample_ic_big<<<nb2, kICBigThreads, 0, st>>>(a);
        } else {
            launch(nb2, 32);   // one walk per warp: queues of n entries for the longest walks
        }
        IM_CUDA(cudaGetLastError());
        IM_CUDA(cudaFreeAsync(q2, st));
        IM_CUDA(cudaMemcpyAsync(hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, st));
        IM_CUDA(cudaStreamSynchronize(st));
        dev_status = (int)(hc[4] & 0xffffffffu);
    }
    if (dev_status != kDevOk) {
        if (dev_status == kDevStageOverflow) {
            set_error("RRR set capacity exceeded while sampling");
            return IM_ERR_CAPACITY;
        }
        return map_dev_status(dev_status, "sampling");
    }
    res->stage_off = (int64_t *)(B + o_soff);
    res->sizes = (int32_t *)(B + o_sizes);
    res->scan_tmp = B + o_scan;
    res->sort_tmp = B + o_sort;
    res->total = cnt;
    res->added = (int64_t)hc[1];
    res->examined = (int64_t)hc[2];
    res->alg_bytes = (int64_t)hc[5];
    return IM_OK;
}

// Copies every set from the stage into dst at seg_off and sorts it ascending.
im_status segmented_sort_sets(int32_t *dst, const int64_t *seg_off, int64_t nseg, const int32_t *stage,
                              const int64_t *stage_off, void *tmp, int64_t n_max, cudaStream_t st) {
    int64_t ngiant = 0;
    im_status rs = segmented_sort_impl<int32_t>(dst, seg_off, nseg, stage, stage_off, tmp,
                                                (size_t)(2 + 2 * nseg) * 8, &ngiant, st,
                                                "sort_sets_warp", "sort_sets_block");
    if (rs != IM_OK) return rs;
    if (ngiant > 0) {
        // giant sets (> block sort cap) need an n-bit bitmap per block
        const int64_t gwords = (n_max + 31) / 32;
        const int blocks3 = (int)std::min<int64_t>(ngiant, num_sms());
        uint32_t *gbm = nullptr;
        IM_CUDA(cudaMallocAsync((void **)&gbm, (size_t)blocks3 * gwords * 4, st));
        IM_CUDA(cudaMemsetAsync(gbm, 0, (size_t)blocks3 * gwords * 4, st));
        unsigned long long *sctr = (unsigned long long *)tmp;
        int64_t *giant = (int64_t *)tmp + 2 + nseg;
        {
            KernelTimer kt(st, "sort_sets_bitmap");
            k_sort_giant<<<blocks3, 1024, 0, st>>>(dst, seg_off, giant, sctr + 1, gbm, gwords);
        }
        IM_CUDA(cudaGetLastError());
        IM_CUDA(cudaFreeAsync(gbm, st));
    }
    return IM_OK;
}

// ---------------------------------------------------------------------------
// Sample(G, count): append sample ids first .. first+count-1 to the pool.
// ---------------------------------------------------------------------------
im_status sample_append(const im_graph *gc, im_model model, uint64_t seed, uint64_t first,
                        uint64_t count, im_pool *pool, cudaStream_t st) {
    im_graph *g = const_cast<im_graph *>(gc);
    if (model == IM_LT) {
        im_status s = build_lt_index(g, st);
        if (s != IM_OK) return s;
        if (!g->lt_valid) {
            set_error("LT sampling needs every vertex's in-weights to sum to at most 2^32");
            return IM_ERR_INVALID_ARG;
        }
    }
    if (count == 0) return IM_OK;
    if (pool->theta + (int64_t)count > pool->max_sets) {
        set_error("pool max_sets exceeded");
        return IM_ERR_CAPACITY;
    }
    const int64_t cnt = (int64_t)count;
    SamplingJob job;
    job.model = model;
    job.views.push_back(query_view(g, seed, first));
    job.counts.push_back(cnt);
    job.n_max = g->n;
    job.stage = pool->set_ids;                      // the index buffer doubles as the stage
    job.stage_cap = pool->max_entries - pool->total;
    pool->index_valid = false;
    SamplingResult r;
    im_status rs = run_sampling(job, [&](size_t b, void **p) { return pool_scratch(pool, b, p); },
                                st, &r);
    if (rs != IM_OK) {
        if (rs == IM_ERR_CAPACITY) set_error("pool max_entries exceeded while sampling");
        return rs;
    }
    // set_off[theta .. theta+cnt] = set_off[theta] + exclusive scan of sizes
    int64_t *so = pool->set_off + pool->theta;
    rs = exclusive_scan_i32_to_i64(r.sizes, so, cnt, so, r.scan_tmp, scan_tmp_bytes(cnt), st);
    if (rs != IM_OK) return rs;
    // copy stage -> members and sort each set ascending
    rs = segmented_sort_sets(pool->members, so, cnt, job.stage, r.stage_off, r.sort_tmp, g->n, st);
    if (rs != IM_OK) return rs;
    pool->theta += cnt;
    pool->total += r.added;
    pool->examined += r.examined;
    pool->sample_bytes += r.alg_bytes;
    IM_CUDA(cudaStreamSynchronize(st));
    return IM_OK;
}

}  // namespace im
