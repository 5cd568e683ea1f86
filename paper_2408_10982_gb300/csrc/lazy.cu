// lazy.cu -- the lazy greedy of Alg. 2 as a grid-wide max-k-cover path.
//
// The greedy's marginal gains only shrink as sets get covered (coverage is
// submodular), so a gain computed earlier is an upper bound on the gain now.
// Alg. 2 keeps these bounds in a priority queue and re-evaluates only the top
// one; a candidate whose freshly computed gain still beats every other bound
// is the standard greedy's pick.  With the ordering key gain << 32 | ~v (ties
// to the smallest id) the seeds, gains and coverage are exactly those of the
// standard greedy (k_greedy in cover.cu): neither path decrements the gains of
// the members of every newly covered set here -- the work that bounds the
// standard greedy -- only S(v) of the few candidates is scanned.
//
// One cooperative persistent launch, one block per SM.  Every block holds the
// same sorted list of the best bounds in shared memory and takes the same
// decisions, so the only grid-wide steps are the evaluation of W candidates
// at once (their S(v) spread over the grid, a barrier) and the cover of a
// picked S(v*) (a barrier).  A candidate evaluated since the last cover has an
// exact gain (it is "fresh"): when the best fresh gain beats every stale bound
// it is picked without another scan.  The list holds the top kLzCap keys of
// the bounds array; vertices outside it are represented by the best key among
// them (bout).  When the list runs dry before a pick can be certified, it is
// rebuilt from the bounds array (exact top-kLzCap selection by histogram
// refinement, ties by smallest id).  Every wait is bounded (grid_sync).
#include <algorithm>

#include "internal.cuh"

namespace im {

namespace {

constexpr int kLzThreads = 1024;
constexpr int kLzCap = 8192;          // sorted bound keys per block (two buffers)
constexpr int kLzMaxW = 32;           // candidates evaluated per round (at most a warp)
constexpr int kLzFresh = 512;         // exact keys kept since the last cover
constexpr int kLzBins = 256;          // histogram bins of one refinement pass
constexpr int kLzU = 4;               // loads in flight per lane in scans

struct LazyArgs {
    int64_t n, theta;
    const int64_t *vtx_off;
    const int32_t *set_ids;
    int32_t k, W;
    int32_t *ub;                     // [n] bound on each vertex's marginal gain; 0 once picked
    uint32_t *covered;               // [ceil(theta/32)]
    unsigned long long *list;        // [kLzCap] list build target
    unsigned int *hist;              // [3][kLzBins]
    unsigned int *tie_cnt;           // [grid]
    unsigned int *fill;              // [1] list build fill counter
    unsigned long long *bout;        // [1] best key outside the list
    unsigned long long *acc;         // [3][kLzMaxW] evaluation counts
    GridBarrier *bar;
    int32_t *seeds;
    int64_t *gains;
    int32_t *nseeds;
    int64_t *coverage;
    long long *stats;                // [4] rounds, evaluations, entries scanned, list builds
    int *status;
    // candidates restricted to the first cand_take seeds of each of cand_parts
    // local solutions (cand_seeds[p * cand_stride + j], j < cand_n[p]); NULL: all of V
    const int32_t *cand_seeds;
    const int32_t *cand_n;
    int32_t cand_parts, cand_take, cand_stride;
};

__device__ __forceinline__ unsigned long long lz_key(uint32_t gain, uint32_t v) {
    return ((unsigned long long)gain << 32) | (0xffffffffu - v);
}
__device__ __forceinline__ uint32_t lz_vertex(unsigned long long key) {
    return 0xffffffffu - (uint32_t)(key & 0xffffffffull);
}
__device__ __forceinline__ uint32_t lz_gain(unsigned long long key) { return (uint32_t)(key >> 32); }

// Number of entries of a[0, len) (sorted descending) greater than x.
__device__ __forceinline__ int lz_count_greater(const unsigned long long *a, int len,
                                                unsigned long long x) {
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] > x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Bitonic sort of s[0, m) descending, m a power of two, by the whole block.
__device__ void lz_sort_desc(unsigned long long *s, int m) {
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (m >> 1); t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool desc = (lo & size) == 0;
                const unsigned long long x = s[lo], y = s[hi];
                if ((x < y) == desc) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

struct LzShared {
    unsigned long long fresh[kLzFresh + kLzMaxW];   // exact keys since the last cover, descending
    unsigned long long fresh2[kLzFresh + kLzMaxW];  // merge target
    unsigned long long nk[kLzMaxW];       // this round's exact keys (0: zero gain)
    unsigned long long nks[kLzMaxW];      // the non-zero ones, descending
    unsigned long long cand[kLzMaxW];     // this round's candidates (stale keys)
    long long off[kLzMaxW];               // their S(v) offsets
    long long pre[kLzMaxW + 1];           // prefix sums of |S(v)|
    unsigned int cnt[kLzMaxW];            // block-local evaluation counts
    unsigned int hist[kLzBins];
    unsigned long long bout;
    unsigned long long bmax;
    long long lo, hi, c_above, tie_base;
    int len, head, nf, nz, nc, pick_fresh, stop, rebuild, split, ok;
    unsigned int t, R;
    long long red[32];
};

// Exact selection of the top kLzCap keys of the bounds array into every
// block's list buf (sorted descending); sh.bout gets the best key left out.
// Every block calls it; it contains grid barriers.  Returns false on a timeout.
__device__ bool lz_build(const LazyArgs &a, LzShared &sh, unsigned long long *buf, int64_t v0,
                         int64_t v1) {
    const uint32_t nb = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    if (blockIdx.x == 0) {
        for (int i = tid; i < 3 * kLzBins; i += blockDim.x) a.hist[i] = 0u;
        if (tid == 0) {
            *a.fill = 0u;
            *a.bout = 0ull;
        }
    }
    if (tid == 0) {
        sh.lo = 1;
        sh.hi = a.theta > 0 ? a.theta : 1;
        sh.c_above = 0;
        sh.split = 0;
    }
    if (!grid_sync(a.bar, nb, a.status)) return false;
    // ---- threshold t: count(bound > t) <= cap < count(bound >= t), or t = 1
    for (int pass = 0;; ++pass) {
        const long long lo = sh.lo, hi = sh.hi;
        const long long w = (hi - lo + kLzBins) / kLzBins;   // ceil((hi - lo + 1) / bins)
        for (int i = tid; i < kLzBins; i += blockDim.x) sh.hist[i] = 0u;
        __syncthreads();
        for (int64_t base = v0; base < v1; base += blockDim.x) {
            const int64_t v = base + tid;
            const long long u = v < v1 ? (long long)__ldcg(a.ub + v) : 0;
            const bool in = u >= lo && u <= hi;
            const int bin = in ? (int)((u - lo) / w) : -1;
            const unsigned grp = __match_any_sync(kFull, bin);
            if (in && lane == __ffs(grp) - 1) atomicAdd(&sh.hist[bin], (unsigned)__popc(grp));
        }
        __syncthreads();
        unsigned int *gh = a.hist + (pass % 3) * kLzBins;
        for (int i = tid; i < kLzBins; i += blockDim.x)
            if (sh.hist[i]) atomicAdd(&gh[i], sh.hist[i]);
        if (blockIdx.x == 0)   // the next pass's buffer: last read two passes ago
            for (int i = tid; i < kLzBins; i += blockDim.x) a.hist[((pass + 1) % 3) * kLzBins + i] = 0u;
        if (!grid_sync(a.bar, nb, a.status)) return false;
        for (int i = tid; i < kLzBins; i += blockDim.x) sh.hist[i] = __ldcg(gh + i);
        __syncthreads();
        if (tid == 0) {
            long long above = sh.c_above, total = 0;
            for (int b = 0; b < kLzBins; ++b) total += sh.hist[b];
            int done = 0;
            if (above + total <= kLzCap) {       // everything in range fits: t = lo
                sh.t = (unsigned)lo;
                sh.split = 0;
                done = 1;
            } else {
                int b = kLzBins - 1;
                while (b >= 0 && above + (long long)sh.hist[b] <= kLzCap) above += sh.hist[b--];
                // bin b overflows the list: refine it
                const long long nlo = lo + (long long)b * w;
                const long long nhi = hi < nlo + w - 1 ? hi : nlo + w - 1;
                sh.c_above = above;
                if (w == 1) {
                    sh.t = (unsigned)nlo;
                    sh.split = 1;
                    sh.R = (unsigned)(kLzCap - above);
                    done = 1;
                } else {
                    sh.lo = nlo;
                    sh.hi = nhi;
                }
            }
            sh.ok = done;
        }
        __syncthreads();
        if (sh.ok) break;
    }
    const unsigned t = sh.t;
    const bool split = sh.split != 0;
    // ---- ties at t (when they do not all fit): ranked by vertex id across blocks
    const int64_t chunk = (v1 - v0 + blockDim.x - 1) / blockDim.x;
    const int64_t c0 = min(v1, v0 + (int64_t)tid * chunk);
    const int64_t c1 = min(v1, c0 + chunk);
    long long my_ties = 0;
    if (split) {
        for (int64_t v = c0; v < c1; ++v) my_ties += (uint32_t)__ldcg(a.ub + v) == t;
        // exclusive scan of the threads' tie counts, in thread (= vertex) order
        long long incl = warp_incl_scan<long long>(my_ties, lane);
        if (lane == 31) sh.red[tid >> 5] = incl;
        __syncthreads();
        if (tid < 32) {
            long long x = tid < (int)(blockDim.x >> 5) ? sh.red[tid] : 0;
            x = warp_incl_scan<long long>(x, tid);
            sh.red[tid] = x;
        }
        __syncthreads();
        const long long wbase = (tid >> 5) ? sh.red[(tid >> 5) - 1] : 0;
        const long long blk_total = sh.red[(blockDim.x >> 5) - 1];
        my_ties = wbase + incl - my_ties;                      // exclusive prefix in the block
        if (tid == 0) a.tie_cnt[blockIdx.x] = (unsigned)blk_total;
        if (!grid_sync(a.bar, nb, a.status)) return false;
        if (tid == 0) {
            long long base = 0;
            for (uint32_t b = 0; b < blockIdx.x; ++b) base += __ldcg(a.tie_cnt + b);
            sh.tie_base = base;
        }
        __syncthreads();
        my_ties += sh.tie_base;                                // global rank of my first tie
    }
    // ---- compaction: keys above t (all), ties in id order up to R, the rest -> bout
    unsigned long long best_out = 0ull;
    for (int64_t v = c0; v < c1; ++v) {
        const uint32_t u = (uint32_t)__ldcg(a.ub + v);
        if (u == 0u) continue;
        const unsigned long long key = lz_key(u, (uint32_t)v);
        bool take = u > t || (u == t && !split);
        if (u == t && split) {
            take = my_ties < (long long)sh.R;
            ++my_ties;
        }
        if (take) {
            const unsigned slot = atomicAdd(a.fill, 1u);
            if (slot < (unsigned)kLzCap) a.list[slot] = key;
            else best_out = key > best_out ? key : best_out;   // cannot happen: counts are exact
        } else {
            best_out = key > best_out ? key : best_out;
        }
    }
    best_out = warp_max_u64(best_out);
    if (lane == 0 && best_out) atomicMax(a.bout, best_out);
    if (!grid_sync(a.bar, nb, a.status)) return false;
    // ---- every block: load and sort the list
    const int len = (int)min(__ldcg(a.fill), (unsigned)kLzCap);
    int m = 64;
    while (m < len) m <<= 1;
    for (int i = tid; i < m; i += blockDim.x) buf[i] = i < len ? __ldcg(a.list + i) : 0ull;
    __syncthreads();
    lz_sort_desc(buf, m);
    if (tid == 0) {
        sh.len = len;
        sh.head = 0;
        sh.bout = __ldcg(a.bout);
        sh.nf = 0;                            // fresh keys are back in the list as bounds
    }
    __syncthreads();
    return true;
}

__global__ void __launch_bounds__(kLzThreads, 1) k_greedy_lazy(LazyArgs a) {
    extern __shared__ unsigned long long lz_dyn[];      // two list buffers of kLzCap keys
    __shared__ LzShared sh;
    unsigned long long *L = lz_dyn, *L2 = lz_dyn + kLzCap;
    unsigned long long *F = sh.fresh, *F2 = sh.fresh2;
    const uint32_t nb = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
    const int64_t stride = (int64_t)nb * blockDim.x;
    const int64_t gwarp = gtid >> 5, nwarps = stride >> 5;
    const int64_t per = (a.n + nb - 1) / nb;
    const int64_t v0 = min(a.n, (int64_t)blockIdx.x * per);
    const int64_t v1 = min(a.n, v0 + per);
    const int64_t words = (a.theta + 31) / 32;
    const int W = a.W < 1 ? 1 : (a.W > kLzMaxW ? kLzMaxW : a.W);

    // bounds: |S(v)| for every vertex, or only for the candidate vertices
    for (int64_t v = v0 + tid; v < v1; v += blockDim.x)
        a.ub[v] = a.cand_seeds ? 0 : (int32_t)(__ldg(a.vtx_off + v + 1) - __ldg(a.vtx_off + v));
    for (int64_t x = gtid; x < words; x += stride) a.covered[x] = 0u;
    if (blockIdx.x == 0)
        for (int i = tid; i < 3 * kLzMaxW; i += blockDim.x) a.acc[i] = 0ull;
    if (a.cand_seeds) {
        if (!grid_sync(a.bar, nb, a.status)) return;
        // the first cand_take seeds of each of cand_parts local solutions
        const int64_t slots = (int64_t)a.cand_parts * a.cand_take;
        for (int64_t q = gtid; q < slots; q += stride) {
            const int32_t p = (int32_t)(q / a.cand_take), jj = (int32_t)(q % a.cand_take);
            if (jj < __ldcg(a.cand_n + p)) {
                const int32_t v = __ldcg(a.cand_seeds + (int64_t)p * a.cand_stride + jj);
                a.ub[v] = (int32_t)(__ldg(a.vtx_off + v + 1) - __ldg(a.vtx_off + v));
            }
        }
    }
    if (!lz_build(a, sh, L, v0, v1)) return;

    long long rounds = 0, evals = 0, scanned = 0, builds = 1;
    int32_t j = 0;
    long long cov = 0;
    int e = 0;                                           // evaluation rounds so far
    while (j < a.k) {
        ++rounds;
        // ---- what this round does (thread 0; every block alike)
        if (tid == 0) {
            const unsigned long long top_stale = sh.head < sh.len ? L[sh.head] : 0ull;
            const unsigned long long bound = top_stale > sh.bout ? top_stale : sh.bout;
            sh.stop = 0;
            sh.rebuild = 0;
            sh.nc = 0;
            sh.pick_fresh = 0;
            if (j == 0 && sh.head < sh.len && top_stale > sh.bout) {
                sh.pick_fresh = 1;        // before the first cover every bound is exact
            } else if (sh.nf && F[0] > bound) {
                sh.pick_fresh = 2;
            } else if (sh.head < sh.len) {
                sh.nc = min(W, sh.len - sh.head);
            } else if (sh.bout == 0ull) {
                if (sh.nf) sh.pick_fresh = 2;            // nothing stale is left anywhere
                else sh.stop = 1;
            } else {
                sh.rebuild = 1;                          // the best bound lies outside the list
            }
        }
        __syncthreads();
        if (sh.stop) break;
        if (sh.rebuild) {
            // fresh keys are exact bounds in ub: the rebuilt list takes them back
            if (!lz_build(a, sh, L, v0, v1)) return;
            ++builds;
            continue;
        }
        const int nc = sh.nc;
        if (nc > 0) {
            // ---- candidates: the next nc stale keys; their S(v) offsets and prefix sums
            if (tid < 32) {
                long long len = 0;
                if (tid < nc) {
                    const unsigned long long key = L[sh.head + tid];
                    const uint32_t v = lz_vertex(key);
                    sh.cand[tid] = key;
                    sh.off[tid] = __ldg(a.vtx_off + v);
                    len = __ldg(a.vtx_off + v + 1) - sh.off[tid];
                }
                const long long incl = warp_incl_scan<long long>(len, tid);
                sh.pre[tid + 1] = incl;
                if (tid == 0) sh.pre[0] = 0;
            }
            if (tid < kLzMaxW) sh.cnt[tid] = 0u;
            __syncthreads();
            // ---- evaluate: |S(c) \ covered| over the whole grid
            const long long tot = sh.pre[nc];
            for (int64_t base = gwarp * (32 * kLzU); base < tot; base += nwarps * (32 * kLzU)) {
                int ci[kLzU];
                bool unc[kLzU];
#pragma unroll
                for (int u = 0; u < kLzU; ++u) {
                    const int64_t p = base + u * 32 + lane;
                    ci[u] = -1;
                    unc[u] = false;
                    if (p < tot) {
                        int lo = 0, hi = nc - 1;         // last c with pre[c] <= p
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (sh.pre[mid] <= p) lo = mid;
                            else hi = mid - 1;
                        }
                        const int32_t id = __ldg(a.set_ids + sh.off[lo] + (p - sh.pre[lo]));
                        unc[u] = !((__ldcg(a.covered + (id >> 5)) >> (id & 31)) & 1u);
                        ci[u] = lo;
                    }
                }
#pragma unroll
                for (int u = 0; u < kLzU; ++u) {
                    const unsigned grp = __match_any_sync(kFull, ci[u]);
                    const unsigned hit = __ballot_sync(kFull, unc[u]);
                    if (ci[u] >= 0 && lane == __ffs(grp) - 1) {
                        const unsigned c = __popc(grp & hit);
                        if (c) atomicAdd(&sh.cnt[ci[u]], c);
                    }
                }
            }
            __syncthreads();
            unsigned long long *acc = a.acc + (e % 3) * kLzMaxW;
            if (tid < nc && sh.cnt[tid]) atomicAdd(acc + tid, (unsigned long long)sh.cnt[tid]);
            if (!grid_sync(a.bar, nb, a.status)) return;
            // the buffer of evaluation round e + 2: every block read it (round e - 1)
            // before this barrier, and none writes it before the next one
            if (blockIdx.x == 0 && tid < kLzMaxW) a.acc[((e + 2) % 3) * kLzMaxW + tid] = 0ull;
            // ---- exact keys of the candidates, sorted, merged into the fresh list
            unsigned long long nk = 0ull;
            if (tid < nc) {
                const uint32_t v = lz_vertex(sh.cand[tid]);
                const uint32_t g = (uint32_t)__ldcg(acc + tid);
                if (blockIdx.x == 0) a.ub[v] = (int32_t)g;
                nk = g ? lz_key(g, v) : 0ull;            // a zero gain is never picked
                sh.nk[tid] = nk;
            }
            __syncthreads();
            if (tid < nc && nk) {                        // rank among the new keys
                int r = 0;
                for (int c = 0; c < nc; ++c) r += sh.nk[c] > nk;
                sh.nks[r] = nk;
            }
            if (tid == 0) {
                int nz = 0;
                for (int c = 0; c < nc; ++c) nz += sh.nk[c] != 0ull;
                sh.nz = nz;
            }
            __syncthreads();
            {
                const int nf = sh.nf, nz = sh.nz;
                for (int i = tid; i < nf; i += blockDim.x) {
                    const unsigned long long x = F[i];
                    F2[i + lz_count_greater(sh.nks, nz, x)] = x;
                }
                for (int i = tid; i < nz; i += blockDim.x) {
                    const unsigned long long x = sh.nks[i];
                    F2[i + lz_count_greater(F, nf, x)] = x;
                }
                __syncthreads();
                unsigned long long *tmp = F;
                F = F2;
                F2 = tmp;
                if (tid == 0) {
                    int m = nf + nz;
                    if (m > kLzFresh) {
                        // no room: the smallest exact keys leave the list; their
                        // vertices are outside it now, represented by bout
                        if (F[kLzFresh] > sh.bout) sh.bout = F[kLzFresh];
                        m = kLzFresh;
                    }
                    sh.nf = m;
                    sh.head += nc;
                    evals += nc;
                    scanned += tot;
                    const unsigned long long top_stale = sh.head < sh.len ? L[sh.head] : 0ull;
                    const unsigned long long bound = top_stale > sh.bout ? top_stale : sh.bout;
                    sh.pick_fresh = (m && F[0] > bound) ? 2 : 0;
                }
                __syncthreads();
            }
            ++e;
        }
        if (sh.pick_fresh == 0) continue;
        // ---- the pick: remove it, turn the fresh keys back into bounds
        unsigned long long pick;
        if (sh.pick_fresh == 1) {
            pick = L[sh.head];
            __syncthreads();
            if (tid == 0) sh.head += 1;
        } else {
            pick = F[0];
            __syncthreads();
            const int nf = sh.nf;
            for (int i = tid + 1; i < nf; i += blockDim.x) F2[i - 1] = F[i];
            __syncthreads();
            unsigned long long *tmp = F;
            F = F2;
            F2 = tmp;
            if (tid == 0) sh.nf = nf - 1;
        }
        __syncthreads();
        const uint32_t vs = lz_vertex(pick);
        const uint32_t gain = lz_gain(pick);
        if (blockIdx.x == 0 && tid == 0) {
            a.seeds[j] = (int32_t)vs;
            a.gains[j] = (int64_t)gain;
            a.ub[vs] = 0;
        }
        ++j;
        cov += gain;
        // merge the fresh keys into the rest of the list (both sorted descending)
        {
            const int head = sh.head, len = sh.len, nf = sh.nf;
            const int rest = len - head;
            if (rest + nf <= kLzCap) {
                for (int i = tid; i < rest; i += blockDim.x) {
                    const unsigned long long x = L[head + i];
                    L2[i + lz_count_greater(F, nf, x)] = x;
                }
                for (int i = tid; i < nf; i += blockDim.x) {
                    const unsigned long long x = F[i];
                    L2[i + lz_count_greater(L + head, rest, x)] = x;
                }
                __syncthreads();
                unsigned long long *tmp = L;
                L = L2;
                L2 = tmp;
                if (tid == 0) {
                    sh.len = rest + nf;
                    sh.head = 0;
                    sh.nf = 0;
                }
            } else if (tid == 0) {
                // no room: the fresh keys stay exact bounds in ub, and the best
                // of them now bounds what lies outside the list
                if (nf && F[0] > sh.bout) sh.bout = F[0];
                sh.nf = 0;
            }
            __syncthreads();
        }
        // ---- cover S(v*) over the whole grid
        const int64_t sb = __ldg(a.vtx_off + vs), se = __ldg(a.vtx_off + vs + 1);
        for (int64_t base = sb + (gtid & ~(int64_t)31); base < se; base += stride) {
            const int64_t t = base + lane;
            warp_bitmap_or(a.covered, t < se ? (int64_t)__ldg(a.set_ids + t) : -1, lane);
        }
        if (!grid_sync(a.bar, nb, a.status)) return;
    }
    if (blockIdx.x == 0 && tid == 0) {
        *a.nseeds = j;
        *a.coverage = cov;
        if (a.stats) {
            a.stats[0] = rounds;
            a.stats[1] = evals;
            a.stats[2] = scanned;
            a.stats[3] = builds;
        }
    }
}

}  // namespace

size_t lazy_greedy_smem() { return (size_t)2 * kLzCap * sizeof(unsigned long long); }

// Scratch of one lazy greedy launch (bytes), for n vertices and theta sets.
size_t lazy_greedy_scratch(int64_t n, int64_t theta) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t words = std::max<int64_t>(1, (theta + 31) / 32);
    return up((size_t)n * 4) + up((size_t)words * 4) + up((size_t)kLzCap * 8) +
           up((size_t)3 * kLzBins * 4) + up((size_t)4096 * 4) + up(64) + up(64) +
           up((size_t)3 * kLzMaxW * 8) + up(sizeof(GridBarrier)) + up(4 * 8);
}

im_status greedy_lazy_launch(int64_t n, int64_t theta, const int64_t *vtx_off,
                             const int32_t *set_ids, int32_t k, int32_t W, void *scratch,
                             int32_t *seeds, int64_t *gains, int32_t *nseeds, int64_t *coverage,
                             long long *stats_out, int *status, cudaStream_t st,
                             const int32_t *cand_seeds, const int32_t *cand_n, int32_t cand_parts,
                             int32_t cand_take, int32_t cand_stride) {
    const size_t smem = lazy_greedy_smem();
    IM_TRY(raise_dyn_smem((const void *)k_greedy_lazy, smem));
    int per_sm = 0;
    IM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy_lazy, kLzThreads, smem));
    if (per_sm < 1) {
        set_error("lazy greedy: kernel does not fit on an SM");
        return IM_ERR_UNSUPPORTED;
    }
    const int grid = std::min(num_sms(), 4096);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t words = std::max<int64_t>(1, (theta + 31) / 32);
    char *B = (char *)scratch;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = B + off;
        off += up(bytes);
        return p;
    };
    LazyArgs a;
    a.n = n;
    a.theta = theta;
    a.vtx_off = vtx_off;
    a.set_ids = set_ids;
    a.k = k;
    a.W = W;
    a.ub = (int32_t *)take((size_t)n * 4);
    a.covered = (uint32_t *)take((size_t)words * 4);
    a.list = (unsigned long long *)take((size_t)kLzCap * 8);
    a.hist = (unsigned int *)take((size_t)3 * kLzBins * 4);
    a.tie_cnt = (unsigned int *)take((size_t)4096 * 4);
    a.fill = (unsigned int *)take(64);
    a.bout = (unsigned long long *)take(64);
    a.acc = (unsigned long long *)take((size_t)3 * kLzMaxW * 8);
    a.bar = (GridBarrier *)take(sizeof(GridBarrier));
    a.stats = (long long *)take(4 * 8);
    a.seeds = seeds;
    a.gains = gains;
    a.nseeds = nseeds;
    a.coverage = coverage;
    a.status = status;
    a.cand_seeds = cand_seeds;
    a.cand_n = cand_n;
    a.cand_parts = cand_parts;
    a.cand_take = cand_take;
    a.cand_stride = cand_stride;
    IM_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), st));
    IM_CUDA(cudaMemsetAsync(a.stats, 0, 4 * 8, st));
    void *args[] = {&a};
    {
        KernelTimer kt(st, "greedy_lazy");
        IM_CUDA(cudaLaunchCooperativeKernel((const void *)k_greedy_lazy, dim3(grid),
                                            dim3(kLzThreads), args, smem, st));
    }
    if (stats_out)
        IM_CUDA(cudaMemcpyAsync(stats_out, a.stats, 4 * 8, cudaMemcpyDeviceToHost, st));
    return IM_OK;
}

im_status greedy_select(im_pool *p, int32_t k, bool lazy, int32_t *d_seeds, int64_t *d_gains,
                        int32_t *d_nseeds, int64_t *d_cov, cudaStream_t st, int *d_status) {
    int32_t W = (int32_t)tune_value(IM_TUNE_GREEDY_EVALS);
    if (!lazy && W == 0) return greedy_plain(p, k, d_seeds, d_gains, d_nseeds, d_cov, st, d_status);
    if (W <= 0) W = 16;
    void *scratch = nullptr;
    im_status s = pool_scratch(p, lazy_greedy_scratch(p->g->n, p->theta), &scratch);
    if (s != IM_OK) return s;
    IM_CUDA(cudaMemsetAsync(d_nseeds, 0, sizeof(int32_t), st));
    IM_CUDA(cudaMemsetAsync(d_cov, 0, sizeof(int64_t), st));
    return greedy_lazy_launch(p->g->n, p->theta, p->vtx_off, p->set_ids, k, W, scratch, d_seeds,
                              d_gains, d_nseeds, d_cov, p->lz_stats, d_status, st);
}

}  // namespace im

using namespace im;

extern "C" im_status im_greedy_stats(const im_pool *p, int64_t *stats) {
    if (!p || !stats) return IM_ERR_INVALID_ARG;
    for (int i = 0; i < 4; ++i) stats[i] = p->lz_stats[i];
    return IM_OK;
}
