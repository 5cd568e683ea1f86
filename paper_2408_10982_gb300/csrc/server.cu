// server.cu -- request loop with continuous batching over resident graphs.
//
// Clients submit queries (im_server_submit) and poll or wait for their
// results.  Worker threads -- each with its own CUDA stream and im_batch
// arena -- take the queued requests in arrival order, admit as many as the
// batch size and the device-memory budget allow (a request's footprint is
// estimated from theta and the members per set seen so far on its graph and
// model), solve them with im_solve_batch, and publish the results.  Requests
// that arrive while batches are on the GPU wait for the next free worker;
// with several workers, batches overlap on the device.  With a heavy lane
// (opts.heavy_members > 0), requests whose estimated RRR members reach that
// bound run on worker 0 only, each by itself through the single-query path
// (sampling into a pool the worker keeps, then max-k-cover), and the other
// workers take the rest in arrival order past them, so a few long queries do
// not hold up the short ones queued behind them.  A result does not depend on
// the batch it ran in.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    im_query q;
    Clock::time_point submitted, finished;
    int64_t footprint = 0;
    bool heavy = false;       // runs on worker 0 only (the heavy lane)
    bool done = false;
    im_status status = IM_OK;
    std::string error;        // the failing batch's message (set in the worker's thread)
    std::vector<int32_t> seeds;
    int64_t coverage = 0;
    int64_t entries = 0;
};

}  // namespace

struct im_server {
    int device = 0;
    im_server_opts opts;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    std::map<std::pair<const im_graph *, int32_t>, double> per_set;   // members per set seen
    std::vector<std::thread> workers;
    int64_t mem_in_use = 0;
    int32_t in_flight = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    // counters
    int64_t batches = 0, batched_queries = 0;
};

namespace {

// device bytes a request needs inside a batch: stage + members + covering
// subsets (12 B per member), set offsets and sizes (20 B per set), the
// covered bitmap, and per-vertex greedy state (24 B per vertex)
int64_t footprint(im_server *s, const im_query &q) {
    auto it = s->per_set.find({q.graph, q.model});
    const double per = it != s->per_set.end() ? it->second : 64.0;
    int64_t rg = 0;
    if (q.cover.algo == IM_RANDGREEDI) {   // per-part bitmaps and per-set bucket masks
        const int64_t P = q.cover.partitions > 0 ? q.cover.partitions : 148;
        rg = P * ((q.theta + 31) / 32) * 4 + q.theta * 8 + q.graph->n * 16;
    }
    return (int64_t)((double)q.theta * per * 1.5 * 12.0) + q.theta * 20 + q.theta / 8 +
           q.graph->n * 24 + rg + 4096;
}

// Estimated RRR members of a request (theta x members per set seen so far).
double est_members(im_server *s, const im_query &q) {
    auto it = s->per_set.find({q.graph, q.model});
    const double per = it != s->per_set.end() ? it->second : 64.0;
    return (double)q.theta * per;
}

// A heavy request on its own, as im_sample_rrr + im_max_k_cover on a pool of
// its graph and model that worker 0 keeps between requests (recreated larger
// when theta or the members outgrow it).  For one large query this is the
// library's fastest path: the per-query kernels, the whole GPU.
im_status solve_alone(std::map<std::pair<const im_graph *, int32_t>, im_pool *> &pools,
                      const im_query &q, int64_t want_entries, int32_t *seeds, im_result *res,
                      cudaStream_t st) {
    im_pool *&p = pools[{q.graph, q.model}];
    want_entries = std::max<int64_t>(want_entries, 1 << 16);
    im_status r = IM_OK;
    for (int attempt = 0; attempt < 8; ++attempt) {
        if (p && (p->max_sets < q.theta || p->max_entries < want_entries)) {
            im_pool_destroy(p);
            p = nullptr;
        }
        if (!p) {
            r = im_pool_create(q.graph, std::max<int64_t>(q.theta, 1), want_entries, &p);
            if (r != IM_OK) return r;
        }
        r = im_pool_reset(p);
        if (r != IM_OK) return r;
        r = im_sample_rrr(q.graph, (im_model)q.model, q.seed, 0, (uint64_t)q.theta, p, st);
        if (r != IM_ERR_CAPACITY) break;
        want_entries *= 4;                        // the sets were larger than estimated
    }
    if (r != IM_OK) return r;
    std::vector<int64_t> gains((size_t)q.k);
    const im_cover_opts *o = q.cover.algo != IM_GREEDY_PLAIN ? &q.cover : nullptr;
    r = im_max_k_cover(p, q.k, o, seeds, gains.data(), &res->num_seeds, &res->coverage, st);
    if (r != IM_OK) return r;
    int64_t theta = 0;
    r = im_pool_info(p, &theta, &res->entries, nullptr);
    res->partitions = o && q.cover.algo == IM_RANDGREEDI ? q.cover.partitions : 0;
    return r;
}

void worker_main(im_server *s, int32_t wid) {
    cudaSetDevice(s->device);
    const bool any = wid == 0 || s->opts.heavy_members <= 0;   // may this worker run heavy ones
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    im_batch *b = nullptr;
    im_batch_create(&b);
    std::map<std::pair<const im_graph *, int32_t>, im_pool *> pools;   // heavy requests alone
    std::vector<uint64_t> ids;
    std::vector<im_query> qs;
    for (;;) {
        std::unique_lock<std::mutex> lk(s->mu);
        // the first queued request this worker may run
        auto first_mine = [&]() {
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
                if (any || !s->reqs[*it].heavy) return it;
            return s->queue.end();
        };
        s->cv_work.wait(lk, [&] {
            const auto it = first_mine();
            if (it == s->queue.end()) return s->stop;
            const Request &r = s->reqs[*it];
            return s->in_flight == 0 || s->mem_in_use + r.footprint <= s->opts.mem_budget;
        });
        // stop requested and nothing left for this worker (worker 0 drains the heavy lane)
        if (first_mine() == s->queue.end()) break;
        // admit in arrival order (past the heavy lane's requests on the other
        // workers) while the batch and the memory budget allow
        ids.clear();
        qs.clear();
        int64_t mem = 0;
        bool alone = false;          // worker 0: a heavy request by itself
        int64_t want_entries = 0;
        for (auto it = s->queue.begin();
             it != s->queue.end() && (int32_t)ids.size() < s->opts.max_batch;) {
            Request &r = s->reqs[*it];
            if (!any && r.heavy) {
                ++it;
                continue;
            }
            // the heavy lane runs a heavy request alone, not inside a batch
            // (a RandGreedi request that leaves its partition count to the
            // batch still goes through one)
            const bool by_itself = r.heavy && s->opts.heavy_members > 0 &&
                                   !(r.q.cover.algo == IM_RANDGREEDI && r.q.cover.partitions <= 0);
            if (by_itself && !ids.empty()) break;
            if (!ids.empty() && s->mem_in_use + mem + r.footprint > s->opts.mem_budget) break;
            mem += r.footprint;
            ids.push_back(*it);
            qs.push_back(r.q);
            it = s->queue.erase(it);
            if (by_itself) {
                alone = true;
                want_entries = (int64_t)(est_members(s, r.q) * 1.25);
                break;
            }
        }
        s->mem_in_use += mem;
        s->in_flight++;
        lk.unlock();

        int32_t kmax = 1;
        for (auto &q : qs) kmax = std::max(kmax, q.k);
        std::vector<int32_t> seeds((size_t)qs.size() * kmax);
        std::vector<im_result> res(qs.size());
        const im_status st_batch =
            alone ? solve_alone(pools, qs[0], want_entries, seeds.data(), res.data(), st)
                  : im_solve_batch(b, qs.data(), (int32_t)qs.size(), kmax, seeds.data(), nullptr,
                                   res.data(), st);
        const std::string err = st_batch == IM_OK ? std::string() : std::string(im_last_error());
        // a batch that failed part way may still have work queued on the stream:
        // let it finish before the arena is reused or the worker leaves
        if (st_batch != IM_OK) cudaStreamSynchronize(st);
        const auto now = Clock::now();

        lk.lock();
        for (size_t i = 0; i < ids.size(); ++i) {
            Request &r = s->reqs[ids[i]];
            r.done = true;
            r.finished = now;
            r.status = st_batch;
            r.error = err;
            if (st_batch == IM_OK) {
                r.seeds.assign(seeds.begin() + (int64_t)i * kmax,
                               seeds.begin() + (int64_t)i * kmax + res[i].num_seeds);
                r.coverage = res[i].coverage;
                r.entries = res[i].entries;
                if (r.q.theta > 0) {
                    double &est = s->per_set[{r.q.graph, r.q.model}];
                    const double seen = (double)res[i].entries / (double)r.q.theta;
                    est = est > 0 ? 0.5 * est + 0.5 * seen : seen;
                }
            }
        }
        s->batches++;
        s->batched_queries += (int64_t)ids.size();
        s->mem_in_use -= mem;
        s->in_flight--;
        lk.unlock();
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    for (auto &kv : pools)
        if (kv.second) im_pool_destroy(kv.second);
    im_batch_destroy(b);
    cudaStreamDestroy(st);
}

im_status take_result(im_server *s, uint64_t ticket, int32_t *seeds, int32_t *num_seeds,
                      int64_t *coverage, double *latency_ms, std::unique_lock<std::mutex> &lk) {
    auto it = s->reqs.find(ticket);
    Request &r = it->second;
    const im_status st = r.status;
    if (st != IM_OK) im::set_error("im_server: the request's batch failed: " + r.error);
    if (st == IM_OK) {
        if (seeds && !r.seeds.empty()) std::memcpy(seeds, r.seeds.data(), r.seeds.size() * 4);
        if (num_seeds) *num_seeds = (int32_t)r.seeds.size();
        if (coverage) *coverage = r.coverage;
    }
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r.finished - r.submitted).count();
    s->reqs.erase(it);
    (void)lk;
    return st;
}

}  // namespace

using namespace im;

extern "C" {

im_status im_server_create(const im_server_opts *opts, im_server **out) {
    if (!opts || !out || opts->workers < 1 || opts->workers > 16 || opts->max_batch < 1 ||
        opts->mem_budget <= 0 || opts->heavy_members < 0 ||
        (opts->heavy_members > 0 && opts->workers < 2)) {
        set_error("im_server_create: bad options");
        return IM_ERR_INVALID_ARG;
    }
    im_server *s = new (std::nothrow) im_server();
    if (!s) return IM_ERR_OOM;
    s->opts = *opts;
    cudaGetDevice(&s->device);
    for (int32_t w = 0; w < opts->workers; ++w) s->workers.emplace_back(worker_main, s, w);
    *out = s;
    return IM_OK;
}

im_status im_server_destroy(im_server *s) {
    if (!s) return IM_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
    return IM_OK;
}

im_status im_server_submit(im_server *s, const im_query *q, uint64_t *ticket) {
    if (!s || !q || !ticket || !q->graph || q->k < 1 || q->k > q->graph->n || q->theta < 0 ||
        (q->model != IM_IC && q->model != IM_LT) || q->graph->device != s->device) {
        set_error("im_server_submit: bad query");
        return IM_ERR_INVALID_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return IM_ERR_INVALID_ARG;
        const uint64_t t = s->next_ticket++;
        Request &r = s->reqs[t];
        r.q = *q;
        r.submitted = Clock::now();
        r.footprint = footprint(s, *q);
        r.heavy = s->opts.heavy_members > 0 &&
                  est_members(s, *q) >= (double)s->opts.heavy_members;
        s->queue.push_back(t);
        *ticket = t;
    }
    s->cv_work.notify_all();   // the right worker for this request may not be the first woken
    return IM_OK;
}

im_status im_server_poll(im_server *s, uint64_t ticket, int32_t *seeds, int32_t *num_seeds,
                         int64_t *coverage, double *latency_ms) {
    if (!s) return IM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("im_server_poll: unknown ticket");
        return IM_ERR_INVALID_ARG;
    }
    if (!it->second.done) return IM_ERR_BUSY;
    return take_result(s, ticket, seeds, num_seeds, coverage, latency_ms, lk);
}

im_status im_server_wait(im_server *s, uint64_t ticket, double timeout_s, int32_t *seeds,
                         int32_t *num_seeds, int64_t *coverage, double *latency_ms) {
    if (!s) return IM_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("im_server_wait: unknown ticket");
        return IM_ERR_INVALID_ARG;
    }
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        auto jt = s->reqs.find(ticket);
        return jt != s->reqs.end() && jt->second.done;
    });
    if (!ok) return IM_ERR_BUSY;
    return take_result(s, ticket, seeds, num_seeds, coverage, latency_ms, lk);
}

im_status im_server_stats(im_server *s, int64_t *batches, int64_t *queries, int64_t *queued) {
    if (!s) return IM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (batches) *batches = s->batches;
    if (queries) *queries = s->batched_queries;
    if (queued) *queued = (int64_t)s->queue.size();
    return IM_OK;
}

}  // extern "C"
