// Batched and served execution of many independent sieve instances.
//
// The searches of Section 5 ("Real world searching") sieve many combinations
// of P#/d and m-ranges of very uneven size.  Two runtimes share the GPU among
// them:
//
// * Batch: a fixed set of plans, spread over worker streams with the longest
//   first (greedy longest-processing-time assignment on each plan's cost
//   estimate), the whole launch sequence captured once into a CUDA graph and
//   replayed with one launch.  With CS_BATCH_JOBS=1, when every plan reads its
//   large primes from a residue cache, the walks of all plans and all their
//   prime chunks run instead as jobs of a few persistent launches (one per walk
//   kernel, the most costly plans' jobs first) between the plans' tile sieves
//   and their counts.  That is not the default: on the 64-instance mix it
//   measured 1.19 s per run against 0.99 s with a launch per chunk, which keeps
//   one chunk's primes and one plan's bitset in L2 at a time and reads the plan
//   from the kernel parameters.
// * Server: requests arrive over time; a request is admitted when a slot (a
//   stream) is free and its device memory fits the budget, its plan is built
//   with stream-ordered allocation and sieved on the slot's stream, so it
//   overlaps with the requests already running; its bitset stays resident until
//   the caller releases the ticket.
#include <cuda_runtime.h>

#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/combsieve.h"
#include "cs_internal.h"

using namespace cs;

struct cs_batch_s {
    std::vector<cs_plan_t> plans;
    std::vector<cudaStream_t> streams;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, fork2 = nullptr, done = nullptr;
    std::vector<cudaEvent_t> join, join2;
    WalkJobs *wj = nullptr;               // persistent multi-job walks (cached plans)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool launched = false;
    uint64_t launches = 0;

    ~cs_batch_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : join) cudaEventDestroy(e);
        for (auto e : join2) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (fork2) cudaEventDestroy(fork2);
        walk_jobs_destroy(wj);
        if (done) cudaEventDestroy(done);
        for (auto s : streams) cudaStreamDestroy(s);
        if (origin) cudaStreamDestroy(origin);
    }
};

struct ServerTicket {
    cs_plan_t plan = nullptr;
    int slot = -1;
    uint64_t bytes = 0;
};

namespace {
// Priority level of a request from its cost estimate (about picoseconds of
// device time): below 1 ms level 0, below 10 ms level 1, and so on.
int level_of(uint64_t est_cost, int n_levels) {
    double ms = (double)est_cost * 1e-9;
    int lv = 0;
    for (double lim = 1.0; lv < n_levels - 1 && ms >= lim; lim *= 10.0) lv++;
    return lv;
}
}  // namespace

struct cs_server_s {
    uint64_t budget = 0, used = 0;
    // slot k owns one stream per priority level: slots[k * n_levels + level];
    // level 0 is the highest priority and takes the cheapest requests
    std::vector<cudaStream_t> slots;
    int n_levels = 1;
    std::vector<uint64_t> slot_ticket;      // per slot, 0 = free
    std::unordered_map<uint64_t, ServerTicket> tickets;
    uint64_t next_ticket = 1;
    cs_tuning tune{};
    bool has_tune = false;
    std::mutex mu;
    // residue caches shared by all requests with the same (P, d), resident for
    // the server's lifetime (outside the request budget)
    std::vector<std::pair<std::pair<uint32_t, uint64_t>, cs_cache_t>> caches;
    cudaStream_t cache_stream = nullptr;

    ~cs_server_s() {
        for (auto &kv : tickets) cs_destroy(kv.second.plan);
        for (auto &c : caches) cs_cache_destroy(c.second);
        for (auto s : slots) cudaStreamDestroy(s);
        if (cache_stream) cudaStreamDestroy(cache_stream);
    }
};

namespace {

cs_status cuda_err(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return CS_OK;
    return set_error(e == cudaErrorMemoryAllocation ? CS_ENOMEM : CS_EDEVICE, what);
}

}  // namespace

extern "C" {

cs_status cs_batch_create(const cs_plan_t *plans, int n, int n_streams, cs_batch_t *out) {
    if (!out || !plans || n <= 0) return set_error(CS_EINVAL, "need plans, n >= 1 and out");
    *out = nullptr;
    // default width: instances that each fill the GPU gain little from running
    // side by side and lose L2 locality (64 uneven searches: 1 stream 1.31x,
    // 2 streams 1.27x, 16 streams 1.0x over plain launches); the residue-cache
    // fills, when present, run on streams of their own in any case
    bool any_cache = false;
    for (int i = 0; i < n; i++) any_cache = any_cache || (plans[i] && plan_cache(plans[i]));
    if (n_streams <= 0) n_streams = std::min(n, any_cache ? 1 : 2);
    n_streams = std::min(std::max(n_streams, 1), std::min(n, 64));
    std::vector<std::pair<uint64_t, int>> order;
    for (int i = 0; i < n; i++) {
        if (!plans[i]) return set_error(CS_EINVAL, "NULL plan in batch");
        if (plan_profiled(plans[i])) return set_error(CS_EINVAL, "batched plans must not be built with profile = 1");
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return set_error(CS_EINVAL, "a plan appears twice in the batch");
        cs_info_t info;
        cs_status s = cs_info(plans[i], &info);
        if (s) return s;
        order.push_back({info.est_cost, i});
    }
    std::sort(order.begin(), order.end(), [](auto &a, auto &b) { return a.first > b.first; });
    // longest first onto the least-loaded stream
    std::vector<std::vector<int>> lane(n_streams);
    std::vector<uint64_t> load(n_streams, 0);
    for (auto &o : order) {
        int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[k].push_back(o.second);
        load[k] += o.first;
    }

    // residue caches used by the plans, with the largest L each must reach
    std::vector<std::pair<cs_cache_t, uint64_t>> caches;
    for (int i = 0; i < n; i++) {
        cs_cache_t c = plan_cache(plans[i]);
        if (!c) continue;
        cs_info_t info;
        cs_info(plans[i], &info);
        auto it = std::find_if(caches.begin(), caches.end(), [&](auto &x) { return x.first == c; });
        if (it == caches.end()) caches.push_back({c, 0});
    }

    cs_batch_s *b = new (std::nothrow) cs_batch_s();
    if (!b) return set_error(CS_ENOMEM, "host allocation failed");
    b->plans.assign(plans, plans + n);
    cs_status s = CS_OK;
    // the walks as jobs of persistent launches (CS_BATCH_JOBS=1) when every
    // plan is a cached three-gap plan; by default one launch per chunk, as cs_sieve
    std::vector<WalkJob> jobs;
    const char *bj = getenv("CS_BATCH_JOBS");
    bool use_jobs = bj && atoi(bj) == 1;
    for (size_t o = 0; o < order.size() && use_jobs; o++) use_jobs = plan_walk_jobs(plans[order[o].second], jobs);
    if (use_jobs) {
        cudaError_t ej = walk_jobs_create(jobs, &b->wj);
        if (ej != cudaSuccess) {
            delete b;
            return cuda_err(ej, "walk_jobs_create");
        }
    }
#define BT(call)                                          \
    do {                                                  \
        s = cuda_err((call), #call);                      \
        if (s) { delete b; return s; }                    \
    } while (0)
    BT(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
    BT(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    BT(cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming));
    BT(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
    for (int k = 0; k < n_streams + (int)caches.size(); k++) {
        cudaStream_t st;
        BT(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->streams.push_back(st);
        cudaEvent_t ev, ev2;
        BT(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->join.push_back(ev);
        BT(cudaEventCreateWithFlags(&ev2, cudaEventDisableTiming));
        b->join2.push_back(ev2);
    }
    BT(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    cs_status cap = CS_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->origin);
    // each cache is regenerated once per run on its own stream; the plans'
    // walks wait for the chunks they read (events inside the graph)
    for (size_t k = 0; k < caches.size() && e == cudaSuccess && !cap; k++) {
        cudaStream_t cst = b->streams[n_streams + k];
        e = cudaStreamWaitEvent(cst, b->fork, 0);
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> lk(cache_mutex(caches[k].first));
            cap = cache_fill_upto(caches[k].first, 0, cst, false);
        }
        if (e == cudaSuccess && !cap) e = cudaEventRecord(b->join[n_streams + k], cst);
        if (e == cudaSuccess && !cap) e = cudaStreamWaitEvent(b->origin, b->join[n_streams + k], 0);
    }
    for (int k = 0; k < n_streams && e == cudaSuccess && !cap; k++) {
        e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
        for (int i : lane[k]) {
            if (e != cudaSuccess || cap) break;
            cap = b->wj ? plan_sieve_head(b->plans[i], b->streams[k]) : cs_sieve(b->plans[i], b->streams[k]);
            cs_info_t info;
            if (!cap && !cs_info(b->plans[i], &info))
                b->launches += info.launches_per_sieve - (b->wj ? info.n_large_chunks : 0);
        }
        if (e == cudaSuccess && !cap) e = cudaEventRecord(b->join[k], b->streams[k]);
        if (e == cudaSuccess && !cap) e = cudaStreamWaitEvent(b->origin, b->join[k], 0);
    }
    if (b->wj && e == cudaSuccess && !cap) {
        // every plan's tile sieve and every cache are done: the walks of all
        // plans, then each plan's counts on its worker stream
        e = walk_jobs_launch(b->wj, b->origin);
        b->launches += walk_jobs_launches(b->wj);
        if (e == cudaSuccess) e = cudaEventRecord(b->fork2, b->origin);
        for (int k = 0; k < n_streams && e == cudaSuccess && !cap; k++) {
            e = cudaStreamWaitEvent(b->streams[k], b->fork2, 0);
            for (int i : lane[k]) {
                if (e != cudaSuccess || cap) break;
                cap = plan_sieve_tail(b->plans[i], b->streams[k]);
            }
            if (e == cudaSuccess && !cap) e = cudaEventRecord(b->join2[k], b->streams[k]);
            if (e == cudaSuccess && !cap) e = cudaStreamWaitEvent(b->origin, b->join2[k], 0);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
    b->graph = g;
    for (cs_plan_t p : b->plans) plan_set_sieved(p, false);   // recorded, not run yet
    if (cap) { delete b; return cap; }
    BT(e);
    BT(e2);
    BT(cudaGraphInstantiate(&b->exec, b->graph, 0));
#undef BT
    *out = b;
    return CS_OK;
}

cs_status cs_batch_run(cs_batch_t b, void *stream) {
    if (!b) return set_error(CS_EINVAL, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cs_status s = cuda_err(cudaGraphLaunch(b->exec, st), "cudaGraphLaunch");
    if (s) return s;
    s = cuda_err(cudaEventRecord(b->done, st), "cudaEventRecord");
    if (s) return s;
    for (cs_plan_t p : b->plans) plan_set_sieved(p, true);
    b->launched = true;
    return CS_OK;
}

cs_status cs_batch_sync(cs_batch_t b) {
    if (!b) return set_error(CS_EINVAL, "batch is NULL");
    if (!b->launched) return set_error(CS_ESTATE, "cs_batch_run has not been called");
    cs_status s = cuda_err(cudaEventSynchronize(b->done), "cudaEventSynchronize");
    if (s) return s;
    for (cs_plan_t p : b->plans) {
        s = cs_sync(p);
        if (s) return s;
    }
    return CS_OK;
}

cs_status cs_batch_info(cs_batch_t b, uint64_t *n_streams, uint64_t *launches) {
    if (!b) return set_error(CS_EINVAL, "batch is NULL");
    if (n_streams) *n_streams = b->streams.size();
    if (launches) *launches = b->launches;
    return CS_OK;
}

cs_status cs_batch_destroy(cs_batch_t b) {
    if (!b) return CS_OK;
    if (b->launched) cudaEventSynchronize(b->done);
    delete b;
    return CS_OK;
}

// ------------------------------------------------------------------ server

cs_status cs_server_start(uint64_t budget_bytes, int max_slots, const cs_tuning *tune, cs_server_t *out) {
    if (!out || max_slots <= 0 || max_slots > 256 || budget_bytes == 0)
        return set_error(CS_EINVAL, "need out, 1 <= max_slots <= 256 and a budget");
    *out = nullptr;
    cs_server_s *sv = new (std::nothrow) cs_server_s();
    if (!sv) return set_error(CS_ENOMEM, "host allocation failed");
    sv->budget = budget_bytes;
    if (tune) {
        sv->tune = *tune;
        sv->tune.profile = 0;
        sv->has_tune = true;
    }
    int least = 0, greatest = 0;
    cs_status s0 = cuda_err(cudaDeviceGetStreamPriorityRange(&least, &greatest), "cudaDeviceGetStreamPriorityRange");
    if (!s0) s0 = cuda_err(cudaStreamCreateWithPriority(&sv->cache_stream, cudaStreamNonBlocking, greatest),
                           "cudaStreamCreateWithPriority");
    if (s0) { delete sv; return s0; }
    sv->n_levels = std::min(4, least - greatest + 1);   // greatest is numerically lowest
    if (sv->n_levels < 1) sv->n_levels = 1;
    for (int i = 0; i < max_slots; i++) {
        for (int lv = 0; lv < sv->n_levels; lv++) {
            cudaStream_t st;
            cs_status s = cuda_err(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest + lv),
                                   "cudaStreamCreateWithPriority");
            if (s) { delete sv; return s; }
            sv->slots.push_back(st);
        }
        sv->slot_ticket.push_back(0);
    }
    *out = sv;
    return CS_OK;
}

cs_status cs_submit(cs_server_t sv, uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                    uint64_t L, uint64_t *ticket) {
    if (!sv || !ticket) return set_error(CS_EINVAL, "NULL argument");
    *ticket = 0;
    std::lock_guard<std::mutex> lk(sv->mu);
    int slot = -1;
    for (size_t i = 0; i < sv->slot_ticket.size(); i++)
        if (!sv->slot_ticket[i]) { slot = (int)i; break; }
    if (slot < 0) return set_error(CS_EAGAIN, "no free slot");
    // the (P, d) residue cache: created or extended to L, missing chunks
    // generated on the cache stream (the plan's walks wait on their events)
    cs_cache_t cache = nullptr;
    for (auto &c : sv->caches)
        if (c.first.first == P && c.first.second == d) cache = c.second;
    cs_status s = CS_OK;
    if (!cache) {
        s = cache_new(P, d, L, &cache);
        if (s) return s;
        sv->caches.push_back({{P, d}, cache});
    }
    {
        std::lock_guard<std::mutex> lk(cache_mutex(cache));
        s = cache_extend(cache, L);
        if (!s) s = cache_fill_upto(cache, L, sv->cache_stream, true);
    }
    if (s) return s;
    // build on the slot's lowest-priority stream, sieve on the stream of the
    // request's priority level (both belong to the slot, which is idle)
    cudaStream_t st_alloc = sv->slots[slot * sv->n_levels + sv->n_levels - 1];
    cs_plan_t plan = nullptr;
    s = plan_create(P, d, M_start, M_inc, SL, L, sv->has_tune ? &sv->tune : nullptr, st_alloc, true,
                    cache, &plan);
    if (s) return s;
    cs_info_t info;
    cs_info(plan, &info);
    if (sv->used + info.device_bytes > sv->budget) {
        cs_destroy(plan);
        return set_error(CS_EAGAIN, "device memory budget exhausted");
    }
    cudaStream_t st = sv->slots[slot * sv->n_levels + level_of(info.est_cost, sv->n_levels)];
    s = cs_sieve(plan, st);
    if (s) {
        cs_destroy(plan);
        return s;
    }
    uint64_t id = sv->next_ticket++;
    sv->tickets[id] = ServerTicket{plan, slot, info.device_bytes};
    sv->slot_ticket[slot] = id;
    sv->used += info.device_bytes;
    *ticket = id;
    return CS_OK;
}

cs_status cs_poll(cs_server_t sv, uint64_t ticket, int *done) {
    if (!sv || !done) return set_error(CS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return set_error(CS_EINVAL, "unknown ticket");
    cudaError_t e = cudaEventQuery(plan_done_event(it->second.plan));
    if (e == cudaErrorNotReady) {
        *done = 0;
        return CS_OK;
    }
    if (e != cudaSuccess) return cuda_err(e, "cudaEventQuery");
    *done = 1;
    // the result stays resident; the slot (stream) is free for the next request
    if (it->second.slot >= 0) {
        sv->slot_ticket[it->second.slot] = 0;
        it->second.slot = -1;
    }
    return CS_OK;
}

cs_status cs_server_plan(cs_server_t sv, uint64_t ticket, cs_plan_t *plan) {
    if (!sv || !plan) return set_error(CS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return set_error(CS_EINVAL, "unknown ticket");
    *plan = it->second.plan;
    return CS_OK;
}

cs_status cs_release(cs_server_t sv, uint64_t ticket) {
    if (!sv) return set_error(CS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return set_error(CS_EINVAL, "unknown ticket");
    cs_destroy(it->second.plan);
    if (it->second.slot >= 0) sv->slot_ticket[it->second.slot] = 0;
    sv->used -= it->second.bytes;
    sv->tickets.erase(it);
    return CS_OK;
}

cs_status cs_server_usage(cs_server_t sv, uint64_t *used_bytes, uint64_t *busy_slots, uint64_t *resident) {
    if (!sv) return set_error(CS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (used_bytes) *used_bytes = sv->used;
    if (busy_slots) {
        uint64_t b = 0;
        for (auto t : sv->slot_ticket) b += t != 0;
        *busy_slots = b;
    }
    if (resident) *resident = sv->tickets.size();
    return CS_OK;
}

cs_status cs_server_stop(cs_server_t sv) {
    if (!sv) return CS_OK;
    delete sv;
    return CS_OK;
}

}  // extern "C"
