// Served allocation loop (continuous batching) behind mapa_serve_* in mapa.h.
//
// One worker thread per server.  Each round it
//   1. applies every departure that is due (explicit DEPART events and jobs
//      whose lifetime ran out) with one release kernel, so later arrivals see
//      the freed accelerators (state management, Sec. 3.6); a queue head that
//      is waiting for accelerators (FIFO, Sec. 4) is retried after one;
//   2. admits the requests that have arrived, in order, up to max_batch;
//   3. decides them together with the batched engine, every request against
//      the same occupancy snapshot (its busy mask is set to the snapshot);
//   4. commits the longest arrival-order prefix of decisions that do not
//      overlap (FIFO, Sec. 4); the requests from the first overlap on are
//      decided again in the same round, in order, by a device-side chain
//      against the live occupancy (see decide_round).
// The occupancy lives on the device; the worker keeps a host copy of it that
// it updates from the committed and released vertex sets.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mapa_ctx.h"
#include "mapa_engine.h"

namespace {

using Clock = std::chrono::steady_clock;

// A decision that holds accelerators once committed: exact, or an anytime
// request's best match past its work budget.
inline bool placed(int32_t status) { return status == MAPA_OK || status == MAPA_INEXACT; }

struct Pending {
    mapa_event ev;
    int32_t rounds = 0;
};

struct Job {
    std::vector<int> verts;
};

}  // namespace

struct mapa_server_s {
    mapa_ctx ctx = nullptr;
    int32_t topo_id = 0;
    int32_t max_batch = 1;
    bool fifo_wait = true;  // a request that does not fit waits (paper's FIFO queue)
    Clock::time_point t0;

    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work;  // new events or stop
    std::condition_variable cv_done;  // finished events
    std::deque<Pending> incoming;     // submitted, in non-decreasing at_ns
    std::deque<mapa_served> done;
    uint64_t submitted = 0;
    uint64_t finished = 0;
    bool stop = false;
    int error = MAPA_OK;
    std::string error_msg;

    // worker-only state
    std::multimap<int64_t, int64_t> expiries;      // due time -> job (lifetimes)
    std::multimap<int64_t, Pending> departs;       // explicit DEPART events by time
    bool blocked = false;                          // head of the queue waits for a departure
    int32_t window = 0;                            // requests admitted per round (adaptive)
    std::unordered_map<int64_t, Job> live;         // committed jobs
    uint32_t occ[MAPA_MASK_WORDS] = {};            // host copy of the device occupancy
    std::atomic<uint64_t> rounds{0}, decisions{0}, conflicts{0};

    // device and pinned buffers, sized for max_batch
    mapa_request *d_reqs = nullptr;
    mapa_result *d_out = nullptr;
    int32_t *d_conflict = nullptr;
    int64_t *d_jobs = nullptr;
    mapa_request *h_reqs = nullptr;
    mapa_result *h_out = nullptr;
    int32_t *h_conflict = nullptr;
    int64_t *h_jobs = nullptr;
    int32_t jobs_cap = 0;

    int64_t now_ns() const {
        return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
    }
};

namespace {

void finish(mapa_server srv, std::vector<mapa_served> &out) {
    if (out.empty()) return;
    std::lock_guard<std::mutex> lock(srv->mu);
    for (auto &d : out) srv->done.push_back(d);
    srv->finished += out.size();
    out.clear();
    srv->cv_done.notify_all();
}

void fail(mapa_server srv, int code, const std::string &msg) {
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->error == MAPA_OK) {
        srv->error = code;
        srv->error_msg = msg;
    }
    srv->stop = true;
    srv->cv_done.notify_all();
}

// Requests a serving chain decides between two host checks of its FIFO-wait flag.
constexpr int32_t kChainSegment = 32;
// Rounds smaller than this skip the parallel pass and go straight to the chain.
constexpr int32_t kSpeculateMin = 16;

mapa_served served_of(const Pending &p, int64_t done_ns, const uint32_t *snap) {
    mapa_served s;
    memset(&s, 0, sizeof(s));
    s.request_id = p.ev.request_id;
    s.arrive_ns = p.ev.at_ns;
    s.done_ns = done_ns;
    s.kind = p.ev.kind;
    s.rounds = p.rounds;
    if (snap) memcpy(s.snapshot, snap, sizeof(s.snapshot));
    return s;
}

// Releases `jobs` on the device (one kernel) and in the host copy.
int release_jobs(mapa_server srv, const std::vector<int64_t> &jobs, std::string *err) {
    if (jobs.empty()) return MAPA_OK;
    mapa_ctx ctx = srv->ctx;
    const mapa::TopoDevice &t = ctx->topos[srv->topo_id].dev;
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    if (static_cast<int32_t>(jobs.size()) > srv->jobs_cap) {
        cudaFree(srv->d_jobs);
        cudaFreeHost(srv->h_jobs);
        srv->d_jobs = nullptr;
        srv->h_jobs = nullptr;
        const int32_t cap = std::max<int32_t>(static_cast<int32_t>(jobs.size()), 1024);
        if (cudaMalloc(&srv->d_jobs, sizeof(int64_t) * cap) != cudaSuccess ||
            cudaMallocHost(&srv->h_jobs, sizeof(int64_t) * cap) != cudaSuccess) {
            if (err) *err = "cannot allocate the release list";
            return MAPA_E_NOMEM;
        }
        srv->jobs_cap = cap;
    }
    cudaStreamSynchronize(st);  // the pinned list may still be read by an earlier release
    for (size_t i = 0; i < jobs.size(); ++i) {
        srv->h_jobs[i] = jobs[i];
        auto it = srv->live.find(jobs[i]);
        if (it == srv->live.end()) continue;
        for (int v : it->second.verts) srv->occ[v >> 5] &= ~(1u << (v & 31));
        srv->live.erase(it);
    }
    if (cudaMemcpyAsync(srv->d_jobs, srv->h_jobs, sizeof(int64_t) * jobs.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
        if (err) *err = "release list copy failed";
        return MAPA_E_CUDA;
    }
    return mapa::engine_release_many(ctx->engine, t, srv->d_jobs, static_cast<int32_t>(jobs.size()), err);
}

void add_mask(uint32_t *m, const mapa_result &r) {
    for (int j = 0; j < r.k; ++j) m[r.verts[j] >> 5] |= 1u << (r.verts[j] & 31);
}

// One round:
//   1. every admitted request is decided in one parallel batch against the
//      same occupancy snapshot;
//   2. the longest prefix, in arrival order, of decisions that do not overlap
//      is committed on the device;
//   3. the requests from the first overlap on are decided again, in arrival
//      order, as a device chain against the live occupancy (each committed
//      before the next is decided), so none is decided more than twice.
//   With FIFO waiting, the first request that does not fit stops the round:
//   it and every later request go back to the head of the queue.
// Every decision equals deciding that request alone with busy = the
// occupancy it was decided against, which is recorded in its snapshot.
int decide_round(mapa_server srv, std::vector<Pending> &round, std::vector<mapa_served> &out, std::string *err) {
    mapa_ctx ctx = srv->ctx;
    const mapa::TopoDevice &t = ctx->topos[srv->topo_id].dev;
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    const int32_t n = static_cast<int32_t>(round.size());
    uint32_t snap[MAPA_MASK_WORDS];
    memcpy(snap, srv->occ, sizeof(snap));
    int rc = MAPA_OK;
    const bool speculate = n >= kSpeculateMin;
    if (speculate) {
        for (int32_t i = 0; i < n; ++i) {
            mapa_request &q = srv->h_reqs[i];
            memset(&q, 0, sizeof(q));
            q.pattern_id = round[i].ev.pattern_id;
            q.policy = round[i].ev.policy;
            memcpy(q.busy, snap, sizeof(snap));
            round[i].rounds += 1;
        }
        if (cudaMemcpyAsync(srv->d_reqs, srv->h_reqs, sizeof(mapa_request) * n, cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
            if (err) *err = "request copy failed";
            return MAPA_E_CUDA;
        }
        rc = mapa::engine_run_batch(ctx->engine, t, ctx->pattern_args, n, srv->d_reqs, srv->d_out, false, err);
        if (rc != MAPA_OK) return rc;
        rc = mapa::engine_commit_round(ctx->engine, t, srv->d_out, n, srv->d_conflict, srv->fifo_wait, err);
        if (rc != MAPA_OK) return rc;
        if (cudaMemcpyAsync(srv->h_out, srv->d_out, sizeof(mapa_result) * n, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(srv->h_conflict, srv->d_conflict, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            if (err) *err = "round result copy failed";
            return MAPA_E_CUDA;
        }
    } else {
        // a small round goes straight to the chain (exact FIFO order)
        for (int32_t i = 0; i < n; ++i) {
            memset(&srv->h_out[i], 0, sizeof(mapa_result));
            srv->h_conflict[i] = 1;
        }
    }
    std::vector<mapa_result> res(srv->h_out, srv->h_out + n);
    std::vector<uint32_t> snaps(static_cast<size_t>(n) * MAPA_MASK_WORDS);
    uint32_t cur[MAPA_MASK_WORDS];
    memcpy(cur, snap, sizeof(cur));
    std::vector<int32_t> chain, chain_pids;
    std::vector<uint8_t> chain_bounded;
    std::vector<char> deferred(n, 0);
    for (int32_t i = 0; i < n; ++i) {
        memcpy(&snaps[static_cast<size_t>(i) * MAPA_MASK_WORDS], snap, sizeof(snap));
        if (srv->h_conflict[i] == 1) {
            chain.push_back(i);
            chain_pids.push_back(round[i].ev.pattern_id);
            chain_bounded.push_back(static_cast<uint8_t>(
                (round[i].ev.policy.mode == MAPA_MODE_BOUNDED ? mapa::kKindBounded : 0) |
                ((round[i].ev.policy.flags & MAPA_POLICY_BW_SENSITIVE) ? mapa::kKindSensitive : 0)));
        } else if (srv->h_conflict[i] == 2) {
            deferred[i] = 1;
        } else if (placed(res[i].status)) {
            add_mask(cur, res[i]);
        }
    }
    // The chain runs in segments; after one that ended waiting (FIFO), the
    // rest of the chain waits too and is not decided.
    const int32_t m_all = static_cast<int32_t>(chain.size());
    bool chain_blocked = false;
    for (int32_t c0 = 0; c0 < m_all; c0 += kChainSegment) {
        const int32_t m = std::min(kChainSegment, m_all - c0);
        if (chain_blocked) {
            for (int32_t j = 0; j < m; ++j) deferred[chain[c0 + j]] = 1;
            continue;
        }
        for (int32_t j = 0; j < m; ++j) {
            mapa_request &q = srv->h_reqs[j];
            memset(&q, 0, sizeof(q));
            q.pattern_id = round[chain[c0 + j]].ev.pattern_id;
            q.policy = round[chain[c0 + j]].ev.policy;
            round[chain[c0 + j]].rounds += 1;
        }
        if (cudaMemcpyAsync(srv->d_reqs, srv->h_reqs, sizeof(mapa_request) * m, cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
            if (err) *err = "request copy failed";
            return MAPA_E_CUDA;
        }
        rc = mapa::engine_run_chain(ctx->engine, t, ctx->pattern_args, m, chain_pids.data() + c0,
                                    chain_bounded.data() + c0, srv->d_reqs, srv->d_out, srv->fifo_wait, srv->h_out,
                                    err);
        if (rc != MAPA_OK) return rc;
        for (int32_t j = 0; j < m; ++j) {
            const int32_t i = chain[c0 + j];
            memcpy(&snaps[static_cast<size_t>(i) * MAPA_MASK_WORDS], cur, sizeof(cur));
            res[i] = srv->h_out[j];
            if (res[i].reserved == mapa::kDeferred) {
                res[i].reserved = 0;
                deferred[i] = 1;
                chain_blocked = true;
                continue;
            }
            if (placed(res[i].status)) add_mask(cur, res[i]);
        }
        if (speculate) srv->conflicts += static_cast<uint64_t>(m);  // decided again after an overlap
    }
    const int64_t done_ns = srv->now_ns();
    srv->rounds += 1;
    // FIFO waiting: the first request that did not fit and every later one go
    // back to the head of the queue.  A request that did not fit although the
    // server holds nothing that could be released gets its MAPA_NO_FIT now.
    std::vector<Pending> requeue;
    bool final_no_fit_done = false;
    for (int32_t i = 0; i < n; ++i) {
        if (!deferred[i]) continue;
        bool committed_this_round = false;
        for (int32_t j = 0; j < n; ++j)
            if (!deferred[j] && placed(res[j].status) && res[j].job_id > 0) committed_this_round = true;
        const bool nothing_to_release = srv->live.empty() && srv->expiries.empty() && srv->departs.empty() &&
                                        !committed_this_round;
        if (!final_no_fit_done && res[i].status == MAPA_NO_FIT && nothing_to_release) {
            deferred[i] = 0;  // answered: it cannot fit on what the server can free
            final_no_fit_done = true;
            continue;
        }
        requeue.push_back(round[i]);
    }
    for (int32_t i = 0; i < n; ++i) {
        if (deferred[i]) continue;
        mapa_served s = served_of(round[i], done_ns, &snaps[static_cast<size_t>(i) * MAPA_MASK_WORDS]);
        s.result = res[i];
        out.push_back(s);
        srv->decisions += 1;
        if (placed(res[i].status) && res[i].job_id > 0) {
            Job job;
            for (int j = 0; j < res[i].k; ++j) job.verts.push_back(res[i].verts[j]);
            srv->live.emplace(res[i].job_id, std::move(job));
            if (round[i].ev.lifetime_ns > 0) srv->expiries.emplace(done_ns + round[i].ev.lifetime_ns, res[i].job_id);
        }
    }
    // Admission window: a round whose decisions all committed from the
    // parallel pass doubles it; one that hit an overlap or had to wait
    // shrinks it towards twice what it committed, so contended stretches
    // spend little on speculative decisions that the chain redoes anyway.
    int32_t prefix = 0;  // decisions the parallel pass committed
    for (int32_t i = 0; i < n; ++i)
        if (speculate && srv->h_conflict[i] == 0) ++prefix;
    if ((!speculate || chain.empty()) && requeue.empty())
        srv->window = std::min(srv->max_batch, std::max(srv->window, 1) * 2);
    else if (speculate)
        srv->window = std::max(std::min(srv->max_batch, 8), std::min(srv->max_batch, 2 * prefix));
    memcpy(srv->occ, cur, sizeof(cur));
    if (!requeue.empty()) {
        std::lock_guard<std::mutex> lock(srv->mu);
        for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) srv->incoming.push_front(*it);
        srv->blocked = !final_no_fit_done;
    }
    return MAPA_OK;
}

void worker_loop(mapa_server srv) {
    if (cudaSetDevice(srv->ctx->device) != cudaSuccess) {
        fail(srv, MAPA_E_CUDA, "cudaSetDevice failed in the serving thread");
        return;
    }
    std::vector<mapa_served> out;
    std::vector<Pending> round;
    std::vector<int64_t> departing;
    std::string err;
    for (;;) {
        round.clear();
        departing.clear();
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            if (srv->stop) return;
            const int64_t now = srv->now_ns();
            // 1. departures that are due: lifetimes that ran out, then DEPART events
            while (!srv->expiries.empty() && srv->expiries.begin()->first <= now) {
                departing.push_back(srv->expiries.begin()->second);
                srv->expiries.erase(srv->expiries.begin());
            }
            while (!srv->departs.empty() && srv->departs.begin()->first <= now) {
                const Pending p = srv->departs.begin()->second;
                srv->departs.erase(srv->departs.begin());
                const int64_t job = p.ev.job_id;
                const bool known = srv->live.count(job) &&
                                   std::find(departing.begin(), departing.end(), job) == departing.end();
                mapa_served d = served_of(p, now, nullptr);
                d.result.status = known ? MAPA_OK : MAPA_E_STATE;
                out.push_back(d);
                if (!known) continue;
                departing.push_back(job);
                for (auto it = srv->expiries.begin(); it != srv->expiries.end(); ++it)
                    if (it->second == job) {
                        srv->expiries.erase(it);
                        break;
                    }
            }
            if (!departing.empty()) srv->blocked = false;
            // 2. arrivals in order, unless the head of the queue waits for a departure
            if (!srv->blocked) {
                while (!srv->incoming.empty() && srv->incoming.front().ev.at_ns <= now &&
                       static_cast<int32_t>(round.size()) < srv->window) {
                    round.push_back(srv->incoming.front());
                    srv->incoming.pop_front();
                }
            }
            if (round.empty() && departing.empty() && out.empty()) {
                int64_t next_due = -1;
                if (!srv->blocked && !srv->incoming.empty()) next_due = srv->incoming.front().ev.at_ns;
                if (!srv->expiries.empty()) {
                    const int64_t e = srv->expiries.begin()->first;
                    next_due = next_due < 0 ? e : std::min(next_due, e);
                }
                if (!srv->departs.empty()) {
                    const int64_t e = srv->departs.begin()->first;
                    next_due = next_due < 0 ? e : std::min(next_due, e);
                }
                if (next_due < 0)
                    srv->cv_work.wait(lock);
                else if (next_due > now)
                    srv->cv_work.wait_until(lock, srv->t0 + std::chrono::nanoseconds(next_due));
                continue;
            }
        }
        int rc = release_jobs(srv, departing, &err);
        if (rc == MAPA_OK && !round.empty()) rc = decide_round(srv, round, out, &err);
        if (rc != MAPA_OK) {
            fail(srv, rc, err);
            return;
        }
        finish(srv, out);
    }
}

}  // namespace

extern "C" {

int mapa_serve_open(mapa_ctx ctx, int32_t topo_id, int32_t max_batch, uint32_t flags, mapa_server *out) {
    if (!ctx || !out) return MAPA_E_INVALID;
    if (flags & ~MAPA_SERVE_REJECT) {
        ctx->last_error = "unknown serving flags";
        return MAPA_E_INVALID;
    }
    *out = nullptr;
    if (topo_id < 0 || topo_id >= static_cast<int32_t>(ctx->topos.size()) || !ctx->topos[topo_id].live) {
        ctx->last_error = "unknown topology id";
        return MAPA_E_INVALID;
    }
    if (max_batch < 1 || max_batch > (1 << 20)) {
        ctx->last_error = "max_batch must be in 1..2^20";
        return MAPA_E_RANGE;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        ctx->last_error = "cudaSetDevice failed";
        return MAPA_E_CUDA;
    }
    mapa_server srv = new mapa_server_s();
    srv->ctx = ctx;
    srv->topo_id = topo_id;
    srv->max_batch = max_batch;
    srv->fifo_wait = (flags & MAPA_SERVE_REJECT) == 0;
    srv->window = max_batch;
    const size_t nb = static_cast<size_t>(max_batch);
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    if (cudaMalloc(&srv->d_reqs, sizeof(mapa_request) * nb) != cudaSuccess ||
        cudaMalloc(&srv->d_out, sizeof(mapa_result) * nb) != cudaSuccess ||
        cudaMalloc(&srv->d_conflict, sizeof(int32_t) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_reqs, sizeof(mapa_request) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_out, sizeof(mapa_result) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_conflict, sizeof(int32_t) * nb) != cudaSuccess ||
        cudaMemcpyAsync(srv->occ, ctx->topos[topo_id].dev.occupancy, sizeof(srv->occ), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        ctx->last_error = "cannot allocate the server's buffers";
        mapa_serve_close(srv);
        return MAPA_E_NOMEM;
    }
    srv->t0 = Clock::now();
    srv->worker = std::thread(worker_loop, srv);
    *out = srv;
    return MAPA_OK;
}

int mapa_serve_submit(mapa_server srv, const mapa_event *events, int32_t n) {
    if (!srv || n < 0 || (n > 0 && !events)) return MAPA_E_INVALID;
    for (int32_t i = 0; i < n; ++i) {
        if (events[i].kind != MAPA_EVENT_ARRIVE && events[i].kind != MAPA_EVENT_DEPART) return MAPA_E_INVALID;
        if (i > 0 && events[i].at_ns < events[i - 1].at_ns) return MAPA_E_INVALID;
    }
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stop) return srv->error != MAPA_OK ? srv->error : MAPA_E_STATE;
    if (n > 0 && !srv->incoming.empty() && events[0].kind == MAPA_EVENT_ARRIVE &&
        events[0].at_ns < srv->incoming.back().ev.at_ns)
        return MAPA_E_INVALID;
    for (int32_t i = 0; i < n; ++i) {
        Pending p;
        p.ev = events[i];
        if (p.ev.kind == MAPA_EVENT_DEPART)
            srv->departs.emplace(p.ev.at_ns, p);
        else
            srv->incoming.push_back(p);
    }
    srv->submitted += static_cast<uint64_t>(n);
    srv->cv_work.notify_one();
    return MAPA_OK;
}

int mapa_serve_poll(mapa_server srv, mapa_served *out, int32_t max, int32_t *got, int32_t timeout_ms) {
    if (!srv || !got || max < 0 || (max > 0 && !out)) return MAPA_E_INVALID;
    std::unique_lock<std::mutex> lock(srv->mu);
    if (timeout_ms > 0 && srv->done.empty())
        srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                              [&] { return !srv->done.empty() || srv->stop; });
    int32_t k = 0;
    while (k < max && !srv->done.empty()) {
        out[k++] = srv->done.front();
        srv->done.pop_front();
    }
    *got = k;
    return srv->error;
}

int mapa_serve_drain(mapa_server srv, int32_t timeout_ms) {
    if (!srv) return MAPA_E_INVALID;
    std::unique_lock<std::mutex> lock(srv->mu);
    auto ready = [&] { return srv->finished >= srv->submitted || srv->stop; };
    if (timeout_ms > 0) {
        if (!srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) return MAPA_E_TIMEOUT;
    } else {
        srv->cv_done.wait(lock, ready);
    }
    return srv->error;
}

int mapa_serve_counters(mapa_server srv, uint64_t *rounds, uint64_t *decisions, uint64_t *conflicts) {
    if (!srv) return MAPA_E_INVALID;
    std::lock_guard<std::mutex> lock(srv->mu);
    if (rounds) *rounds = srv->rounds.load();
    if (decisions) *decisions = srv->decisions.load();
    if (conflicts) *conflicts = srv->conflicts.load();
    return MAPA_OK;
}

int mapa_serve_close(mapa_server srv) {
    if (!srv) return MAPA_E_INVALID;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    const int rc = srv->error;
    if (rc != MAPA_OK && srv->ctx) srv->ctx->last_error = srv->error_msg;
    if (srv->ctx) cudaStreamSynchronize(mapa::engine_stream(srv->ctx->engine));
    cudaFree(srv->d_reqs);
    cudaFree(srv->d_out);
    cudaFree(srv->d_conflict);
    cudaFree(srv->d_jobs);
    if (srv->h_reqs) cudaFreeHost(srv->h_reqs);
    if (srv->h_out) cudaFreeHost(srv->h_out);
    if (srv->h_conflict) cudaFreeHost(srv->h_conflict);
    if (srv->h_jobs) cudaFreeHost(srv->h_jobs);
    delete srv;
    return rc;
}

}  // extern "C"
