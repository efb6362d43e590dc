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
// The occupancy lives on the device, and so do the lifetimes: a commit
// stamps its vertices with the device clock plus the job's lifetime, and
// every chain step frees the vertices whose time has passed before the next
// decision, logging what it freed.  The worker keeps a host copy of the
// occupancy that it updates from the committed vertex sets and that log; its
// own schedule of lifetimes only tells it when to look (and releases a job
// itself should the device not have done so a millisecond later).
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
    std::multimap<int64_t, int64_t> expiries;      // host time a lifetime ends -> job (when to look)
    std::unordered_map<int64_t, std::multimap<int64_t, int64_t>::iterator> expiry_of;  // job -> its entry
    std::multimap<int64_t, Pending> departs;       // explicit DEPART events by time
    bool blocked = false;                          // head of the queue waits for a departure
    int32_t window = 0;                            // requests admitted per round (adaptive)
    int32_t spec_skip = 0;                         // large rounds left that go straight to the chain
    int32_t deg_max = 0;                           // largest vertex degree of the topology
    int32_t spec_backoff = 0;                      // their number after the next parallel pass that fails
    double chain_ns = 100000.0;                    // device chain time per decision (running mean)
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
    // device lifetimes: per request of a call, and the log of freed vertices
    int64_t *d_life = nullptr, *h_life = nullptr;
    int64_t *d_log_job = nullptr, *h_log_job = nullptr;
    int32_t *d_log_pos = nullptr, *h_log_pos = nullptr;
    uint32_t *d_log_n = nullptr, *h_log_n = nullptr;

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

// Longest run of requests a serving chain decides between two host checks
// of its FIFO-wait flag; each segment's decisions are published when it
// ends, so a round of n requests runs segments of n/4 (1..8): a small round
// publishes every decision at once, a long one saves host round trips.
constexpr int32_t kChainSegment = 8;
// Rounds smaller than this skip the parallel pass and go straight to the chain.
constexpr int32_t kSpeculateMin = 16;
// Requests admitted per round while the parallel pass is backed off.
constexpr int32_t kChainRound = 64;
// Longest back-off of the parallel pass, in rounds.
constexpr int32_t kMaxBackoff = 64;
// Entries of the log of vertices freed on the device: one chain segment or
// one expiry pass frees each vertex at most once per step.
constexpr uint32_t kLogCap = 256 * (kChainSegment + 2);
// Entries read back with the log's count (more take a second copy).
constexpr uint32_t kLogFirst = 256;

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

// Frontier memory one request of the pattern can hold under the context's
// work budget B (0 when there is none): it stores at most B partial matches
// before it is cut, and the level that crosses B holds at most (1 + the
// largest degree) x B entries, each 8 + 4 W + 4 ceil(k/4) bytes (score,
// request, free-set words, tuple words).
uint64_t frontier_estimate(mapa_server srv, int32_t pattern_id) {
    mapa_ctx ctx = srv->ctx;
    const uint64_t B = mapa::engine_work_budget(ctx->engine);
    if (B == 0 || pattern_id < 0 || pattern_id >= static_cast<int32_t>(ctx->pattern_args.size())) return 0;
    const int W = ctx->topos[srv->topo_id].dev.W;
    const int k = ctx->pattern_args[pattern_id].k;
    const uint64_t entry = 8 + 4 * static_cast<uint64_t>(W) + 4 * static_cast<uint64_t>((k + 3) / 4);
    return (1 + static_cast<uint64_t>(srv->deg_max)) * B * entry;
}

// Requests a round admits: the window, or while the parallel pass is backed
// off a whole chain of up to kChainRound.
int32_t admit_limit(mapa_server srv) {
    return srv->spec_skip > 0 ? std::max(srv->window, std::min(srv->max_batch, kChainRound)) : srv->window;
}

// Moves the requests that have arrived by `now` from the queue into round,
// in order, while the round holds fewer than limit requests and, under a
// work budget, while the round's requests can all hold their largest
// frontier at once (mem: the round's frontier bytes so far).  The caller
// holds srv->mu.
void admit_arrivals(mapa_server srv, std::vector<Pending> &round, int32_t limit, int64_t now, uint64_t &mem) {
    const uint64_t mem_cap = mapa::engine_frontier_budget(srv->ctx->engine);
    while (!srv->incoming.empty() && srv->incoming.front().ev.at_ns <= now &&
           static_cast<int32_t>(round.size()) < limit) {
        const uint64_t est = frontier_estimate(srv, srv->incoming.front().ev.pattern_id);
        if (!round.empty() && mem + est > mem_cap) break;
        mem += est;
        round.push_back(srv->incoming.front());
        srv->incoming.pop_front();
    }
}

mapa::ServeLife life_args(mapa_server srv) {
    mapa::ServeLife lf;
    lf.life = srv->d_life;
    lf.log_job = srv->d_log_job;
    lf.log_pos = srv->d_log_pos;
    lf.n_log = srv->d_log_n;
    lf.cap = kLogCap;
    return lf;
}

// Empties the device log (enqueued).
int clear_log(mapa_server srv, std::string *err) {
    if (cudaMemsetAsync(srv->d_log_n, 0, sizeof(uint32_t), mapa::engine_stream(srv->ctx->engine)) != cudaSuccess) {
        if (err) *err = "log reset failed";
        return MAPA_E_CUDA;
    }
    return MAPA_OK;
}

// Reads the device log back (synchronises the stream): (position, job) pairs
// in the order the device wrote them.  copied: the count and the first
// kLogFirst entries are already in the pinned host copies.
int read_log(mapa_server srv, std::vector<std::pair<int32_t, int64_t>> &entries, std::string *err,
             bool copied = false) {
    cudaStream_t st = mapa::engine_stream(srv->ctx->engine);
    entries.clear();
    if (!copied &&
        (cudaMemcpyAsync(srv->h_log_n, srv->d_log_n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaMemcpyAsync(srv->h_log_job, srv->d_log_job, sizeof(int64_t) * kLogFirst, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaMemcpyAsync(srv->h_log_pos, srv->d_log_pos, sizeof(int32_t) * kLogFirst, cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess)) {
        if (err) *err = "log copy failed";
        return MAPA_E_CUDA;
    }
    const uint32_t n = *srv->h_log_n;
    if (n > kLogCap) {
        if (err) *err = "the device log of freed vertices overflowed";
        return MAPA_E_STATE;
    }
    if (n > kLogFirst) {
        const size_t rest = n - kLogFirst;
        if (cudaMemcpyAsync(srv->h_log_job + kLogFirst, srv->d_log_job + kLogFirst, sizeof(int64_t) * rest,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(srv->h_log_pos + kLogFirst, srv->d_log_pos + kLogFirst, sizeof(int32_t) * rest,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            if (err) *err = "log copy failed";
            return MAPA_E_CUDA;
        }
    }
    for (uint32_t i = 0; i < n; ++i) entries.emplace_back(srv->h_log_pos[i], srv->h_log_job[i]);
    return MAPA_OK;
}

// A job the device freed: forget it and clear its vertices from mask m.
// Returns false when the job is not (or no longer) live.
bool forget_job(mapa_server srv, int64_t job, uint32_t *m) {
    auto it = srv->live.find(job);
    if (it == srv->live.end()) return false;
    for (int v : it->second.verts) m[v >> 5] &= ~(1u << (v & 31));
    srv->live.erase(it);
    auto e = srv->expiry_of.find(job);
    if (e != srv->expiry_of.end()) {
        srv->expiries.erase(e->second);
        srv->expiry_of.erase(e);
    }
    return true;
}

// Frees on the device every vertex whose lifetime has ended and applies the
// log to the host state (host mask m); sets *freed when anything was freed.
int expire_on_device(mapa_server srv, uint32_t *m, bool *freed, std::string *err) {
    mapa_ctx ctx = srv->ctx;
    const mapa::TopoDevice &t = ctx->topos[srv->topo_id].dev;
    int rc = clear_log(srv, err);
    if (rc == MAPA_OK) rc = mapa::engine_expire(ctx->engine, t, life_args(srv), err);
    std::vector<std::pair<int32_t, int64_t>> log;
    if (rc == MAPA_OK) rc = read_log(srv, log, err);
    if (rc != MAPA_OK) return rc;
    for (const auto &en : log)
        if (forget_job(srv, en.second, m) && freed) *freed = true;
    return MAPA_OK;
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
    // n grows when requests that arrive during the round's chain join it;
    // n0 is the round as admitted (the parallel pass's requests)
    int32_t n = static_cast<int32_t>(round.size());
    const int32_t n0 = n;
    // lifetimes that ended before the round: freed before its snapshot (the
    // device ends a lifetime no later than the host schedule says)
    int rc = MAPA_OK;
    if (!srv->expiries.empty() && srv->expiries.begin()->first <= srv->now_ns())
        rc = expire_on_device(srv, srv->occ, nullptr, err);
    if (rc != MAPA_OK) return rc;
    uint32_t snap[MAPA_MASK_WORDS];
    memcpy(snap, srv->occ, sizeof(snap));
    // The parallel pass pays when most of its decisions commit; after one
    // where fewer than half did, the next large rounds skip it (exponential
    // back-off), since the chain redoes what overlaps anyway.
    // It also pays only when requests arrive faster than the chain decides
    // them (otherwise the chain keeps up, and publishes each decision sooner).
    const double gap = n > 1 ? static_cast<double>(round.back().ev.at_ns - round.front().ev.at_ns) / (n - 1) : 0.0;
    const bool speculate = n >= kSpeculateMin && srv->spec_skip == 0 && gap < srv->chain_ns;
    if (n >= kSpeculateMin && srv->spec_skip > 0) --srv->spec_skip;
    std::vector<int64_t> done_at(n, -1);
    // jobs of this round that the device freed before they were published
    std::unordered_map<int64_t, int32_t> round_job;  // job -> request
    std::vector<char> gone(n, 0);
    // Publishes the decisions in idx that are final (not deferred, not yet
    // out); the host schedule looks for a committed job's end one lifetime
    // after its publication (the device ends it one lifetime after commit).
    auto publish = [&](const std::vector<int32_t> &idx, const std::vector<mapa_result> &res,
                       const std::vector<uint32_t> &snaps, const std::vector<char> &deferred) {
        const int64_t now = srv->now_ns();
        for (const int32_t i : idx) {
            if (deferred[i] || done_at[i] >= 0) continue;
            done_at[i] = now;
            mapa_served sv = served_of(round[i], now, &snaps[static_cast<size_t>(i) * MAPA_MASK_WORDS]);
            sv.result = res[i];
            out.push_back(sv);
            srv->decisions += 1;
            if (placed(res[i].status) && res[i].job_id > 0 && !gone[i]) {
                Job job;
                for (int j = 0; j < res[i].k; ++j) job.verts.push_back(res[i].verts[j]);
                srv->live.emplace(res[i].job_id, std::move(job));
                if (round[i].ev.lifetime_ns > 0)
                    srv->expiry_of[res[i].job_id] =
                        srv->expiries.emplace(now + round[i].ev.lifetime_ns, res[i].job_id);
            }
        }
        finish(srv, out);
    };
    if (speculate) {
        for (int32_t i = 0; i < n; ++i) {
            mapa_request &q = srv->h_reqs[i];
            memset(&q, 0, sizeof(q));
            q.pattern_id = round[i].ev.pattern_id;
            q.policy = round[i].ev.policy;
            memcpy(q.busy, snap, sizeof(snap));
            srv->h_life[i] = round[i].ev.lifetime_ns;
            round[i].rounds += 1;
        }
        if (cudaMemcpyAsync(srv->d_reqs, srv->h_reqs, sizeof(mapa_request) * n, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(srv->d_life, srv->h_life, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
            if (err) *err = "request copy failed";
            return MAPA_E_CUDA;
        }
        rc = mapa::engine_run_batch(ctx->engine, t, ctx->pattern_args, n, srv->d_reqs, srv->d_out, false, err);
        if (rc != MAPA_OK) return rc;
        const mapa::ServeLife lf = life_args(srv);
        rc = mapa::engine_commit_round(ctx->engine, t, srv->d_out, n, srv->d_conflict, srv->fifo_wait, &lf, err);
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
    std::vector<int32_t> first_pass;
    for (int32_t i = 0; i < n; ++i) {
        memcpy(&snaps[static_cast<size_t>(i) * MAPA_MASK_WORDS], snap, sizeof(snap));
        if (speculate && srv->h_conflict[i] == 0) first_pass.push_back(i);
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
    // what the parallel pass committed (and its no-fits) is final now
    if (!first_pass.empty()) publish(first_pass, res, snaps, deferred);
    // The chain runs in segments; after one that ended waiting (FIFO), the
    // rest of the chain waits too and is not decided.
    const int32_t seg = std::max(1, std::min(kChainSegment, n / 4));
    bool chain_blocked = false;
    // Continuous batching: requests that arrive while the chain runs join
    // its end between segments (they are later than every request of the
    // round, so arrival order holds), up to the round's admission limit and
    // at most kChainRound requests unless the round began larger.
    const int32_t grow_limit = std::min(admit_limit(srv), std::max(n0, kChainRound));
    uint64_t round_mem = 0;
    for (const Pending &p : round) round_mem += frontier_estimate(srv, p.ev.pattern_id);
    auto join_arrivals = [&]() {
        const size_t before = round.size();
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            if (srv->stop) return;
            admit_arrivals(srv, round, grow_limit, srv->now_ns(), round_mem);
        }
        for (size_t i = before; i < round.size(); ++i) {
            chain.push_back(static_cast<int32_t>(i));
            chain_pids.push_back(round[i].ev.pattern_id);
            chain_bounded.push_back(static_cast<uint8_t>(
                (round[i].ev.policy.mode == MAPA_MODE_BOUNDED ? mapa::kKindBounded : 0) |
                ((round[i].ev.policy.flags & MAPA_POLICY_BW_SENSITIVE) ? mapa::kKindSensitive : 0)));
        }
        n = static_cast<int32_t>(round.size());
        res.resize(n);
        snaps.resize(static_cast<size_t>(n) * MAPA_MASK_WORDS, 0u);
        deferred.resize(n, 0);
        done_at.resize(n, -1);
        gone.resize(n, 0);
    };
    for (int32_t c0 = 0;; c0 += seg) {
        if (!chain_blocked) join_arrivals();
        const int32_t m_all = static_cast<int32_t>(chain.size());
        if (c0 >= m_all) break;
        const int32_t m = std::min(seg, m_all - c0);
        if (chain_blocked) {
            for (int32_t j = 0; j < m; ++j) deferred[chain[c0 + j]] = 1;
            continue;
        }
        for (int32_t j = 0; j < m; ++j) {
            mapa_request &q = srv->h_reqs[j];
            memset(&q, 0, sizeof(q));
            q.pattern_id = round[chain[c0 + j]].ev.pattern_id;
            q.policy = round[chain[c0 + j]].ev.policy;
            srv->h_life[j] = round[chain[c0 + j]].ev.lifetime_ns;
            round[chain[c0 + j]].rounds += 1;
        }
        if (cudaMemcpyAsync(srv->d_reqs, srv->h_reqs, sizeof(mapa_request) * m, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(srv->d_life, srv->h_life, sizeof(int64_t) * m, cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
            if (err) *err = "request copy failed";
            return MAPA_E_CUDA;
        }
        // each step frees the lifetimes that ended before the next decision
        mapa::ServeLife lf = life_args(srv);
        lf.host_n_log = srv->h_log_n;
        lf.host_log_job = srv->h_log_job;
        lf.host_log_pos = srv->h_log_pos;
        lf.host_first = kLogFirst;
        const int64_t t_seg0 = srv->now_ns();
        rc = clear_log(srv, err);
        if (rc == MAPA_OK)
            rc = mapa::engine_run_chain(ctx->engine, t, ctx->pattern_args, m, chain_pids.data() + c0,
                                        chain_bounded.data() + c0, srv->d_reqs, srv->d_out, srv->fifo_wait,
                                        srv->h_out, &lf, err);
        std::vector<std::pair<int32_t, int64_t>> log;
        if (rc == MAPA_OK) rc = read_log(srv, log, err, true);
        if (rc != MAPA_OK) return rc;
        const int64_t t_seg = srv->now_ns();
        srv->chain_ns = 0.9 * srv->chain_ns + 0.1 * static_cast<double>(t_seg - t_seg0) / m;
        // replay the segment on the host mask in device order: what was
        // freed before decision j, then decision j
        size_t li = 0;
        auto freed_before = [&](int32_t pos) {
            for (; li < log.size() && log[li].first <= pos; ++li) {
                const int64_t job = log[li].second;
                if (forget_job(srv, job, cur)) continue;
                auto rj = round_job.find(job);  // committed earlier in this round, not yet published
                if (rj == round_job.end() || gone[rj->second]) continue;
                gone[rj->second] = 1;
                const mapa_result &r = res[rj->second];
                for (int q = 0; q < r.k; ++q) cur[r.verts[q] >> 5] &= ~(1u << (r.verts[q] & 31));
            }
        };
        for (int32_t j = 0; j < m; ++j) {
            const int32_t i = chain[c0 + j];
            freed_before(j);
            memcpy(&snaps[static_cast<size_t>(i) * MAPA_MASK_WORDS], cur, sizeof(cur));
            res[i] = srv->h_out[j];
            if (res[i].reserved == mapa::kDeferred) {
                res[i].reserved = 0;
                deferred[i] = 1;
                chain_blocked = true;
                continue;
            }
            if (placed(res[i].status)) {
                add_mask(cur, res[i]);
                if (res[i].job_id > 0) round_job[res[i].job_id] = i;
            }
        }
        freed_before(m);
        if (speculate)  // decided again after an overlap (not the requests that joined the chain)
            for (int32_t j = 0; j < m; ++j) srv->conflicts += chain[c0 + j] < n0 ? 1u : 0u;
        publish(std::vector<int32_t>(chain.begin() + c0, chain.begin() + c0 + m), res, snaps, deferred);
    }
    srv->rounds += 1;
    // FIFO waiting: the first request that did not fit and every later one go
    // back to the head of the queue.  A request that did not fit although the
    // server holds nothing that could be released gets its MAPA_NO_FIT now.
    std::vector<Pending> requeue;
    bool final_no_fit_done = false;
    for (int32_t i = 0; i < n; ++i) {
        if (!deferred[i]) continue;
        // the jobs this round committed are live by now (published), unless
        // the device already ended their lifetime
        const bool nothing_to_release = srv->live.empty() && srv->expiries.empty() && srv->departs.empty();
        if (!final_no_fit_done && res[i].status == MAPA_NO_FIT && nothing_to_release) {
            deferred[i] = 0;  // answered: it cannot fit on what the server can free
            final_no_fit_done = true;
            continue;
        }
        requeue.push_back(round[i]);
    }
    // the rest (no-fits answered at the end of the round)
    std::vector<int32_t> rest;
    for (int32_t i = 0; i < n; ++i)
        if (!deferred[i] && done_at[i] < 0) rest.push_back(i);
    if (!rest.empty()) publish(rest, res, snaps, deferred);
    // Admission window: a round whose decisions all committed from the
    // parallel pass doubles it; one that hit an overlap or had to wait
    // shrinks it towards twice what it committed, so contended stretches
    // spend little on speculative decisions that the chain redoes anyway.
    int32_t prefix = 0;  // decisions the parallel pass committed
    for (int32_t i = 0; i < n0; ++i)
        if (speculate && srv->h_conflict[i] == 0) ++prefix;
    if (speculate) {
        if (2 * prefix >= n0) {
            srv->spec_backoff = 0;
        } else {
            srv->spec_backoff = std::min(kMaxBackoff, std::max(1, 2 * srv->spec_backoff));
            srv->spec_skip = srv->spec_backoff;
        }
    }
    int32_t redone = 0;  // chain requests from the parallel pass
    for (const int32_t i : chain) redone += i < n0 ? 1 : 0;
    if ((!speculate || redone == 0) && requeue.empty())
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
    // Host time by which the device must have ended a lifetime before the
    // worker releases the job itself.
    constexpr int64_t kLifeGraceNs = 1000000;
    for (;;) {
        round.clear();
        departing.clear();
        // 1a. lifetimes: the device ends them by its clock; look when one is due
        bool due = false;
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            if (srv->stop) return;
            due = !srv->expiries.empty() && srv->expiries.begin()->first <= srv->now_ns();
        }
        if (due) {
            bool freed = false;
            int rc = expire_on_device(srv, srv->occ, &freed, &err);
            if (rc != MAPA_OK) {
                fail(srv, rc, err);
                return;
            }
            if (freed) {
                std::lock_guard<std::mutex> lock(srv->mu);
                srv->blocked = false;
            }
        }
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            if (srv->stop) return;
            const int64_t now = srv->now_ns();
            // 1b. a lifetime the device has not ended well after its time
            // (clocks that disagree), then DEPART events
            while (!srv->expiries.empty() && srv->expiries.begin()->first + kLifeGraceNs <= now) {
                const int64_t job = srv->expiries.begin()->second;
                departing.push_back(job);
                srv->expiry_of.erase(job);
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
                auto e = srv->expiry_of.find(job);
                if (e != srv->expiry_of.end()) {
                    srv->expiries.erase(e->second);
                    srv->expiry_of.erase(e);
                }
            }
            if (!departing.empty()) srv->blocked = false;
            // 2. arrivals in order, unless the head of the queue waits for a departure
            if (!srv->blocked) {
                uint64_t mem = 0;
                admit_arrivals(srv, round, admit_limit(srv), now, mem);
            }
            // a head that waits for accelerators while nothing can be released
            // any more is decided again (and answered MAPA_NO_FIT)
            if (srv->blocked && srv->live.empty() && srv->expiries.empty() && srv->departs.empty())
                srv->blocked = false;
            if (round.empty() && departing.empty() && out.empty()) {
                int64_t next_due = -1;
                if (!srv->blocked && !srv->incoming.empty()) next_due = srv->incoming.front().ev.at_ns;
                if (!srv->expiries.empty()) {
                    // a lifetime already looked for: wake at its grace time
                    int64_t e = srv->expiries.begin()->first;
                    if (e <= now) e += kLifeGraceNs;
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
    {
        const mapa::TopoEntry &te = ctx->topos[topo_id];
        const int32_t n = te.dev.n;
        for (int32_t a = 0; a < n; ++a) {
            int32_t d = 0;
            for (int32_t b = 0; b < n; ++b) d += (a != b && te.wm[static_cast<size_t>(a) * n + b] != 0) ? 1 : 0;
            srv->deg_max = std::max(srv->deg_max, d);
        }
    }
    const size_t nb = static_cast<size_t>(max_batch);
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    if (cudaMalloc(&srv->d_reqs, sizeof(mapa_request) * nb) != cudaSuccess ||
        cudaMalloc(&srv->d_out, sizeof(mapa_result) * nb) != cudaSuccess ||
        cudaMalloc(&srv->d_conflict, sizeof(int32_t) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_reqs, sizeof(mapa_request) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_out, sizeof(mapa_result) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_conflict, sizeof(int32_t) * nb) != cudaSuccess ||
        cudaMalloc(&srv->d_life, sizeof(int64_t) * nb) != cudaSuccess ||
        cudaMallocHost(&srv->h_life, sizeof(int64_t) * nb) != cudaSuccess ||
        cudaMalloc(&srv->d_log_job, sizeof(int64_t) * kLogCap) != cudaSuccess ||
        cudaMalloc(&srv->d_log_pos, sizeof(int32_t) * kLogCap) != cudaSuccess ||
        cudaMalloc(&srv->d_log_n, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&srv->h_log_job, sizeof(int64_t) * kLogCap) != cudaSuccess ||
        cudaMallocHost(&srv->h_log_pos, sizeof(int32_t) * kLogCap) != cudaSuccess ||
        cudaMallocHost(&srv->h_log_n, sizeof(uint32_t)) != cudaSuccess ||
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
    cudaFree(srv->d_life);
    cudaFree(srv->d_log_job);
    cudaFree(srv->d_log_pos);
    cudaFree(srv->d_log_n);
    if (srv->h_life) cudaFreeHost(srv->h_life);
    if (srv->h_log_job) cudaFreeHost(srv->h_log_job);
    if (srv->h_log_pos) cudaFreeHost(srv->h_log_pos);
    if (srv->h_log_n) cudaFreeHost(srv->h_log_n);
    if (srv->h_reqs) cudaFreeHost(srv->h_reqs);
    if (srv->h_out) cudaFreeHost(srv->h_out);
    if (srv->h_conflict) cudaFreeHost(srv->h_conflict);
    if (srv->h_jobs) cudaFreeHost(srv->h_jobs);
    delete srv;
    return rc;
}

}  // extern "C"
