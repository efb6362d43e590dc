// Simulator of Sec. 6 behind mapa_simulate in mapa.h.
//
// A dispatcher reads the job file in order into a FIFO queue; a cycle-based
// execution engine models which accelerators are busy.  At every cycle where
// something happens (an arrival or the end of a job) the engine
//   1. frees the accelerators of every job that has finished,
//   2. allocates the queue head while it has arrived and fits under the
//      policy, starting it at this cycle; a head that does not fit waits for
//      the next job to finish (FIFO: nothing behind it is tried), and one
//      that does not fit on the idle machine is logged as MAPA_NO_FIT,
//   3. advances to the next arrival or end of job.
// Decisions other than BASELINE go to the GPU path, one request against the
// simulator's own occupancy.  The logger computes AggBW (Eq. 1), PreservedBW
// (Eq. 3) and Predicted EffBW (Eq. 2) of every allocation from a host copy
// of the link weights.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <string>
#include <vector>

#include "mapa_ctx.h"
#include "mapa_internal.h"

namespace {

struct Running {
    int64_t end;
    int32_t job;
    bool operator>(const Running &o) const { return end != o.end ? end > o.end : job > o.job; }
};

int fail(mapa_ctx ctx, int rc, const std::string &msg) {
    ctx->last_error = msg;
    return rc;
}

// Logger: Eq. 1, Eq. 2 and Eq. 3 of an allocation.
void log_metrics(const mapa::TopoEntry &te, const mapa::PatternArgs &pat, const std::vector<char> &busy,
                 mapa_sim_record *r) {
    const int n = te.dev.n;
    const auto w = [&](int a, int b) { return te.wm[static_cast<size_t>(a) * n + b]; };
    int64_t agg = 0;
    int counts[3] = {0, 0, 0};
    for (int v = 0; v < pat.k; ++v)
        for (uint32_t m = pat.back[v]; m; m &= m - 1u) {
            const int32_t x = w(r->verts[__builtin_ctz(m)], r->verts[v]);
            agg += x;
            const int32_t code = mapa::effbw_class_code(x);
            if (code == mapa::kEffbwRadix * mapa::kEffbwRadix) ++counts[0];
            else if (code == mapa::kEffbwRadix) ++counts[1];
            else if (code == 1) ++counts[2];
        }
    int64_t pres = 0;
    for (int a = 0; a < n; ++a)
        if (!busy[a])
            for (int b = a + 1; b < n; ++b)
                if (!busy[b]) pres += w(a, b);
    r->agg = static_cast<int32_t>(agg);
    r->pres = static_cast<int32_t>(pres);
    r->effbw_milli = static_cast<int32_t>(std::llround(1000.0 * mapa::effbw_predict(counts[0], counts[1], counts[2])));
}

}  // namespace

extern "C" int mapa_simulate(mapa_ctx ctx, int32_t topo_id, int32_t policy, int32_t njobs, const mapa_sim_job *jobs,
                             mapa_sim_record *out) {
    if (!ctx) return MAPA_E_INVALID;
    if (topo_id < 0 || topo_id >= static_cast<int32_t>(ctx->topos.size()) || !ctx->topos[topo_id].live)
        return fail(ctx, MAPA_E_INVALID, "unknown topology id");
    if (policy < MAPA_SIM_BASELINE || policy > MAPA_SIM_EFFBW) return fail(ctx, MAPA_E_INVALID, "unknown policy");
    if (njobs < 0 || (njobs > 0 && (!jobs || !out))) return fail(ctx, MAPA_E_INVALID, "bad job arrays");
    const int32_t npat = static_cast<int32_t>(ctx->patterns.size());
    for (int32_t i = 0; i < njobs; ++i) {
        if (jobs[i].pattern_id < 0 || jobs[i].pattern_id >= npat) return fail(ctx, MAPA_E_INVALID, "unknown pattern id");
        if (jobs[i].duration < 0) return fail(ctx, MAPA_E_INVALID, "negative duration");
        if (i > 0 && jobs[i].arrive < jobs[i - 1].arrive) return fail(ctx, MAPA_E_INVALID, "arrivals out of order");
    }
    const mapa::TopoEntry &te = ctx->topos[topo_id];
    const int n = te.dev.n;
    std::vector<char> busy(static_cast<size_t>(n), 0);
    std::priority_queue<Running, std::vector<Running>, std::greater<Running>> running;
    int32_t head = 0;
    int64_t t = njobs > 0 ? jobs[0].arrive : 0;

    // One decision for job j against the current occupancy: MAPA_OK with
    // out[j].verts filled, MAPA_NO_FIT, or a negative error for the job.
    auto decide = [&](int32_t j) -> int {
        const mapa::PatternArgs &pat = ctx->patterns[jobs[j].pattern_id].args;
        mapa_sim_record &r = out[j];
        if (policy == MAPA_SIM_BASELINE) {
            int got = 0;
            for (int v = 0; v < n && got < pat.k; ++v)
                if (!busy[v]) r.verts[got++] = static_cast<uint8_t>(v);
            return got == pat.k ? MAPA_OK : MAPA_NO_FIT;
        }
        mapa_request q;
        memset(&q, 0, sizeof(q));
        q.pattern_id = jobs[j].pattern_id;
        q.policy.mode = MAPA_MODE_EXHAUSTIVE;
        const bool sens = policy == MAPA_SIM_EFFBW || (policy == MAPA_SIM_PRESERVE && jobs[j].sensitive);
        if (sens) {
            q.policy.flags = MAPA_POLICY_BW_SENSITIVE;
        } else if (policy == MAPA_SIM_GREEDY) {
            q.policy.alpha = 1;
        } else {
            q.policy.beta = 1;
        }
        for (int v = 0; v < n; ++v)
            if (busy[v]) q.busy[v >> 5] |= 1u << (v & 31);
        mapa_result res;
        const int rc = mapa_allocate_batch(ctx, topo_id, 1, &q, &res, MAPA_BATCH_INDEPENDENT);
        if (rc != MAPA_OK) return rc;
        if (res.status == MAPA_OK) memcpy(r.verts, res.verts, sizeof(r.verts));
        return res.status;
    };

    while (head < njobs || !running.empty()) {
        while (!running.empty() && running.top().end <= t) {
            const mapa_sim_record &r = out[running.top().job];
            for (int i = 0; i < r.k; ++i) busy[r.verts[i]] = 0;
            running.pop();
        }
        while (head < njobs && jobs[head].arrive <= t) {
            mapa_sim_record &r = out[head];
            memset(&r, 0, sizeof(r));
            r.job_id = jobs[head].job_id;
            r.k = ctx->patterns[jobs[head].pattern_id].args.k;
            const int st = decide(head);
            if (st == MAPA_OK) {
                for (int i = 0; i < r.k; ++i) busy[r.verts[i]] = 1;
                r.status = MAPA_OK;
                r.start = t;
                r.end = t + jobs[head].duration;
                log_metrics(te, ctx->patterns[jobs[head].pattern_id].args, busy, &r);
                running.push(Running{r.end, head});
                ++head;
            } else if (st == MAPA_NO_FIT && !running.empty()) {
                memset(r.verts, 0, sizeof(r.verts));
                break;  // the head waits for a job to finish
            } else if (st < 0 && st != MAPA_E_RANGE && st != MAPA_E_BUDGET) {
                return st;  // the call failed as a whole (mapa_last_error holds why)
            } else {
                // never fits (idle machine), or refused for this job
                r.status = st;
                r.start = r.end = t;
                memset(r.verts, 0, sizeof(r.verts));
                ++head;
            }
        }
        int64_t next = INT64_MAX;
        if (!running.empty()) next = running.top().end;
        if (head < njobs && jobs[head].arrive > t) next = std::min(next, jobs[head].arrive);
        if (next == INT64_MAX) break;
        t = std::max(next, t);
    }
    return MAPA_OK;
}
