// Host runtime and C ABI of the MAPA allocation engine (declared in include/mapa.h).
//
// Responsibilities on the host: validate inputs, turn the hardware graph
// (Sec. 3.2) into per-vertex adjacency and weight-class bitsets, analyse each
// application graph (Sec. 3.1) for its automorphism group and the order
// constraints that keep one match per distinct subgraph (Sec. 3.3), stage
// requests and drive the device engine (mapa_engine.cu).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "mapa_ctx.h"
#include "mapa_internal.h"

static_assert(sizeof(mapa_policy) == 24, "mapa_policy layout");
static_assert(sizeof(mapa_request) == 64, "mapa_request layout");
static_assert(sizeof(mapa_result) == 80, "mapa_result layout");

namespace {

thread_local std::string g_create_error;

using mapa::PatternEntry;
using mapa::TopoEntry;

}  // namespace

namespace mapa {

// ---------------------------------------------------------------------------
// Pattern analysis: Aut(P) by orbit search under a chain of pointwise
// stabilisers.  For v = 0, 1, ..., k-1 (with 0..v-1 already fixed) the orbit
// of v under the stabiliser is found by asking, for each later vertex u,
// whether some automorphism fixes 0..v-1 and sends v to u.  Every such u
// gets the constraint phi(v) < phi(u); |Aut(P)| is the product of the orbit
// sizes (orbit-stabiliser theorem).  Choosing v in increasing id order makes
// the one surviving map of each class its lexicographically smallest member.

namespace {

struct AutSearch {
    int k = 0;
    uint32_t adj[kMaxK] = {};
    int deg[kMaxK] = {};
    int sigma[kMaxK] = {};
    uint32_t taken = 0;
    int fixed = 0;  // sigma(i) = i for i < fixed
    int v = 0, u = 0;
    uint64_t nodes = 0;
    uint64_t budget = 50'000'000;
    bool exhausted = false;

    bool consistent(int i, int j) const {
        // i -> j must agree with every earlier assignment on adjacency
        for (int a = 0; a < i; ++a) {
            const bool pi = (adj[a] >> i) & 1u;
            const bool pj = (adj[sigma[a]] >> j) & 1u;
            if (pi != pj) return false;
        }
        return true;
    }

    bool dfs(int i) {
        if (i == k) return true;
        if (++nodes > budget) {
            exhausted = true;
            return false;
        }
        if (i < fixed || i == v) {
            const int j = i < fixed ? i : u;
            if ((taken >> j) & 1u) return false;
            if (deg[j] != deg[i] || !consistent(i, j)) return false;
            sigma[i] = j;
            taken |= 1u << j;
            if (dfs(i + 1)) return true;
            taken &= ~(1u << j);
            return false;
        }
        for (int j = 0; j < k; ++j) {
            if ((taken >> j) & 1u) continue;
            if (deg[j] != deg[i] || !consistent(i, j)) continue;
            sigma[i] = j;
            taken |= 1u << j;
            if (dfs(i + 1)) return true;
            taken &= ~(1u << j);
            if (exhausted) return false;
        }
        return false;
    }
};

}  // namespace

int analyze_pattern(int32_t k, const std::vector<std::pair<int, int>> &edges, PatternArgs *out, uint64_t *aut_order,
                    std::string *err) {
    if (k < 1 || k > kMaxK) {
        if (err) *err = "pattern size must be in 1..32";
        return MAPA_E_RANGE;
    }
    uint32_t adj[kMaxK] = {};
    for (const auto &e : edges) {
        const int a = e.first, b = e.second;
        if (a < 0 || b < 0 || a >= k || b >= k) {
            if (err) *err = "pattern edge endpoint out of range";
            return MAPA_E_INVALID;
        }
        if (a == b) {
            if (err) *err = "pattern self-loop";
            return MAPA_E_INVALID;
        }
        if ((adj[a] >> b) & 1u) {
            if (err) *err = "duplicate pattern edge";
            return MAPA_E_INVALID;
        }
        adj[a] |= 1u << b;
        adj[b] |= 1u << a;
    }
    PatternArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.k = k;
    for (int i = 0; i < k; ++i) pa.back[i] = adj[i] & ((i == 0) ? 0u : ((1u << i) - 1u));
    for (int l = 0; l <= k; ++l)
        for (const auto &e : edges) {
            const int lo = std::min(e.first, e.second), hi = std::max(e.first, e.second);
            if (lo >= l) ++pa.e_in[l];
            else if (hi >= l) ++pa.e_cross[l];
        }
    for (int i = 0; i < k; ++i) {
        pa.fdeg[i] = static_cast<uint8_t>(__builtin_popcount(i + 1 < 32 ? adj[i] >> (i + 1) : 0u));
        pa.dist0[i] = 255;
    }
    {
        // breadth-first distances from pattern vertex 0
        uint32_t seen = 1u, layer = 1u;
        pa.dist0[0] = 0;
        for (int d = 1; layer; ++d) {
            uint32_t next = 0u;
            for (uint32_t m = layer; m; m &= m - 1u) next |= adj[__builtin_ctz(m)];
            next &= ~seen;
            for (uint32_t m = next; m; m &= m - 1u) pa.dist0[__builtin_ctz(m)] = static_cast<uint8_t>(d);
            seen |= next;
            layer = next;
        }
    }
    AutSearch s;
    s.k = k;
    for (int i = 0; i < k; ++i) {
        s.adj[i] = adj[i];
        s.deg[i] = __builtin_popcount(adj[i]);
    }
    uint64_t order = 1;
    bool saturated = false;
    for (int v = 0; v < k; ++v) {
        uint64_t orbit = 1;
        for (int u = v + 1; u < k; ++u) {
            if (s.deg[u] != s.deg[v]) continue;
            s.fixed = v;
            s.v = v;
            s.u = u;
            s.taken = 0;
            s.nodes = 0;
            s.exhausted = false;
            const bool found = s.dfs(0);
            if (s.exhausted) {
                if (err) *err = "automorphism search of the pattern exceeded its budget";
                return MAPA_E_RANGE;
            }
            if (found) {
                pa.lo[u] |= 1u << v;
                ++orbit;
            }
        }
        if (!saturated) {
            if (order > UINT64_MAX / orbit) {
                saturated = true;
                order = UINT64_MAX;
            } else {
                order *= orbit;
            }
        }
    }
    pa.above0 = k > 1;
    for (int i = 1; i < k; ++i)
        if (!((pa.lo[i] >> 0) & 1u)) pa.above0 = 0;
    *out = pa;
    if (aut_order) *aut_order = order;
    return MAPA_OK;
}

}  // namespace mapa

// ---------------------------------------------------------------------------
// C ABI

namespace {

int fail(mapa_ctx ctx, int code, const std::string &msg) {
    if (ctx)
        ctx->last_error = msg;
    else
        g_create_error = msg;
    return code;
}

#define CTX_CUDA(ctx, x)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) return fail(ctx, MAPA_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

std::vector<std::pair<int, int>> builtin_edges(int kind, int k) {
    std::vector<std::pair<int, int>> e;
    switch (kind) {
        case MAPA_RING:
            if (k == 2) e.push_back({0, 1});
            if (k >= 3) {
                for (int i = 0; i + 1 < k; ++i) e.push_back({i, i + 1});
                e.push_back({0, k - 1});
            }
            break;
        case MAPA_TREE:
            for (int i = 1; i < k; ++i) e.push_back({(i - 1) / 2, i});
            break;
        case MAPA_CLIQUE:
            for (int i = 0; i < k; ++i)
                for (int j = i + 1; j < k; ++j) e.push_back({i, j});
            break;
        case MAPA_PATH:
            for (int i = 0; i + 1 < k; ++i) e.push_back({i, i + 1});
            break;
        default:
            break;
    }
    return e;
}

int add_pattern(mapa_ctx ctx, int32_t k, const std::vector<std::pair<int, int>> &edges, int32_t *pattern_id) {
    PatternEntry pe;
    std::string err;
    const int rc = mapa::analyze_pattern(k, edges, &pe.args, &pe.aut_order, &err);
    if (rc != MAPA_OK) return fail(ctx, rc, err);
    pe.args.id = static_cast<int32_t>(ctx->patterns.size());
    ctx->patterns.push_back(pe);
    ctx->pattern_args.push_back(pe.args);
    *pattern_id = static_cast<int32_t>(ctx->patterns.size() - 1);
    return MAPA_OK;
}

TopoEntry *get_topo(mapa_ctx ctx, int32_t topo_id) {
    if (topo_id < 0 || topo_id >= static_cast<int32_t>(ctx->topos.size()) || !ctx->topos[topo_id].live)
        return nullptr;
    return &ctx->topos[topo_id];
}

void free_topo(mapa::TopoDevice &t) {
    cudaFree(t.adj);
    cudaFree(t.clsv);
    cudaFree(t.wc);
    cudaFree(t.occupancy);
    cudaFree(t.owner);
    cudaFree(t.expire);
    cudaFree(t.next_job);
    cudaFree(t.scratch);
    cudaFree(t.wc_effbw);
    t = mapa::TopoDevice();
}

}  // namespace

extern "C" {

const char *mapa_version(void) { return "mapa-gb300 0.1 (sm_103a)"; }

int mapa_ctx_create(int device, uint64_t frontier_mem_cap, mapa_ctx *out) {
    if (!out) return fail(nullptr, MAPA_E_INVALID, "out is NULL");
    *out = nullptr;
    std::string err;
    mapa::Engine *e = mapa::engine_create(device, frontier_mem_cap, &err);
    if (!e) return fail(nullptr, MAPA_E_CUDA, err);
    mapa_ctx ctx = new mapa_ctx_s();
    ctx->engine = e;
    ctx->device = device;
    *out = ctx;
    return MAPA_OK;
}

void mapa_ctx_destroy(mapa_ctx ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    for (auto &t : ctx->topos)
        if (t.live) free_topo(t.dev);
    mapa::engine_destroy(ctx->engine);
    delete ctx;
}

int mapa_ctx_set_stream(mapa_ctx ctx, void *cuda_stream) {
    if (!ctx) return MAPA_E_INVALID;
    mapa::engine_set_stream(ctx->engine, static_cast<cudaStream_t>(cuda_stream));
    return MAPA_OK;
}

const char *mapa_last_error(mapa_ctx ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->last_error.c_str();
}

int mapa_topology_load(mapa_ctx ctx, int32_t n, int32_t m, const int32_t *u, const int32_t *v, const int32_t *w,
                       int32_t fill_weight, int32_t *topo_id) {
    if (!ctx || !topo_id) return MAPA_E_INVALID;
    if (n < 1 || n > MAPA_MAX_N) return fail(ctx, MAPA_E_RANGE, "topology size must be in 1..256");
    if (m < 0 || (m > 0 && (!u || !v || !w))) return fail(ctx, MAPA_E_INVALID, "bad edge arrays");
    if (fill_weight < 0 || fill_weight >= MAPA_MAX_WEIGHT) return fail(ctx, MAPA_E_RANGE, "fill weight out of range");
    std::vector<int32_t> wm(static_cast<size_t>(n) * n, 0);
    for (int32_t e = 0; e < m; ++e) {
        const int32_t a = u[e], b = v[e], x = w[e];
        if (a < 0 || b < 0 || a >= n || b >= n) return fail(ctx, MAPA_E_INVALID, "link endpoint out of range");
        if (a == b) return fail(ctx, MAPA_E_INVALID, "self-loop in hardware graph");
        if (x <= 0 || x >= MAPA_MAX_WEIGHT) return fail(ctx, MAPA_E_RANGE, "link weight must be in 1..2^20-1");
        if (wm[a * n + b] != 0) return fail(ctx, MAPA_E_INVALID, "duplicate link in hardware graph");
        wm[a * n + b] = x;
        wm[b * n + a] = x;
    }
    if (fill_weight > 0)
        for (int32_t a = 0; a < n; ++a)
            for (int32_t b = 0; b < n; ++b)
                if (a != b && wm[a * n + b] == 0) wm[a * n + b] = fill_weight;
    std::map<int32_t, int> cls;
    int64_t total = 0;
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = a + 1; b < n; ++b)
            if (wm[a * n + b] > 0) {
                cls.emplace(wm[a * n + b], 0);
                total += wm[a * n + b];
            }
    if (cls.size() > MAPA_MAX_CLASSES) return fail(ctx, MAPA_E_RANGE, "more than 8 distinct link weights");
    int ci = 0;
    std::vector<int32_t> wc;
    for (auto &kv : cls) {
        kv.second = ci++;
        wc.push_back(kv.first);
    }
    const int C = static_cast<int>(wc.size());
    const int W = n <= 32 ? 1 : n <= 64 ? 2 : n <= 128 ? 4 : 8;
    std::vector<uint32_t> adj(static_cast<size_t>(n) * W, 0u), clsv(static_cast<size_t>(n) * std::max(C, 1) * W, 0u);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = 0; b < n; ++b) {
            const int32_t x = wm[a * n + b];
            if (x <= 0) continue;
            adj[a * W + (b >> 5)] |= 1u << (b & 31);
            clsv[(static_cast<size_t>(a) * C + cls[x]) * W + (b >> 5)] |= 1u << (b & 31);
        }
    CTX_CUDA(ctx, cudaSetDevice(ctx->device));
    TopoEntry te;
    mapa::TopoDevice &t = te.dev;
    t.n = n;
    t.W = W;
    t.C = C;
    t.total_weight = total;
    t.wmin = wc.empty() ? 0 : wc.front();
    t.wmax = wc.empty() ? 0 : wc.back();
    for (int32_t a = 0; a < n; ++a) {
        int64_t d = 0;
        for (int32_t b = 0; b < n; ++b) d += wm[a * n + b];
        t.dmax = static_cast<int32_t>(std::max<int64_t>(t.dmax, d));
    }
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    if (cudaMalloc(&t.adj, adj.size() * 4) != cudaSuccess || cudaMalloc(&t.clsv, clsv.size() * 4) != cudaSuccess ||
        cudaMalloc(&t.wc, std::max(C, 1) * 4) != cudaSuccess || cudaMalloc(&t.occupancy, 8 * 4) != cudaSuccess ||
        cudaMalloc(&t.owner, n * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&t.expire, n * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&t.next_job, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&t.scratch, 64) != cudaSuccess || cudaMalloc(&t.wc_effbw, std::max(C, 1) * 4) != cudaSuccess) {
        free_topo(t);
        return fail(ctx, MAPA_E_NOMEM, "cannot allocate topology on the device");
    }
    std::vector<int32_t> codes(wc.size());
    for (size_t c = 0; c < wc.size(); ++c) codes[c] = mapa::effbw_class_code(wc[c]);
    CTX_CUDA(ctx, cudaMemcpyAsync(t.adj, adj.data(), adj.size() * 4, cudaMemcpyHostToDevice, st));
    CTX_CUDA(ctx, cudaMemcpyAsync(t.clsv, clsv.data(), clsv.size() * 4, cudaMemcpyHostToDevice, st));
    if (C > 0) CTX_CUDA(ctx, cudaMemcpyAsync(t.wc, wc.data(), C * 4, cudaMemcpyHostToDevice, st));
    if (C > 0) CTX_CUDA(ctx, cudaMemcpyAsync(t.wc_effbw, codes.data(), C * 4, cudaMemcpyHostToDevice, st));
    CTX_CUDA(ctx, cudaMemsetAsync(t.occupancy, 0, 8 * 4, st));
    CTX_CUDA(ctx, cudaMemsetAsync(t.owner, 0, n * sizeof(int64_t), st));
    CTX_CUDA(ctx, cudaMemsetAsync(t.expire, 0, n * sizeof(int64_t), st));
    CTX_CUDA(ctx, cudaMemsetAsync(t.next_job, 0, sizeof(unsigned long long), st));
    CTX_CUDA(ctx, cudaStreamSynchronize(st));
    te.live = true;
    te.wm = std::move(wm);
    t.id = static_cast<int32_t>(ctx->topos.size());
    ctx->topos.push_back(te);
    *topo_id = static_cast<int32_t>(ctx->topos.size() - 1);
    return MAPA_OK;
}

int mapa_pattern_load(mapa_ctx ctx, int32_t k, int32_t m, const int32_t *a, const int32_t *b, int32_t *pattern_id) {
    if (!ctx || !pattern_id) return MAPA_E_INVALID;
    if (m < 0 || (m > 0 && (!a || !b))) return fail(ctx, MAPA_E_INVALID, "bad pattern edge arrays");
    std::vector<std::pair<int, int>> edges;
    for (int32_t i = 0; i < m; ++i) edges.push_back({a[i], b[i]});
    return add_pattern(ctx, k, edges, pattern_id);
}

int mapa_pattern_builtin(mapa_ctx ctx, int32_t kind, int32_t k, int32_t *pattern_id) {
    if (!ctx || !pattern_id) return MAPA_E_INVALID;
    if (kind < MAPA_RING || kind > MAPA_PATH) return fail(ctx, MAPA_E_INVALID, "unknown pattern kind");
    if (k < 1 || k > MAPA_MAX_K) return fail(ctx, MAPA_E_RANGE, "pattern size must be in 1..32");
    return add_pattern(ctx, k, builtin_edges(kind, k), pattern_id);
}

int mapa_allocate_batch(mapa_ctx ctx, int32_t topo_id, int32_t nreq, const mapa_request *reqs, mapa_result *out,
                        uint32_t flags) {
    if (!ctx) return MAPA_E_INVALID;
    TopoEntry *te = get_topo(ctx, topo_id);
    if (!te) return fail(ctx, MAPA_E_INVALID, "unknown topology id");
    if (nreq < 0 || (nreq > 0 && (!reqs || !out))) return fail(ctx, MAPA_E_INVALID, "bad request arrays");
    if (flags & ~(MAPA_BATCH_SEQUENTIAL | MAPA_BATCH_DEVICE)) return fail(ctx, MAPA_E_INVALID, "unknown flags");
    if (nreq == 0) return MAPA_OK;
    const bool sequential = (flags & MAPA_BATCH_SEQUENTIAL) != 0;
    const bool device = (flags & MAPA_BATCH_DEVICE) != 0;
    CTX_CUDA(ctx, cudaSetDevice(ctx->device));
    std::string err;
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    const mapa_request *reqs_dev = reqs;
    mapa_result *out_dev = out;
    if (!device) {
        mapa_request *rd = nullptr;
        mapa_result *od = nullptr;
        const int rc = mapa::engine_stage(ctx->engine, nreq, &rd, &od, &err);
        if (rc != MAPA_OK) return fail(ctx, rc, err);
        CTX_CUDA(ctx, cudaMemcpyAsync(rd, reqs, sizeof(mapa_request) * nreq, cudaMemcpyHostToDevice, st));
        reqs_dev = rd;
        out_dev = od;
    }
    int rc = mapa::engine_run_batch(ctx->engine, te->dev, ctx->pattern_args, nreq, reqs_dev, out_dev, sequential, &err);
    if (rc != MAPA_OK) return fail(ctx, rc, err);
    if (!device) {
        CTX_CUDA(ctx, cudaMemcpyAsync(out, out_dev, sizeof(mapa_result) * nreq, cudaMemcpyDeviceToHost, st));
    }
    CTX_CUDA(ctx, cudaStreamSynchronize(st));
    return MAPA_OK;
}

int mapa_allocate(mapa_ctx ctx, int32_t topo_id, int32_t pattern_id, const mapa_policy *policy, mapa_result *out) {
    if (!ctx || !out) return MAPA_E_INVALID;
    memset(out, 0, sizeof(*out));
    out->status = MAPA_E_INVALID;
    if (pattern_id < 0 || pattern_id >= static_cast<int32_t>(ctx->patterns.size()))
        return fail(ctx, MAPA_E_INVALID, "unknown pattern id");
    mapa_request q;
    memset(&q, 0, sizeof(q));
    q.pattern_id = pattern_id;
    if (policy)
        q.policy = *policy;
    else {
        q.policy.alpha = 1;
        q.policy.beta = 1;
    }
    const int rc = mapa_allocate_batch(ctx, topo_id, 1, &q, out, MAPA_BATCH_SEQUENTIAL);
    if (rc != MAPA_OK) {
        out->status = rc;
        return rc;
    }
    return out->status;
}

int mapa_release(mapa_ctx ctx, int32_t topo_id, int64_t job_id) {
    if (!ctx) return MAPA_E_INVALID;
    TopoEntry *te = get_topo(ctx, topo_id);
    if (!te) return fail(ctx, MAPA_E_INVALID, "unknown topology id");
    if (job_id <= 0) return fail(ctx, MAPA_E_STATE, "not a live job id");
    std::string err;
    int32_t freed = 0;
    const int rc = mapa::engine_release(ctx->engine, te->dev, job_id, &freed, &err);
    if (rc != MAPA_OK) return fail(ctx, rc, err);
    if (freed == 0) return fail(ctx, MAPA_E_STATE, "not a live job id");
    return MAPA_OK;
}

int mapa_occupancy_get(mapa_ctx ctx, int32_t topo_id, uint32_t *busy_out) {
    if (!ctx || !busy_out) return MAPA_E_INVALID;
    TopoEntry *te = get_topo(ctx, topo_id);
    if (!te) return fail(ctx, MAPA_E_INVALID, "unknown topology id");
    cudaStream_t st = mapa::engine_stream(ctx->engine);
    CTX_CUDA(ctx, cudaMemcpyAsync(busy_out, te->dev.occupancy, 8 * 4, cudaMemcpyDeviceToHost, st));
    CTX_CUDA(ctx, cudaStreamSynchronize(st));
    return MAPA_OK;
}

int mapa_allocate_batch_noalloc(mapa_ctx ctx, int32_t topo_id, int32_t pattern_id, int32_t nreq,
                                const mapa_request *reqs_dev, mapa_result *out_dev) {
    if (!ctx) return MAPA_E_INVALID;
    TopoEntry *te = get_topo(ctx, topo_id);
    if (!te) return fail(ctx, MAPA_E_INVALID, "unknown topology id");
    if (pattern_id < 0 || pattern_id >= static_cast<int32_t>(ctx->patterns.size()))
        return fail(ctx, MAPA_E_INVALID, "unknown pattern id");
    if (nreq > 0 && (!reqs_dev || !out_dev)) return fail(ctx, MAPA_E_INVALID, "bad request arrays");
    CTX_CUDA(ctx, cudaSetDevice(ctx->device));
    std::string err;
    const int rc = mapa::noalloc_decide(te->dev, ctx->pattern_args[pattern_id], pattern_id, nreq, reqs_dev, out_dev,
                                        mapa::engine_stream(ctx->engine), &err);
    if (rc != MAPA_OK) return fail(ctx, rc, err);
    return MAPA_OK;
}

int mapa_autotune(mapa_ctx ctx, int32_t topo_id, int32_t nreq, const mapa_request *reqs, int32_t *chosen) {
    if (!ctx) return MAPA_E_INVALID;
    TopoEntry *te = get_topo(ctx, topo_id);
    if (!te) return fail(ctx, MAPA_E_INVALID, "unknown topology id");
    if (nreq < 0 || (nreq > 0 && (!reqs || !chosen))) return fail(ctx, MAPA_E_INVALID, "bad arrays");
    CTX_CUDA(ctx, cudaSetDevice(ctx->device));
    std::vector<int32_t> tmp(ctx->pattern_args.size() + 1, 0);
    std::string err;
    const int rc = mapa::engine_autotune(ctx->engine, te->dev, ctx->pattern_args, nreq, reqs, tmp.data(), &err);
    if (rc != MAPA_OK) return fail(ctx, rc, err);
    for (size_t p = 0; p < ctx->pattern_args.size(); ++p) chosen[p] = tmp[p];
    return MAPA_OK;
}

int mapa_stats_get(mapa_ctx ctx, mapa_stats *out) {
    if (!ctx || !out) return MAPA_E_INVALID;
    return mapa::engine_stats(ctx->engine, out);
}

int mapa_stats_reset(mapa_ctx ctx) {
    if (!ctx) return MAPA_E_INVALID;
    mapa::engine_stats_reset(ctx->engine);
    return MAPA_OK;
}

int mapa_ctx_set_timing(mapa_ctx ctx, int on) {
    if (!ctx) return MAPA_E_INVALID;
    mapa::engine_set_timing(ctx->engine, on != 0);
    return MAPA_OK;
}

int mapa_ctx_set_work_budget(mapa_ctx ctx, uint64_t max_partials) {
    if (!ctx) return MAPA_E_INVALID;
    mapa::engine_set_work_budget(ctx->engine, max_partials);
    return MAPA_OK;
}

int mapa_autotune_level_limit(mapa_ctx ctx, int32_t topo_id, int32_t pattern_id, uint64_t *entries) {
    if (!ctx || !entries) return MAPA_E_INVALID;
    *entries = mapa::engine_tuned_chunk(ctx->engine, topo_id, pattern_id);
    return MAPA_OK;
}

int mapa_result_merge(int32_t nparts, const mapa_result *parts, mapa_result *out) {
    if (nparts < 1 || !parts || !out) return MAPA_E_INVALID;
    mapa_result best;
    memset(&best, 0, sizeof(best));
    best.k = parts[0].k;
    bool have = false, inexact = false;
    uint64_t count = 0;
    for (int32_t i = 0; i < nparts; ++i) {
        const mapa_result &p = parts[i];
        if (p.k != best.k) return MAPA_E_INVALID;  // shares of different requests
        if (p.status < 0) {
            memset(out, 0, sizeof(*out));
            out->status = p.status;
            out->k = p.k;
            return MAPA_OK;
        }
        count += p.count;
        if (p.status != MAPA_OK && p.status != MAPA_INEXACT) continue;
        inexact |= p.status == MAPA_INEXACT;
        // larger score first, then the lexicographically smaller tuple
        bool take = !have || p.score > best.score;
        if (have && p.score == best.score)
            take = std::lexicographical_compare(p.verts, p.verts + p.k, best.verts, best.verts + best.k);
        if (take) {
            best = p;
            have = true;
        }
    }
    best.status = !have ? MAPA_NO_FIT : (inexact ? MAPA_INEXACT : MAPA_OK);
    if (!have) {
        memset(&best, 0, sizeof(best));
        best.status = MAPA_NO_FIT;
        best.k = parts[0].k;
    }
    best.count = count;
    best.job_id = 0;
    *out = best;
    return MAPA_OK;
}

int mapa_pattern_analyze(int32_t k, int32_t m, const int32_t *a, const int32_t *b, uint64_t *aut_order,
                         uint32_t *back_masks, uint32_t *lo_masks) {
    if (m < 0 || (m > 0 && (!a || !b))) return MAPA_E_INVALID;
    std::vector<std::pair<int, int>> edges;
    for (int32_t i = 0; i < m; ++i) edges.push_back({a[i], b[i]});
    mapa::PatternArgs pa;
    std::string err;
    const int rc = mapa::analyze_pattern(k, edges, &pa, aut_order, &err);
    if (rc != MAPA_OK) return rc;
    for (int i = 0; i < k; ++i) {
        if (back_masks) back_masks[i] = pa.back[i];
        if (lo_masks) lo_masks[i] = pa.lo[i];
    }
    return MAPA_OK;
}

}  // extern "C"
