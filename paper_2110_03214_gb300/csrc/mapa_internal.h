// Internal declarations shared by the host runtime (mapa_capi.cpp) and the
// device engine (mapa_engine.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mapa.h"

namespace mapa {

constexpr int kMaxN = MAPA_MAX_N;
constexpr int kMaxK = MAPA_MAX_K;
constexpr int kMaxClasses = MAPA_MAX_CLASSES;

// Level kernels: 256 threads, each warp owns 32 * kIpt consecutive parents.
constexpr int kTpb = 256;
constexpr int kWarps = kTpb / 32;
constexpr int kIpt = 4;
constexpr int kTile = kTpb * kIpt;

// Largest request group enumerated together (larger groups are sliced).
constexpr int kMaxGroup = 1 << 20;

// Capacity limit of a stored level: with at most 8 columns per field, every
// column offset j * cap + p stays below 2^31 (kernels index in 32 bits).
// Larger frontiers are produced in chunks.
constexpr uint64_t kMaxLevelEntries = 1ull << 28;

// Pattern as the device sees it: vertex i is matched at level i; back[i] holds
// the earlier neighbours of i, lo[i] the earlier vertices j with the
// symmetry-breaking constraint phi(j) < phi(i).
// For the bounded mode, level l (pattern vertices 0..l-1 placed) has
// e_cross[l] pattern edges between a placed and an unplaced vertex and
// e_in[l] pattern edges between two unplaced ones.
struct PatternArgs {
    int32_t k;
    int32_t id;  // pattern id in its context (keys the tuned tail depth)
    uint32_t back[kMaxK];
    uint32_t lo[kMaxK];
    uint16_t e_cross[kMaxK + 1];
    uint16_t e_in[kMaxK + 1];
    // Feasibility filters of the anytime seed dive (necessary conditions on
    // any match): fdeg[i] = neighbours of i with a larger id; dist0[i] =
    // distance from vertex 0 to i in the pattern (255: not connected).
    uint8_t fdeg[kMaxK];
    uint8_t dist0[kMaxK];
    int32_t above0;  // 1: every other pattern vertex has the constraint phi(0) < phi(i)
};

// Hardware graph in device memory.
//   adj[v * W + w]            bit u of word w: link v-u exists
//   clsv[(v * C + c) * W + w] bit u: link v-u has weight class c
//   wc[c]                     weight of class c
struct TopoArgs {
    int32_t n;
    int32_t W;  // words per vertex mask: 1, 2, 4 or 8
    int32_t C;  // distinct link weights
    const uint32_t *adj;
    const uint32_t *clsv;
    const int32_t *wc;
    int32_t wmin, wmax;  // smallest and largest link weight
    int32_t dmax;        // largest weighted degree of a vertex
};

// One frontier level in structure-of-arrays form, `cap` entries per column.
//   S[i]                      partial score of entry i
//   r[i]                      request index within the group
//   R[i * W + w]              free vertices not yet used (word w; an entry's words together)
//   T[j * cap + i]            tuple bytes 4j..4j+3 (phi of pattern vertices)
//   root != 0 (level 0 only): T[i] holds the request's range of phi(0),
//   root_lo | root_hi << 16 (root_hi = 0: no restriction)
struct LevelView {
    int32_t *S;
    uint32_t *r;
    uint32_t *R;
    uint32_t *T;
    uint64_t cap;
    int32_t root;
};

// Per-request state of a group being enumerated.
struct GroupArgs {
    int32_t size;              // requests in the group
    const int32_t *req_index;  // group slot -> position in the batch
    const mapa_request *reqs;  // the batch (device)
    mapa_result *out;          // results (device), indexed by batch position
    int32_t *alpha;            // [size]
    int32_t *beta;             // [size]
    uint64_t *key;             // [size] argmax key of the current last-level chunk
    unsigned long long *count; // [size] matches found
    int32_t *best_s;           // [size]
    int32_t *best_valid;       // [size]
    uint32_t *best_t;          // [size * 8] best tuple bytes
    const uint32_t *occupancy; // device occupancy or nullptr (request masks only)
    int64_t total_weight;      // for the int32 range check
    int32_t *error;            // device error word (0 = fine)
    // Bounded mode: score of a match already found per request (partials whose
    // completions all score below it are skipped); INT_MIN = no cut-off,
    // INT_MAX = proven to have no match.  nullptr when no request of the
    // group is bounded.
    int32_t *thr;              // [size]
    // Work budget (0 = none): partial matches stored per request so far; a
    // request past work_budget gets thr = INT_MAX (every later partial is
    // cut) and ends with MAPA_E_BUDGET.  nullptr when no budget is set.
    unsigned long long *work;  // [size]
    unsigned long long work_budget;
    // Anytime requests: the seed dive's best complete match (score INT_MIN
    // = none) and its tuple bytes.
    int32_t *dive_s;           // [size]
    uint32_t *dive_t;          // [size * 8]
    // Bandwidth-sensitive group (Algorithm 1, first branch): scores are the
    // link-count index (x * R + y) * R + z of the match, ranked through
    // effbw_rank; sens_ok = 0 when the pattern has more edges than R - 1.
    int32_t sens;
    int32_t sens_ok;
    const int32_t *effbw_rank;   // [R^3] dense rank of Eq. 2 at each index
    const int32_t *effbw_milli;  // [R^3] round(1000 * EffBW)
    const int32_t *effbw_code;   // [C] index weight of each link class
};

// Bandwidth-sensitive scoring (mapa_effbw.cpp): link counts per type below
// kEffbwRadix, indexed (x * R + y) * R + z.
constexpr int kEffbwRadix = 64;
double effbw_predict(int x, int y, int z);
int32_t effbw_class_code(int32_t weight);
void effbw_tables(std::vector<int32_t> *rank, std::vector<int32_t> *milli);

// Device-side error codes written to the error word.
enum DeviceError : int32_t {
    kDevOk = 0,
    kDevScoreMismatch = 1,  // finalize found a score that disagrees with its tuple
    kDevResolveMiss = 2,    // resolve could not re-find the argmax tail
    kDevLookbackTimeout = 3,  // a bounded look-back wait gave up
};

struct Engine;  // device buffers + launch helpers (mapa_engine.h)

Engine *engine_create(int device, uint64_t frontier_cap, std::string *err);
void engine_destroy(Engine *e);
void engine_set_stream(Engine *e, cudaStream_t s);
cudaStream_t engine_stream(Engine *e);

struct TopoDevice {
    int32_t id = -1;  // topology id in its context
    int32_t n = 0, W = 1, C = 0;
    int32_t wmin = 0, wmax = 0, dmax = 0;
    int64_t total_weight = 0;
    uint32_t *adj = nullptr;
    uint32_t *clsv = nullptr;
    int32_t *wc = nullptr;
    uint32_t *occupancy = nullptr;  // [8]
    int64_t *owner = nullptr;       // [n] job id holding each vertex, 0 = free
    int64_t *expire = nullptr;      // [n] device-clock ns when the vertex's job ends (0 = held until released)
    unsigned long long *next_job = nullptr;
    int32_t *scratch = nullptr;     // small per-topology scratch (release count)
    int32_t *wc_effbw = nullptr;    // [C] effbw_class_code of each class weight
    TopoArgs args() const { return TopoArgs{n, W, C, adj, clsv, wc, wmin, wmax, dmax}; }
    // The same graph with the class weights replaced by the link-count codes.
    TopoArgs args_effbw() const { return TopoArgs{n, W, C, adj, clsv, wc_effbw, 0, 0, 0}; }
};

// Runs one batch on the device.  reqs/out are device arrays of nreq entries.
// sequential: process in order against the topology occupancy and commit.
int engine_run_batch(Engine *e, const TopoDevice &t, const std::vector<PatternArgs> &patterns, int32_t nreq,
                     const mapa_request *reqs_dev, mapa_result *out_dev, bool sequential, std::string *err);

int engine_stats(Engine *e, mapa_stats *out);

// Autotuner: times every fused tail depth for each pattern present in the
// host batch reqs[0..nreq) and keeps the fastest per (topology, pattern).
// chosen[p] receives the depth for pattern id p (0 if p is not in the batch).
int engine_autotune(Engine *e, const TopoDevice &t, const std::vector<PatternArgs> &patterns, int32_t nreq,
                    const mapa_request *reqs_host, int32_t *chosen, std::string *err);
void engine_stats_reset(Engine *e);
void engine_set_timing(Engine *e, bool on);
void engine_set_work_budget(Engine *e, uint64_t max_partials);
uint64_t engine_tuned_chunk(const Engine *e, int32_t topo_id, int32_t pattern_id);
// Frontier memory the concurrent groups of a batch may hold (all slots) and
// the context's work budget (stored partial matches per request, 0 = none).
uint64_t engine_frontier_budget(const Engine *e);
uint64_t engine_work_budget(const Engine *e);

// Allocation-free single-kernel decision (mapa_noalloc.cu).
int noalloc_decide(const TopoDevice &t, const PatternArgs &pat, int32_t pattern_id, int32_t nreq,
                   const mapa_request *reqs_dev, mapa_result *out_dev, cudaStream_t stream, std::string *err);

int engine_release(Engine *e, const TopoDevice &t, int64_t job_id, int32_t *freed, std::string *err);

// Serving: commit a round's decisions in order with conflict flags, and
// release a list of jobs (device array); both enqueue only.
// Internal mark (mapa_result.reserved) of a chain decision deferred by FIFO waiting.
constexpr int32_t kDeferred = 2;

// Lifetimes kept on the device (served loop): life[i] is the lifetime in ns
// of the job that request i of the call commits (0 = until released); the
// job's vertices end at the device clock of the commit plus life[i].  Before
// each later decision of a chain the vertices whose end has passed are freed
// and every freed (job, vertex) is appended to the log with the chain
// position it was freed before (n = after the last decision, -1 = freed by
// engine_expire).  The log holds cap entries; n_log counts every entry, so
// *n_log > cap means entries were lost (a caller error: cap too small).
struct ServeLife {
    const int64_t *life = nullptr;
    int64_t *log_job = nullptr;
    int32_t *log_pos = nullptr;
    uint32_t *n_log = nullptr;
    uint32_t cap = 0;
    // optional pinned host copies engine_run_chain fills before it returns:
    // the count and the first host_first entries
    uint32_t *host_n_log = nullptr;
    int64_t *host_log_job = nullptr;
    int32_t *host_log_pos = nullptr;
    uint32_t host_first = 0;
};

int engine_commit_round(Engine *e, const TopoDevice &t, mapa_result *out_dev, int32_t n, int32_t *conflict_dev,
                        bool fifo_wait, const ServeLife *life, std::string *err);
// Frees every vertex whose job's lifetime has ended (log position -1).
int engine_expire(Engine *e, const TopoDevice &t, const ServeLife &life, std::string *err);
// kinds[i]: bit 0 = request i is in bounded mode, bit 1 = bandwidth-sensitive
// (nullptr = neither, for every request).
constexpr uint8_t kKindBounded = 1, kKindSensitive = 2;
// out_host (may be null): pinned host copy of the n results, filled before
// the call returns.
int engine_run_chain(Engine *e, const TopoDevice &t, const std::vector<PatternArgs> &patterns, int32_t n,
                     const int32_t *pattern_ids, const uint8_t *kinds, const mapa_request *reqs_dev,
                     mapa_result *out_dev, bool fifo_wait, mapa_result *out_host, const ServeLife *life,
                     std::string *err);
int engine_release_many(Engine *e, const TopoDevice &t, const int64_t *jobs_dev, int32_t njobs, std::string *err);

// Scratch for staging host batches.
int engine_stage(Engine *e, int32_t nreq, mapa_request **reqs_dev, mapa_result **out_dev, std::string *err);

// Host-side pattern analysis (automorphisms and order constraints).
int analyze_pattern(int32_t k, const std::vector<std::pair<int, int>> &edges, PatternArgs *out,
                    uint64_t *aut_order, std::string *err);

}  // namespace mapa
