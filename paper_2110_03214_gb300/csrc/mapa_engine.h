// Internal engine state shared by the batch driver (mapa_engine.cu) and the
// per-mask-width runner translation units (mapa_engine_w*.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "mapa_internal.h"

namespace mapa {

#define MAPA_CUDA_TRY(x)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                         \
            if (err) *err = std::string(#x) + ": " + cudaGetErrorString(e_) + " (" +     \
                            __FILE__ + ":" + std::to_string(__LINE__) + ")";             \
            return MAPA_E_CUDA;                                                          \
        }                                                                                \
    } while (0)

constexpr int kStatWords = 8;

// Memory and stream of one request group in flight.  The groups of an
// independent batch run concurrently, one per slot (round robin beyond
// kSlots); every other path uses slot 0 on the engine's stream.
struct Slot {
    char *arena = nullptr;      // frontier levels and their control words
    uint64_t arena_bytes = 0;
    char *group_mem = nullptr;  // per-request group arrays
    uint64_t group_bytes = 0;
    cudaStream_t stream = nullptr;  // concurrent groups (created on first use)
    cudaEvent_t done = nullptr;
    // eager anytime dives (and a detached run's finalize) of the slot's
    // host-driven runs (created on first use); side_busy: work on it that the
    // engine's stream has not joined yet
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    bool side_busy = false;
};
constexpr int kSlots = 4;

struct Engine {
    int device = 0;
    int sm_count = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t frontier_cap = 0;
    Slot slots[kSlots];
    cudaEvent_t fork = nullptr;  // start of the concurrent groups of a batch
    mapa_request *stage_reqs = nullptr;
    mapa_result *stage_out = nullptr;
    int32_t stage_cap = 0;
    int32_t *order = nullptr;
    int32_t order_cap = 0;
    int32_t *hist = nullptr;
    int32_t hist_cap = 0;
    int32_t *overflow = nullptr;  // one flag per request group of a batch
    int32_t overflow_cap = 0;
    int32_t *d_error = nullptr;
    unsigned long long *d_stats = nullptr;  // kStatWords counters of the current batch
    int32_t *d_blocked = nullptr;           // FIFO-wait flag of a commit chain (= d_chain + 2)
    int32_t *d_chain = nullptr;             // [3] commit chain: cursor, step overflow flag, FIFO-wait flag
    int32_t *effbw_rank = nullptr;          // [kEffbwRadix^3] (built on first use)
    int32_t *effbw_milli = nullptr;
    unsigned long long *h_pinned = nullptr;  // small pinned scratch
    mapa_stats st{};
    bool timing = false;
    int tail_override = 0;  // 0 = automatic tail depth
    int tail_blocks_per_sm = 0;  // 0 = from the occupancy calculator
    int dive_steps = 32;         // bounded mode: node expansions of a request's seed dive
    int degree_min_m = 6;        // bounded mode: degree term only where >= this many pattern vertices remain
    uint64_t work_budget = 0;    // stored partial matches a request may produce (0 = no limit)
    bool chunk_single_pass = true;  // chunked levels by single-pass k_expand (MAPA_CHUNK_SINGLE_PASS=0: count + write)
    bool tail_sorted = false;    // short fused tail: parents of a tile ordered by estimated subtree size (MAPA_TAIL_SORT=1)
    int dive_block = 2;          // guided dives on blocks: 0 never, 1 always, 2 groups below 2 x SMs (MAPA_DIVE_BLOCK)
    // host-driven runs under a work budget start the anytime dives at once on
    // their slot's side stream, beside their own enumeration (MAPA_DIVE_EAGER=0:
    // after it)
    bool dive_eager = true;
    // (topology, pattern) -> (batches left that run the group straight on the
    // chunked path because its device-driven run overflowed, the current wait
    // between retries) (MAPA_HOST_HINT=0: off)
    bool host_hint_on = true;
    std::map<std::pair<int32_t, int32_t>, std::pair<int, int>> host_hint;
    std::map<std::pair<int32_t, int32_t>, int> tail_table;  // (topology, pattern) -> tuned depth
    // (topology, pattern) -> tuned largest entries of a stored level (0 = as
    // many as the frontier cap allows): smaller levels make the chunked path
    // produce a level in smaller chunks that stay in L2 between passes
    std::map<std::pair<int32_t, int32_t>, uint64_t> chunk_table;
    // Captured launch sequences of independent batches, keyed by batch shape.
    bool use_graphs = true;
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        mapa_stats delta{};  // host-side counters the captured launches account for
    };
    std::map<std::vector<int64_t>, GraphEntry> graphs;
    std::map<std::vector<int64_t>, int> shapes_seen;  // shapes run once without a graph
    void clear_graphs() {
        for (auto &kv : graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        graphs.clear();
        shapes_seen.clear();
    }
    std::vector<cudaEvent_t> events;  // pairs around timed launches
    std::vector<uint8_t> pair_kind;   // per pair: 0 = fused last level, 1 = level expansion
    size_t events_used = 0;

    cudaEvent_t next_event() {
        if (events_used == events.size()) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            events.push_back(ev);
        }
        return events[events_used++];
    }
    // Two events bracketing one timed launch of the given kind.
    void timed_pair(uint8_t kind, cudaEvent_t *ev0, cudaEvent_t *ev1) {
        if (pair_kind.size() <= events_used / 2) pair_kind.resize(events_used / 2 + 1);
        pair_kind[events_used / 2] = kind;
        *ev0 = next_event();
        *ev1 = next_event();
    }
};

int ensure_device(char **ptr, uint64_t *have, uint64_t need, std::string *err);

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline uint64_t align_up(uint64_t a, uint64_t b) { return (a + b - 1) / b * b; }
inline uint64_t entry_bytes(int ell, int W) { return 4ull * (2 + W + ((ell + 3) / 4)); }

// One request group (all requests of one pattern in a batch slice).
struct GroupRun {
    const PatternArgs *pat;
    GroupArgs g;
    int tail;               // fused tail depth T
    int32_t *overflow;      // device flag for this group (device-driven path)
    bool bounded = false;   // some request of the group is in bounded mode (g.thr set)
    bool sens = false;      // the group's requests are bandwidth-sensitive
    bool redo = false;      // rerun of a group whose device-driven run overflowed (on the chunked path)
    bool detach = false;    // host-driven: finish the group on its slot's side stream (the caller joins it)
    int slot = 0;           // arena of the group
    cudaStream_t stream = nullptr;  // stream of its launches (nullptr = the engine's)
};

// Per-mask-width entry points (mapa_engine_w{1,2,4,8}.cu).
//   run_group_device_*: enqueue the whole group without host synchronisation;
//   run_group_host_*:   host-driven, chunked so any frontier fits.
#define MAPA_DECLARE_W(W)                                                                                  \
    int run_group_device_w##W(Engine *e, const TopoDevice &t, const GroupRun &gr, std::string *err);      \
    int run_group_host_w##W(Engine *e, const TopoDevice &t, const GroupRun &gr, std::string *err);
MAPA_DECLARE_W(1)
MAPA_DECLARE_W(2)
MAPA_DECLARE_W(4)
MAPA_DECLARE_W(8)
#undef MAPA_DECLARE_W

}  // namespace mapa
