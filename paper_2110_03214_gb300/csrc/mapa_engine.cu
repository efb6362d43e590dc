// Batch driver of the MAPA allocation engine: context state, frontier arena
// planning, grouping of requests by pattern, state management kernels and
// the per-batch control flow.  The level kernels live in mapa_kernels.cuh and
// are instantiated per mask width in mapa_engine_w{1,2,4,8}.cu.
//
// Control flow of one independent batch (MAPA_BATCH_INDEPENDENT):
//   1. k_histogram counts requests per pattern; the host reads the counts
//      (one synchronisation) and k_scatter lays out each pattern's requests
//      contiguously.
//   2. Every group (requests of one pattern, sliced to <= 2^20) is enqueued
//      device-driven: level sizes stay on the device, so the whole batch is
//      one asynchronous launch sequence.
//   3. One synchronisation at the end; a group whose frontier outgrew its
//      level capacity is redone with the host-driven path, which produces
//      levels in chunks that fit (depth first).
// Sequential batches (and mapa_allocate) decide one request at a time
// against the device occupancy and commit each result (state management,
// Sec. 3.6).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "mapa_engine.h"
#include "mapa_runner.cuh"

namespace mapa {

// ----------------------------------------------------------------------------
// Non-templated kernels

// Exclusive scan of per-block child counts (one block); off[nb] = total.
__global__ void __launch_bounds__(1024) k_scan(const unsigned long long *cnt, unsigned long long *off, uint64_t nb) {
    __shared__ unsigned long long s_warp[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < nb; base += 1024) {
        const uint64_t i = base + threadIdx.x;
        const unsigned long long v = i < nb ? cnt[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long y = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(kFull, y, o);
                if (lane >= o) y += t;
            }
            s_warp[lane] = y;
        }
        __syncthreads();
        const unsigned long long before = (warp ? s_warp[warp - 1] : 0ull) + s_carry;
        if (i < nb) off[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[nb] = s_carry;
}

void launch_scan(const unsigned long long *cnt, unsigned long long *off, uint64_t nb, cudaStream_t s) {
    k_scan<<<1, 1024, 0, s>>>(cnt, off, nb);
}

__device__ __forceinline__ long long device_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return static_cast<long long>(t);
}

// Frees (one warp) every held vertex whose job's end time has passed and
// logs it with log position pos.
__device__ void expire_pass(int n, uint32_t *occ, int64_t *owner, int64_t *expire, const ServeLife &lf, int32_t pos,
                            int lane) {
    const long long now = device_clock_ns();
    for (int v = lane; v < n; v += 32) {
        const long long end = expire[v];
        if (end == 0 || end > now) continue;
        expire[v] = 0;
        const long long job = owner[v];
        if (job == 0) continue;
        owner[v] = 0;
        atomicAnd(occ + (v >> 5), ~(1u << (v & 31)));
        const uint32_t slot = atomicAdd(lf.n_log, 1u);
        if (slot < lf.cap) {
            lf.log_job[slot] = job;
            lf.log_pos[slot] = pos;
        }
    }
}

// Marks the k vertices of res busy under job (with its end time, 0 = none).
__device__ __forceinline__ void hold(const mapa_result &res, uint32_t *occ, int64_t *owner, int64_t *expire,
                                     long long job, long long end) {
    for (int i = 0; i < res.k; ++i) {
        const int v = res.verts[i];
        occ[v >> 5] |= 1u << (v & 31);
        owner[v] = job;
        expire[v] = end;
    }
}

__global__ void k_expire(int n, uint32_t *occ, int64_t *owner, int64_t *expire, ServeLife lf) {
    expire_pass(n, occ, owner, expire, lf, -1, threadIdx.x & 31);
}

// State management (Sec. 3.6): mark the chosen vertices busy under a new job id.
// With `blocked` (FIFO waiting): once a request of the chain did not fit,
// it and every later one are marked deferred (reserved = kDeferred) and
// nothing more is committed.
__global__ void k_commit(mapa_result *res, uint32_t *occ, int64_t *owner, int64_t *expire, unsigned long long *next_job,
                         int32_t *blocked) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (blocked) {
        if (*blocked || res->status == MAPA_NO_FIT) {
            *blocked = 1;
            res->reserved = kDeferred;
            return;
        }
    }
    if (res->status != MAPA_OK && res->status != MAPA_INEXACT) return;
    const long long job = static_cast<long long>(atomicAdd(next_job, 1ull)) + 1;
    hold(*res, occ, owner, expire, job, 0);
    res->job_id = job;
}

// One step of a commit chain, last kernel of the step (one warp): commits the
// decision at batch position *cursor as k_commit does (with its end time when
// lifetimes are kept on the device), logs the step's overflow flag for that
// position and clears it, moves the cursor to the next request, and then
// frees the vertices whose lifetime has ended before the next decision.
// Every kernel of a step reads its request through the cursor, so the launch
// sequence of a step is the same for every request of a pattern and can be
// replayed from one captured graph.
__global__ void k_commit_step(int n, mapa_result *out, int32_t *chain, uint32_t *occ, int64_t *owner, int64_t *expire,
                              unsigned long long *next_job, int32_t *blocked, int32_t *ovf_log, ServeLife lf) {
    const int lane = threadIdx.x & 31;
    const int32_t pos = chain[0];
    __syncwarp();
    if (lane == 0) {
        mapa_result *res = out + pos;
        ovf_log[pos] = chain[1];
        chain[1] = 0;
        chain[0] = pos + 1;
        bool commit = true;
        if (blocked) {
            if (*blocked || res->status == MAPA_NO_FIT) {
                *blocked = 1;
                res->reserved = kDeferred;
                commit = false;
            }
        }
        if (commit && (res->status == MAPA_OK || res->status == MAPA_INEXACT)) {
            const long long job = static_cast<long long>(atomicAdd(next_job, 1ull)) + 1;
            const long long life = lf.life ? lf.life[pos] : 0;
            hold(*res, occ, owner, expire, job, life > 0 ? device_clock_ns() + life : 0);
            res->job_id = job;
        }
    }
    __syncwarp();
    if (lf.life) expire_pass(n, occ, owner, expire, lf, pos + 1, lane);
}

// State management (Sec. 3.6): return a job's vertices to the free pool.
__global__ void k_release(int n, long long job, uint32_t *occ, int64_t *owner, int64_t *expire, int32_t *freed) {
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        if (owner[v] == job) {
            owner[v] = 0;
            expire[v] = 0;
            atomicAnd(occ + (v >> 5), ~(1u << (v & 31)));
            atomicAdd(freed, 1);
        }
    }
}

// Serving round commit (Sec. 3.6 state management, FIFO order of Sec. 4):
// decisions of one round were taken against the same occupancy snapshot;
// commit the longest prefix, in arrival order, whose decisions do not overlap
// one another.  conflict[i] = 1 from the first overlapping decision on (the
// server decides those again, in order, against the live occupancy);
// with fifo_wait, conflict[i] = 2 from the first request that did not fit on
// (it and everything behind it wait at the head of the queue).
__global__ void k_commit_round(mapa_result *res, int32_t n, uint32_t *occ, int64_t *owner, int64_t *expire,
                               unsigned long long *next_job, int32_t *conflict, int32_t fifo_wait,
                               const int64_t *life) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const long long now = device_clock_ns();
    uint32_t cur[MAPA_MASK_WORDS];
    for (int w = 0; w < MAPA_MASK_WORDS; ++w) cur[w] = occ[w];
    int32_t stop = 0;
    for (int i = 0; i < n; ++i) {
        conflict[i] = stop;
        if (stop) continue;
        if (fifo_wait && res[i].status == MAPA_NO_FIT) {
            stop = conflict[i] = 2;
            continue;
        }
        if (res[i].status != MAPA_OK && res[i].status != MAPA_INEXACT) continue;
        uint32_t mask[MAPA_MASK_WORDS] = {};
        for (int j = 0; j < res[i].k; ++j) {
            const int v = res[i].verts[j];
            mask[v >> 5] |= 1u << (v & 31);
        }
        bool clash = false;
        for (int w = 0; w < MAPA_MASK_WORDS; ++w) clash |= (mask[w] & cur[w]) != 0u;
        if (clash) {
            stop = conflict[i] = 1;
            continue;
        }
        const long long job = static_cast<long long>(atomicAdd(next_job, 1ull)) + 1;
        for (int w = 0; w < MAPA_MASK_WORDS; ++w) cur[w] |= mask[w];
        const long long lt = life ? life[i] : 0;
        for (int j = 0; j < res[i].k; ++j) {
            owner[res[i].verts[j]] = job;
            expire[res[i].verts[j]] = lt > 0 ? now + lt : 0;
        }
        res[i].job_id = job;
    }
    for (int w = 0; w < MAPA_MASK_WORDS; ++w) occ[w] = cur[w];
}

// Returns the vertices of several jobs to the free pool (Sec. 3.6).
__global__ void k_release_many(int n, const int64_t *jobs, int32_t njobs, uint32_t *occ, int64_t *owner,
                               int64_t *expire) {
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        const int64_t o = owner[v];
        if (o == 0) continue;
        for (int j = 0; j < njobs; ++j) {
            if (o == jobs[j]) {
                owner[v] = 0;
                expire[v] = 0;
                atomicAnd(occ + (v >> 5), ~(1u << (v & 31)));
                break;
            }
        }
    }
}

// Group key of a request: its pattern, and whether it is bandwidth-sensitive
// (scored by Eq. 2) -- npat * 2 keys.
__device__ __forceinline__ int32_t group_key(const mapa_request &q, int32_t npat) {
    return q.pattern_id + ((q.policy.flags & MAPA_POLICY_BW_SENSITIVE) ? npat : 0);
}

// Group requests by key: histogram (hist[key], then bounded-mode requests at
// hist[2 npat + key]), then scatter into per-key runs.
__global__ void k_histogram(const mapa_request *reqs, int32_t nreq, int32_t npat, int32_t *hist, mapa_result *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nreq; i += gridDim.x * blockDim.x) {
        const int32_t pid = reqs[i].pattern_id;
        if (pid < 0 || pid >= npat) {
            mapa_result res;
            memset(&res, 0, sizeof(res));
            res.status = MAPA_E_INVALID;
            out[i] = res;
        } else {
            const int32_t key = group_key(reqs[i], npat);
            atomicAdd(hist + key, 1);
            if (reqs[i].policy.mode == MAPA_MODE_BOUNDED) atomicAdd(hist + 2 * npat + key, 1);
        }
    }
}

__global__ void k_scatter(const mapa_request *reqs, int32_t nreq, int32_t npat, int32_t *cursor, int32_t *order) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nreq; i += gridDim.x * blockDim.x) {
        const int32_t pid = reqs[i].pattern_id;
        if (pid < 0 || pid >= npat) continue;
        order[atomicAdd(cursor + group_key(reqs[i], npat), 1)] = i;
    }
}

// ----------------------------------------------------------------------------
// Engine lifecycle

int ensure_device(char **ptr, uint64_t *have, uint64_t need, std::string *err) {
    if (*have >= need) return MAPA_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *have = 0;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), need);
    if (e != cudaSuccess) {
        if (err) *err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return MAPA_E_NOMEM;
    }
    *have = need;
    return MAPA_OK;
}

Engine *engine_create(int device, uint64_t frontier_cap, std::string *err) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        if (err)
            *err = std::string("no usable CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "bad index");
        return nullptr;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        if (err) *err = "cudaSetDevice failed";
        return nullptr;
    }
    Engine *en = new Engine();
    en->device = device;
    en->frontier_cap = frontier_cap ? frontier_cap : (4ull << 30);
    cudaDeviceGetAttribute(&en->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (en->sm_count < 1) en->sm_count = 1;
    if (const char *ov = std::getenv("MAPA_TAIL_DEPTH")) en->tail_override = std::atoi(ov);
    if (const char *ov = std::getenv("MAPA_TAIL_BLOCKS_PER_SM")) en->tail_blocks_per_sm = std::atoi(ov);
    if (const char *ov = std::getenv("MAPA_GRAPHS")) en->use_graphs = std::atoi(ov) != 0;
    if (const char *ov = std::getenv("MAPA_TAIL_SORT")) en->tail_sorted = std::atoi(ov) != 0;
    if (const char *ov = std::getenv("MAPA_CHUNK_SINGLE_PASS")) en->chunk_single_pass = std::atoi(ov) != 0;
    if (const char *ov = std::getenv("MAPA_DIVE_BLOCK")) en->dive_block = std::max(0, std::min(std::atoi(ov), 2));
    if (const char *ov = std::getenv("MAPA_DIVE_EAGER")) en->dive_eager = std::atoi(ov) != 0;
    if (const char *ov = std::getenv("MAPA_HOST_HINT")) en->host_hint_on = std::atoi(ov) != 0;
    if (const char *ov = std::getenv("MAPA_DIVE_STEPS")) en->dive_steps = std::max(0, std::min(std::atoi(ov), 1 << 20));
    if (const char *ov = std::getenv("MAPA_BOUND_DEGREE_MIN_M")) en->degree_min_m = std::max(0, std::atoi(ov));
    if (cudaStreamCreateWithFlags(&en->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&en->d_error, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&en->d_stats, kStatWords * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&en->d_chain, 3 * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&en->h_pinned, 64 * sizeof(unsigned long long)) != cudaSuccess) {
        if (err) *err = "context allocation failed";
        engine_destroy(en);
        return nullptr;
    }
    en->d_blocked = en->d_chain + 2;
    en->stream = en->own_stream;
    cudaMemset(en->d_error, 0, sizeof(int32_t));
    cudaMemset(en->d_stats, 0, kStatWords * sizeof(unsigned long long));
    return en;
}

void engine_destroy(Engine *e) {
    if (!e) return;
    cudaSetDevice(e->device);
    for (Slot &sl : e->slots) {
        if (sl.side) {
            cudaStreamSynchronize(sl.side);
            cudaStreamDestroy(sl.side);
        }
        if (sl.side_fork) cudaEventDestroy(sl.side_fork);
        if (sl.side_join) cudaEventDestroy(sl.side_join);
    }
    if (e->stream) cudaStreamSynchronize(e->stream);
    e->clear_graphs();
    for (Slot &sl : e->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        cudaFree(sl.arena);
        cudaFree(sl.group_mem);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (e->fork) cudaEventDestroy(e->fork);
    cudaFree(e->stage_reqs);
    cudaFree(e->stage_out);
    cudaFree(e->order);
    cudaFree(e->hist);
    cudaFree(e->overflow);
    cudaFree(e->d_error);
    cudaFree(e->d_stats);
    cudaFree(e->d_chain);
    cudaFree(e->effbw_rank);
    cudaFree(e->effbw_milli);
    for (cudaEvent_t ev : e->events) cudaEventDestroy(ev);
    if (e->h_pinned) cudaFreeHost(e->h_pinned);
    if (e->own_stream) cudaStreamDestroy(e->own_stream);
    delete e;
}

void engine_set_stream(Engine *e, cudaStream_t s) { e->stream = s ? s : e->own_stream; }
cudaStream_t engine_stream(Engine *e) { return e->stream; }

int engine_stats(Engine *e, mapa_stats *out) {
    *out = e->st;
    return MAPA_OK;
}

void engine_stats_reset(Engine *e) { e->st = mapa_stats{}; }

void engine_set_timing(Engine *e, bool on) { e->timing = on; }

void engine_set_work_budget(Engine *e, uint64_t max_partials) { e->work_budget = max_partials; }

uint64_t engine_tuned_chunk(const Engine *e, int32_t topo_id, int32_t pattern_id) {
    return chunk_limit(e, topo_id, pattern_id);
}

uint64_t engine_frontier_budget(const Engine *e) { return e->frontier_cap * static_cast<uint64_t>(kSlots); }

uint64_t engine_work_budget(const Engine *e) { return e->work_budget; }

int engine_stage(Engine *e, int32_t nreq, mapa_request **reqs_dev, mapa_result **out_dev, std::string *err) {
    if (nreq > e->stage_cap) {
        cudaFree(e->stage_reqs);
        cudaFree(e->stage_out);
        e->stage_reqs = nullptr;
        e->stage_out = nullptr;
        e->stage_cap = 0;
        const int32_t cap = std::max(nreq, 1024);
        if (cudaMalloc(&e->stage_reqs, sizeof(mapa_request) * cap) != cudaSuccess ||
            cudaMalloc(&e->stage_out, sizeof(mapa_result) * cap) != cudaSuccess) {
            if (err) *err = "cannot allocate request staging buffers";
            return MAPA_E_NOMEM;
        }
        e->stage_cap = cap;
    }
    *reqs_dev = e->stage_reqs;
    *out_dev = e->stage_out;
    return MAPA_OK;
}

// ----------------------------------------------------------------------------
// Frontier arena: levels 0..L carved from one allocation of frontier_cap
// bytes.  Level 0 holds the group's roots; levels 1..L share capacity E.

int plan_layout(Engine *e, int slot, int32_t group_size, int k, int T, int W, bool device_mode, int n,
                LayoutPlan *lay, std::string *err, uint64_t max_entries) {
    lay->L = k - T;
    const uint64_t cap = e->frontier_cap;
    const uint64_t lvl0 = static_cast<uint64_t>(std::max(group_size, 1));
    uint64_t per_entry = 0;
    for (int ell = 1; ell <= lay->L; ++ell) per_entry += entry_bytes(ell, W);
    const uint64_t scr_x1024 = device_mode ? 32 : 208;  // control bytes per 1024 entries of a level
    const uint64_t fixed = lvl0 * entry_bytes(0, W) + (lvl0 / 256 + 4) * 48 + 64 * 1024 + 4096 * (lay->L + 2);
    uint64_t E = 0;
    if (lay->L >= 1) {
        if (cap <= fixed) {
            if (err) *err = "frontier memory cap too small for this group";
            return MAPA_E_NOMEM;
        }
        E = (cap - fixed) * 1024 / (per_entry * 1024 + scr_x1024 * lay->L + 1);
        E = std::min<uint64_t>(E, kMaxLevelEntries);
        // a tuned level-size limit, never below one tile of children
        if (max_entries) E = std::min<uint64_t>(E, std::max<uint64_t>(max_entries, uint64_t(kTile) * n));
        E = E / kTile * kTile;
        if (E < static_cast<uint64_t>(kTile) * static_cast<uint64_t>(n)) {
            if (err) *err = "frontier memory cap too small (needs room for one tile of children per level)";
            return MAPA_E_NOMEM;
        }
    }
    lay->E = E;
    uint64_t total = 0;
    auto bump = [&](uint64_t bytes) {
        const uint64_t at = total;
        total = align_up(total + std::max<uint64_t>(bytes, 1), 256);
        return at;
    };
    uint64_t off_level[kMaxK + 1][4];
    uint64_t off_scr[kMaxK + 1][4];
    for (int ell = 0; ell <= lay->L; ++ell) {
        const uint64_t c = ell == 0 ? lvl0 : E;
        const int nwt = (ell + 3) / 4;
        off_level[ell][0] = bump(c * 4);
        off_level[ell][1] = bump(c * 4);
        off_level[ell][2] = bump(c * 4 * W);
        off_level[ell][3] = bump(c * 4 * std::max(nwt, 1));
        if (!device_mode && ell < lay->L) {
            const uint64_t nb = ceil_div(c, kTile) + 1;
            off_scr[ell][0] = bump(nb * kWarps * 4);
            off_scr[ell][1] = bump(nb * 8);
            off_scr[ell][2] = bump((nb + 1) * 8);
            off_scr[ell][3] = bump(nb * 32 * 4);
        }
    }
    // Level l of a group holds at most group_size * n^l entries (each entry
    // has fewer than n children), and never more than its capacity.
    lay->bound[0] = lvl0;
    for (int ell = 1; ell <= lay->L; ++ell) {
        const uint64_t b = lay->bound[ell - 1];
        lay->bound[ell] = b > E / static_cast<uint64_t>(std::max(n, 1)) ? E : std::min<uint64_t>(E, b * n);
    }
    const uint64_t ctrl_begin = total;
    const uint64_t off_counts = bump(8ull * (lay->L + 1));
    const uint64_t off_tiles = bump(4ull * (lay->L + 1));
    uint64_t off_status[kMaxK + 1];
    // look-back status words: device mode sized by the level bound, host
    // mode (chunks of at most a level's capacity) by the capacity
    for (int ell = 0; ell < lay->L; ++ell) {
        const uint64_t c = device_mode ? lay->bound[ell] : (ell == 0 ? lvl0 : E);
        off_status[ell] = bump(8ull * (c / kTpb + 2));
    }
    const uint64_t off_hctrl = bump(32ull * (lay->L + 1));
    const uint64_t ctrl_end = total;
    Slot &sl = e->slots[slot];
    uint64_t have = sl.arena_bytes;
    if (have < total) e->clear_graphs();  // captured launches point into the old arena
    const int rc = ensure_device(&sl.arena, &have, std::max<uint64_t>(total, 1), err);
    if (rc != MAPA_OK) return rc;
    sl.arena_bytes = have;
    char *base = sl.arena;
    for (int ell = 0; ell <= lay->L; ++ell) {
        LevelView &lv = lay->level[ell];
        lv.cap = ell == 0 ? lvl0 : E;
        lv.root = ell == 0;
        lv.S = reinterpret_cast<int32_t *>(base + off_level[ell][0]);
        lv.r = reinterpret_cast<uint32_t *>(base + off_level[ell][1]);
        lv.R = reinterpret_cast<uint32_t *>(base + off_level[ell][2]);
        lv.T = reinterpret_cast<uint32_t *>(base + off_level[ell][3]);
        if (!device_mode && ell < lay->L) {
            lay->warp_cnt[ell] = reinterpret_cast<uint32_t *>(base + off_scr[ell][0]);
            lay->blk_cnt[ell] = reinterpret_cast<unsigned long long *>(base + off_scr[ell][1]);
            lay->blk_off[ell] = reinterpret_cast<unsigned long long *>(base + off_scr[ell][2]);
            lay->cut_bits[ell] = reinterpret_cast<uint32_t *>(base + off_scr[ell][3]);
        }
        if (ell < lay->L) lay->status[ell] = reinterpret_cast<unsigned long long *>(base + off_status[ell]);
    }
    lay->hctrl = reinterpret_cast<unsigned long long *>(base + off_hctrl);
    lay->counts = reinterpret_cast<unsigned long long *>(base + off_counts);
    lay->tiles = reinterpret_cast<unsigned int *>(base + off_tiles);
    lay->ctrl = base + ctrl_begin;
    lay->ctrl_bytes = ctrl_end - ctrl_begin;
    return MAPA_OK;
}

// ----------------------------------------------------------------------------
// Batch driver

// Fused tail depth of a pattern.  The stored level k - T must hold more than
// the requests' roots when k >= 2, or one thread would walk a whole request.
static int tail_depth(const Engine *e, const TopoDevice &t, const PatternArgs &p) {
    if (e->tail_override > 0) return std::max(1, std::min({e->tail_override, 3, p.k}));
    const auto it = e->tail_table.find({t.id, p.id});
    if (it != e->tail_table.end()) return std::max(1, std::min(it->second, p.k));
    return p.k >= 3 ? 2 : 1;
}

static int ensure_effbw(Engine *e, std::string *err) {
    if (e->effbw_rank) return MAPA_OK;
    std::vector<int32_t> rank, milli;
    effbw_tables(&rank, &milli);
    const size_t bytes = rank.size() * sizeof(int32_t);
    MAPA_CUDA_TRY(cudaMalloc(&e->effbw_rank, bytes));
    MAPA_CUDA_TRY(cudaMalloc(&e->effbw_milli, bytes));
    MAPA_CUDA_TRY(cudaMemcpyAsync(e->effbw_rank, rank.data(), bytes, cudaMemcpyHostToDevice, e->stream));
    MAPA_CUDA_TRY(cudaMemcpyAsync(e->effbw_milli, milli.data(), bytes, cudaMemcpyHostToDevice, e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    return MAPA_OK;
}

static int run_group(Engine *e, const TopoDevice &t, const GroupRun &gr_in, bool device, std::string *err) {
    GroupRun gr = gr_in;
    gr.g.sens = 0;
    if (gr.sens) {
        // Eq. 2 ranks replace the score: no cut-offs, tail depth 1
        const int rc = ensure_effbw(e, err);
        if (rc != MAPA_OK) return rc;
        gr.bounded = false;
        gr.tail = 1;
        int edges = 0;
        for (int v = 0; v < gr.pat->k; ++v) edges += __builtin_popcount(gr.pat->back[v]);
        gr.g.sens = 1;
        gr.g.sens_ok = edges < kEffbwRadix;
        gr.g.effbw_rank = e->effbw_rank;
        gr.g.effbw_milli = e->effbw_milli;
        gr.g.effbw_code = t.wc_effbw;
    }
    // The work budget cuts a request through its threshold, so a budgeted
    // group keeps the threshold array even when no request is bounded.
    gr.g.work_budget = e->work_budget;
    if (!gr.g.work_budget) gr.g.work = nullptr;
    if (!gr.bounded && !gr.g.work) gr.g.thr = nullptr;
    switch (t.W) {
        case 1: return device ? run_group_device_w1(e, t, gr, err) : run_group_host_w1(e, t, gr, err);
        case 2: return device ? run_group_device_w2(e, t, gr, err) : run_group_host_w2(e, t, gr, err);
        case 4: return device ? run_group_device_w4(e, t, gr, err) : run_group_host_w4(e, t, gr, err);
        case 8: return device ? run_group_device_w8(e, t, gr, err) : run_group_host_w8(e, t, gr, err);
        default:
            if (err) *err = "internal: bad word count";
            return MAPA_E_INVALID;
    }
}

// Per-request group arrays (alpha, beta, key, count, best) of a slot for up
// to `size` requests.
static int group_arrays(Engine *e, int slot, int32_t size, GroupArgs *g, std::string *err) {
    const uint64_t n = static_cast<uint64_t>(std::max(size, 1));
    const uint64_t bytes = align_up(n * 4, 256) * 6 + align_up(n * 8, 256) * 3 + align_up(n * 32, 256) * 2;
    Slot &sl = e->slots[slot];
    uint64_t have = sl.group_bytes;
    if (have < bytes) e->clear_graphs();
    const int rc = ensure_device(&sl.group_mem, &have, bytes, err);
    if (rc != MAPA_OK) return rc;
    sl.group_bytes = have;
    char *p = sl.group_mem;
    auto take = [&](uint64_t b) {
        char *q = p;
        p += align_up(b, 256);
        return q;
    };
    g->alpha = reinterpret_cast<int32_t *>(take(n * 4));
    g->beta = reinterpret_cast<int32_t *>(take(n * 4));
    g->best_s = reinterpret_cast<int32_t *>(take(n * 4));
    g->best_valid = reinterpret_cast<int32_t *>(take(n * 4));
    g->thr = reinterpret_cast<int32_t *>(take(n * 4));
    g->key = reinterpret_cast<uint64_t *>(take(n * 8));
    g->count = reinterpret_cast<unsigned long long *>(take(n * 8));
    g->work = reinterpret_cast<unsigned long long *>(take(n * 8));
    g->dive_s = reinterpret_cast<int32_t *>(take(n * 4));
    g->dive_t = reinterpret_cast<uint32_t *>(take(n * 32));
    g->best_t = reinterpret_cast<uint32_t *>(take(n * 32));
    return MAPA_OK;
}

static int ensure_i32(Engine *e, int32_t **ptr, int32_t *cap, int64_t need, std::string *err) {
    uint64_t have = static_cast<uint64_t>(*cap) * 4;
    if (have < static_cast<uint64_t>(std::max<int64_t>(need, 1)) * 4) e->clear_graphs();
    char *p = reinterpret_cast<char *>(*ptr);
    const int rc = ensure_device(&p, &have, static_cast<uint64_t>(std::max<int64_t>(need, 1)) * 4, err);
    *ptr = reinterpret_cast<int32_t *>(p);
    *cap = static_cast<int32_t>(have / 4);
    return rc;
}

static int begin_batch(Engine *e, std::string *err) {
    e->events_used = 0;
    MAPA_CUDA_TRY(cudaMemsetAsync(e->d_stats, 0, kStatWords * sizeof(unsigned long long), e->stream));
    return MAPA_OK;
}

// After the batch's work: fold device counters and event times into the
// context stats and report device-side errors.
static int end_batch(Engine *e, std::string *err) {
    MAPA_CUDA_TRY(cudaMemcpyAsync(e->h_pinned, e->d_stats, kStatWords * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, e->stream));
    MAPA_CUDA_TRY(cudaMemcpyAsync(e->h_pinned + kStatWords, e->d_error, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    const unsigned long long *s = e->h_pinned;
    e->st.tail_nodes += s[kStatNodes];
    e->st.tail_leaves += s[kStatLeaves];
    e->st.embeddings += s[kStatLeaves];
    e->st.tail_parents += s[kStatParents];
    e->st.tail_int_ops += s[kStatOps];
    e->st.spill_entries += s[kStatSpill];
    e->st.spill_bytes += s[kStatSpillBytes];
    e->st.expand_bytes += s[kStatExpandBytes];
    if (e->timing) {
        for (size_t i = 0; i + 1 < e->events_used; i += 2) {
            float ms = 0.f;
            MAPA_CUDA_TRY(cudaEventElapsedTime(&ms, e->events[i], e->events[i + 1]));
            if (e->pair_kind[i / 2] == 1) e->st.expand_ms += ms;
            else e->st.tail_ms += ms;
        }
    }
    e->events_used = 0;
    int32_t h = 0;
    memcpy(&h, e->h_pinned + kStatWords, sizeof(int32_t));
    if (h != kDevOk) {
        cudaMemsetAsync(e->d_error, 0, sizeof(int32_t), e->stream);
        cudaStreamSynchronize(e->stream);
        if (h == kDevLookbackTimeout) {
            if (err) *err = "a bounded device wait gave up (frontier look-back)";
            return MAPA_E_TIMEOUT;
        }
        if (err)
            *err = h == kDevScoreMismatch ? "internal check failed: score disagrees with its tuple"
                                          : "internal check failed: argmax tail not re-found";
        return MAPA_E_STATE;
    }
    return MAPA_OK;
}

int engine_run_batch(Engine *e, const TopoDevice &t, const std::vector<PatternArgs> &patterns, int32_t nreq,
                     const mapa_request *reqs_dev, mapa_result *out_dev, bool sequential, std::string *err) {
    MAPA_CUDA_TRY(cudaSetDevice(e->device));
    if (nreq == 0) return MAPA_OK;
    const int32_t npat = static_cast<int32_t>(patterns.size());
    GroupArgs g;
    memset(&g, 0, sizeof(g));
    g.reqs = reqs_dev;
    g.out = out_dev;
    g.total_weight = t.total_weight;
    g.error = e->d_error;
    int rc = begin_batch(e, err);
    if (rc != MAPA_OK) return rc;

    if (sequential) {
        // One request at a time against the device occupancy, committing each.
        rc = group_arrays(e, 0, 1, &g, err);
        if (rc != MAPA_OK) return rc;
        rc = ensure_i32(e, &e->order, &e->order_cap, nreq, err);
        if (rc != MAPA_OK) return rc;
        rc = ensure_i32(e, &e->overflow, &e->overflow_cap, 1, err);
        if (rc != MAPA_OK) return rc;
        std::vector<int32_t> idx(nreq);
        for (int32_t i = 0; i < nreq; ++i) idx[i] = i;
        MAPA_CUDA_TRY(cudaMemcpyAsync(e->order, idx.data(), sizeof(int32_t) * nreq, cudaMemcpyHostToDevice, e->stream));
        std::vector<mapa_request> hreq(nreq);
        MAPA_CUDA_TRY(cudaMemcpyAsync(hreq.data(), reqs_dev, sizeof(mapa_request) * nreq, cudaMemcpyDeviceToHost,
                                      e->stream));
        MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
        g.occupancy = t.occupancy;
        g.size = 1;
        for (int32_t i = 0; i < nreq; ++i) {
            const int32_t pid = hreq[i].pattern_id;
            if (pid < 0 || pid >= npat) {
                mapa_result bad;
                memset(&bad, 0, sizeof(bad));
                bad.status = MAPA_E_INVALID;
                MAPA_CUDA_TRY(cudaMemcpyAsync(out_dev + i, &bad, sizeof(bad), cudaMemcpyHostToDevice, e->stream));
                MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
                continue;
            }
            g.req_index = e->order + i;
            GroupRun gr{&patterns[pid], g, tail_depth(e, t, patterns[pid]), e->overflow,
                        hreq[i].policy.mode == MAPA_MODE_BOUNDED,
                        (hreq[i].policy.flags & MAPA_POLICY_BW_SENSITIVE) != 0};
            MAPA_CUDA_TRY(cudaMemsetAsync(e->overflow, 0, sizeof(int32_t), e->stream));
            rc = run_group(e, t, gr, true, err);
            if (rc != MAPA_OK) return rc;
            MAPA_CUDA_TRY(cudaMemcpyAsync(e->h_pinned + 16, e->overflow, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                          e->stream));
            MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
            int32_t ovf = 0;
            memcpy(&ovf, e->h_pinned + 16, sizeof(int32_t));
            if (ovf) {
                GroupRun redo = gr;
                redo.redo = true;
                rc = run_group(e, t, redo, false, err);
                if (rc != MAPA_OK) return rc;
            }
            k_commit<<<1, 32, 0, e->stream>>>(out_dev + i, t.occupancy, t.owner, t.expire, t.next_job, nullptr);
            MAPA_CUDA_TRY(cudaGetLastError());
            e->st.kernel_launches += 1;
        }
        return end_batch(e, err);
    }

    // Independent requests: group by (pattern, sensitivity) on the device.
    const int32_t nkey = 2 * npat;
    rc = ensure_i32(e, &e->hist, &e->hist_cap, 2 * nkey + 1, err);
    if (rc != MAPA_OK) return rc;
    rc = ensure_i32(e, &e->order, &e->order_cap, nreq, err);
    if (rc != MAPA_OK) return rc;
    MAPA_CUDA_TRY(cudaMemsetAsync(e->hist, 0, sizeof(int32_t) * (2 * nkey + 1), e->stream));
    const unsigned hgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(nreq, 256), 1024));
    k_histogram<<<hgrid, 256, 0, e->stream>>>(reqs_dev, nreq, npat, e->hist, out_dev);
    std::vector<int32_t> hist(2 * nkey + 1);  // requests per key, then bounded-mode requests per key
    MAPA_CUDA_TRY(
        cudaMemcpyAsync(hist.data(), e->hist, sizeof(int32_t) * 2 * nkey, cudaMemcpyDeviceToHost, e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    std::vector<int32_t> start(nkey + 1, 0);
    for (int32_t p = 0; p < nkey; ++p) start[p + 1] = start[p] + hist[p];
    MAPA_CUDA_TRY(cudaMemcpyAsync(e->hist, start.data(), sizeof(int32_t) * nkey, cudaMemcpyHostToDevice, e->stream));
    k_scatter<<<hgrid, 256, 0, e->stream>>>(reqs_dev, nreq, npat, e->hist, e->order);
    MAPA_CUDA_TRY(cudaGetLastError());
    e->st.kernel_launches += 2;

    std::vector<GroupRun> runs;
    for (int32_t key = 0; key < nkey; ++key) {
        const int32_t p = key % npat;
        const bool sens = key >= npat;
        for (int32_t s0 = 0; s0 < hist[key]; s0 += kMaxGroup) {
            GroupArgs gs = g;
            gs.size = std::min(kMaxGroup, hist[key] - s0);
            gs.req_index = e->order + start[key] + s0;
            runs.push_back(GroupRun{&patterns[p], gs, tail_depth(e, t, patterns[p]), nullptr,
                                    hist[nkey + key] > 0, sens});
        }
    }
    if (runs.empty()) return end_batch(e, err);
    // A group whose device-driven run overflowed in one of the last batches
    // goes straight to the chunked path (the same result, without the
    // overflowing pass); every kHostHintBatches batches it tries again.
    constexpr int kHostHintBatches = 16, kHostHintMax = 1024;
    std::vector<char> direct(runs.size(), 0);
    if (e->host_hint_on)
        for (size_t i = 0; i < runs.size(); ++i) {
            auto h = e->host_hint.find({t.id, runs[i].pat->id});
            direct[i] = h != e->host_hint.end() && h->second.first > 0;
        }
    // The groups are independent: they run concurrently, one per slot (own
    // stream, arena and group arrays; round robin beyond kSlots), so one
    // group's small early levels overlap another's large ones.
    // With per-kernel timing on, groups run one after another so each timed
    // kernel has the GPU to itself.
    const int nslots = e->timing ? 1 : static_cast<int>(std::min<size_t>(kSlots, runs.size()));
    int32_t largest_in[kSlots] = {0, 0, 0, 0};
    for (size_t i = 0; i < runs.size(); ++i)
        largest_in[i % nslots] = std::max(largest_in[i % nslots], runs[i].g.size);
    GroupArgs arrays[kSlots];
    for (int s = 0; s < nslots; ++s) {
        rc = group_arrays(e, s, largest_in[s], &arrays[s], err);
        if (rc != MAPA_OK) return rc;
        Slot &sl = e->slots[s];
        if (nslots > 1 && !sl.stream) {
            MAPA_CUDA_TRY(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
            MAPA_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        }
    }
    if (nslots > 1 && !e->fork) MAPA_CUDA_TRY(cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming));
    rc = ensure_i32(e, &e->overflow, &e->overflow_cap, static_cast<int64_t>(runs.size()), err);
    if (rc != MAPA_OK) return rc;
    for (size_t i = 0; i < runs.size(); ++i) {
        GroupRun &gr = runs[i];
        gr.slot = static_cast<int>(i % nslots);
        gr.stream = nslots > 1 ? e->slots[gr.slot].stream : nullptr;
        const GroupArgs &a = arrays[gr.slot];
        gr.g.alpha = a.alpha;
        gr.g.beta = a.beta;
        gr.g.best_s = a.best_s;
        gr.g.best_valid = a.best_valid;
        gr.g.key = a.key;
        gr.g.count = a.count;
        gr.g.best_t = a.best_t;
        gr.g.thr = a.thr;
        gr.g.work = a.work;
        gr.g.dive_s = a.dive_s;
        gr.g.dive_t = a.dive_t;
        gr.overflow = e->overflow + i;
    }
    // Every group of the batch, device-driven.  A batch whose shape was seen
    // before (same topology, buffers, per-pattern sizes and tail depths)
    // replays its captured graph; a new shape is captured, then replayed.
    auto enqueue_all = [&]() -> int {
        MAPA_CUDA_TRY(cudaMemsetAsync(e->overflow, 0, sizeof(int32_t) * runs.size(), e->stream));
        if (nslots > 1) {
            MAPA_CUDA_TRY(cudaEventRecord(e->fork, e->stream));
            for (int s = 0; s < nslots; ++s) MAPA_CUDA_TRY(cudaStreamWaitEvent(e->slots[s].stream, e->fork, 0));
        }
        for (size_t i = 0; i < runs.size(); ++i) {
            if (direct[i]) continue;
            const int r = run_group(e, t, runs[i], true, err);
            if (r != MAPA_OK) return r;
        }
        if (nslots > 1) {
            for (int s = 0; s < nslots; ++s) {
                MAPA_CUDA_TRY(cudaEventRecord(e->slots[s].done, e->slots[s].stream));
                MAPA_CUDA_TRY(cudaStreamWaitEvent(e->stream, e->slots[s].done, 0));
            }
        }
        return MAPA_OK;
    };
    if (!e->use_graphs || e->timing) {
        rc = enqueue_all();
        if (rc != MAPA_OK) return rc;
    } else {
        std::vector<int64_t> key = {t.id, reinterpret_cast<int64_t>(reqs_dev), reinterpret_cast<int64_t>(out_dev),
                                    nreq, reinterpret_cast<int64_t>(e->overflow), reinterpret_cast<int64_t>(e->order),
                                    reinterpret_cast<int64_t>(e->stream), nslots,
                                    static_cast<int64_t>(e->work_budget)};
        for (int s = 0; s < nslots; ++s) {
            const Slot &sl = e->slots[s];
            key.push_back(reinterpret_cast<int64_t>(sl.arena));
            key.push_back(static_cast<int64_t>(sl.arena_bytes));
            key.push_back(reinterpret_cast<int64_t>(sl.group_mem));
            key.push_back(reinterpret_cast<int64_t>(sl.stream));
        }
        for (size_t i = 0; i < runs.size(); ++i) key.push_back(direct[i]);
        for (const GroupRun &gr : runs) {
            key.push_back(gr.pat->id);
            key.push_back(gr.g.size);
            key.push_back(gr.tail);
            key.push_back(gr.g.req_index - e->order);
            key.push_back(gr.bounded);
            key.push_back(gr.sens);
            key.push_back(static_cast<int64_t>(chunk_limit(e, t.id, gr.pat->id)));
        }
        auto it = e->graphs.find(key);
        const bool repeat = it != e->graphs.end() || e->shapes_seen.count(key) > 0;
        if (!repeat) {
            // first sighting of this shape: run it directly, capture if it recurs
            if (e->shapes_seen.size() >= 256) e->shapes_seen.clear();
            e->shapes_seen[key] = 1;
            rc = enqueue_all();
            if (rc != MAPA_OK) return rc;
        } else if (it == e->graphs.end()) {
            if (e->graphs.size() >= 32) e->clear_graphs();
            // plan every group once outside capture so no allocation happens inside it
            for (const GroupRun &gr : runs) {
                LayoutPlan lay;
                rc = plan_layout(e, gr.slot, gr.g.size, gr.pat->k, gr.tail, t.W, true, t.n, &lay, err,
                                 chunk_limit(e, t.id, gr.pat->id));
                if (rc != MAPA_OK) return rc;
            }
            const mapa_stats before = e->st;
            cudaGraph_t graph = nullptr;
            MAPA_CUDA_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeRelaxed));
            rc = enqueue_all();
            const cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
            if (rc != MAPA_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            Engine::GraphEntry entry;
            cudaError_t ie = ce;
            if (ce == cudaSuccess) ie = cudaGraphInstantiate(&entry.exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            const mapa_stats delta_src = e->st;
            e->st = before;
            if (ie != cudaSuccess) {
                // capture not possible here: drop graphs for this context, run directly
                cudaGetLastError();
                e->use_graphs = false;
                rc = enqueue_all();
                if (rc != MAPA_OK) return rc;
            } else {
                entry.delta.kernel_launches = delta_src.kernel_launches - before.kernel_launches;
                entry.delta.tail_launches = delta_src.tail_launches - before.tail_launches;
                entry.delta.requests = delta_src.requests - before.requests;
                it = e->graphs.emplace(key, entry).first;
            }
        }
        if (e->use_graphs && it != e->graphs.end()) {
            MAPA_CUDA_TRY(cudaGraphLaunch(it->second.exec, e->stream));
            e->st.kernel_launches += it->second.delta.kernel_launches;
            e->st.tail_launches += it->second.delta.tail_launches;
            e->st.requests += it->second.delta.requests;
        }
    }
    std::vector<int32_t> ovf(runs.size());
    MAPA_CUDA_TRY(cudaMemcpyAsync(ovf.data(), e->overflow, sizeof(int32_t) * runs.size(), cudaMemcpyDeviceToHost,
                                  e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    for (size_t i = 0; i < runs.size(); ++i) {
        if (!ovf[i] && !direct[i]) continue;
        // redo on the engine's stream (the slot's memory is free by now), so
        // its results are in place before anything later on that stream
        GroupRun redo = runs[i];
        redo.stream = nullptr;
        redo.redo = true;
        redo.detach = true;  // its dives and finish overlap the next redo
        rc = run_group(e, t, redo, false, err);
        if (rc != MAPA_OK) return rc;
    }
    for (Slot &sl : e->slots)
        if (sl.side_busy) {
            MAPA_CUDA_TRY(cudaStreamWaitEvent(e->stream, sl.side_join, 0));
            sl.side_busy = false;
        }
    // a retry that overflows again doubles the wait before the next one
    if (e->host_hint_on)
        for (size_t i = 0; i < runs.size(); ++i) {
            auto &h = e->host_hint[{t.id, runs[i].pat->id}];  // (batches left, period)
            if (ovf[i]) {
                h.second = h.second ? std::min(2 * h.second, kHostHintMax) : kHostHintBatches;
                h.first = h.second;
            } else if (direct[i] && h.first > 0) {
                --h.first;
            }
        }
    return end_batch(e, err);
}

// Decides reqs_dev[0..n) one after another against the live device
// occupancy, committing each before the next is decided (FIFO, Sec. 3.6),
// with every launch enqueued and a single synchronisation at the end.  A
// request whose frontier outgrows the arena makes the call fail with
// MAPA_E_NOMEM (its commit would not be trustworthy).
int engine_run_chain(Engine *e, const TopoDevice &t, const std::vector<PatternArgs> &patterns, int32_t n,
                     const int32_t *pattern_ids, const uint8_t *kinds, const mapa_request *reqs_dev,
                     mapa_result *out_dev, bool fifo_wait, mapa_result *out_host, const ServeLife *life,
                     std::string *err) {
    const ServeLife lf = life ? *life : ServeLife{};
    MAPA_CUDA_TRY(cudaSetDevice(e->device));
    if (n <= 0) return MAPA_OK;
    const int32_t npat = static_cast<int32_t>(patterns.size());
    for (int32_t i = 0; i < n; ++i)
        if (pattern_ids[i] < 0 || pattern_ids[i] >= npat) {
            if (err) *err = "unknown pattern id in a served request";
            return MAPA_E_INVALID;
        }
    GroupArgs g;
    memset(&g, 0, sizeof(g));
    g.reqs = reqs_dev;
    g.out = out_dev;
    g.total_weight = t.total_weight;
    g.error = e->d_error;
    g.occupancy = t.occupancy;
    g.size = 1;
    g.req_index = e->d_chain;  // the cursor: batch position of the step's request
    int rc = begin_batch(e, err);
    if (rc == MAPA_OK) rc = group_arrays(e, 0, 1, &g, err);
    if (rc == MAPA_OK) rc = ensure_i32(e, &e->overflow, &e->overflow_cap, n, err);
    if (rc != MAPA_OK) return rc;
    // cursor, step overflow flag and FIFO-wait flag; every step writes its
    // own entry of the overflow log
    MAPA_CUDA_TRY(cudaMemsetAsync(e->d_chain, 0, 3 * sizeof(int32_t), e->stream));
    int32_t *blocked = fifo_wait ? e->d_blocked : nullptr;
    auto step = [&](const GroupRun &gr) -> int {
        const int r = run_group(e, t, gr, true, err);
        if (r != MAPA_OK) return r;
        k_commit_step<<<1, 32, 0, e->stream>>>(t.n, out_dev, e->d_chain, t.occupancy, t.owner, t.expire, t.next_job,
                                                blocked, e->overflow, lf);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 1;
        return MAPA_OK;
    };
    for (int32_t i = 0; i < n; ++i) {
        const PatternArgs &pat = patterns[pattern_ids[i]];
        const bool bounded = kinds != nullptr && (kinds[i] & kKindBounded) != 0;
        const bool sens = kinds != nullptr && (kinds[i] & kKindSensitive) != 0;
        const GroupRun gr{&pat, g, tail_depth(e, t, pat), e->d_chain + 1, bounded, sens};
        if (!e->use_graphs || e->timing) {
            rc = step(gr);
            if (rc != MAPA_OK) return rc;
            continue;
        }
        // the launches of a step depend only on these: replay them from a
        // graph once a step of the same kind has run directly
        const Slot &sl = e->slots[0];
        const std::vector<int64_t> key = {-1, t.id, pat.id, gr.tail, bounded, sens, fifo_wait,
                                          reinterpret_cast<int64_t>(reqs_dev), reinterpret_cast<int64_t>(out_dev),
                                          reinterpret_cast<int64_t>(sl.arena), static_cast<int64_t>(sl.arena_bytes),
                                          reinterpret_cast<int64_t>(sl.group_mem), reinterpret_cast<int64_t>(e->overflow),
                                          reinterpret_cast<int64_t>(e->stream),
                                          static_cast<int64_t>(e->work_budget),
                                          reinterpret_cast<int64_t>(lf.life), reinterpret_cast<int64_t>(lf.log_job)};
        auto it = e->graphs.find(key);
        if (it == e->graphs.end() && e->shapes_seen.count(key)) {
            if (e->graphs.size() >= 64) e->clear_graphs();
            const mapa_stats before = e->st;
            cudaGraph_t graph = nullptr;
            MAPA_CUDA_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeRelaxed));
            rc = step(gr);
            const cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
            if (rc != MAPA_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            Engine::GraphEntry entry;
            cudaError_t ie = ce;
            if (ce == cudaSuccess) ie = cudaGraphInstantiate(&entry.exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            const mapa_stats delta_src = e->st;
            e->st = before;
            if (ie != cudaSuccess) {
                cudaGetLastError();
                e->use_graphs = false;  // capture not possible here: direct launches from now on
                rc = step(gr);
                if (rc != MAPA_OK) return rc;
                continue;
            }
            entry.delta.kernel_launches = delta_src.kernel_launches - before.kernel_launches;
            entry.delta.tail_launches = delta_src.tail_launches - before.tail_launches;
            entry.delta.requests = delta_src.requests - before.requests;
            it = e->graphs.emplace(key, entry).first;
        }
        if (it != e->graphs.end()) {
            MAPA_CUDA_TRY(cudaGraphLaunch(it->second.exec, e->stream));
            e->st.kernel_launches += it->second.delta.kernel_launches;
            e->st.tail_launches += it->second.delta.tail_launches;
            e->st.requests += it->second.delta.requests;
        } else {
            if (e->shapes_seen.size() >= 256) e->shapes_seen.clear();
            e->shapes_seen[key] = 1;
            rc = step(gr);
            if (rc != MAPA_OK) return rc;
        }
    }
    std::vector<int32_t> ovf(n);
    MAPA_CUDA_TRY(cudaMemcpyAsync(ovf.data(), e->overflow, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, e->stream));
    if (out_host)
        MAPA_CUDA_TRY(
            cudaMemcpyAsync(out_host, out_dev, sizeof(mapa_result) * n, cudaMemcpyDeviceToHost, e->stream));
    if (lf.host_n_log) {
        MAPA_CUDA_TRY(cudaMemcpyAsync(lf.host_n_log, lf.n_log, sizeof(uint32_t), cudaMemcpyDeviceToHost, e->stream));
        MAPA_CUDA_TRY(cudaMemcpyAsync(lf.host_log_job, lf.log_job, sizeof(int64_t) * lf.host_first,
                                      cudaMemcpyDeviceToHost, e->stream));
        MAPA_CUDA_TRY(cudaMemcpyAsync(lf.host_log_pos, lf.log_pos, sizeof(int32_t) * lf.host_first,
                                      cudaMemcpyDeviceToHost, e->stream));
    }
    rc = end_batch(e, err);
    if (rc != MAPA_OK) return rc;
    for (int32_t i = 0; i < n; ++i)
        if (ovf[i]) {
            if (err) *err = "a served request outgrew the frontier arena; raise frontier_mem_cap";
            return MAPA_E_NOMEM;
        }
    return MAPA_OK;
}

int engine_commit_round(Engine *e, const TopoDevice &t, mapa_result *out_dev, int32_t n, int32_t *conflict_dev,
                        bool fifo_wait, const ServeLife *life, std::string *err) {
    if (n <= 0) return MAPA_OK;
    k_commit_round<<<1, 32, 0, e->stream>>>(out_dev, n, t.occupancy, t.owner, t.expire, t.next_job, conflict_dev,
                                            fifo_wait ? 1 : 0, life ? life->life : nullptr);
    MAPA_CUDA_TRY(cudaGetLastError());
    e->st.kernel_launches += 1;
    return MAPA_OK;
}

int engine_release_many(Engine *e, const TopoDevice &t, const int64_t *jobs_dev, int32_t njobs, std::string *err) {
    if (njobs <= 0) return MAPA_OK;
    k_release_many<<<1, 256, 0, e->stream>>>(t.n, jobs_dev, njobs, t.occupancy, t.owner, t.expire);
    MAPA_CUDA_TRY(cudaGetLastError());
    e->st.kernel_launches += 1;
    return MAPA_OK;
}

int engine_expire(Engine *e, const TopoDevice &t, const ServeLife &life, std::string *err) {
    k_expire<<<1, 32, 0, e->stream>>>(t.n, t.occupancy, t.owner, t.expire, life);
    MAPA_CUDA_TRY(cudaGetLastError());
    e->st.kernel_launches += 1;
    return MAPA_OK;
}

int engine_autotune(Engine *e, const TopoDevice &t, const std::vector<PatternArgs> &patterns, int32_t nreq,
                    const mapa_request *reqs_host, int32_t *chosen, std::string *err) {
    MAPA_CUDA_TRY(cudaSetDevice(e->device));
    const int32_t npat = static_cast<int32_t>(patterns.size());
    for (int32_t p = 0; p < npat; ++p) chosen[p] = 0;
    if (e->tail_override > 0) {
        if (err) *err = "the tail depth is fixed by MAPA_TAIL_DEPTH";
        return MAPA_E_STATE;
    }
    std::vector<std::vector<mapa_request>> by_pattern(npat);
    for (int32_t i = 0; i < nreq; ++i) {
        const int32_t pid = reqs_host[i].pattern_id;
        if (pid >= 0 && pid < npat) by_pattern[pid].push_back(reqs_host[i]);
    }
    mapa_request *d_reqs = nullptr;
    mapa_result *d_out = nullptr;
    int rc = engine_stage(e, std::max(nreq, 1), &d_reqs, &d_out, err);
    if (rc != MAPA_OK) return rc;
    cudaEvent_t ev0, ev1;
    MAPA_CUDA_TRY(cudaEventCreate(&ev0));
    MAPA_CUDA_TRY(cudaEventCreate(&ev1));
    const bool timing = e->timing, graphs = e->use_graphs, hint = e->host_hint_on;
    // every trial runs the device-driven pass first: a setting whose levels
    // overflow pays for it here as it does whenever its group is retried
    e->host_hint_on = false;
    e->timing = false;
    e->use_graphs = false;  // time the launches themselves, not graph capture and instantiation
    const mapa_stats saved = e->st;
    for (int32_t p = 0; p < npat && rc == MAPA_OK; ++p) {
        const auto &rs = by_pattern[p];
        if (rs.empty()) continue;
        const int32_t n = static_cast<int32_t>(rs.size());
        rc = cudaMemcpyAsync(d_reqs, rs.data(), sizeof(mapa_request) * n, cudaMemcpyHostToDevice, e->stream) ==
                     cudaSuccess
                 ? MAPA_OK
                 : MAPA_E_CUDA;
        float best_ms = 0.f;
        int best_t = 0;
        for (int T = 1; T <= std::min(3, patterns[p].k) && rc == MAPA_OK; ++T) {
            e->tail_table[{t.id, p}] = T;
            float ms_min = 0.f;
            for (int rep = 0; rep < 3 && rc == MAPA_OK; ++rep) {  // first pass warms the arena and caches
                cudaEventRecord(ev0, e->stream);
                rc = engine_run_batch(e, t, patterns, n, d_reqs, d_out, false, err);
                cudaEventRecord(ev1, e->stream);
                cudaEventSynchronize(ev1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                if (rep == 1 || (rep > 1 && ms < ms_min)) ms_min = ms;
            }
            if (rc == MAPA_OK && (best_t == 0 || ms_min < best_ms)) {
                best_ms = ms_min;
                best_t = T;
            }
        }
        if (best_t) {
            e->tail_table[{t.id, p}] = best_t;
            chosen[p] = best_t;
            // then the level-size limit at that depth: none, 4M or 1M entries
            uint64_t best_c = 0;
            for (uint64_t lim : {uint64_t(1) << 22, uint64_t(1) << 20}) {
                if (rc != MAPA_OK) break;
                e->chunk_table[{t.id, p}] = lim;
                float ms_min = 0.f;
                for (int rep = 0; rep < 3 && rc == MAPA_OK; ++rep) {
                    cudaEventRecord(ev0, e->stream);
                    rc = engine_run_batch(e, t, patterns, n, d_reqs, d_out, false, err);
                    cudaEventRecord(ev1, e->stream);
                    cudaEventSynchronize(ev1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev0, ev1);
                    if (rep == 1 || (rep > 1 && ms < ms_min)) ms_min = ms;
                }
                if (rc == MAPA_OK && ms_min < 0.97f * best_ms) {  // keep a limit only for a clear gain
                    best_ms = ms_min;
                    best_c = lim;
                }
            }
            if (best_c) e->chunk_table[{t.id, p}] = best_c;
            else e->chunk_table.erase({t.id, p});
        }
    }
    e->st = saved;
    e->timing = timing;
    e->use_graphs = graphs;
    e->host_hint_on = hint;
    e->host_hint.clear();  // overflows seen while trying settings say nothing about the kept ones
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    return rc;
}

int engine_release(Engine *e, const TopoDevice &t, int64_t job_id, int32_t *freed, std::string *err) {
    MAPA_CUDA_TRY(cudaSetDevice(e->device));
    MAPA_CUDA_TRY(cudaMemsetAsync(t.scratch, 0, sizeof(int32_t), e->stream));
    k_release<<<1, 256, 0, e->stream>>>(t.n, static_cast<long long>(job_id), t.occupancy, t.owner, t.expire,
                                        t.scratch);
    MAPA_CUDA_TRY(cudaGetLastError());
    MAPA_CUDA_TRY(cudaMemcpyAsync(freed, t.scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    e->st.kernel_launches += 1;
    return MAPA_OK;
}

}  // namespace mapa
