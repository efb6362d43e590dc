// Host drivers of one request group, templated on the mask width W, the
// weight-class count CT and the fused tail depth T.  Included by the
// per-width translation units mapa_engine_w*.cu.
#pragma once

#include <algorithm>
#include <vector>

#include "mapa_engine.h"
#include "mapa_kernels.cuh"

namespace mapa {

// Frontier arena layout of one group run.
struct LayoutPlan {
    int L = 0;       // last stored level (= k - T)
    uint64_t E = 0;  // capacity of levels 1..L
    LevelView level[kMaxK + 1];
    // host-driven path: per-level block counts and offsets
    uint32_t *warp_cnt[kMaxK + 1];
    unsigned long long *blk_cnt[kMaxK + 1];
    unsigned long long *blk_off[kMaxK + 1];
    uint32_t *cut_bits[kMaxK + 1];  // count pass's cut decisions, 32 words per block
    // device-driven path: level counts, tile tickets, look-back status words
    unsigned long long *counts = nullptr;   // [L + 1]
    unsigned int *tiles = nullptr;          // [L + 1]
    unsigned long long *status[kMaxK + 1];  // [bound_l / kTpb + 2] per level l < L
    // host-driven single-pass chunks, per level: tile counter, stop tile,
    // resume record, child count (4 words)
    unsigned long long *hctrl = nullptr;
    uint64_t bound[kMaxK + 1];              // upper bound on the entries of level l (<= its capacity)
    char *ctrl = nullptr;                   // contiguous control region (zeroed per run)
    uint64_t ctrl_bytes = 0;
};

int plan_layout(Engine *e, int slot, int32_t group_size, int k, int T, int W, bool device_mode, int n,
                LayoutPlan *lay, std::string *err, uint64_t max_entries = 0);

// Tuned level-size limit of a (topology, pattern) (0 = none).
inline uint64_t chunk_limit(const Engine *e, int32_t topo_id, int32_t pattern_id) {
    const auto it = e->chunk_table.find({topo_id, pattern_id});
    return it == e->chunk_table.end() ? 0 : it->second;
}
void launch_scan(const unsigned long long *cnt, unsigned long long *off, uint64_t nb, cudaStream_t s);

inline TailArgs make_tail_args(const PatternArgs &pat, int T, int W, int C) {
    TailArgs ta{};
    ta.ell = pat.k - T;
    const uint32_t old = ta.ell == 0 ? 0u : ((ta.ell >= 32) ? ~0u : ((1u << ta.ell) - 1u));
    uint64_t backs = 0, los = 0;
    for (int t = 0; t < T; ++t) {
        const int v = ta.ell + t;
        ta.back_old[t] = pat.back[v] & old;
        ta.lo_old[t] = pat.lo[v] & old;
        ta.back_tail[t] = (pat.back[v] >> ta.ell) & ((1u << t) - 1u);
        ta.lo_tail[t] = (pat.lo[v] >> ta.ell) & ((1u << t) - 1u);
        backs += __builtin_popcount(ta.back_old[t]);
        los += __builtin_popcount(ta.lo_old[t]);
    }
    // Algorithmic integer operations per unit (the method's own work): a
    // parent at level i costs (|back[i]| + 3) W word operations for its
    // candidate mask, a generated child 2 C W + |back[i]| + 4 for its score
    // increment, and a complete match one more for the argmax compare.  A
    // node of the first tail level is a child of the parent and the parent
    // of the next level; a leaf is a child of the last level.
    (void)backs;
    (void)los;
    const uint64_t w = static_cast<uint64_t>(W), c = static_cast<uint64_t>(C);
    auto nback = [&](int v) { return static_cast<uint64_t>(__builtin_popcount(pat.back[v])); };
    const int last = pat.k - 1;
    ta.cost_parent = (nback(ta.ell) + 3) * w;
    ta.cost_node = T >= 2 ? (2 * c * w + nback(ta.ell) + 4) + (nback(ta.ell + 1) + 3) * w : 0;
    ta.cost_leaf = 2 * c * w + nback(last) + 4 + 1;
    ta.bound = level_bound(pat, ta.ell);
    return ta;
}

template <typename K>
inline int blocks_per_sm(K kernel, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kTpb, smem) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

template <int W, int CT, int T>
struct Runner {
    Engine *e;
    const TopoDevice &t;
    const GroupRun &gr;
    const PatternArgs &pat;
    GroupArgs g;
    TopoArgs targs;  // the graph as the scoring kernels see it (class codes for a sensitive group)
    cudaStream_t st;  // stream of the group's launches
    LayoutPlan lay;
    TailArgs ta;
    size_t smem_adj, smem_all;
    std::string *err;

    Runner(Engine *e_, const TopoDevice &t_, const GroupRun &gr_, std::string *err_)
        : e(e_), t(t_), gr(gr_), pat(*gr_.pat), g(gr_.g), targs(gr_.sens ? t_.args_effbw() : t_.args()),
          st(gr_.stream ? gr_.stream : e_->stream), err(err_) {
        smem_adj = topo_smem_bytes(t.n, W, t.C, false);
        smem_all = topo_smem_bytes(t.n, W, t.C, true);
        ta = make_tail_args(pat, T, W, t.C);
        ta.bound.degrees = ta.bound.m >= e->degree_min_m;
    }

    // Bound of the partials stored at level l (the degree term only where its
    // scan of R pays for itself: at least degree_min_m pattern vertices left).
    LevelBound bound_at(int l) const {
        LevelBound b = level_bound(pat, l);
        b.degrees = b.m >= e->degree_min_m;
        return b;
    }

    int allow_smem() {
        if (smem_all <= 48 * 1024) return MAPA_OK;
        const int b = static_cast<int>(smem_all);
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_setup<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_dive<W, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_dive_block<W, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_count<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_write<W, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_expand<W, CT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_expand<W, CT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_last<W, CT, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_last<W, CT, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        if constexpr (T <= 2 && W <= 2) {
            MAPA_CUDA_TRY(
                cudaFuncSetAttribute(k_last_short<W, CT, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
            MAPA_CUDA_TRY(cudaFuncSetAttribute(k_last_short<W, CT, T, false, true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        }
        if constexpr (T == 3 && W <= 2)
            MAPA_CUDA_TRY(cudaFuncSetAttribute(k_last_coop3<W, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        if constexpr (T == 1)
            MAPA_CUDA_TRY(
                cudaFuncSetAttribute(k_last_short<W, CT, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_resolve<W, CT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_finalize<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        return MAPA_OK;
    }

    // The dives of the group: one warp per request, or for guided (anytime)
    // requests one block each where the group is too small to fill the GPU
    // with warps (a served chain: one request); the outcome is the same.
    int dives(int fallback, const int32_t *overflow, cudaStream_t s) {
        const unsigned dgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, kWarps), 4096));
        const bool block_guided = e->dive_block == 1 || (e->dive_block == 2 && g.size < 2 * e->sm_count);
        k_dive<W, CT><<<dgrid, kTpb, smem_all, s>>>(targs, pat, g, lay.level[0], e->dive_steps, fallback, overflow,
                                                    block_guided ? 1 : 0);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 1;
        if (block_guided) {
            const unsigned bgrid = static_cast<unsigned>(std::min<uint64_t>(g.size, 8192));
            k_dive_block<W, CT><<<bgrid, kTpb, smem_all, s>>>(targs, pat, g, lay.level[0], e->dive_steps, fallback,
                                                              overflow);
            MAPA_CUDA_TRY(cudaGetLastError());
            e->st.kernel_launches += 1;
        }
        return MAPA_OK;
    }

    int setup(unsigned long long *count0) {
        const unsigned sgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, kWarps), 4096));
        k_setup<W><<<sgrid, kTpb, smem_all, st>>>(targs, g, lay.level[0], count0);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 1;
        MAPA_CUDA_TRY(cudaGetLastError());
        if (gr.bounded && !gr.sens) {
            // bounded mode: seed scores for the cut-offs (and the fallback
            // match of anytime requests); one warp per request, others skip
            const int rc = dives(0, nullptr, st);
            if (rc != MAPA_OK) return rc;
        }
        return MAPA_OK;
    }

    // Work budget: count the stored partials of each request in a level just
    // written and mark the requests past the budget.
    int budget(const LevelView &lv, const unsigned long long *count_dev, unsigned long long count_host) {
        if (!g.work) return MAPA_OK;
        const unsigned bgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, 256), 4096));
        k_budget<<<bgrid, 256, 0, st>>>(lv, count_dev, count_host, g);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 1;
        return MAPA_OK;
    }

    // eager: the anytime dives were started beside the enumeration on the
    // slot's side stream; finish after them -- on the side stream itself when
    // the run is detached (once the enumeration on st is done), else on st.
    int finalize(bool eager = false) {
        cudaStream_t fs = st;
        if (eager) {
            Slot &sl = e->slots[gr.slot];
            if (gr.detach) {
                MAPA_CUDA_TRY(cudaEventRecord(sl.side_fork, st));
                MAPA_CUDA_TRY(cudaStreamWaitEvent(sl.side, sl.side_fork, 0));
                fs = sl.side;
                sl.side_busy = true;
            } else {
                MAPA_CUDA_TRY(cudaStreamWaitEvent(st, sl.side_join, 0));
            }
        } else if (g.work && !gr.sens) {
            // exhaustive anytime requests past the budget: their fallback dive
            const int rc = dives(1, gr.redo ? nullptr : gr.overflow, st);
            if (rc != MAPA_OK) return rc;
        }
        // one warp per request, eight per block, at most two blocks per SM
        // (each block stages the topology once for all its requests)
        const unsigned fgrid =
            static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, kWarps), uint64_t(2) * e->sm_count));
        k_finalize<W><<<fgrid, kTpb, smem_all, fs>>>(t.args(), pat, g);  // real weights: AggBW, PreservedBW
        MAPA_CUDA_TRY(cudaGetLastError());
        if (fs != st) MAPA_CUDA_TRY(cudaEventRecord(e->slots[gr.slot].side_join, fs));
        e->st.kernel_launches += 1;
        e->st.requests += static_cast<uint64_t>(g.size);
        return MAPA_OK;
    }

    // Fused last levels over the stored level L (count on the device or given).
    int last_level(const unsigned long long *count_dev, unsigned long long count_host, unsigned int *tile_ctr,
                   uint64_t max_parents) {
        const LevelView &in = lay.level[lay.L];
        static int nb_last = 0;
        if (!nb_last) nb_last = blocks_per_sm(k_last<W, CT, T, false>, smem_all);
        const int per_sm = e->tail_blocks_per_sm > 0 ? e->tail_blocks_per_sm : nb_last;
        const unsigned grid = static_cast<unsigned>(
            std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(max_parents, kTile), uint64_t(e->sm_count) * per_sm)));
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (e->timing) {
            e->timed_pair(0, &ev0, &ev1);
            MAPA_CUDA_TRY(cudaEventRecord(ev0, st));
        }
        bool launched = false;
        const unsigned sgrid =
            static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(ceil_div(max_parents, kTile), 1u << 30)));
        if constexpr (T == 1) {
            if (g.sens) {
                // bandwidth-sensitive group: argmax over Eq. 2 ranks
                k_last_short<W, CT, 1, true><<<sgrid, kTpb, smem_all, st>>>(
                    targs, in, count_dev, count_host, ta, g.alpha, g.beta, g.key, g.count, e->d_stats, g.effbw_rank);
                launched = true;
            }
        }
        if constexpr (T == 3 && W <= 2) {
            if (!g.thr && !launched) {
                // depth 3: the first tail level handed out across lanes
                static int nb3 = 0;
                if (!nb3) nb3 = blocks_per_sm(k_last_coop3<W, CT>, smem_all);
                const unsigned cgrid = static_cast<unsigned>(std::max<uint64_t>(
                    1, std::min<uint64_t>(ceil_div(max_parents, kTpb), uint64_t(e->sm_count) * nb3)));
                k_last_coop3<W, CT><<<cgrid, kTpb, smem_all, st>>>(targs, in, count_dev, count_host, ta, g.alpha,
                                                                     g.beta, g.key, g.count, tile_ctr, e->d_stats);
                launched = true;
            }
        }
        if constexpr (T <= 2 && W <= 2) {
            if (!g.thr && !launched) {
                // masks of at most 64 vertices: one tile of parents per block
                auto tail = e->tail_sorted ? k_last_short<W, CT, T, false, true> : k_last_short<W, CT, T, false>;
                tail<<<sgrid, kTpb, smem_all, st>>>(targs, in, count_dev, count_host, ta, g.alpha, g.beta, g.key,
                                                    g.count, e->d_stats, nullptr);
                launched = true;
            }
        }
        if (launched) {
        } else if (g.thr) {
            k_last<W, CT, T, true><<<grid, kTpb, smem_all, st>>>(
                targs, in, count_dev, count_host, ta, g.alpha, g.beta, g.key, g.count, tile_ctr, e->d_stats, g.thr);
        } else {
            k_last<W, CT, T, false><<<grid, kTpb, smem_all, st>>>(
                targs, in, count_dev, count_host, ta, g.alpha, g.beta, g.key, g.count, tile_ctr, e->d_stats, g.thr);
        }
        MAPA_CUDA_TRY(cudaGetLastError());
        if (e->timing) MAPA_CUDA_TRY(cudaEventRecord(ev1, st));
        const unsigned rgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, 256), 1024));
        k_resolve<W, CT, T><<<rgrid, 256, smem_all, st>>>(targs, in, count_dev, count_host, ta, g);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 2;
        e->st.tail_launches += 1;
        return MAPA_OK;
    }

    // ---- device-driven: every launch enqueued, no host synchronisation
    int run_device() {
        int rc = allow_smem();
        if (rc != MAPA_OK) return rc;
        rc = plan_layout(e, gr.slot, g.size, pat.k, T, W, true, t.n, &lay, err, chunk_limit(e, t.id, pat.id));
        if (rc != MAPA_OK) return rc;
        MAPA_CUDA_TRY(cudaMemsetAsync(lay.ctrl, 0, lay.ctrl_bytes, st));
        rc = setup(lay.counts);
        if (rc != MAPA_OK) return rc;
        static int nb_expand = 0;
        if (!nb_expand) nb_expand = blocks_per_sm(k_expand<W, CT, false>, smem_all);
        auto expand = g.thr ? k_expand<W, CT, true> : k_expand<W, CT, false>;
        for (int ell = 0; ell < lay.L; ++ell) {
            const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(
                1, std::min<uint64_t>(ceil_div(lay.bound[ell], kTpb), uint64_t(e->sm_count) * nb_expand)));
            cudaEvent_t ev0 = nullptr, ev1 = nullptr;
            if (e->timing) {
                e->timed_pair(1, &ev0, &ev1);
                MAPA_CUDA_TRY(cudaEventRecord(ev0, st));
            }
            expand<<<grid, kTpb, smem_all, st>>>(
                targs, lay.level[ell], lay.level[ell + 1], ell, pat.back[ell], pat.lo[ell], lay.counts + ell,
                lay.counts + ell + 1, lay.level[ell + 1].cap, lay.tiles + ell, lay.status[ell], gr.overflow, g.alpha,
                g.beta, e->d_error, e->d_stats, entry_bytes(ell + 1, W), entry_bytes(ell, W), g.thr, bound_at(ell),
                0ull, 0, nullptr, nullptr);
            MAPA_CUDA_TRY(cudaGetLastError());
            if (e->timing) MAPA_CUDA_TRY(cudaEventRecord(ev1, st));
            e->st.kernel_launches += 1;
            e->st.expand_launches += 1;
            rc = budget(lay.level[ell + 1], lay.counts + ell + 1, 0ull);
            if (rc != MAPA_OK) return rc;
        }
        rc = last_level(lay.counts + lay.L, 0ull, lay.tiles + lay.L, lay.bound[lay.L]);
        if (rc != MAPA_OK) return rc;
        return finalize();
    }

    // ---- host-driven, single pass per chunk: k_expand writes the children
    // of a prefix of the parents [p0, p0 + P) that fits the level capacity
    // and reports where it stopped; that chunk is descended depth first,
    // then the level continues from the first unwritten parent.  Parents are
    // read once (a tile that did not fit is read again in the next chunk).
    int process_sp(int ell, uint64_t P) {
        if (P == 0) return MAPA_OK;
        if (ell == lay.L) {
            MAPA_CUDA_TRY(cudaMemsetAsync(lay.tiles, 0, sizeof(unsigned int), st));
            return last_level(nullptr, P, lay.tiles, P);
        }
        const LevelView &in = lay.level[ell];
        const LevelView &out = lay.level[ell + 1];
        unsigned long long *ctl = lay.hctrl + 4 * ell;  // tile counter, stop, resume, child count
        static int nb_expand = 0;
        if (!nb_expand) nb_expand = blocks_per_sm(k_expand<W, CT, false>, smem_all);
        auto expand = g.thr ? k_expand<W, CT, true> : k_expand<W, CT, false>;
        uint64_t p0 = 0;
        while (p0 < P) {
            const uint64_t pc = P - p0;
            const uint64_t nt = ceil_div(pc, kTpb);
            MAPA_CUDA_TRY(cudaMemsetAsync(lay.status[ell], 0, 8 * (nt + 2), st));
            MAPA_CUDA_TRY(cudaMemsetAsync(ctl, 0, 8, st));
            MAPA_CUDA_TRY(cudaMemsetAsync(ctl + 1, 0xFF, 16, st));
            const unsigned grid = static_cast<unsigned>(
                std::max<uint64_t>(1, std::min<uint64_t>(nt, uint64_t(e->sm_count) * nb_expand)));
            cudaEvent_t ev0 = nullptr, ev1 = nullptr;
            if (e->timing) {
                e->timed_pair(1, &ev0, &ev1);
                MAPA_CUDA_TRY(cudaEventRecord(ev0, st));
            }
            expand<<<grid, kTpb, smem_all, st>>>(
                targs, in, out, ell, pat.back[ell], pat.lo[ell], nullptr, ctl + 3, out.cap,
                reinterpret_cast<unsigned int *>(ctl), lay.status[ell], nullptr, g.alpha, g.beta, e->d_error, nullptr,
                entry_bytes(ell + 1, W), entry_bytes(ell, W), g.thr, bound_at(ell), pc, p0,
                reinterpret_cast<unsigned int *>(ctl + 1), ctl + 2);
            MAPA_CUDA_TRY(cudaGetLastError());
            if (e->timing) MAPA_CUDA_TRY(cudaEventRecord(ev1, st));
            MAPA_CUDA_TRY(
                cudaMemcpyAsync(e->h_pinned, ctl + 2, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            MAPA_CUDA_TRY(cudaStreamSynchronize(st));
            const unsigned long long resume = e->h_pinned[0], written_all = e->h_pinned[1];
            uint64_t consumed = pc, children = written_all;
            if (resume != ~0ull) {
                consumed = (resume >> 32) * kTpb;
                children = resume & 0xFFFFFFFFull;
            }
            if (consumed == 0) {
                if (err) *err = "internal: one tile's children exceed the level capacity";
                return MAPA_E_NOMEM;
            }
            e->st.kernel_launches += 1;
            e->st.expand_launches += 1;
            e->st.spill_entries += children;
            e->st.spill_bytes += 2 * children * entry_bytes(ell + 1, W);
            e->st.expand_bytes += consumed * entry_bytes(ell, W) + children * entry_bytes(ell + 1, W);
            int rc = budget(out, nullptr, children);
            if (rc != MAPA_OK) return rc;
            rc = process_sp(ell + 1, children);
            if (rc != MAPA_OK) return rc;
            p0 += consumed;
        }
        return MAPA_OK;
    }

    // ---- host-driven: counts read back per level, children produced in
    // chunks that fit the level capacity, depth first.
    int process(int ell, uint64_t P) {
        if (P == 0) return MAPA_OK;
        if (ell == lay.L) {
            MAPA_CUDA_TRY(cudaMemsetAsync(lay.tiles, 0, sizeof(unsigned int), st));
            return last_level(nullptr, P, lay.tiles, P);
        }
        const LevelView &in = lay.level[ell];
        const LevelView &out = lay.level[ell + 1];
        const uint64_t nb = ceil_div(P, kTile);
        cudaEvent_t cev0 = nullptr, cev1 = nullptr;
        if (e->timing) {
            e->timed_pair(1, &cev0, &cev1);
            MAPA_CUDA_TRY(cudaEventRecord(cev0, st));
        }
        k_count<W><<<static_cast<unsigned>(nb), kTpb, g.thr ? smem_all : smem_adj, st>>>(
            targs, in, P, pat.back[ell], pat.lo[ell], lay.warp_cnt[ell], lay.blk_cnt[ell], g.thr, g.alpha, g.beta,
            bound_at(ell), lay.cut_bits[ell]);
        MAPA_CUDA_TRY(cudaGetLastError());
        launch_scan(lay.blk_cnt[ell], lay.blk_off[ell], nb, st);
        MAPA_CUDA_TRY(cudaGetLastError());
        if (e->timing) MAPA_CUDA_TRY(cudaEventRecord(cev1, st));
        e->st.kernel_launches += 2;
        e->st.expand_launches += 1;
        e->st.expand_bytes += P * entry_bytes(ell, W);  // the parents, read once (algorithmically)
        MAPA_CUDA_TRY(cudaMemcpyAsync(e->h_pinned, lay.blk_off[ell] + nb, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, st));
        MAPA_CUDA_TRY(cudaStreamSynchronize(st));
        const unsigned long long total = e->h_pinned[0];
        if (total == 0) return MAPA_OK;
        std::vector<unsigned long long> off;
        if (total > lay.E) {
            off.resize(nb + 1);
            MAPA_CUDA_TRY(cudaMemcpyAsync(off.data(), lay.blk_off[ell], sizeof(unsigned long long) * (nb + 1),
                                          cudaMemcpyDeviceToHost, st));
            MAPA_CUDA_TRY(cudaStreamSynchronize(st));
        }
        uint64_t b0 = 0;
        while (b0 < nb) {
            uint64_t b1 = nb;
            if (total > lay.E) {
                b1 = std::upper_bound(off.begin() + b0 + 1, off.end(), off[b0] + lay.E) - off.begin() - 1;
                if (b1 <= b0) {
                    if (err) *err = "internal: one block's children exceed the level capacity";
                    return MAPA_E_NOMEM;
                }
            }
            const uint64_t children = total > lay.E ? off[b1] - off[b0] : total;
            cudaEvent_t wev0 = nullptr, wev1 = nullptr;
            if (e->timing) {
                e->timed_pair(1, &wev0, &wev1);
                MAPA_CUDA_TRY(cudaEventRecord(wev0, st));
            }
            k_write<W, CT><<<static_cast<unsigned>(b1 - b0), kTpb, smem_all, st>>>(
                targs, in, P, ell, pat.back[ell], pat.lo[ell], out, lay.warp_cnt[ell], lay.blk_off[ell], b0,
                g.alpha, g.beta, g.thr, lay.cut_bits[ell]);
            MAPA_CUDA_TRY(cudaGetLastError());
            if (e->timing) MAPA_CUDA_TRY(cudaEventRecord(wev1, st));
            e->st.kernel_launches += 1;
            e->st.expand_launches += 1;
            e->st.expand_bytes += children * entry_bytes(ell + 1, W);
            e->st.spill_entries += children;
            e->st.spill_bytes += 2 * children * entry_bytes(ell + 1, W);
            int rc = budget(out, nullptr, children);
            if (rc != MAPA_OK) return rc;
            rc = process(ell + 1, children);
            if (rc != MAPA_OK) return rc;
            b0 = b1;
        }
        return MAPA_OK;
    }

    int run_host() {
        Slot &slot = e->slots[gr.slot];
        if (slot.side_busy) {  // a detached run still uses the slot's memory
            MAPA_CUDA_TRY(cudaStreamSynchronize(slot.side));
            slot.side_busy = false;
        }
        int rc = allow_smem();
        if (rc != MAPA_OK) return rc;
        rc = plan_layout(e, gr.slot, g.size, pat.k, T, W, false, t.n, &lay, err, chunk_limit(e, t.id, pat.id));
        if (rc != MAPA_OK) return rc;
        rc = setup(nullptr);
        if (rc != MAPA_OK) return rc;
        // Under a work budget the anytime dives depend only on the request,
        // so they start now on a side stream, beside the enumeration (a dive
        // of a request that ends within its budget is not used).
        const bool eager = e->dive_eager && g.work && !gr.sens;
        if (eager) {
            // the slot's own side stream: the dives of the batch's host-driven
            // runs (one slot each) overlap one another as well
            Slot &sl = e->slots[gr.slot];
            if (!sl.side) {
                MAPA_CUDA_TRY(cudaStreamCreateWithFlags(&sl.side, cudaStreamNonBlocking));
                MAPA_CUDA_TRY(cudaEventCreateWithFlags(&sl.side_fork, cudaEventDisableTiming));
                MAPA_CUDA_TRY(cudaEventCreateWithFlags(&sl.side_join, cudaEventDisableTiming));
            }
            MAPA_CUDA_TRY(cudaEventRecord(sl.side_fork, st));
            MAPA_CUDA_TRY(cudaStreamWaitEvent(sl.side, sl.side_fork, 0));
            rc = dives(2, nullptr, sl.side);
            if (rc != MAPA_OK) return rc;
            MAPA_CUDA_TRY(cudaEventRecord(sl.side_join, sl.side));
        }
        rc = e->chunk_single_pass ? process_sp(0, static_cast<uint64_t>(g.size))
                                  : process(0, static_cast<uint64_t>(g.size));
        if (rc != MAPA_OK) return rc;
        return finalize(eager);
    }
};

// Picks the class-count specialisation and tail depth for a group.
template <int W, int CT>
inline int dispatch_tail(Engine *e, const TopoDevice &t, const GroupRun &gr, bool device, std::string *err) {
    switch (gr.tail) {
        case 1: {
            Runner<W, CT, 1> r(e, t, gr, err);
            return device ? r.run_device() : r.run_host();
        }
        case 2: {
            Runner<W, CT, 2> r(e, t, gr, err);
            return device ? r.run_device() : r.run_host();
        }
        case 3: {
            Runner<W, CT, 3> r(e, t, gr, err);
            return device ? r.run_device() : r.run_host();
        }
        default:
            if (err) *err = "internal: tail depth must be 1..3";
            return MAPA_E_INVALID;
    }
}

template <int W>
inline int dispatch_group(Engine *e, const TopoDevice &t, const GroupRun &gr, bool device, std::string *err) {
    if constexpr (W <= 2) {
        switch (t.C) {
            case 1: return dispatch_tail<W, 1>(e, t, gr, device, err);
            case 2: return dispatch_tail<W, 2>(e, t, gr, device, err);
            case 3: return dispatch_tail<W, 3>(e, t, gr, device, err);
            default: break;
        }
    } else {
        // wider masks: the two- and three-class graphs (the dragonfly and
        // boards workloads) get unrolled score increments too
        switch (t.C) {
            case 2: return dispatch_tail<W, 2>(e, t, gr, device, err);
            case 3: return dispatch_tail<W, 3>(e, t, gr, device, err);
            default: break;
        }
    }
    return dispatch_tail<W, 0>(e, t, gr, device, err);
}

}  // namespace mapa

#define MAPA_DEFINE_W(W)                                                                                        \
    namespace mapa {                                                                                           \
    int run_group_device_w##W(Engine *e, const TopoDevice &t, const GroupRun &gr, std::string *err) {         \
        return dispatch_group<W>(e, t, gr, true, err);                                                         \
    }                                                                                                          \
    int run_group_host_w##W(Engine *e, const TopoDevice &t, const GroupRun &gr, std::string *err) {           \
        return dispatch_group<W>(e, t, gr, false, err);                                                        \
    }                                                                                                          \
    }
