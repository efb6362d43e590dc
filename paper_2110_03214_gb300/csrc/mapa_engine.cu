// Device engine of the MAPA allocation hot path (sm_103a).
//
// What is computed (MAPA, arXiv 2110.03214, Sec. 3.3-3.6): for each request,
// every match phi of the pattern P in the free part F of the hardware graph
// (injective, adjacency-preserving, Sec. 3.3), its int32 score
//     S = alpha * AggBW(phi) + beta * PreservedBW(phi)          (Eq. 1, Eq. 3)
// and the argmax with the lexicographically smallest tuple among equal scores
// (Algorithm 1's strict ">" scan over a lexicographic enumeration).
//
// How (our design; the paper has no GPU kernel):
//   * Matches are grown one pattern vertex per level in pattern-id order.
//     A partial match at level l stores, in structure-of-arrays columns, its
//     running score S, its request r, R = F minus the vertices used so far,
//     and its tuple bytes.  Automorphism symmetry breaking keeps one map per
//     class: phi(j) < phi(i) for every j in lo[i].  With constraints chosen
//     in increasing id order the surviving map of each class is its
//     lexicographically smallest one, so the argmax tuple is exactly the one
//     a plain lexicographic scan over all maps would choose.
//   * Candidates of a partial: R & (AND over earlier neighbours b of adj[phi b])
//     & (bits above max over lo of phi), on bitsets held in shared memory.
//   * Incremental score of adding v with back-neighbour image set B and
//     remaining free set R (the sums run over weight classes c):
//         dS = sum_c w_c * (alpha * popc(B & cls_c[v]) - beta * popc(R & cls_c[v]))
//     The first term is v's share of Eq. 1, the second the links of v to
//     still-free vertices that Eq. 3 loses; the root starts at beta * W(F).
//   * Non-final levels are spilled to HBM: a count pass, a scan of per-block
//     counts and a write pass that expands children warp-cooperatively (each
//     lane emits one child, consecutive lanes write consecutive entries), so
//     every level stays in lexicographic order.  Frontiers larger than the
//     level capacity are processed in chunks, depth first.
//   * The last T levels (T = 1 or 2) are fused: no frontier write; each
//     thread scores its parent's subtree in registers and keeps the best
//     score; a warp-then-block reduction feeds one 64-bit atomicMax per
//     request of key = (biased S << 32) | ~parent.  Lexicographic order of
//     parents makes the smallest parent index the lexicographic tie-break;
//     a resolve pass re-walks the winning parent's subtree to recover the
//     tail in lexicographic order.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mapa_internal.h"

namespace mapa {

#define MAPA_CUDA_TRY(x)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                         \
            if (err) *err = std::string(#x) + ": " + cudaGetErrorString(e_);             \
            return MAPA_E_CUDA;                                                          \
        }                                                                                \
    } while (0)

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kNoReq = 0xFFFFFFFFu;

// ----------------------------------------------------------------------------
// Small device helpers

__device__ __forceinline__ uint32_t biased(int32_t s) { return static_cast<uint32_t>(s) ^ 0x80000000u; }
__device__ __forceinline__ int32_t unbiased(uint32_t b) { return static_cast<int32_t>(b ^ 0x80000000u); }

__host__ __device__ __forceinline__ uint32_t valid_word(int n, int w) {
    int lo = 32 * w;
    if (n >= lo + 32) return ~0u;
    if (n <= lo) return 0u;
    return (1u << (n - lo)) - 1u;
}

template <int W>
__device__ __forceinline__ void set_bit(uint32_t (&m)[W], int v) {
#pragma unroll
    for (int w = 0; w < W; ++w) m[w] |= ((v >> 5) == w) ? (1u << (v & 31)) : 0u;
}

template <int W>
__device__ __forceinline__ void clear_bit(uint32_t (&m)[W], int v) {
#pragma unroll
    for (int w = 0; w < W; ++w) m[w] &= ((v >> 5) == w) ? ~(1u << (v & 31)) : ~0u;
}

template <int W>
__device__ __forceinline__ int popc_mask(const uint32_t (&m)[W]) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popc(m[w]);
    return c;
}

// Keeps only vertices > lb (lb = -1 keeps all).
template <int W>
__device__ __forceinline__ void and_above(uint32_t (&c)[W], int lb) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int base = 32 * w;
        uint32_t m;
        if (lb < base)
            m = ~0u;
        else if (lb >= base + 31)
            m = 0u;
        else
            m = ~0u << (lb - base + 1);
        c[w] &= m;
    }
}

// Removes and returns the lowest set vertex of a W-word mask (-1 if empty).
template <int W>
__device__ __forceinline__ int pop_lowest(uint32_t (&m)[W]) {
    int v = -1;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        if (v < 0 && m[w] != 0u) {
            v = 32 * w + __ffs(m[w]) - 1;
            m[w] &= m[w] - 1u;
        }
    }
    return v;
}

// Position of the rank-th (0-based) set bit of x (x has more than rank bits set).
__device__ __forceinline__ int nth_bit32(uint32_t x, int rank) {
    int pos = 0;
    int c = __popc(x & 0xFFFFu);
    if (rank >= c) { rank -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xFFu);
    if (rank >= c) { rank -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xFu);
    if (rank >= c) { rank -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (rank >= c) { rank -= c; x >>= 2; pos += 2; }
    if (rank >= static_cast<int>(x & 1u)) pos += 1;
    return pos;
}

template <int W>
__device__ __forceinline__ int nth_bit(const uint32_t (&m)[W], int rank) {
    int v = 0;
    bool done = false;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int c = __popc(m[w]);
        if (!done) {
            if (rank < c) {
                v = 32 * w + nth_bit32(m[w], rank);
                done = true;
            } else {
                rank -= c;
            }
        }
    }
    return v;
}

// Topology bitsets staged in shared memory.
struct SmemTopo {
    const uint32_t *adj;
    const uint32_t *cls;
    const int32_t *wc;
    int n, C;
};

__host__ __device__ inline size_t topo_smem_bytes(int n, int W, int C, bool with_cls) {
    size_t words = static_cast<size_t>(n) * W;
    if (with_cls) words += static_cast<size_t>(n) * C * W + C;
    return words * 4;
}

template <int W>
__device__ __forceinline__ SmemTopo stage_topology(const TopoArgs &t, bool with_cls) {
    extern __shared__ uint32_t smem_words[];
    uint32_t *adj = smem_words;
    uint32_t *cls = adj + t.n * W;
    int32_t *wc = reinterpret_cast<int32_t *>(cls + (with_cls ? t.n * t.C * W : 0));
    for (int i = threadIdx.x; i < t.n * W; i += blockDim.x) adj[i] = t.adj[i];
    if (with_cls) {
        for (int i = threadIdx.x; i < t.n * t.C * W; i += blockDim.x) cls[i] = t.clsv[i];
        for (int i = threadIdx.x; i < t.C; i += blockDim.x) wc[i] = t.wc[i];
    }
    __syncthreads();
    return SmemTopo{adj, cls, wc, t.n, t.C};
}

__device__ __forceinline__ int tuple_byte(const LevelView &L, uint64_t p, int j) {
    return static_cast<int>((L.T[static_cast<uint64_t>(j >> 2) * L.cap + p] >> ((j & 3) * 8)) & 0xFFu);
}

// Intersection of the adjacency rows of the placed back-neighbours (A), the
// set of their images (B) and the lower bound from the order constraints.
template <int W>
__device__ __forceinline__ void level_masks(const LevelView &L, uint64_t p, uint32_t back, uint32_t lo,
                                            const uint32_t *s_adj, uint32_t (&A)[W], uint32_t (&B)[W], int &lb) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        A[w] = ~0u;
        B[w] = 0u;
    }
    lb = -1;
    while (back) {
        const int b = __ffs(back) - 1;
        back &= back - 1u;
        const int x = tuple_byte(L, p, b);
#pragma unroll
        for (int w = 0; w < W; ++w) A[w] &= s_adj[x * W + w];
        set_bit<W>(B, x);
    }
    while (lo) {
        const int a = __ffs(lo) - 1;
        lo &= lo - 1u;
        lb = max(lb, tuple_byte(L, p, a));
    }
}

// Score change from adding vertex v (see the file header).
template <int W>
__device__ __forceinline__ int32_t delta(const SmemTopo &s, int v, const uint32_t (&B)[W], const uint32_t (&Rr)[W],
                                         int32_t alpha, int32_t beta) {
    const uint32_t *x = s.cls + static_cast<size_t>(v) * s.C * W;
    int32_t acc = 0;
    for (int c = 0; c < s.C; ++c) {
        int pb = 0, pr = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t xw = x[c * W + w];
            pb += __popc(B[w] & xw);
            pr += __popc(Rr[w] & xw);
        }
        acc += s.wc[c] * (alpha * pb - beta * pr);
    }
    return acc;
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Tail description for the fused last levels.
struct TailArgs {
    int32_t ell;     // level of the stored parents (= k - T)
    uint32_t back0;  // earlier neighbours of pattern vertex ell
    uint32_t lo0;
    uint32_t back1;  // of vertex ell + 1 (T == 2)
    uint32_t lo1;
};

// ----------------------------------------------------------------------------
// Kernels

// Per request: free set F, root entry (S = beta * W(F), R = F), accumulators.
template <int W>
__global__ void k_setup(TopoArgs topo, GroupArgs g, LevelView L0) {
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31;
    const int gw = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = static_cast<int>((gridDim.x * blockDim.x) >> 5);
    for (int i = gw; i < g.size; i += nw) {
        const mapa_request &q = g.reqs[g.req_index[i]];
        uint32_t F[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint32_t busy = q.busy[w];
            if (g.occupancy) busy |= g.occupancy[w];
            F[w] = ~busy & valid_word(s.n, w);
        }
        long long acc = 0;
        for (int v = lane; v < s.n; v += 32) {
            if (!((F[v >> 5] >> (v & 31)) & 1u)) continue;
            const uint32_t *x = s.cls + static_cast<size_t>(v) * s.C * W;
            for (int c = 0; c < s.C; ++c) {
                int pc = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) pc += __popc(x[c * W + w] & F[w]);
                acc += static_cast<long long>(s.wc[c]) * pc;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) {
            const int32_t al = q.policy.alpha, be = q.policy.beta;
            const long long mag = (llabs(static_cast<long long>(al)) + llabs(static_cast<long long>(be))) *
                                  static_cast<long long>(g.total_weight);
            int32_t state = 0;
            if (q.policy.mode != MAPA_MODE_EXHAUSTIVE) state = -3;
            else if (mag >= (1LL << 31)) state = -2;
            const long long wfree = acc / 2;
            L0.S[i] = state == 0 ? static_cast<int32_t>(be * wfree) : 0;
            L0.r[i] = static_cast<uint32_t>(i);
#pragma unroll
            for (int w = 0; w < W; ++w) L0.R[w * L0.cap + i] = state == 0 ? F[w] : 0u;
            g.alpha[i] = al;
            g.beta[i] = be;
            g.key[i] = 0ull;
            g.count[i] = 0ull;
            g.best_valid[i] = state;
        }
    }
}

// Count pass: children of every parent, summed per warp and per block.
template <int W>
__global__ void __launch_bounds__(kTpb) k_count(TopoArgs topo, LevelView in, uint64_t P, uint32_t back, uint32_t lo,
                                                uint32_t *warp_cnt, unsigned long long *blk_cnt) {
    const SmemTopo s = stage_topology<W>(topo, false);
    __shared__ uint32_t s_w[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t wbase = static_cast<uint64_t>(blockIdx.x) * kTile + static_cast<uint64_t>(warp) * 32 * kIpt;
    int wsum = 0;
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint64_t p = wbase + j * 32 + lane;
        int cnt = 0;
        if (p < P) {
            uint32_t A[W], B[W], c[W];
            int lb;
            level_masks<W>(in, p, back, lo, s.adj, A, B, lb);
#pragma unroll
            for (int w = 0; w < W; ++w) c[w] = in.R[w * in.cap + p] & A[w];
            and_above<W>(c, lb);
            cnt = popc_mask<W>(c);
        }
        wsum += warp_sum_int(cnt);
    }
    if (lane == 0) {
        warp_cnt[static_cast<uint64_t>(blockIdx.x) * kWarps + warp] = static_cast<uint32_t>(wsum);
        s_w[warp] = static_cast<uint32_t>(wsum);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kWarps; ++w) t += s_w[w];
        blk_cnt[blockIdx.x] = t;
    }
}

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

// Write pass: load-balanced child expansion.  Each warp owns 32 * kIpt
// consecutive parents; for each group of 32 parents the warp scans their
// child counts and then emits children 32 at a time, lane c taking child c:
// it finds its parent by a binary search over the scanned counts, fetches the
// parent's masks by shuffle and writes one entry, so the stores of a warp are
// consecutive in every column and children keep lexicographic order.
template <int W>
__global__ void __launch_bounds__(kTpb) k_write(TopoArgs topo, LevelView in, uint64_t P, int ell, uint32_t back,
                                                uint32_t lo, LevelView out, const uint32_t *warp_cnt,
                                                const unsigned long long *blk_off, uint64_t blk_first,
                                                const int32_t *alpha, const int32_t *beta) {
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t b = blk_first + blockIdx.x;
    uint64_t obase = blk_off[b] - blk_off[blk_first];
    for (int w2 = 0; w2 < warp; ++w2) obase += warp_cnt[b * kWarps + w2];
    const uint64_t wbase = b * kTile + static_cast<uint64_t>(warp) * 32 * kIpt;
    const int nw_in = (ell + 3) >> 2;
    const int new_word = ell >> 2;
    const uint32_t new_shift = (ell & 3) * 8;
    for (int j = 0; j < kIpt; ++j) {
        const uint64_t p = wbase + j * 32 + lane;
        uint32_t cand[W], B[W], R[W];
        int32_t S = 0;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cand[w] = B[w] = R[w] = 0u;
        if (p < P) {
            uint32_t A[W];
            int lb;
            level_masks<W>(in, p, back, lo, s.adj, A, B, lb);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                R[w] = in.R[w * in.cap + p];
                cand[w] = R[w] & A[w];
            }
            and_above<W>(cand, lb);
            S = in.S[p];
            r = in.r[p];
        }
        const int cnt = popc_mask<W>(cand);
        const int incl = warp_incl_scan(cnt, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        for (int c0 = 0; c0 < total; c0 += 32) {
            const int c = c0 + lane;
            int src = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int t = __shfl_sync(kFull, incl, src + step - 1);
                if (t <= c) src += step;
            }
            const int incl_s = __shfl_sync(kFull, incl, src);
            const int cnt_s = __shfl_sync(kFull, cnt, src);
            uint32_t cs[W], Bs[W], Rs[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                cs[w] = __shfl_sync(kFull, cand[w], src);
                Bs[w] = __shfl_sync(kFull, B[w], src);
                Rs[w] = __shfl_sync(kFull, R[w], src);
            }
            const int32_t Ss = __shfl_sync(kFull, S, src);
            const uint32_t rs = __shfl_sync(kFull, r, src);
            if (c < total) {
                const int v = nth_bit<W>(cs, c - (incl_s - cnt_s));
                const int32_t d = delta<W>(s, v, Bs, Rs, alpha[rs], beta[rs]);
                const uint64_t o = obase + c;
                const uint64_t ps = wbase + j * 32 + src;
                out.S[o] = Ss + d;
                out.r[o] = rs;
                clear_bit<W>(Rs, v);
#pragma unroll
                for (int w = 0; w < W; ++w) out.R[w * out.cap + o] = Rs[w];
                for (int jw = 0; jw < nw_in; ++jw) {
                    uint32_t word = in.T[jw * in.cap + ps];
                    if (jw == new_word) word |= static_cast<uint32_t>(v) << new_shift;
                    out.T[jw * out.cap + o] = word;
                }
                if (new_shift == 0) out.T[new_word * out.cap + o] = static_cast<uint32_t>(v);
            }
        }
        obase += total;
    }
}

// Enumerates the fused tail (T levels) of parent p and reports, for every
// complete match, its score to `leaf(score)`; returns false as soon as
// `leaf` returns false.
template <int W, int T, typename Leaf>
__device__ __forceinline__ bool walk_tail(const SmemTopo &s, const LevelView &in, uint64_t p, const TailArgs &ta,
                                          int32_t al, int32_t be, Leaf &&leaf, uint32_t *nodes = nullptr) {
    const int32_t S = in.S[p];
    uint32_t R[W], A[W], B[W], c1[W];
    int lb;
    level_masks<W>(in, p, ta.back0, ta.lo0, s.adj, A, B, lb);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        R[w] = in.R[w * in.cap + p];
        c1[w] = R[w] & A[w];
    }
    and_above<W>(c1, lb);
    if constexpr (T == 1) {
        int v;
        while ((v = pop_lowest<W>(c1)) >= 0) {
            if (!leaf(S + delta<W>(s, v, B, R, al, be), v, -1)) return false;
        }
    } else {
        const uint32_t newbit = 1u << ta.ell;
        uint32_t A2[W], B2[W];
        int lb2;
        level_masks<W>(in, p, ta.back1 & ~newbit, ta.lo1 & ~newbit, s.adj, A2, B2, lb2);
        const bool nb = (ta.back1 & newbit) != 0u;
        const bool nl = (ta.lo1 & newbit) != 0u;
        int v1;
        while ((v1 = pop_lowest<W>(c1)) >= 0) {
            if (nodes) ++*nodes;
            const int32_t s1 = S + delta<W>(s, v1, B, R, al, be);
            uint32_t R1[W], c2[W], B2n[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                R1[w] = R[w];
                B2n[w] = B2[w];
            }
            clear_bit<W>(R1, v1);
            if (nb) set_bit<W>(B2n, v1);
#pragma unroll
            for (int w = 0; w < W; ++w) c2[w] = R1[w] & A2[w] & (nb ? s.adj[v1 * W + w] : ~0u);
            and_above<W>(c2, nl ? max(lb2, v1) : lb2);
            int v2;
            while ((v2 = pop_lowest<W>(c2)) >= 0) {
                if (!leaf(s1 + delta<W>(s, v2, B2n, R1, al, be), v1, v2)) return false;
            }
        }
    }
    return true;
}

__device__ __forceinline__ void flush_request(uint64_t *key, unsigned long long *count, uint32_t r, uint64_t k,
                                              unsigned long long c) {
    if (c == 0ull) return;
    atomicMax(reinterpret_cast<unsigned long long *>(key + r), static_cast<unsigned long long>(k));
    atomicAdd(count + r, c);
}

// Fused last levels: count and argmax key per request, no frontier write.
template <int W, int T>
__global__ void __launch_bounds__(kTpb) k_last(TopoArgs topo, LevelView in, uint64_t P, TailArgs ta,
                                               const int32_t *alpha, const int32_t *beta, uint64_t *key,
                                               unsigned long long *count, unsigned long long *stats) {
    const SmemTopo s = stage_topology<W>(topo, true);
    __shared__ uint32_t s_r[kWarps];
    __shared__ unsigned long long s_key[kWarps];
    __shared__ unsigned long long s_cnt[kWarps];
    __shared__ unsigned long long s_nodes;
    if (threadIdx.x == 0) s_nodes = 0ull;
    uint32_t nodes = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t wbase = static_cast<uint64_t>(blockIdx.x) * kTile + static_cast<uint64_t>(warp) * 32 * kIpt;
    uint32_t r_cur = kNoReq;
    unsigned long long bkey = 0ull, bcnt = 0ull;
    for (int j = 0; j < kIpt; ++j) {
        const uint64_t p = wbase + j * 32 + lane;
        if (p >= P) continue;
        const uint32_t r = in.r[p];
        if (r != r_cur) {
            if (r_cur != kNoReq) flush_request(key, count, r_cur, bkey, bcnt);
            r_cur = r;
            bkey = 0ull;
            bcnt = 0ull;
        }
        int32_t smax = INT_MIN;
        uint32_t leaves = 0;
        walk_tail<W, T>(
            s, in, p, ta, alpha[r], beta[r],
            [&](int32_t sc, int, int) {
                smax = max(smax, sc);
                ++leaves;
                return true;
            },
            &nodes);
        if (leaves) {
            const unsigned long long k64 =
                (static_cast<unsigned long long>(biased(smax)) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(p));
            bkey = max(bkey, k64);
            bcnt += leaves;
        }
    }
    // warp, then block aggregation of (request, key, count)
    const int wn = warp_sum_int(static_cast<int>(nodes));
    if (lane == 0) {
        s_r[warp] = kNoReq;
        if (wn) atomicAdd(&s_nodes, static_cast<unsigned long long>(wn));
    }
    const unsigned act = __ballot_sync(kFull, bcnt > 0ull);
    if (act) {
        const int lead = __ffs(act) - 1;
        const uint32_t rl = __shfl_sync(kFull, r_cur, lead);
        const bool uniform = __all_sync(kFull, bcnt == 0ull || r_cur == rl);
        if (uniform) {
            unsigned long long k = bkey, c = bcnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                k = max(k, __shfl_xor_sync(kFull, k, o));
                c += __shfl_xor_sync(kFull, c, o);
            }
            if (lane == 0) {
                s_r[warp] = rl;
                s_key[warp] = k;
                s_cnt[warp] = c;
            }
        } else if (bcnt) {
            flush_request(key, count, r_cur, bkey, bcnt);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r = kNoReq;
        unsigned long long k = 0ull, c = 0ull;
        for (int w = 0; w < kWarps; ++w) {
            if (s_r[w] == kNoReq) continue;
            if (s_r[w] != r) {
                if (r != kNoReq) flush_request(key, count, r, k, c);
                r = s_r[w];
                k = 0ull;
                c = 0ull;
            }
            k = max(k, s_key[w]);
            c += s_cnt[w];
        }
        if (r != kNoReq) flush_request(key, count, r, k, c);
        if (s_nodes) atomicAdd(stats, s_nodes);
    }
}

// Per request present in a last-level chunk: decode the chunk's argmax key,
// re-walk the winning parent's tail in lexicographic order to recover the
// first tail reaching that score, and merge into the running best with a
// strict ">" (chunks arrive in lexicographic order).
template <int W, int T>
__global__ void k_resolve(TopoArgs topo, LevelView in, uint64_t P, TailArgs ta, GroupArgs g) {
    const SmemTopo s = stage_topology<W>(topo, true);
    if (P == 0) return;
    const uint32_t r_lo = in.r[0], r_hi = in.r[P - 1];
    for (uint64_t rr = r_lo + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; rr <= r_hi;
         rr += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t r = static_cast<uint32_t>(rr);
        const unsigned long long k64 = g.key[r];
        if (k64 == 0ull) continue;
        g.key[r] = 0ull;
        const int32_t target = unbiased(static_cast<uint32_t>(k64 >> 32));
        const uint64_t p = 0xFFFFFFFFu - static_cast<uint32_t>(k64 & 0xFFFFFFFFull);
        int t1 = -1, t2 = -1;
        walk_tail<W, T>(s, in, p, ta, g.alpha[r], g.beta[r], [&](int32_t sc, int v1, int v2) {
            if (sc == target) {
                t1 = v1;
                t2 = v2;
                return false;
            }
            return true;
        });
        if (t1 < 0) {
            atomicExch(g.error, kDevResolveMiss);
            continue;
        }
        if (g.best_valid[r] == 0 || (g.best_valid[r] == 1 && target > g.best_s[r])) {
            g.best_s[r] = target;
            g.best_valid[r] = 1;
            const int nw = (ta.ell + 3) >> 2;
            uint32_t words[8];
#pragma unroll
            for (int jw = 0; jw < 8; ++jw) words[jw] = jw < nw ? in.T[jw * in.cap + p] : 0u;
            // insert tail bytes at positions ell (and ell + 1)
#pragma unroll
            for (int jw = 0; jw < 8; ++jw) {
                if (jw == (ta.ell >> 2)) words[jw] |= static_cast<uint32_t>(t1) << ((ta.ell & 3) * 8);
                if (T == 2 && jw == ((ta.ell + 1) >> 2)) words[jw] |= static_cast<uint32_t>(t2) << (((ta.ell + 1) & 3) * 8);
            }
#pragma unroll
            for (int jw = 0; jw < 8; ++jw) g.best_t[static_cast<uint64_t>(r) * 8 + jw] = words[jw];
        }
    }
}

__device__ __forceinline__ int32_t link_weight(const SmemTopo &s, int W, int x, int y) {
    const uint32_t *row = s.cls + static_cast<size_t>(x) * s.C * W;
    for (int c = 0; c < s.C; ++c)
        if ((row[c * W + (y >> 5)] >> (y & 31)) & 1u) return s.wc[c];
    return 0;
}

// Writes the result of every request of the group: the chosen tuple's AggBW
// (Eq. 1) and PreservedBW (Eq. 3) recomputed from their definitions on the
// bitsets, checked against the enumerated score.
template <int W>
__global__ void k_finalize(TopoArgs topo, PatternArgs pat, GroupArgs g) {
    const SmemTopo s = stage_topology<W>(topo, true);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.size; i += gridDim.x * blockDim.x) {
        const int32_t bi = g.req_index[i];
        const mapa_request &q = g.reqs[bi];
        mapa_result res;
        memset(&res, 0, sizeof(res));
        res.k = pat.k;
        res.count = g.count[i];
        const int32_t state = g.best_valid[i];
        if (state == -2) {
            res.status = MAPA_E_RANGE;
            res.count = 0;
        } else if (state == -3) {
            res.status = MAPA_E_INVALID;
            res.count = 0;
        } else if (q.policy.max_embeddings > 0 && res.count > q.policy.max_embeddings) {
            res.status = MAPA_E_BUDGET;
        } else if (state != 1) {
            res.status = MAPA_NO_FIT;
        } else {
            uint8_t t[kMaxK];
            for (int j = 0; j < pat.k; ++j) t[j] = static_cast<uint8_t>((g.best_t[static_cast<uint64_t>(i) * 8 + (j >> 2)] >> ((j & 3) * 8)) & 0xFFu);
            long long agg = 0;
            for (int v = 0; v < pat.k; ++v) {
                uint32_t m = pat.back[v];
                while (m) {
                    const int a = __ffs(m) - 1;
                    m &= m - 1u;
                    agg += link_weight(s, W, t[a], t[v]);
                }
            }
            uint32_t rem[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint32_t busy = q.busy[w];
                if (g.occupancy) busy |= g.occupancy[w];
                rem[w] = ~busy & valid_word(s.n, w);
            }
            for (int j = 0; j < pat.k; ++j) clear_bit<W>(rem, t[j]);
            long long twice = 0;
            for (int v = 0; v < s.n; ++v) {
                if (!((rem[v >> 5] >> (v & 31)) & 1u)) continue;
                const uint32_t *x = s.cls + static_cast<size_t>(v) * s.C * W;
                for (int c = 0; c < s.C; ++c) {
                    int pc = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) pc += __popc(x[c * W + w] & rem[w]);
                    twice += static_cast<long long>(s.wc[c]) * pc;
                }
            }
            const long long pres = twice / 2;
            const long long score = static_cast<long long>(g.alpha[i]) * agg + static_cast<long long>(g.beta[i]) * pres;
            if (score != g.best_s[i]) atomicExch(g.error, kDevScoreMismatch);
            res.status = MAPA_OK;
            res.score = g.best_s[i];
            res.agg = static_cast<int32_t>(agg);
            res.pres = static_cast<int32_t>(pres);
            for (int j = 0; j < pat.k; ++j) res.verts[j] = t[j];
        }
        g.out[bi] = res;
    }
}

// State management (Sec. 3.6): mark the chosen vertices busy under a new job id.
__global__ void k_commit(mapa_result *res, uint32_t *occ, int64_t *owner, unsigned long long *next_job) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (res->status != MAPA_OK) return;
    const long long job = static_cast<long long>(atomicAdd(next_job, 1ull)) + 1;
    for (int i = 0; i < res->k; ++i) {
        const int v = res->verts[i];
        occ[v >> 5] |= 1u << (v & 31);
        owner[v] = job;
    }
    res->job_id = job;
}

// State management (Sec. 3.6): return a job's vertices to the free pool.
__global__ void k_release(int n, long long job, uint32_t *occ, int64_t *owner, int32_t *freed) {
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        if (owner[v] == job) {
            owner[v] = 0;
            atomicAnd(occ + (v >> 5), ~(1u << (v & 31)));
            atomicAdd(freed, 1);
        }
    }
}

// Group requests by pattern: histogram, then scatter into per-pattern runs.
__global__ void k_histogram(const mapa_request *reqs, int32_t nreq, int32_t npat, int32_t *hist, mapa_result *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nreq; i += gridDim.x * blockDim.x) {
        const int32_t pid = reqs[i].pattern_id;
        if (pid < 0 || pid >= npat) {
            mapa_result res;
            memset(&res, 0, sizeof(res));
            res.status = MAPA_E_INVALID;
            out[i] = res;
        } else {
            atomicAdd(hist + pid, 1);
        }
    }
}

__global__ void k_scatter(const mapa_request *reqs, int32_t nreq, int32_t npat, int32_t *cursor, int32_t *order) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nreq; i += gridDim.x * blockDim.x) {
        const int32_t pid = reqs[i].pattern_id;
        if (pid < 0 || pid >= npat) continue;
        order[atomicAdd(cursor + pid, 1)] = i;
    }
}

// Sum of the per-request match counts of a group (telemetry).
__global__ void __launch_bounds__(1024) k_sum_counts(const unsigned long long *count, int32_t n,
                                                     unsigned long long *out) {
    unsigned long long acc = 0ull;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += count[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// ----------------------------------------------------------------------------
// Host side

struct Engine {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t frontier_cap = 0;
    char *arena = nullptr;
    uint64_t arena_bytes = 0;
    char *group_mem = nullptr;
    uint64_t group_bytes = 0;
    mapa_request *stage_reqs = nullptr;
    mapa_result *stage_out = nullptr;
    int32_t stage_cap = 0;
    int32_t *order = nullptr;
    int32_t order_cap = 0;
    int32_t *hist = nullptr;  // [kMaxPatternsPerBatch + 1]
    int32_t hist_cap = 0;
    int32_t *d_error = nullptr;
    unsigned long long *d_stats = nullptr;  // [0] tail nodes of the current group
    unsigned long long *h_pinned = nullptr;  // small pinned scratch
    mapa_stats st{};
    bool timing = false;
    std::vector<cudaEvent_t> events;  // pairs around fused last-level launches
    size_t events_used = 0;

    cudaEvent_t next_event() {
        if (events_used == events.size()) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            events.push_back(ev);
        }
        return events[events_used++];
    }
};

static int ensure_device(char **ptr, uint64_t *have, uint64_t need, std::string *err) {
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
        if (err) *err = std::string("no usable CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "bad index");
        return nullptr;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        if (err) *err = "cudaSetDevice failed";
        return nullptr;
    }
    Engine *en = new Engine();
    en->device = device;
    en->frontier_cap = frontier_cap ? frontier_cap : (4ull << 30);
    if (cudaStreamCreateWithFlags(&en->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&en->d_error, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&en->d_stats, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&en->h_pinned, 64 * sizeof(unsigned long long)) != cudaSuccess) {
        if (err) *err = "context allocation failed";
        engine_destroy(en);
        return nullptr;
    }
    en->stream = en->own_stream;
    cudaMemset(en->d_error, 0, sizeof(int32_t));
    return en;
}

void engine_destroy(Engine *e) {
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    cudaFree(e->arena);
    cudaFree(e->group_mem);
    cudaFree(e->stage_reqs);
    cudaFree(e->stage_out);
    cudaFree(e->order);
    cudaFree(e->hist);
    cudaFree(e->d_error);
    cudaFree(e->d_stats);
    for (cudaEvent_t ev : e->events) cudaEventDestroy(ev);
    if (e->h_pinned) cudaFreeHost(e->h_pinned);
    if (e->own_stream) cudaStreamDestroy(e->own_stream);
    delete e;
}

void engine_set_stream(Engine *e, cudaStream_t s) { e->stream = s ? s : e->own_stream; }

int engine_stats(Engine *e, mapa_stats *out) {
    *out = e->st;
    return MAPA_OK;
}

void engine_stats_reset(Engine *e) { e->st = mapa_stats{}; }

void engine_set_timing(Engine *e, bool on) { e->timing = on; }
cudaStream_t engine_stream(Engine *e) { return e->stream; }

int engine_stage(Engine *e, int32_t nreq, mapa_request **reqs_dev, mapa_result **out_dev, std::string *err) {
    if (nreq > e->stage_cap) {
        cudaFree(e->stage_reqs);
        cudaFree(e->stage_out);
        e->stage_reqs = nullptr;
        e->stage_out = nullptr;
        e->stage_cap = 0;
        int32_t cap = std::max(nreq, 1024);
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

static inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
static inline uint64_t align_up(uint64_t a, uint64_t b) { return (a + b - 1) / b * b; }

// Frontier layout of one group run.
struct RunLayout {
    int L = 0;                 // last stored level (= k - T)
    uint64_t E = 0;            // capacity of levels 1..L
    LevelView level[kMaxK];
    uint32_t *warp_cnt[kMaxK];
    unsigned long long *blk_cnt[kMaxK];
    unsigned long long *blk_off[kMaxK];
};

static uint64_t entry_bytes(int ell, int W) { return 4ull * (2 + W + ((ell + 3) / 4)); }

template <int W, int T>
struct GroupRunner {
    Engine *e;
    const TopoDevice &t;
    const PatternArgs &pat;
    GroupArgs g;
    RunLayout lay;
    size_t smem_adj, smem_all;
    std::string *err;

    GroupRunner(Engine *e_, const TopoDevice &t_, const PatternArgs &p_, std::string *err_)
        : e(e_), t(t_), pat(p_), err(err_) {
        smem_adj = topo_smem_bytes(t.n, W, t.C, false);
        smem_all = topo_smem_bytes(t.n, W, t.C, true);
    }

    int plan(int32_t group_size) {
        lay.L = pat.k - T;
        // Per-level columns carved out of one arena of frontier_cap bytes.
        const uint64_t cap = e->frontier_cap;
        const uint64_t lvl0 = static_cast<uint64_t>(group_size);
        uint64_t per_entry = 0;  // bytes per unit of E over levels 1..L (with scratch)
        for (int ell = 1; ell <= lay.L; ++ell) per_entry += entry_bytes(ell, W);
        const uint64_t fixed = lvl0 * entry_bytes(0, W) + 64 * 1024 + (ceil_div(lvl0, kTile) + 2) * 48 + 4096 * (lay.L + 2);
        uint64_t E = 0;
        if (lay.L >= 1) {
            if (cap <= fixed) {
                if (err) *err = "frontier memory cap too small for this group";
                return MAPA_E_NOMEM;
            }
            const uint64_t scratch_per_entry_x1024 = 48ull * lay.L;  // warp/blk counts per 1024 entries
            E = (cap - fixed) * 1024 / (per_entry * 1024 + scratch_per_entry_x1024 + 1);
            E = std::min<uint64_t>(E, 1ull << 31);
            E = E / kTile * kTile;
            const uint64_t need = static_cast<uint64_t>(kTile) * static_cast<uint64_t>(t.n);
            if (E < need) {
                if (err) *err = "frontier memory cap too small (needs room for one tile of children per level)";
                return MAPA_E_NOMEM;
            }
        }
        lay.E = E;
        // carve
        uint64_t total = 0;
        auto bump = [&](uint64_t bytes) {
            const uint64_t at = total;
            total = align_up(total + bytes, 256);
            return at;
        };
        uint64_t off_level[kMaxK][4];
        uint64_t off_scr[kMaxK][3];
        for (int ell = 0; ell <= lay.L; ++ell) {
            const uint64_t c = ell == 0 ? lvl0 : E;
            const int nwt = (ell + 3) / 4;
            off_level[ell][0] = bump(c * 4);
            off_level[ell][1] = bump(c * 4);
            off_level[ell][2] = bump(c * 4 * W);
            off_level[ell][3] = nwt ? bump(c * 4 * nwt) : 0;
            if (ell < lay.L) {
                const uint64_t nb = ceil_div(c, kTile) + 1;
                off_scr[ell][0] = bump(nb * kWarps * 4);
                off_scr[ell][1] = bump(nb * 8);
                off_scr[ell][2] = bump((nb + 1) * 8);
            }
        }
        uint64_t have = e->arena_bytes;
        int rc = ensure_device(&e->arena, &have, std::max<uint64_t>(total, 1), err);
        if (rc != MAPA_OK) return rc;
        e->arena_bytes = have;
        char *base = e->arena;
        for (int ell = 0; ell <= lay.L; ++ell) {
            LevelView &lv = lay.level[ell];
            lv.cap = ell == 0 ? lvl0 : E;
            lv.S = reinterpret_cast<int32_t *>(base + off_level[ell][0]);
            lv.r = reinterpret_cast<uint32_t *>(base + off_level[ell][1]);
            lv.R = reinterpret_cast<uint32_t *>(base + off_level[ell][2]);
            lv.T = reinterpret_cast<uint32_t *>(base + off_level[ell][3]);
            if (ell < lay.L) {
                lay.warp_cnt[ell] = reinterpret_cast<uint32_t *>(base + off_scr[ell][0]);
                lay.blk_cnt[ell] = reinterpret_cast<unsigned long long *>(base + off_scr[ell][1]);
                lay.blk_off[ell] = reinterpret_cast<unsigned long long *>(base + off_scr[ell][2]);
            }
        }
        return MAPA_OK;
    }

    TailArgs tail() const {
        TailArgs ta;
        ta.ell = lay.L;
        ta.back0 = pat.back[lay.L];
        ta.lo0 = pat.lo[lay.L];
        ta.back1 = T == 2 ? pat.back[lay.L + 1] : 0u;
        ta.lo1 = T == 2 ? pat.lo[lay.L + 1] : 0u;
        return ta;
    }

    int last_level(uint64_t P) {
        const TailArgs ta = tail();
        const LevelView &in = lay.level[lay.L];
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (e->timing) {
            ev0 = e->next_event();
            ev1 = e->next_event();
            MAPA_CUDA_TRY(cudaEventRecord(ev0, e->stream));
        }
        k_last<W, T><<<static_cast<unsigned>(ceil_div(P, kTile)), kTpb, smem_all, e->stream>>>(
            t.args(), in, P, ta, g.alpha, g.beta, g.key, g.count, e->d_stats);
        if (e->timing) MAPA_CUDA_TRY(cudaEventRecord(ev1, e->stream));
        const unsigned rgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, 256), 1024));
        k_resolve<W, T><<<rgrid, 256, smem_all, e->stream>>>(t.args(), in, P, ta, g);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 2;
        e->st.tail_launches += 1;
        e->st.tail_parents += P;
        return MAPA_OK;
    }

    // Algorithmic integer operations per unit of the fused tail (see DESIGN).
    void tail_op_costs(uint64_t *per_parent, uint64_t *per_node, uint64_t *per_leaf) const {
        const TailArgs ta = tail();
        const uint64_t C = static_cast<uint64_t>(t.C);
        const uint32_t nb = 1u << ta.ell;
        const uint64_t backs = __builtin_popcount(ta.back0) + (T == 2 ? __builtin_popcount(ta.back1 & ~nb) : 0);
        const uint64_t los = __builtin_popcount(ta.lo0) + (T == 2 ? __builtin_popcount(ta.lo1 & ~nb) : 0);
        *per_parent = backs * (2 + 2 * W) + 3 * los + 3 * W + 1;
        *per_node = 4 * C * W + 3 * C + 5 * W + 1;
        *per_leaf = 4 * C * W + 3 * C + 3;
    }

    void note_spill(int ell, uint64_t children) {
        e->st.kernel_launches += 1;
        e->st.spill_entries += children;
        e->st.spill_bytes += 2 * children * entry_bytes(ell + 1, W);
    }

    int process(int ell, uint64_t P) {
        if (P == 0) return MAPA_OK;
        if (ell == lay.L) return last_level(P);
        const LevelView &in = lay.level[ell];
        const LevelView &out = lay.level[ell + 1];
        const uint64_t nb = ceil_div(P, kTile);
        k_count<W><<<static_cast<unsigned>(nb), kTpb, smem_adj, e->stream>>>(t.args(), in, P, pat.back[ell],
                                                                             pat.lo[ell], lay.warp_cnt[ell],
                                                                             lay.blk_cnt[ell]);
        k_scan<<<1, 1024, 0, e->stream>>>(lay.blk_cnt[ell], lay.blk_off[ell], nb);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 2;
        MAPA_CUDA_TRY(cudaMemcpyAsync(e->h_pinned, lay.blk_off[ell] + nb, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, e->stream));
        MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
        const unsigned long long total = e->h_pinned[0];
        if (total == 0) return MAPA_OK;
        if (total <= lay.E) {
            k_write<W><<<static_cast<unsigned>(nb), kTpb, smem_all, e->stream>>>(
                t.args(), in, P, ell, pat.back[ell], pat.lo[ell], out, lay.warp_cnt[ell], lay.blk_off[ell], 0,
                g.alpha, g.beta);
            MAPA_CUDA_TRY(cudaGetLastError());
            note_spill(ell, total);
            return process(ell + 1, total);
        }
        // Depth-first over chunks of whole blocks whose children fit.
        std::vector<unsigned long long> off(nb + 1);
        MAPA_CUDA_TRY(cudaMemcpyAsync(off.data(), lay.blk_off[ell], sizeof(unsigned long long) * (nb + 1),
                                      cudaMemcpyDeviceToHost, e->stream));
        MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
        uint64_t b0 = 0;
        while (b0 < nb) {
            uint64_t b1 = std::upper_bound(off.begin() + b0 + 1, off.end(), off[b0] + lay.E) - off.begin() - 1;
            if (b1 <= b0) {
                if (err) *err = "internal: one block's children exceed the level capacity";
                return MAPA_E_NOMEM;
            }
            k_write<W><<<static_cast<unsigned>(b1 - b0), kTpb, smem_all, e->stream>>>(
                t.args(), in, P, ell, pat.back[ell], pat.lo[ell], out, lay.warp_cnt[ell], lay.blk_off[ell], b0,
                g.alpha, g.beta);
            MAPA_CUDA_TRY(cudaGetLastError());
            note_spill(ell, off[b1] - off[b0]);
            const int rc = process(ell + 1, off[b1] - off[b0]);
            if (rc != MAPA_OK) return rc;
            b0 = b1;
        }
        return MAPA_OK;
    }

    // Kernels staging more than 48 KB of topology need the opt-in limit.
    int allow_smem() {
        if (smem_all <= 48 * 1024) return MAPA_OK;
        const int b = static_cast<int>(smem_all);
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_setup<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_write<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_last<W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_resolve<W, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        MAPA_CUDA_TRY(cudaFuncSetAttribute(k_finalize<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        return MAPA_OK;
    }

    int run(const GroupArgs &ga) {
        g = ga;
        int rc = allow_smem();
        if (rc != MAPA_OK) return rc;
        rc = plan(g.size);
        if (rc != MAPA_OK) return rc;
        const unsigned sgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, kWarps), 4096));
        MAPA_CUDA_TRY(cudaMemsetAsync(e->d_stats, 0, 8 * sizeof(unsigned long long), e->stream));
        k_setup<W><<<sgrid, kTpb, smem_all, e->stream>>>(t.args(), g, lay.level[0]);
        MAPA_CUDA_TRY(cudaGetLastError());
        const uint64_t parents0 = e->st.tail_parents;
        e->events_used = 0;
        rc = process(0, static_cast<uint64_t>(g.size));
        if (rc != MAPA_OK) return rc;
        const unsigned fgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(g.size, 128), 4096));
        k_finalize<W><<<fgrid, 128, smem_all, e->stream>>>(t.args(), pat, g);
        MAPA_CUDA_TRY(cudaGetLastError());
        e->st.kernel_launches += 2;
        e->st.requests += static_cast<uint64_t>(g.size);
        // group totals: leaves = matches scored, nodes from the device counter
        MAPA_CUDA_TRY(cudaMemcpyAsync(e->h_pinned, e->d_stats, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                      e->stream));
        unsigned long long *leaves_h = e->h_pinned + 8;
        MAPA_CUDA_TRY(cudaMemsetAsync(e->d_stats + 1, 0, sizeof(unsigned long long), e->stream));
        k_sum_counts<<<1, 1024, 0, e->stream>>>(g.count, g.size, e->d_stats + 1);
        MAPA_CUDA_TRY(cudaMemcpyAsync(leaves_h, e->d_stats + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                      e->stream));
        MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
        e->st.kernel_launches += 1;
        const uint64_t nodes = e->h_pinned[0], leaves = leaves_h[0];
        uint64_t cp, cn, cl;
        tail_op_costs(&cp, &cn, &cl);
        e->st.tail_nodes += nodes;
        e->st.tail_leaves += leaves;
        e->st.embeddings += leaves;
        e->st.tail_int_ops += (e->st.tail_parents - parents0) * cp + nodes * cn + leaves * cl;
        if (e->timing) {
            for (size_t i = 0; i + 1 < e->events_used; i += 2) {
                float ms = 0.f;
                MAPA_CUDA_TRY(cudaEventElapsedTime(&ms, e->events[i], e->events[i + 1]));
                e->st.tail_ms += ms;
            }
        }
        e->events_used = 0;
        return MAPA_OK;
    }
};

static int tail_depth(const PatternArgs &p) { return p.k >= 2 ? 2 : 1; }

template <int W>
static int run_group_w(Engine *e, const TopoDevice &t, const PatternArgs &p, const GroupArgs &g, std::string *err) {
    if (tail_depth(p) == 2) {
        GroupRunner<W, 2> runner(e, t, p, err);
        return runner.run(g);
    }
    GroupRunner<W, 1> runner(e, t, p, err);
    return runner.run(g);
}

static int run_group(Engine *e, const TopoDevice &t, const PatternArgs &p, const GroupArgs &g, std::string *err) {
    switch (t.W) {
        case 1: return run_group_w<1>(e, t, p, g, err);
        case 2: return run_group_w<2>(e, t, p, g, err);
        case 4: return run_group_w<4>(e, t, p, g, err);
        case 8: return run_group_w<8>(e, t, p, g, err);
        default:
            if (err) *err = "internal: bad word count";
            return MAPA_E_INVALID;
    }
}

// Per-request group arrays (alpha, beta, key, count, best) for up to `size` requests.
static int group_arrays(Engine *e, int32_t size, GroupArgs *g, std::string *err) {
    const uint64_t n = static_cast<uint64_t>(std::max(size, 1));
    const uint64_t bytes = align_up(n * 4, 256) * 4 + align_up(n * 8, 256) * 2 + align_up(n * 32, 256);
    uint64_t have = e->group_bytes;
    const int rc = ensure_device(&e->group_mem, &have, bytes, err);
    if (rc != MAPA_OK) return rc;
    e->group_bytes = have;
    char *p = e->group_mem;
    auto take = [&](uint64_t b) {
        char *q = p;
        p += align_up(b, 256);
        return q;
    };
    g->alpha = reinterpret_cast<int32_t *>(take(n * 4));
    g->beta = reinterpret_cast<int32_t *>(take(n * 4));
    g->best_s = reinterpret_cast<int32_t *>(take(n * 4));
    g->best_valid = reinterpret_cast<int32_t *>(take(n * 4));
    g->key = reinterpret_cast<uint64_t *>(take(n * 8));
    g->count = reinterpret_cast<unsigned long long *>(take(n * 8));
    g->best_t = reinterpret_cast<uint32_t *>(take(n * 32));
    return MAPA_OK;
}

static int check_device_error(Engine *e, std::string *err) {
    int32_t h = 0;
    MAPA_CUDA_TRY(cudaMemcpyAsync(&h, e->d_error, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (h != kDevOk) {
        cudaMemsetAsync(e->d_error, 0, sizeof(int32_t), e->stream);
        if (err) *err = h == kDevScoreMismatch ? "internal check failed: score disagrees with its tuple"
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
    if (sequential) {
        // One request at a time against the device occupancy, committing each.
        int rc = group_arrays(e, 1, &g, err);
        if (rc != MAPA_OK) return rc;
        uint64_t have = static_cast<uint64_t>(e->order_cap) * 4;
        char *ord = reinterpret_cast<char *>(e->order);
        rc = ensure_device(&ord, &have, static_cast<uint64_t>(std::max(nreq, 1)) * 4, err);
        if (rc != MAPA_OK) return rc;
        e->order = reinterpret_cast<int32_t *>(ord);
        e->order_cap = static_cast<int32_t>(have / 4);
        std::vector<int32_t> idx(nreq), pids(nreq);
        for (int32_t i = 0; i < nreq; ++i) idx[i] = i;
        MAPA_CUDA_TRY(cudaMemcpyAsync(e->order, idx.data(), sizeof(int32_t) * nreq, cudaMemcpyHostToDevice, e->stream));
        // pattern ids are needed on the host to pick the kernel shape
        std::vector<mapa_request> hreq(nreq);
        MAPA_CUDA_TRY(cudaMemcpyAsync(hreq.data(), reqs_dev, sizeof(mapa_request) * nreq, cudaMemcpyDeviceToHost, e->stream));
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
            rc = run_group(e, t, patterns[pid], g, err);
            if (rc != MAPA_OK) return rc;
            k_commit<<<1, 32, 0, e->stream>>>(out_dev + i, t.occupancy, t.owner, t.next_job);
            MAPA_CUDA_TRY(cudaGetLastError());
        }
        return check_device_error(e, err);
    }

    // Independent requests: group by pattern on the device.
    uint64_t have = static_cast<uint64_t>(e->hist_cap) * 4;
    char *hp = reinterpret_cast<char *>(e->hist);
    int rc = ensure_device(&hp, &have, static_cast<uint64_t>(npat + 1) * 4, err);
    if (rc != MAPA_OK) return rc;
    e->hist = reinterpret_cast<int32_t *>(hp);
    e->hist_cap = static_cast<int32_t>(have / 4);
    have = static_cast<uint64_t>(e->order_cap) * 4;
    char *ord = reinterpret_cast<char *>(e->order);
    rc = ensure_device(&ord, &have, static_cast<uint64_t>(nreq) * 4, err);
    if (rc != MAPA_OK) return rc;
    e->order = reinterpret_cast<int32_t *>(ord);
    e->order_cap = static_cast<int32_t>(have / 4);

    MAPA_CUDA_TRY(cudaMemsetAsync(e->hist, 0, sizeof(int32_t) * (npat + 1), e->stream));
    const unsigned hgrid = static_cast<unsigned>(std::min<uint64_t>(ceil_div(nreq, 256), 1024));
    k_histogram<<<hgrid, 256, 0, e->stream>>>(reqs_dev, nreq, npat, e->hist, out_dev);
    std::vector<int32_t> hist(npat + 1);
    MAPA_CUDA_TRY(cudaMemcpyAsync(hist.data(), e->hist, sizeof(int32_t) * npat, cudaMemcpyDeviceToHost, e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    std::vector<int32_t> start(npat + 1, 0);
    for (int32_t p = 0; p < npat; ++p) start[p + 1] = start[p] + hist[p];
    MAPA_CUDA_TRY(cudaMemcpyAsync(e->hist, start.data(), sizeof(int32_t) * npat, cudaMemcpyHostToDevice, e->stream));
    k_scatter<<<hgrid, 256, 0, e->stream>>>(reqs_dev, nreq, npat, e->hist, e->order);
    MAPA_CUDA_TRY(cudaGetLastError());
    int32_t largest = 0;
    for (int32_t p = 0; p < npat; ++p) largest = std::max(largest, hist[p]);
    rc = group_arrays(e, std::min(largest, kMaxGroup), &g, err);
    if (rc != MAPA_OK) return rc;
    g.occupancy = nullptr;
    for (int32_t p = 0; p < npat; ++p) {
        for (int32_t s0 = 0; s0 < hist[p]; s0 += kMaxGroup) {
            g.size = std::min(kMaxGroup, hist[p] - s0);
            g.req_index = e->order + start[p] + s0;
            rc = run_group(e, t, patterns[p], g, err);
            if (rc != MAPA_OK) return rc;
        }
    }
    return check_device_error(e, err);
}

int engine_release(Engine *e, const TopoDevice &t, int64_t job_id, int32_t *freed, std::string *err) {
    MAPA_CUDA_TRY(cudaSetDevice(e->device));
    MAPA_CUDA_TRY(cudaMemsetAsync(t.scratch, 0, sizeof(int32_t), e->stream));
    k_release<<<1, 256, 0, e->stream>>>(t.n, static_cast<long long>(job_id), t.occupancy, t.owner, t.scratch);
    MAPA_CUDA_TRY(cudaGetLastError());
    MAPA_CUDA_TRY(cudaMemcpyAsync(freed, t.scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    MAPA_CUDA_TRY(cudaStreamSynchronize(e->stream));
    return MAPA_OK;
}

}  // namespace mapa
