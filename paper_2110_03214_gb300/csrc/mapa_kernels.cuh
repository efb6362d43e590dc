// Device kernels of the MAPA allocation hot path (sm_103a), templated on the
// mask width W (32-bit words per vertex set), the number of weight classes CT
// (1..3 specialised, 0 = any) and the fused tail depth T.
//
// What is computed (MAPA, arXiv 2110.03214, Sec. 3.3-3.6): for each request,
// every match phi of the pattern P in the free part F of the hardware graph
// (injective, adjacency-preserving, Sec. 3.3), its int32 score
//     S = alpha * AggBW(phi) + beta * PreservedBW(phi)          (Eq. 1, Eq. 3)
// and the argmax with the lexicographically smallest tuple among equal scores
// (Algorithm 1's strict ">" scan over a lexicographic enumeration).
//
// How (our design; the paper has no GPU kernel):
//   * Matches grow one pattern vertex per level in pattern-id order.  A
//     partial match at level l stores, in structure-of-arrays columns, its
//     running score S, its request r, R = F minus the vertices used so far,
//     and its tuple bytes.  Order constraints phi(j) < phi(i) for j in lo[i]
//     keep one map per automorphism class; chosen in increasing id order they
//     keep the lexicographically smallest map of each class, so the argmax
//     tuple is the one a plain lexicographic scan over all maps would choose.
//   * Candidates: R & (AND over earlier neighbours b of adj[phi b]) & (vertices
//     above max over lo of phi), on bitsets staged in shared memory.
//   * Score increment of adding v (B = images of v's earlier neighbours,
//     R = still-free vertices), summed over weight classes c:
//         dS = sum_c w_c * (alpha * popc(B & cls_c[v]) - beta * popc(R & cls_c[v]))
//     The first term is v's share of Eq. 1, the second the links from v to
//     free vertices that Eq. 3 loses; a request's root starts at beta * W(F).
//   * Non-final levels are written to HBM by k_expand, a single-pass kernel:
//     each 256-parent tile counts its children, learns its output offset by
//     a decoupled look-back over earlier tiles (tiles are handed out in
//     increasing order, so a tile only waits on tiles already running), and
//     writes its children warp-cooperatively (lane c emits child c of the
//     warp, so consecutive lanes store consecutive entries of every column).
//     Levels therefore stay in lexicographic order.
//   * The last T levels are fused in k_last: no frontier write; each thread
//     walks its parent's subtree in registers, keeps the best score, and a
//     warp-then-block reduction feeds one 64-bit atomicMax per request of
//     key = (biased S << 32) | ~parent.  Lexicographic order of parents makes
//     the smallest parent index the lexicographic tie-break; k_resolve re-walks
//     the winning parent's subtree to recover the tail.
//   * Every wait (the look-back) is bounded: after kSpinLimit polls the kernel
//     records an error word and stops writing, so a fault can never hang.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "mapa_internal.h"

namespace mapa {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kNoReq = 0xFFFFFFFFu;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
constexpr unsigned kSpinLimit = 1u << 24;
// dive_s of an anytime request whose fallback dive proved it has no match
constexpr int32_t kDiveNoMatch = INT_MIN + 1;

// Device stats slots (summed over a batch, read once at its end).
enum StatSlot {
    kStatNodes = 0, kStatLeaves, kStatParents, kStatOps, kStatSpill, kStatSpillBytes,
    kStatExpandBytes,  // algorithmic bytes of the level expansions: parents read + children written
    kStatSlots
};

// ----------------------------------------------------------------------------
// Mask helpers

__device__ __forceinline__ uint32_t biased(int32_t s) { return static_cast<uint32_t>(s) ^ 0x80000000u; }
__device__ __forceinline__ int32_t unbiased(uint32_t b) { return static_cast<int32_t>(b ^ 0x80000000u); }

__host__ __device__ __forceinline__ uint32_t valid_word(int n, int w) {
    const int lo = 32 * w;
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

// Keeps only vertices < hb (hb <= 0 keeps none).
template <int W>
__device__ __forceinline__ void and_below(uint32_t (&c)[W], int hb) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int base = 32 * w;
        uint32_t m;
        if (hb <= base)
            m = 0u;
        else if (hb >= base + 32)
            m = ~0u;
        else
            m = (1u << (hb - base)) - 1u;
        c[w] &= m;
    }
}

// Highest set vertex of a W-word mask (-1 if empty).
template <int W>
__device__ __forceinline__ int highest_bit(const uint32_t (&m)[W]) {
    int v = -1;
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (m[w] != 0u) v = 32 * w + 31 - __clz(m[w]);
    return v;
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

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
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

// ----------------------------------------------------------------------------
// Topology in shared memory

// The topology in shared memory: vertex v's adjacency row at adj + v *
// adj_stride(W), its C class rows at cls + v * cs (class c at c * W).  Both
// strides are odd, so lanes reading rows of different vertices spread over
// the 32 banks (a stride of W words would put word w of every vertex in one
// of 32 / W banks).
struct SmemTopo {
    const uint32_t *adj;
    const uint32_t *cls;
    const int32_t *wc;
    int n, C;
    int32_t wmin, wmax, dmax;
    int cs;  // words per vertex of cls: (C W) | 1
};

__host__ __device__ constexpr int adj_stride(int W) { return W | 1; }
__host__ __device__ constexpr int cls_stride(int C, int W) { return (C * W) | 1; }

__host__ __device__ inline size_t topo_smem_bytes(int n, int W, int C, bool with_cls) {
    size_t words = static_cast<size_t>(n) * adj_stride(W);
    if (with_cls) words += static_cast<size_t>(n) * cls_stride(C, W) + C;
    return words * 4;
}

template <int W>
__device__ __forceinline__ SmemTopo stage_topology(const TopoArgs &t, bool with_cls) {
    extern __shared__ uint32_t smem_words[];
    constexpr int as = adj_stride(W);
    const int cs = cls_stride(t.C, W);
    uint32_t *adj = smem_words;
    uint32_t *cls = adj + t.n * as;
    int32_t *wc = reinterpret_cast<int32_t *>(cls + (with_cls ? t.n * cs : 0));
    for (int i = threadIdx.x; i < t.n * W; i += blockDim.x) adj[(i / W) * as + i % W] = t.adj[i];
    if (with_cls) {
        const int row = t.C * W;
        for (int i = threadIdx.x; i < t.n * row; i += blockDim.x) cls[(i / row) * cs + i % row] = t.clsv[i];
        for (int i = threadIdx.x; i < t.C; i += blockDim.x) wc[i] = t.wc[i];
    }
    __syncthreads();
    return SmemTopo{adj, cls, wc, t.n, t.C, t.wmin, t.wmax, t.dmax, cs};
}

// Offset of entry p in column j of a level: capacities are at most
// kMaxLevelEntries and fields at most 8 columns wide, so it fits 32 bits.
__device__ __forceinline__ uint32_t col_at(const LevelView &L, uint32_t j, uint32_t p) {
    return j * static_cast<uint32_t>(L.cap) + p;
}

// The free set R of entry p: its W words are stored together at R + p W
// (entry-major), so a thread moves them with W / 4 16-byte accesses (8 or
// 4 bytes for W = 2, 1) and a warp's accesses to 32 consecutive entries
// cover 128 W contiguous bytes.  Arena columns start 256-byte aligned.
template <int W>
__device__ __forceinline__ void load_R(const LevelView &L, uint64_t p, uint32_t (&R)[W]) {
    if constexpr (W % 4 == 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(L.R + p * W);
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            const uint4 x = src[q];
            R[4 * q] = x.x;
            R[4 * q + 1] = x.y;
            R[4 * q + 2] = x.z;
            R[4 * q + 3] = x.w;
        }
    } else if constexpr (W == 2) {
        const uint2 x = reinterpret_cast<const uint2 *>(L.R)[p];
        R[0] = x.x;
        R[1] = x.y;
    } else {
        R[0] = L.R[p];
    }
}

template <int W>
__device__ __forceinline__ void store_R(const LevelView &L, uint64_t p, const uint32_t (&R)[W]) {
    if constexpr (W % 4 == 0) {
        uint4 *dst = reinterpret_cast<uint4 *>(L.R + p * W);
#pragma unroll
        for (int q = 0; q < W / 4; ++q) dst[q] = make_uint4(R[4 * q], R[4 * q + 1], R[4 * q + 2], R[4 * q + 3]);
    } else if constexpr (W == 2) {
        reinterpret_cast<uint2 *>(L.R)[p] = make_uint2(R[0], R[1]);
    } else {
        L.R[p] = R[0];
    }
}

__device__ __forceinline__ int tuple_byte(const LevelView &L, uint32_t p, int j) {
    return static_cast<int>((L.T[col_at(L, static_cast<uint32_t>(j >> 2), p)] >> ((j & 3) * 8)) & 0xFFu);
}

// Intersection of the adjacency rows of placed back-neighbours (A), the set of
// their images (B) and the lower bound from the order constraints (lb).
template <int W>
__device__ __forceinline__ void level_masks(const LevelView &L, uint32_t p, uint32_t back, uint32_t lo,
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
        for (int w = 0; w < W; ++w) A[w] &= s_adj[x * adj_stride(W) + w];
        set_bit<W>(B, x);
    }
    while (lo) {
        const int a = __ffs(lo) - 1;
        lo &= lo - 1u;
        lb = max(lb, tuple_byte(L, p, a));
    }
}

// Range of phi(0) of a split request (level 0 only; see LevelView): narrows
// the candidates of pattern vertex 0 to [root_lo, root_hi).  Call only where
// pattern vertex 0 is being placed.
template <int W>
__device__ __forceinline__ void root_range(const LevelView &L, uint32_t p, uint32_t (&A)[W], int &lb) {
    if (!L.root) return;
    const uint32_t t = L.T[p];
    const int hi = static_cast<int>(t >> 16);
    if (hi == 0) return;
    lb = max(lb, static_cast<int>(t & 0xFFFFu) - 1);
    and_below<W>(A, hi);
}

// Score increments (see the file header).  CT > 0: the class count is known at
// compile time and alpha*w_c, beta*w_c live in registers.
template <int W, int CT>
struct Scorer {
    const uint32_t *cls;
    const int32_t *wc;
    int C, cs;
    int32_t al, be;
    int32_t aw[CT > 0 ? CT : 1];
    int32_t bw[CT > 0 ? CT : 1];

    __device__ __forceinline__ Scorer(const SmemTopo &s, int32_t al_, int32_t be_)
        : cls(s.cls), wc(s.wc), C(CT > 0 ? CT : s.C), cs(s.cs), al(al_), be(be_) {
        if constexpr (CT > 0) {
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                aw[c] = al_ * s.wc[c];
                bw[c] = be_ * s.wc[c];
            }
        }
    }

    __device__ __forceinline__ int32_t delta(int v, const uint32_t (&B)[W], const uint32_t (&R)[W]) const {
        int32_t acc = 0;
        if constexpr (CT > 0) {
            const uint32_t *x = cls + v * cls_stride(CT, W);
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                int pb = 0, pr = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const uint32_t xw = x[c * W + w];
                    pb += __popc(B[w] & xw);
                    pr += __popc(R[w] & xw);
                }
                acc += aw[c] * pb - bw[c] * pr;
            }
        } else {
            const uint32_t *x = cls + static_cast<size_t>(v) * cs;
            for (int c = 0; c < C; ++c) {
                int pb = 0, pr = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const uint32_t xw = x[c * W + w];
                    pb += __popc(B[w] & xw);
                    pr += __popc(R[w] & xw);
                }
                acc += wc[c] * (al * pb - be * pr);
            }
        }
        return acc;
    }
};

// ----------------------------------------------------------------------------
// Bounded mode: an upper bound on the final score of every completion of a
// partial match with score S, R = free vertices not yet used and m = k - l
// unplaced pattern vertices (l placed).  Counting each link once, completing
// the match adds
//   +alpha * w          for a pattern edge from a placed to an unplaced vertex,
//   (alpha - beta) * w  for a pattern edge between two unplaced vertices,
//   -beta * w           for every other link between the unplaced images U and R.
// The links between U and R weigh at least the sum over u in U of
//   g(d_u) = max(d_u / 2, d_u - (m - 1) * wmax / 2),
// d_u the weight of u's links into R (a link inside U is met from both ends,
// and at most m - 1 of u's links stay inside U).  With D the sum of the m
// smallest 2 g(d_u) over u in R -- bounded below by the four smallest and
// m - 4 more copies of the fourth -- and alpha, beta >= 0, every completion
// scores at most S + min(B1, B2):
//   B1 = alpha * wmax * e_cross + e_in * max((alpha - beta) * wmax, (alpha - beta) * wmin)
//   B2 = alpha * wmax * (e_cross + e_in) - ceil(beta * D / 2).
// Fewer than m vertices left in R: no completion at all.  The degree term
// needs a scan of R; it is skipped when even its largest value (D <= 2 m
// dmax, dmax the largest weighted degree of G) cannot reach thr.

struct LevelBound {
    int32_t e_cross, e_in, m;
    int32_t degrees;  // 0: skip the degree term (B1 only)
};

__host__ __device__ inline LevelBound level_bound(const PatternArgs &p, int l) {
    return LevelBound{p.e_cross[l], p.e_in[l], p.k - l, 1};
}

// Keeps the four smallest values seen in t[0] <= t[1] <= t[2] <= t[3].
__device__ __forceinline__ void keep4(int32_t (&t)[4], int32_t x) {
    if (x >= t[3]) return;
    t[3] = x;
#pragma unroll
    for (int j = 3; j > 0; --j)
        if (t[j] < t[j - 1]) {
            const int32_t y = t[j];
            t[j] = t[j - 1];
            t[j - 1] = y;
        }
}

// 2 g(d_u) for vertex u of R.
template <int W>
__device__ __forceinline__ int32_t twice_floor_loss(const SmemTopo &s, const uint32_t (&R)[W], int u, int32_t cap) {
    const uint32_t *x = s.cls + static_cast<size_t>(u) * s.cs;
    int32_t d = 0;
    for (int c = 0; c < s.C; ++c) {
        int pc = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) pc += __popc(x[c * W + w] & R[w]);
        d += s.wc[c] * pc;
    }
    return max(d, 2 * d - cap);
}

// First stage of the bound (no per-vertex work): returns 1 = cut, 0 = keep,
// -1 = decide with the degree term.
__device__ __forceinline__ int cut_first(const SmemTopo &s, int nR, int32_t S, int32_t al, int32_t be, int32_t thr,
                                         const LevelBound &lb, long long &base2) {
    // INT_MAX: nothing is left to find (no match exists, or the request is
    // past its work budget), whatever the signs of alpha and beta
    if (thr == INT_MAX) return 1;
    if (thr == INT_MIN || al < 0 || be < 0) return 0;
    if (nR < lb.m) return 1;
    const long long wmax = s.wmax, wmin = s.wmin, ab = static_cast<long long>(al) - be;
    const long long b1 = al * wmax * lb.e_cross + lb.e_in * max(ab * wmax, ab * wmin);
    if (S + b1 < thr) return 1;
    if (be == 0 || lb.m == 0 || !lb.degrees) return 0;
    base2 = S + al * wmax * (lb.e_cross + lb.e_in);
    // D <= 2 m dmax: when even that cannot cut, skip the per-vertex scan
    if (base2 - static_cast<long long>(be) * lb.m * s.dmax >= thr) return 0;
    return -1;
}

__device__ __forceinline__ bool cut_second(long long base2, int32_t be, const int32_t (&t)[4], int m, int32_t thr) {
    long long D = t[0];
    if (m >= 2) D += t[1];
    if (m >= 3) D += t[2];
    if (m >= 4) D += static_cast<long long>(t[3]) * (m - 3);
    return base2 - (static_cast<long long>(be) * D + 1) / 2 < thr;
}

// True when no completion of the partial can reach thr (one thread).
template <int W>
__device__ __forceinline__ bool cut_off(const SmemTopo &s, const uint32_t (&R)[W], int32_t S, int32_t al, int32_t be,
                                        int32_t thr, const LevelBound &lb) {
    long long base2 = 0;
    const int first = cut_first(s, popc_mask<W>(R), S, al, be, thr, lb, base2);
    if (first >= 0) return first == 1;
    const int32_t cap = (lb.m - 1) * s.wmax;
    int32_t t[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    uint32_t rem[W];
#pragma unroll
    for (int w = 0; w < W; ++w) rem[w] = R[w];
    int u;
    while ((u = pop_lowest<W>(rem)) >= 0) keep4(t, twice_floor_loss<W>(s, R, u, cap));
    return cut_second(base2, be, t, lb.m, thr);
}

// The same test evaluated by a whole warp on one partial (warp-uniform
// arguments and result).
template <int W>
__device__ __forceinline__ bool cut_off_warp(const SmemTopo &s, const uint32_t (&R)[W], int32_t S, int32_t al,
                                             int32_t be, int32_t thr, const LevelBound &lb, int lane) {
    long long base2 = 0;
    const int first = cut_first(s, popc_mask<W>(R), S, al, be, thr, lb, base2);
    if (first >= 0) return first == 1;
    const int32_t cap = (lb.m - 1) * s.wmax;
    int32_t t[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
#pragma unroll
    for (int w = 0; w < W; ++w)
        if ((R[w] >> lane) & 1u) keep4(t, twice_floor_loss<W>(s, R, 32 * w + lane, cap));
    // the four smallest of the warp: each round takes the least head of the
    // lanes' sorted lists and pops it from the lowest lane holding it (the
    // same multiset as merging the lists pairwise)
    int32_t low[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    const int rounds = min(lb.m, 4);
    for (int j = 0; j < rounds; ++j) {
        const int32_t m = __reduce_min_sync(kFull, t[0]);
        low[j] = m;
        const uint32_t holders = __ballot_sync(kFull, t[0] == m);
        if (lane == __ffs(holders) - 1) {
            t[0] = t[1];
            t[1] = t[2];
            t[2] = t[3];
            t[3] = INT_MAX;
        }
    }
    return cut_second(base2, be, low, lb.m, thr);
}

// ----------------------------------------------------------------------------
// Fused tail: the last T pattern vertices ell .. ell+T-1 of a stored parent.

struct TailArgs {
    int32_t ell;              // level of the stored parents (= k - T)
    uint32_t back_old[3];     // earlier neighbours among stored vertices (< ell), per tail level
    uint32_t lo_old[3];       // order constraints from stored vertices, per tail level
    uint32_t back_tail[3];    // bit j: tail vertex ell+j is an earlier neighbour
    uint32_t lo_tail[3];      // bit j: constraint phi(ell+j) < phi(this)
    uint64_t cost_parent;     // algorithmic integer ops per parent, tail node, leaf (telemetry)
    uint64_t cost_node;
    uint64_t cost_leaf;
    LevelBound bound;         // bounded mode: edge counts of the stored level ell
};

template <int W, int T>
struct TailPre {
    uint32_t A[T][W];
    uint32_t B[T][W];
    int lb[T];
};

template <int W, int T>
__device__ __forceinline__ void tail_precompute(const LevelView &in, uint64_t p, const TailArgs &ta,
                                                const uint32_t *s_adj, TailPre<W, T> &pre) {
#pragma unroll
    for (int t = 0; t < T; ++t) level_masks<W>(in, p, ta.back_old[t], ta.lo_old[t], s_adj, pre.A[t], pre.B[t], pre.lb[t]);
    root_range<W>(in, static_cast<uint32_t>(p), pre.A[0], pre.lb[0]);
}

// Walks tail level t (pattern vertex ell + t) below the tail prefix tv[0..t-1].
// Leaf provides add(count) for every level-(T-1) candidate set and
// visit(score, tv, v) for every complete match (return false to stop).
template <int W, int CT, int T, int t, typename Leaf>
__device__ __forceinline__ bool tail_walk(const SmemTopo &s, const Scorer<W, CT> &sc, const TailArgs &ta,
                                          const TailPre<W, T> &pre, const uint32_t (&R)[W], int32_t S, int (&tv)[T],
                                          Leaf &leaf, uint32_t &nodes) {
    uint32_t c[W], B[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        c[w] = R[w] & pre.A[t][w];
        B[w] = pre.B[t][w];
    }
    int lb = pre.lb[t];
#pragma unroll
    for (int j = 0; j < t; ++j) {
        if ((ta.back_tail[t] >> j) & 1u) {
#pragma unroll
            for (int w = 0; w < W; ++w) c[w] &= s.adj[tv[j] * adj_stride(W) + w];
            set_bit<W>(B, tv[j]);
        }
        if ((ta.lo_tail[t] >> j) & 1u) lb = max(lb, tv[j]);
    }
    and_above<W>(c, lb);
    if constexpr (t == T - 1) {
        leaf.add(popc_mask<W>(c));
        int v;
        while ((v = pop_lowest<W>(c)) >= 0) {
            if (!leaf.visit(S + sc.delta(v, B, R), tv, v)) return false;
        }
    } else {
        int v;
        while ((v = pop_lowest<W>(c)) >= 0) {
            ++nodes;
            const int32_t s1 = S + sc.delta(v, B, R);
            uint32_t R1[W];
#pragma unroll
            for (int w = 0; w < W; ++w) R1[w] = R[w];
            clear_bit<W>(R1, v);
            tv[t] = v;
            if (!tail_walk<W, CT, T, t + 1>(s, sc, ta, pre, R1, s1, tv, leaf, nodes)) return false;
        }
    }
    return true;
}

// ----------------------------------------------------------------------------
// Kernels

// Per request: free set F, root entry (S = beta * W(F), R = F), accumulators.
template <int W>
__global__ void k_setup(TopoArgs topo, GroupArgs g, LevelView L0, unsigned long long *count0) {
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31;
    const int gw = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = static_cast<int>((gridDim.x * blockDim.x) >> 5);
    if (count0 && blockIdx.x == 0 && threadIdx.x == 0) *count0 = static_cast<unsigned long long>(g.size);
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
            const uint32_t *x = s.cls + static_cast<size_t>(v) * s.cs;
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
            // a bandwidth-sensitive group scores link-count indices: alpha 1 on
            // the class codes, no preserved-bandwidth term
            const int32_t al = g.sens ? 1 : q.policy.alpha, be = g.sens ? 0 : q.policy.beta;
            const long long mag = (llabs(static_cast<long long>(al)) + llabs(static_cast<long long>(be))) *
                                  static_cast<long long>(g.total_weight);
            int32_t state = 0;
            if (q.policy.mode != MAPA_MODE_EXHAUSTIVE && q.policy.mode != MAPA_MODE_BOUNDED)
                state = -3;
            else if (g.sens ? !g.sens_ok : mag >= (1LL << 31))
                state = -2;
            const long long wfree = acc / 2;
            L0.S[i] = state == 0 ? static_cast<int32_t>(be * wfree) : 0;
            L0.r[i] = static_cast<uint32_t>(i);
            uint32_t F0[W];
#pragma unroll
            for (int w = 0; w < W; ++w) F0[w] = state == 0 ? F[w] : 0u;
            store_R<W>(L0, i, F0);
            L0.T[i] = q.root_hi ? (static_cast<uint32_t>(q.root_lo) | (static_cast<uint32_t>(q.root_hi) << 16)) : 0u;
            g.alpha[i] = al;
            g.beta[i] = be;
            if (g.thr) g.thr[i] = INT_MIN;
            if (g.work) g.work[i] = 0ull;
            if (g.dive_s) g.dive_s[i] = INT_MIN;
            g.key[i] = 0ull;
            g.count[i] = 0ull;
            g.best_valid[i] = state;
        }
    }
}

// Work budget: adds to each request's count of stored partial matches its
// entries in level lv (P entries, ordered by request, so two binary searches
// per request find them), and marks every request past the budget with
// thr = INT_MAX, which cuts all its later partials.  Runs between level
// launches, so which requests are cut does not depend on timing.
static __global__ void k_budget(LevelView lv, const unsigned long long *count_dev, unsigned long long count_host,
                         GroupArgs g) {
    const unsigned long long P = count_dev ? *count_dev : count_host;
    if (P == 0ull) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.size; i += gridDim.x * blockDim.x) {
        auto first_at_least = [&](uint32_t key) {
            // the ends first: a group of one request (a served chain step)
            // needs no search at all
            if (lv.r[P - 1] < key) return P;
            if (lv.r[0] >= key) return 0ull;
            unsigned long long lo = 0ull, hi = P;
            while (lo < hi) {
                const unsigned long long mid = (lo + hi) >> 1;
                if (lv.r[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            return lo;
        };
        const unsigned long long nr = first_at_least(static_cast<uint32_t>(i) + 1u) - first_at_least(static_cast<uint32_t>(i));
        if (nr == 0ull) continue;
        const unsigned long long w = g.work[i] + nr;
        g.work[i] = w;
        if (w > g.work_budget) g.thr[i] = INT_MAX;
    }
}

// Bounded mode, seed score: one warp per request runs a depth-first branch
// and bound for at most `steps` node expansions.  Lane j holds the node at
// depth j (pattern vertices 0..j-1 placed): its score, its free set and the
// children not yet tried; my_v is the vertex chosen for pattern vertex j.
// Children are tried best score first (ties: smaller vertex); a child whose
// bound cannot beat the best complete score so far is skipped.  On return,
// inc/found hold the best complete score; the result is true when the whole
// search space was finished within the step limit.
// Guided dive (anytime requests): two necessary conditions on any match
// narrow the candidates of pattern vertex j -- its image lies within
// distance dist0[j] of phi(0) in the free graph (the pattern path from 0 to
// j maps onto a walk through free vertices), and has at least fdeg[j] free
// unused neighbours (its later pattern neighbours need distinct images).
// Neither removes a vertex of any match, so they only steer the descent away
// from dead ends.  Keeps of cand[w] the bits whose vertex has >= need
// neighbours in R (warp-uniform masks; lane l tests bit l of every word).
template <int W>
__device__ __forceinline__ void degree_filter(const SmemTopo &s, uint32_t (&cand)[W], const uint32_t (&R)[W],
                                              int need, int lane) {
    if (need <= 0) return;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        bool pass = false;
        if ((cand[w] >> lane) & 1u) {
            const uint32_t *row = s.adj + (32 * w + lane) * adj_stride(W);
            int c = 0;
#pragma unroll
            for (int x = 0; x < W; ++x) c += __popc(row[x] & R[x]);
            pass = c >= need;
        }
        cand[w] = __ballot_sync(kFull, pass);
    }
}

// Lane d receives ball = the vertices of F within distance d of root in G[F].
template <int W>
__device__ __forceinline__ void distance_balls(const SmemTopo &s, const uint32_t (&F)[W], int root, int lane,
                                               uint32_t (&ball)[W]) {
    uint32_t cur[W];
#pragma unroll
    for (int w = 0; w < W; ++w) cur[w] = (root >> 5) == w ? 1u << (root & 31) : 0u;
    for (int d = 0; d < 32; ++d) {
        if (lane == d)
#pragma unroll
            for (int w = 0; w < W; ++w) ball[w] = cur[w];
        uint32_t acc[W];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[w] = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w)
            if ((cur[w] >> lane) & 1u)
#pragma unroll
                for (int x = 0; x < W; ++x) acc[x] |= s.adj[(32 * w + lane) * adj_stride(W) + x];
#pragma unroll
        for (int x = 0; x < W; ++x) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[x] |= __shfl_xor_sync(kFull, acc[x], o);
            cur[x] = (cur[x] | acc[x]) & F[x];
        }
    }
}

// Node-expansion limits of the guided dive: until the first match, at most
// kRootSteps steps below one choice of phi(0), then the next one (an
// abandoned subtree means the dive no longer proves that no match exists);
// after the first match, at most kImproveSteps more steps to improve on it.
constexpr int kRootSteps = 1024, kImproveSteps = 256;
// dive_run outcomes
constexpr int kDiveDone = 0;     // the search space is finished (proof only when nothing was abandoned)
constexpr int kDiveCap = 1;      // step limit (or the improvement limit) reached
constexpr int kDiveRootEnd = 2;  // one-root mode: the root's subtree ended (this step not taken)
constexpr int kDiveFound = 3;    // one-root mode: the first match (its step taken)
constexpr int kDiveAbort = 4;    // one-root mode: an earlier choice of phi(0) found a match

// One warp's depth-first dive; lane j holds the node at depth j (pattern
// vertices 0..j-1 placed): its score, its free set and the children not yet
// tried; my_v is the vertex chosen for pattern vertex j, rec_v (lane j) the
// vertex of pattern vertex j in the best complete match so far.
template <int W>
struct Dive {
    int32_t my_S;
    int my_v, rec_v;
    uint32_t my_R[W], my_rem[W], ball[W];
    int32_t inc;
    bool found, abandoned, picked;
    int j, step, root_steps, found_at;
};

// Candidates of pattern vertex 0 (warp-uniform): the free set, within the
// root range of a split request's share, and for a guided dive with enough
// free neighbours for vertex 0's pattern degree.
template <int W>
__device__ __forceinline__ void dive_root_candidates(const SmemTopo &s, const PatternArgs &pat, const uint32_t (&F)[W],
                                                     bool guided, int root_lo, int root_hi, int lane,
                                                     uint32_t (&root_cand)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) root_cand[w] = F[w];  // pattern vertex 0: no earlier neighbour, no constraint
    if (root_hi > 0) {  // a share of a split request: phi(0) in [root_lo, root_hi)
        and_above<W>(root_cand, root_lo - 1);
        and_below<W>(root_cand, root_hi);
    }
    if (guided) degree_filter<W>(s, root_cand, F, pat.fdeg[0], lane);
}

// A fresh dive whose depth-0 node has the children root_rem left to try.
template <int W>
__device__ __forceinline__ void dive_init(Dive<W> &d, const uint32_t (&F)[W], const uint32_t (&root_rem)[W], int32_t S0,
                                          int lane) {
    d.my_S = S0;
    d.my_v = 0;
    d.rec_v = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        d.my_R[w] = F[w];
        d.my_rem[w] = lane == 0 ? root_rem[w] : 0u;
        d.ball[w] = 0u;
    }
    d.inc = INT_MIN;
    d.found = d.abandoned = d.picked = false;
    d.j = d.step = d.root_steps = d.found_at = 0;
}

// Bounded mode, seed score, and anytime fallback: a depth-first branch and
// bound, one node expansion per step, until d.step reaches steps.  Children
// are tried best score first (ties: smaller vertex); a child whose bound
// cannot beat the best complete score so far is skipped.  d.inc / d.found
// hold the best complete score.
// Guided dive (anytime requests): two necessary conditions on any match
// narrow the candidates of pattern vertex j -- its image lies within
// distance dist0[j] of phi(0) in the free graph (the pattern path from 0 to
// j maps onto a walk through free vertices), and has at least fdeg[j] free
// unused neighbours (its later pattern neighbours need distinct images).
// Neither removes a vertex of any match, so they only steer the descent away
// from dead ends; until the first match the child with the most free unused
// neighbours is taken first (feasibility before score: a score-first
// descent picks low-degree vertices, which end long patterns in dead ends).
// one_root: stop when the subtree of the first choice of phi(0) ends (the
// next choice is not taken) or at its first match (taken); and, when
// *first (a shared word) drops below my_q, because the search of an earlier
// choice found a match, which makes this one's steps irrelevant.
template <int W, int CT>
__device__ int dive_run(Dive<W> &d, const SmemTopo &s, const PatternArgs &pat, const uint32_t (&F)[W], int32_t al,
                        int32_t be, int lane, int steps, bool guided, bool one_root, const int *first = nullptr,
                        int my_q = 0) {
    const Scorer<W, CT> sc(s, al, be);
    const int k = pat.k;
    for (; d.step < steps; ++d.step) {
        if (one_root && d.picked && d.j == 0) return kDiveRootEnd;
        if (first && __shfl_sync(kFull, *reinterpret_cast<const volatile int *>(first), 0) < my_q) return kDiveAbort;
        if (guided && !d.found && d.j > 0 && ++d.root_steps > kRootSteps) {
            d.abandoned = true;
            if (one_root) return kDiveRootEnd;
            d.j = 0;
            d.root_steps = 0;
        }
        if (guided && d.found && d.step - d.found_at > kImproveSteps) return kDiveCap;
        const int j = d.j;
        uint32_t rem[W], R[W];
        bool any = false;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            rem[w] = __shfl_sync(kFull, d.my_rem[w], j);
            R[w] = __shfl_sync(kFull, d.my_R[w], j);
            any |= rem[w] != 0u;
        }
        const int32_t S = __shfl_sync(kFull, d.my_S, j);
        if (!any) {
            if (j == 0) return kDiveDone;
            --d.j;
            continue;
        }
        uint32_t B[W];
#pragma unroll
        for (int w = 0; w < W; ++w) B[w] = 0u;
        for (uint32_t bm = pat.back[j]; bm; bm &= bm - 1u) set_bit<W>(B, __shfl_sync(kFull, d.my_v, __ffs(bm) - 1));
        // the warp's pick: (most room, before the first match), then best
        // score, then smaller vertex; before the first match only the
        // children with the warp's most room are scored (the same pick)
        const bool by_room = guided && !d.found;
        int mr = 0;
        if (by_room) {
            int lroom = -1;  // -1: no child in this lane
#pragma unroll
            for (int w = 0; w < W; ++w)
                if ((rem[w] >> lane) & 1u) {
                    const int v = 32 * w + lane;
                    int room = 0;
#pragma unroll
                    for (int y = 0; y < W; ++y) room += __popc(s.adj[v * adj_stride(W) + y] & R[y]);
                    lroom = max(lroom, room);
                }
            mr = __reduce_max_sync(kFull, lroom);
        }
        int32_t best = INT_MIN;
        int bv = INT_MAX;
#pragma unroll
        for (int w = 0; w < W; ++w)
            if ((rem[w] >> lane) & 1u) {
                const int v = 32 * w + lane;
                if (by_room) {
                    int room = 0;
#pragma unroll
                    for (int y = 0; y < W; ++y) room += __popc(s.adj[v * adj_stride(W) + y] & R[y]);
                    if (room != mr) continue;
                }
                const int32_t x = S + sc.delta(v, B, R);
                if (x > best) {  // a lane's children come in increasing vertex order
                    best = x;
                    bv = v;
                }
            }
        {
            const int32_t ms = __reduce_max_sync(kFull, bv == INT_MAX ? INT_MIN : best);
            bv = __reduce_min_sync(kFull, (bv != INT_MAX && best == ms) ? bv : INT_MAX);
            best = ms;
        }
        if (lane == j) {
            clear_bit<W>(d.my_rem, bv);
            d.my_v = bv;
        }
        if (j == 0) d.picked = true;
        if (j + 1 == k) {
            const bool first = !d.found;
            if (first) d.found_at = d.step;
            if (first || best > d.inc) d.rec_v = d.my_v;  // lanes < k hold the path, lane j its last vertex
            d.inc = first ? best : max(d.inc, best);
            d.found = true;
            if (one_root && first) {
                ++d.step;
                return kDiveFound;
            }
            continue;
        }
        uint32_t R1[W];
#pragma unroll
        for (int w = 0; w < W; ++w) R1[w] = R[w];
        clear_bit<W>(R1, bv);
        // only the score matters here, so ties with the incumbent are cut too
        if (d.found && cut_off_warp<W>(s, R1, best, al, be, d.inc == INT_MAX ? INT_MAX : d.inc + 1,
                                       level_bound(pat, j + 1), lane))
            continue;
        uint32_t cand[W];
#pragma unroll
        for (int w = 0; w < W; ++w) cand[w] = R1[w];
        int lbv = -1;
        for (uint32_t bm = pat.back[j + 1]; bm; bm &= bm - 1u) {
            const int b = __ffs(bm) - 1;
            const int vb = b == j ? bv : __shfl_sync(kFull, d.my_v, b);
#pragma unroll
            for (int w = 0; w < W; ++w) cand[w] &= s.adj[vb * adj_stride(W) + w];
        }
        for (uint32_t lm = pat.lo[j + 1]; lm; lm &= lm - 1u) {
            const int a = __ffs(lm) - 1;
            lbv = max(lbv, a == j ? bv : __shfl_sync(kFull, d.my_v, a));
        }
        and_above<W>(cand, lbv);
        if (guided) {
            if (j == 0) {
                // phi(0) = bv from here on; where every other pattern vertex
                // is ordered above vertex 0, its match lies in the vertices
                // above bv, so distances are taken there
                uint32_t reach[W];
#pragma unroll
                for (int w = 0; w < W; ++w) reach[w] = F[w];
                if (pat.above0) {
                    and_above<W>(reach, bv);
                    set_bit<W>(reach, bv);
                }
                distance_balls<W>(s, reach, bv, lane, d.ball);
                d.root_steps = 0;
                // fewer than k vertices reachable: no match below this root
                int reachable = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) reachable += __popc(__shfl_sync(kFull, d.ball[w], 31));
                if (reachable < k) continue;
            }
            const int dd = pat.dist0[j + 1];
            if (dd < 32) {
#pragma unroll
                for (int w = 0; w < W; ++w) cand[w] &= __shfl_sync(kFull, d.ball[w], dd);
            }
            degree_filter<W>(s, cand, R1, pat.fdeg[j + 1], lane);
        }
        if (lane == j + 1) {
            d.my_S = best;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                d.my_R[w] = R1[w];
                d.my_rem[w] = cand[w];
            }
        }
        ++d.j;
    }
    return kDiveCap;
}

// The whole dive on one warp, for at most `steps` node expansions.  On
// return, inc/found hold the best complete score and lane j of rec_v the
// vertex of pattern vertex j in that match; the result is true when the
// whole search space was finished within the step limit (nothing abandoned).
template <int W, int CT>
__device__ bool dive_warp(const SmemTopo &s, const PatternArgs &pat, int32_t S0, const uint32_t (&F)[W], int32_t al,
                          int32_t be, int lane, int steps, bool guided, int root_lo, int root_hi, int32_t &inc,
                          bool &found, int &rec_v) {
    uint32_t root_cand[W];
    dive_root_candidates<W>(s, pat, F, guided, root_lo, root_hi, lane, root_cand);
    Dive<W> d;
    dive_init<W>(d, F, root_cand, S0, lane);
    const int code = dive_run<W, CT>(d, s, pat, F, al, be, lane, steps, guided, false);
    inc = d.inc;
    found = d.found;
    rec_v = d.rec_v;
    return code == kDiveDone && !d.abandoned;
}

// The guided dive of one request on a block of kWarps warps, with the same
// result as dive_warp.  Until its first match the dive takes the choices of
// phi(0) in a fixed order (most free neighbours in F, then score, then
// vertex: the depth-0 node never changes), and the search below a choice
// depends only on which choices came before it.  So the block takes the
// choices in waves of kWarps, warp w searching choice w of the wave as the
// one warp would after the earlier ones; the steps each took, summed in
// order, tell which choice the one warp would have reached within its step
// limit and where it would have found its first match, and that warp goes
// on from there as the one warp would.  Returns done (as dive_warp) on
// every thread; inc / found / rec_v are those of warp *winner (or of warp 0
// when nothing was found).
template <int W, int CT>
__device__ bool dive_block(const SmemTopo &s, const PatternArgs &pat, int32_t S0, const uint32_t (&F)[W], int32_t al,
                           int32_t be, int steps, int root_lo, int root_hi, int32_t &inc, bool &found, int &rec_v,
                           int *winner) {
    __shared__ int s_root[kWarps], s_used[kWarps], s_code[kWarps], s_fat[kWarps], s_ab[kWarps];
    __shared__ int s_state, s_win, s_start, s_abandoned, s_first;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();  // the previous request's dive is done with the shared words
    const Scorer<W, CT> sc(s, al, be);
    uint32_t root_cand[W], taken[W];  // taken: choices of phi(0) before this wave
    dive_root_candidates<W>(s, pat, F, true, root_lo, root_hi, lane, root_cand);
#pragma unroll
    for (int w = 0; w < W; ++w) taken[w] = 0u;
    Dive<W> d;
    dive_init<W>(d, F, root_cand, S0, lane);
    int start = 0;  // steps the one warp would have taken before this wave
    bool abandoned = false;
    int state = 0, win = -1;
    for (;;) {
        // warp 0: the next kWarps choices of phi(0), in the one warp's order
        if (threadIdx.x == 0) s_first = kWarps;  // no choice of the wave has found a match yet
        if (warp == 0) {
            uint32_t left[W];
#pragma unroll
            for (int w = 0; w < W; ++w) left[w] = root_cand[w] & ~taken[w];
            for (int q = 0; q < kWarps; ++q) {
                int32_t best = INT_MIN;
                int bv = INT_MAX, broom = -1;
#pragma unroll
                for (int w = 0; w < W; ++w)
                    if ((left[w] >> lane) & 1u) {
                        const int v = 32 * w + lane;
                        uint32_t none[W];
#pragma unroll
                        for (int y = 0; y < W; ++y) none[y] = 0u;
                        const int32_t x = S0 + sc.delta(v, none, F);
                        int room = 0;
#pragma unroll
                        for (int y = 0; y < W; ++y) room += __popc(s.adj[v * adj_stride(W) + y] & F[y]);
                        if (room > broom || (room == broom && x > best)) {
                            best = x;
                            bv = v;
                            broom = room;
                        }
                    }
                const int mr = __reduce_max_sync(kFull, broom);
                const int32_t ms = __reduce_max_sync(kFull, broom == mr ? best : INT_MIN);
                bv = __reduce_min_sync(kFull, (broom == mr && best == ms) ? bv : INT_MAX);
                const int v = mr < 0 ? -1 : bv;
                if (lane == 0) s_root[q] = v;
                if (v >= 0) clear_bit<W>(left, v);
            }
        }
        __syncthreads();
        // warp w: choice w of the wave, after the earlier ones
        const int my_root = s_root[warp];
        if (my_root >= 0) {
            uint32_t rem0[W];
#pragma unroll
            for (int w = 0; w < W; ++w) rem0[w] = root_cand[w] & ~taken[w];
            for (int q = 0; q < warp; ++q) clear_bit<W>(rem0, s_root[q]);
            dive_init<W>(d, F, rem0, S0, lane);
            const int code =
                dive_run<W, CT>(d, s, pat, F, al, be, lane, 2 * kRootSteps + 2, true, true, &s_first, warp);
            if (code == kDiveFound && lane == 0) atomicMin(&s_first, warp);
            if (lane == 0) {
                s_code[warp] = code;
                s_used[warp] = d.step;
                s_fat[warp] = d.found_at;
                s_ab[warp] = d.abandoned || code == kDiveCap;
            }
        }
        __syncthreads();
        // the one warp's accounting, in order
        // states: 0 = next wave, 1 = choice s_win found the first match,
        // 2 = no choice left (the search is finished), 3 = step limit
        if (threadIdx.x == 0) {
            int st = start, sw = 0, wq = -1, ab = 0;
            for (int q = 0; q < kWarps; ++q) {
                if (s_root[q] < 0) {  // no choice left: the one warp's next step ends the search
                    sw = st < steps ? 2 : 3;
                    break;
                }
                if (st >= steps) {
                    sw = 3;
                    break;
                }
                if (s_code[q] == kDiveFound && st + s_fat[q] < steps) {
                    wq = q;
                    sw = 1;
                    break;
                }
                st += s_used[q];
                ab |= s_ab[q];  // a choice abandoned before the outcome
            }
            if (sw == 0 && st >= steps) sw = 3;
            s_state = sw;
            s_win = wq;
            s_start = st;
            s_abandoned = ab;
        }
        __syncthreads();
        state = s_state;
        win = s_win;
        start = s_start;
        abandoned = abandoned || s_abandoned != 0;
        if (state != 0) break;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) set_bit<W>(taken, s_root[q]);
        __syncthreads();  // the shared words are rewritten by the next wave
    }
    *winner = state == 1 ? win : 0;
    const bool done = state == 2 && !abandoned;
    if (state == 1 && warp == win) {
        // the one warp goes on from its first match
        d.step += start;
        d.found_at += start;
        dive_run<W, CT>(d, s, pat, F, al, be, lane, steps, true, false);
    }
    if (state != 1) {
        d.found = false;
        d.inc = INT_MIN;
    }
    inc = d.inc;
    found = d.found;
    rec_v = d.rec_v;
    return done;
}

// Per bounded request (one warp each): the seed dive.  thr = the best
// complete score it found (the seed of the cut-offs); INT_MAX when it
// finished the whole search space without a match (there is none); INT_MIN
// otherwise (no cut-offs).  An anytime request also keeps the dive's best
// match as its fallback.
//
// fallback = 1 (run after the enumeration, exhaustive mode): only anytime
// requests that went past the work budget dive, for their fallback match
// alone (no threshold is written); nothing runs when the device-driven pass
// overflowed (*overflow: the chunked redo decides the group instead).
// fallback = 2 (eager, beside the enumeration): every anytime request of an
// exhaustive group dives, whether or not it will pass its budget (the match
// is used only if it does).
// Returns 0 when request i does not dive, 1 for an unguided dive, 2 for a
// guided one (anytime: it keeps the dive's match as its fallback).
__device__ __forceinline__ int dive_kind(const GroupArgs &g, const mapa_request &q, int i, int fallback) {
    const int32_t al = g.alpha[i], be = g.beta[i];
    const bool bounded = q.policy.mode == MAPA_MODE_BOUNDED;
    const bool anytime = (q.policy.flags & MAPA_POLICY_ANYTIME) != 0 && g.dive_s != nullptr;
    if (g.sens || al < 0 || be < 0) return 0;
    if (!fallback && (!bounded || g.best_valid[i] != 0)) return 0;
    if (fallback && (bounded || !anytime || !g.work || g.best_valid[i] < 0)) return 0;
    if (fallback == 1 && g.work[i] <= g.work_budget) return 0;
    return anytime ? 2 : 1;
}

// Writes a dive's outcome for request i (one warp; lane j of rec_v holds
// phi(j) of the match).
__device__ __forceinline__ void dive_outcome(const GroupArgs &g, const PatternArgs &pat, int i, int fallback,
                                             bool anytime, bool done, bool found, int32_t inc, int rec_v, int lane) {
    // a finished dive without a match proves there is none (cut every
    // partial, in either mode); a found score seeds the cut-offs of the
    // bounded mode only (an exhaustive request must count every match)
    if (lane == 0 && !fallback) g.thr[i] = found ? inc : (done ? INT_MAX : INT_MIN);
    // a fallback dive that finished its whole search without a match
    // proves there is none: the request is a no-fit, not a budget end
    if (fallback && done && !found && lane == 0) g.dive_s[i] = kDiveNoMatch;
    if (anytime && found) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            uint32_t word = 0u;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                word |= static_cast<uint32_t>(__shfl_sync(kFull, rec_v, 4 * w + b) & 0xFF) << (8 * b);
            if (lane == 0) g.dive_t[static_cast<uint64_t>(i) * 8 + w] = 4 * w < pat.k ? word : 0u;
        }
        if (lane == 0) g.dive_s[i] = inc;
    }
}

// One warp per request.  block_guided: the guided dives are left to
// k_dive_block.  An anytime request gets enough steps for several complete
// descents (256 per pattern vertex).
template <int W, int CT>
__global__ void __launch_bounds__(kTpb) k_dive(TopoArgs topo, PatternArgs pat, GroupArgs g, LevelView L0, int steps,
                                               int fallback, const int32_t *overflow, int block_guided) {
    if (fallback && overflow && *overflow) return;
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31;
    const int gw = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = static_cast<int>((gridDim.x * blockDim.x) >> 5);
    for (int i = gw; i < g.size; i += nw) {
        const mapa_request &q = g.reqs[g.req_index[i]];
        const int kind = dive_kind(g, q, i, fallback);
        if (kind == 0 || (kind == 2 && block_guided)) continue;
        const bool anytime = kind == 2;
        uint32_t F[W];
        load_R<W>(L0, i, F);
        int32_t inc;
        bool found;
        int rec_v;
        const int my_steps = anytime ? max(steps, 256 * pat.k) : steps;
        const bool done = dive_warp<W, CT>(s, pat, L0.S[i], F, g.alpha[i], g.beta[i], lane, my_steps, anytime,
                                           q.root_lo, q.root_hi, inc, found, rec_v);
        dive_outcome(g, pat, i, fallback, anytime, done, found, inc, rec_v, lane);
    }
}

// The guided dives (anytime requests), one block per request (dive_block:
// the same outcome as the one-warp dive, with the choices of phi(0) taken
// kWarps at a time).
template <int W, int CT>
__global__ void __launch_bounds__(kTpb) k_dive_block(TopoArgs topo, PatternArgs pat, GroupArgs g, LevelView L0,
                                                     int steps, int fallback, const int32_t *overflow) {
    if (fallback && overflow && *overflow) return;
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = blockIdx.x; i < g.size; i += gridDim.x) {
        const mapa_request &q = g.reqs[g.req_index[i]];
        if (dive_kind(g, q, i, fallback) != 2) continue;  // the same for the whole block
        uint32_t F[W];
        load_R<W>(L0, i, F);
        int32_t inc;
        bool found;
        int rec_v, winner;
        const bool done = dive_block<W, CT>(s, pat, L0.S[i], F, g.alpha[i], g.beta[i], max(steps, 256 * pat.k),
                                            q.root_lo, q.root_hi, inc, found, rec_v, &winner);
        if (warp == winner) dive_outcome(g, pat, i, fallback, true, done, found, inc, rec_v, lane);
    }
}

// Count pass of the host-driven (chunked) path: children per warp and block.
// With thresholds (bounded mode, work budget) it also records which parents
// it cut, one bit per parent in cut_bits[block * 32 + warp * kIpt + j], bit
// lane: the write pass applies exactly these decisions, because a request's
// threshold can change between this pass and a later chunk's write pass (the
// work budget marks requests while deeper levels of earlier chunks run), and
// the write pass must produce exactly the children counted here.
template <int W>
__global__ void __launch_bounds__(kTpb, W >= 4 ? 4 : 1) k_count(TopoArgs topo, LevelView in, uint64_t P, uint32_t back, uint32_t lo,
                                                uint32_t *warp_cnt, unsigned long long *blk_cnt, const int32_t *thr,
                                                const int32_t *alpha, const int32_t *beta, LevelBound lbd,
                                                uint32_t *cut_bits) {
    const SmemTopo s = stage_topology<W>(topo, thr != nullptr);
    __shared__ uint32_t s_w[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t wbase = static_cast<uint64_t>(blockIdx.x) * kTile + static_cast<uint64_t>(warp) * 32 * kIpt;
    int wsum = 0;
#pragma unroll
    for (int j = 0; j < kIpt; ++j) {
        const uint64_t p = wbase + j * 32 + lane;
        int cnt = 0;
        bool cut = false;
        if (p < P) {
            uint32_t A[W], B[W], c[W];
            int lb;
            level_masks<W>(in, p, back, lo, s.adj, A, B, lb);
            root_range<W>(in, static_cast<uint32_t>(p), A, lb);
            uint32_t R[W];
            load_R<W>(in, p, R);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                c[w] = R[w] & A[w];
            }
            and_above<W>(c, lb);
            cnt = popc_mask<W>(c);
            if (thr && cnt) {
                const uint32_t r = in.r[p];
                if (cut_off<W>(s, R, in.S[p], alpha[r], beta[r], thr[r], lbd)) {
                    cnt = 0;
                    cut = true;
                }
            }
        }
        if (thr) {
            const unsigned bits = __ballot_sync(kFull, cut);
            if (lane == 0) cut_bits[static_cast<uint64_t>(blockIdx.x) * 32 + warp * kIpt + j] = bits;
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

// Emits the children of one group of 32 parents (one per lane) at
// out[obase + c], c = 0 .. total-1, lane c taking child c of each round.
template <int W, int CT>
__device__ __forceinline__ void emit_children(const SmemTopo &s, const LevelView &in, const LevelView &out, int ell,
                                              uint64_t p_first, int lane, const uint32_t (&cand)[W],
                                              const uint32_t (&B)[W], const uint32_t (&R)[W], int32_t S, uint32_t r,
                                              int cnt, int incl, int total, uint64_t obase, const int32_t *alpha,
                                              const int32_t *beta) {
    const int nw_in = (ell + 3) >> 2;
    const int new_word = ell >> 2;
    const uint32_t new_shift = (ell & 3) * 8;
    for (int c0 = 0; c0 < total; c0 += 32) {
        const int c = c0 + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const int t = __shfl_sync(kFull, incl, src + step - 1);
            if (t <= c) src += step;
        }
        const int start_s = __shfl_sync(kFull, incl - cnt, src);
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
            const int v = nth_bit<W>(cs, c - start_s);
            const Scorer<W, CT> sc(s, alpha[rs], beta[rs]);
            const int32_t d = sc.delta(v, Bs, Rs);
            const uint32_t o = static_cast<uint32_t>(obase) + static_cast<uint32_t>(c);
            const uint32_t ps = static_cast<uint32_t>(p_first) + static_cast<uint32_t>(src);
            out.S[o] = Ss + d;
            out.r[o] = rs;
            clear_bit<W>(Rs, v);
            store_R<W>(out, o, Rs);
            for (int jw = 0; jw < nw_in; ++jw) {
                uint32_t word = in.T[col_at(in, jw, ps)];
                if (jw == new_word) word |= static_cast<uint32_t>(v) << new_shift;
                out.T[col_at(out, jw, o)] = word;
            }
            if (new_shift == 0) out.T[col_at(out, new_word, o)] = static_cast<uint32_t>(v);
        }
    }
}

template <int W>
__device__ __forceinline__ void parent_state(const SmemTopo &s, const LevelView &in, uint32_t p, uint32_t back,
                                             uint32_t lo, uint32_t (&cand)[W], uint32_t (&B)[W], uint32_t (&R)[W],
                                             int32_t &S, uint32_t &r) {
    uint32_t A[W];
    int lb;
    level_masks<W>(in, p, back, lo, s.adj, A, B, lb);
    root_range<W>(in, p, A, lb);
    load_R<W>(in, p, R);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        cand[w] = R[w] & A[w];
    }
    and_above<W>(cand, lb);
    S = in.S[p];
    r = in.r[p];
}

// Write pass of the host-driven (chunked) path.
template <int W, int CT>
__global__ void __launch_bounds__(kTpb, W >= 4 ? 4 : 1) k_write(TopoArgs topo, LevelView in, uint64_t P, int ell, uint32_t back,
                                                uint32_t lo, LevelView out, const uint32_t *warp_cnt,
                                                const unsigned long long *blk_off, uint64_t blk_first,
                                                const int32_t *alpha, const int32_t *beta, const int32_t *thr,
                                                const uint32_t *cut_bits) {
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t b = blk_first + blockIdx.x;
    uint64_t obase = blk_off[b] - blk_off[blk_first];
    for (int w2 = 0; w2 < warp; ++w2) obase += warp_cnt[b * kWarps + w2];
    const uint64_t wbase = b * kTile + static_cast<uint64_t>(warp) * 32 * kIpt;
    for (int j = 0; j < kIpt; ++j) {
        const uint64_t p = wbase + j * 32 + lane;
        uint32_t cand[W], B[W], R[W];
        int32_t S = 0;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cand[w] = B[w] = R[w] = 0u;
        int32_t al = 0, be = 0;
        if (p < P) {
            parent_state<W>(s, in, p, back, lo, cand, B, R, S, r);
            al = alpha[r];
            be = beta[r];
            // the count pass's cut decision, not a new one (see k_count)
            if (thr && ((cut_bits[b * 32 + warp * kIpt + j] >> lane) & 1u)) {
#pragma unroll
                for (int w = 0; w < W; ++w) cand[w] = 0u;
            }
        }
        const int cnt = popc_mask<W>(cand);
        const int incl = warp_incl_scan(cnt, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        emit_children<W, CT>(s, in, out, ell, wbase + j * 32, lane, cand, B, R, S, r, cnt, incl, total, obase, alpha,
                             beta);
        obase += total;
    }
}

// Decoupled look-back (warp 0 of a block): publishes this tile's total and
// returns the sum of all earlier tiles' totals.  Bounded: after kSpinLimit
// polls of a predecessor it records an error and returns a value past any
// capacity so the tile writes nothing.
__device__ __forceinline__ unsigned long long look_back(unsigned long long *status, unsigned long long t,
                                                        unsigned long long total, int lane, int32_t *err) {
    if (t == 0) {
        if (lane == 0) atomicExch(status, kFlagPrefix | total);
        return 0ull;
    }
    if (lane == 0) atomicExch(status + t, kFlagAgg | total);
    unsigned long long excl = 0ull;
    long long pred = static_cast<long long>(t) - 1;
    bool failed = false;
    for (;;) {
        const long long idx = pred - lane;
        unsigned long long word = 0ull;
        if (idx >= 0) {
            unsigned spins = 0;
            word = *reinterpret_cast<volatile unsigned long long *>(status + idx);
            while ((word >> 62) == 0ull && spins < kSpinLimit) {
                if (spins > 32) __nanosleep(64);
                ++spins;
                word = *reinterpret_cast<volatile unsigned long long *>(status + idx);
            }
            if ((word >> 62) == 0ull) failed = true;
        }
        const unsigned prefix = __ballot_sync(kFull, idx >= 0 && (word & kFlagPrefix));
        const int stop = prefix ? __ffs(prefix) - 1 : 31;
        const unsigned long long v = (idx >= 0 && lane <= stop) ? (word & kValueMask) : 0ull;
        excl += warp_sum_u64(v);
        if (__any_sync(kFull, failed)) {
            if (lane == 0) atomicExch(err, kDevLookbackTimeout);
            return kValueMask;
        }
        if (prefix || pred < 32) break;
        pred -= 32;
    }
    if (lane == 0) atomicExch(status + t, kFlagPrefix | (excl + total));
    return excl;
}

// Single-pass level expansion of the device-driven path: parents are read
// from `in` (count at *count_in), children go to `out` (capacity cap_out),
// the child count to *count_out.  If the children do not fit, nothing past
// the capacity is written, *count_out = 0 and *overflow = 1 (the host then
// redoes the group with the chunked path).
template <int W, int CT, bool Bnd>
__global__ void __launch_bounds__(kTpb, W >= 4 ? 4 : 1) k_expand(TopoArgs topo, LevelView in, LevelView out, int ell, uint32_t back,
                                                 uint32_t lo, const unsigned long long *count_in,
                                                 unsigned long long *count_out, unsigned long long cap_out,
                                                 unsigned int *tile_ctr, unsigned long long *status, int32_t *overflow,
                                                 const int32_t *alpha, const int32_t *beta, int32_t *err,
                                                 unsigned long long *stats, unsigned long long child_bytes,
                                                 unsigned long long parent_bytes, const int32_t *thr,
                                                 LevelBound lbd, unsigned long long count_host, uint64_t p0,
                                                 unsigned int *stop, unsigned long long *resume) {
    // Chunked use (host-driven path; stop and resume non-null): the P
    // parents from p0 on are expanded tile by tile until the children no
    // longer fit; the first tile that does not fit records (tile << 32 |
    // children written before it) in *resume (atomicMin) and lowers *stop.
    // A tile picked after that skips its parents but still takes part in
    // the look-back, with a total of cap_out + 1, so no later tile fits and
    // none waits on it.  The written tiles are a prefix of the range, so
    // the host continues from the first unwritten parent.
    const unsigned long long P = count_in ? *count_in : count_host;
    const unsigned long long ntiles = (P + kTpb - 1) / kTpb;
    if (ntiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *count_out = 0ull;
        return;
    }
    if (static_cast<unsigned long long>(blockIdx.x) >= ntiles) return;  // no tile will be left for this block
    const SmemTopo s = stage_topology<W>(topo, true);
    __shared__ unsigned int s_tile;
    __shared__ int s_skip;
    __shared__ int s_wtot[kWarps];
    __shared__ unsigned long long s_excl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = atomicAdd(tile_ctr, 1u);
            s_skip = stop != nullptr && s_tile > *reinterpret_cast<volatile unsigned int *>(stop);
        }
        __syncthreads();
        const unsigned long long t = s_tile;
        if (t >= ntiles) break;
        const bool skip = s_skip != 0;  // past a tile that did not fit
        const uint64_t p = p0 + t * kTpb + threadIdx.x;
        uint32_t cand[W], B[W], R[W];
        int32_t S = 0;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cand[w] = B[w] = R[w] = 0u;
        int32_t al = 0, be = 0;
        if (p < p0 + P && !skip) {
            parent_state<W>(s, in, static_cast<uint32_t>(p), back, lo, cand, B, R, S, r);
            al = alpha[r];
            be = beta[r];
            if constexpr (Bnd) {
                if (popc_mask<W>(cand) && cut_off<W>(s, R, S, al, be, thr[r], lbd)) {
#pragma unroll
                    for (int w = 0; w < W; ++w) cand[w] = 0u;
                }
            }
        }
        const int cnt = popc_mask<W>(cand);
        const int incl = warp_incl_scan(cnt, lane);
        const int wtot = __shfl_sync(kFull, incl, 31);
        if (lane == 0) s_wtot[warp] = wtot;
        __syncthreads();
        int woff = 0, ttot = 0;
#pragma unroll
        for (int w2 = 0; w2 < kWarps; ++w2) {
            const int v = s_wtot[w2];
            woff += w2 < warp ? v : 0;
            ttot += v;
        }
        if (warp == 0) {
            const unsigned long long agg = skip ? cap_out + 1 : static_cast<unsigned long long>(ttot);
            const unsigned long long ex = look_back(status, t, agg, lane, err);
            if (lane == 0) s_excl = ex;
        }
        __syncthreads();
        const unsigned long long excl = s_excl;
        const bool fits = !skip && excl + static_cast<unsigned long long>(ttot) <= cap_out;
        if (threadIdx.x == 0) {
            if (!fits && overflow) atomicExch(overflow, 1);
            if (!fits && resume) {
                atomicMin(resume, (t << 32) | min(excl, 0xFFFFFFFFull));
                atomicMin(stop, static_cast<unsigned int>(t));
            }
            if (t == ntiles - 1) {
                const unsigned long long total = excl + static_cast<unsigned long long>(ttot);
                *count_out = fits ? total : 0ull;
                if (fits && stats) {
                    atomicAdd(stats + kStatSpill, total);
                    atomicAdd(stats + kStatSpillBytes, 2ull * total * child_bytes);
                    atomicAdd(stats + kStatExpandBytes, P * parent_bytes + total * child_bytes);
                }
            }
        }
        if (fits)
            emit_children<W, CT>(s, in, out, ell, p0 + t * kTpb + static_cast<uint64_t>(warp) * 32, lane, cand, B, R,
                                 S, r, cnt, incl, wtot, excl + woff, alpha, beta);
        __syncthreads();
    }
}

__device__ __forceinline__ void flush_request(uint64_t *key, unsigned long long *count, uint32_t r, uint64_t k,
                                              unsigned long long c) {
    if (c == 0ull) return;
    atomicMax(reinterpret_cast<unsigned long long *>(key + r), static_cast<unsigned long long>(k));
    atomicAdd(count + r, c);
}

struct MaxLeaf {
    int32_t smax = INT_MIN;
    uint32_t leaves = 0;
    __device__ __forceinline__ void add(int n) { leaves += static_cast<uint32_t>(n); }
    template <int T>
    __device__ __forceinline__ bool visit(int32_t sc, const int (&)[T], int) {
        smax = max(smax, sc);
        return true;
    }
};

// Fused last T levels: count and argmax key per request, no frontier write.
// Each warp takes chunks of 32 * kIpt consecutive parents from *tile_ctr
// (dynamic load balance without block barriers: a warp whose subtrees were
// small simply takes the next chunk); P is *count_in (device-driven) or
// count_host (host-driven).
template <int W, int CT, int T, bool Bnd>
__global__ void __launch_bounds__(kTpb) k_last(TopoArgs topo, LevelView in, const unsigned long long *count_in,
                                               unsigned long long count_host, TailArgs ta, const int32_t *alpha,
                                               const int32_t *beta, uint64_t *key, unsigned long long *count,
                                               unsigned int *tile_ctr, unsigned long long *stats, const int32_t *thr) {
    {
        const unsigned long long P0 = count_in ? *count_in : count_host;
        if (static_cast<unsigned long long>(blockIdx.x) * kWarps * 32 * kIpt >= P0) return;  // nothing for this block
    }
    const SmemTopo s = stage_topology<W>(topo, true);
    __shared__ uint32_t s_r[kWarps];
    __shared__ unsigned long long s_key[kWarps];
    __shared__ unsigned long long s_cnt[kWarps];
    __shared__ unsigned long long s_nodes, s_leaves, s_parents;
    if (threadIdx.x == 0) {
        s_nodes = 0ull;
        s_leaves = 0ull;
        s_parents = 0ull;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long P = count_in ? *count_in : count_host;
    constexpr unsigned kChunk = 32 * kIpt;
    const unsigned long long nchunks = (P + kChunk - 1) / kChunk;
    uint32_t r_cur = kNoReq;
    unsigned long long bkey = 0ull, bcnt = 0ull, parents = 0ull, leaves_total = 0ull;
    uint32_t nodes = 0;
    for (;;) {
        unsigned int chunk = 0;
        if (lane == 0) chunk = atomicAdd(tile_ctr, 1u);
        chunk = __shfl_sync(kFull, chunk, 0);
        if (chunk >= nchunks) break;
        const uint64_t wbase = static_cast<uint64_t>(chunk) * kChunk;
        for (int j = 0; j < kIpt; ++j) {
            const uint64_t p = wbase + j * 32 + lane;
            if (p >= P) continue;
            ++parents;
            const uint32_t r = in.r[p];
            if (r != r_cur) {
                if (r_cur != kNoReq) flush_request(key, count, r_cur, bkey, bcnt);
                r_cur = r;
                bkey = 0ull;
                bcnt = 0ull;
            }
            uint32_t R[W];
            load_R<W>(in, p, R);
            if constexpr (Bnd) {
                if (cut_off<W>(s, R, in.S[p], alpha[r], beta[r], thr[r], ta.bound)) continue;
            }
            TailPre<W, T> pre;
            tail_precompute<W, T>(in, p, ta, s.adj, pre);
            const Scorer<W, CT> sc(s, alpha[r], beta[r]);
            MaxLeaf leaf;
            int tv[T];
            tail_walk<W, CT, T, 0>(s, sc, ta, pre, R, in.S[p], tv, leaf, nodes);
            if (leaf.leaves) {
                const unsigned long long k64 = (static_cast<unsigned long long>(biased(leaf.smax)) << 32) |
                                               (0xFFFFFFFFu - static_cast<uint32_t>(p));
                bkey = max(bkey, k64);
                bcnt += leaf.leaves;
                leaves_total += leaf.leaves;
            }
        }
    }
    // warp, then block aggregation of (request, key, count)
    const unsigned long long wn = warp_sum_u64(nodes);
    const unsigned long long wl = warp_sum_u64(leaves_total);
    const unsigned long long wp = warp_sum_u64(parents);
    if (lane == 0) {
        s_r[warp] = kNoReq;
        if (wn) atomicAdd(&s_nodes, wn);
        if (wl) atomicAdd(&s_leaves, wl);
        if (wp) atomicAdd(&s_parents, wp);
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
        if (stats && (s_parents || s_nodes || s_leaves)) {
            atomicAdd(stats + kStatNodes, s_nodes);
            atomicAdd(stats + kStatLeaves, s_leaves);
            atomicAdd(stats + kStatParents, s_parents);
            atomicAdd(stats + kStatOps,
                      ta.cost_parent * s_parents + ta.cost_node * s_nodes + ta.cost_leaf * s_leaves);
        }
    }
}

// ----------------------------------------------------------------------------
// Fused tail of depth 1 or 2 (exhaustive mode; masks of at most 64
// vertices, and every bandwidth-sensitive group): the same result as k_last,
// laid out for these shapes.  One block takes one tile of kTile
// consecutive parents (grid = tiles) and each thread walks its parents' last
// one or two levels with explicit loops.  The score increment loops over the
// weight classes: unrolled when the class count CT (1 to 3) is a template
// argument, rolled otherwise.  Measured on the 32-vertex regular workload,
// this form of the walk issues markedly fewer warp instructions than the
// generic recursive walk, and the unrolled increment made it 15% faster
// than the rolled one.

template <int W>
__device__ __forceinline__ int32_t delta_rolled(const SmemTopo &s, int v, const uint32_t (&B)[W],
                                                const uint32_t (&R)[W], int32_t al, int32_t be) {
    const uint32_t *x = s.cls + static_cast<size_t>(v) * s.cs;
    int32_t acc = 0;
#pragma unroll 1
    for (int c = 0; c < s.C; ++c) {
        int pb = 0, pr = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t xw = x[c * W + w];
            pb += __popc(B[w] & xw);
            pr += __popc(R[w] & xw);
        }
        acc += s.wc[c] * (al * pb - be * pr);
    }
    return acc;
}

// The same, unrolled over a class count CT known at compile time (CT > 0).
template <int W, int CT>
__device__ __forceinline__ int32_t delta_c(const SmemTopo &s, int v, const uint32_t (&B)[W], const uint32_t (&R)[W],
                                           int32_t al, int32_t be) {
    if constexpr (CT == 0) {
        return delta_rolled<W>(s, v, B, R, al, be);
    } else {
        const uint32_t *x = s.cls + v * cls_stride(CT, W);
        int32_t acc = 0;
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            int pb = 0, pr = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint32_t xw = x[c * W + w];
                pb += __popc(B[w] & xw);
                pr += __popc(R[w] & xw);
            }
            acc += s.wc[c] * (al * pb - be * pr);
        }
        return acc;
    }
}

// Walks the last T (1 or 2) levels below parent p; leaf(score) for every
// complete match.
// First level of the explicit tail walk of parent p: its score S, free set
// R, the masks of both tail levels (A, B, lb for pattern vertex ell; A2, B2,
// lb2 for ell + 1 when T = 2) and the candidates c1 of the first tail level,
// filtered when T = 2 by necessary conditions for a node to have a leaf.
template <int W, int T>
struct ShortTailState {
    int32_t S;
    uint32_t R[W], A[W], B[W], c1[W];
    int lb;
    uint32_t A2[W], B2[W];
    int lb2;
    bool nb, nl;
    int nodes;  // first-level candidates before the filter (telemetry)
};

template <int W, int T>
__device__ __forceinline__ void short_tail_first(const SmemTopo &s, const LevelView &in, uint32_t p,
                                                 const TailArgs &ta, ShortTailState<W, T> &st) {
    st.S = in.S[p];
    level_masks<W>(in, p, ta.back_old[0], ta.lo_old[0], s.adj, st.A, st.B, st.lb);
    root_range<W>(in, p, st.A, st.lb);
    load_R<W>(in, p, st.R);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        st.c1[w] = st.R[w] & st.A[w];
    }
    and_above<W>(st.c1, st.lb);
    st.nodes = popc_mask<W>(st.c1);
    if constexpr (T == 2) {
        level_masks<W>(in, p, ta.back_old[1], ta.lo_old[1], s.adj, st.A2, st.B2, st.lb2);
        st.nb = (ta.back_tail[1] & 1u) != 0u;
        st.nl = (ta.lo_tail[1] & 1u) != 0u;
        if (st.nb || st.nl) {
            // Necessary conditions for a node to have a leaf, given the free
            // last-level candidates x (the node itself aside): if the last
            // vertex must come after the node's, the node lies below the
            // highest x; if it is adjacent to the node's, the node neighbours
            // some x (on ring patterns this leaves exactly the nodes with
            // leaves).  The per-node test of the walk stays exact.
            uint32_t x[W];
#pragma unroll
            for (int w = 0; w < W; ++w) x[w] = st.R[w] & st.A2[w];
            and_above<W>(x, st.lb2);
            if (st.nl) and_below<W>(st.c1, highest_bit<W>(x));
            if (st.nb) {
                uint32_t N[W];
#pragma unroll
                for (int w = 0; w < W; ++w) N[w] = 0u;
                int u;
                while ((u = pop_lowest<W>(x)) >= 0) {
#pragma unroll
                    for (int w = 0; w < W; ++w) N[w] |= s.adj[u * adj_stride(W) + w];
                }
#pragma unroll
                for (int w = 0; w < W; ++w) st.c1[w] &= N[w];
            }
        }
    }
}

template <int W, int CT, int T, typename Leaf>
__device__ __forceinline__ void walk_short_tail(const SmemTopo &s, const LevelView &in, uint32_t p, const TailArgs &ta,
                                                int32_t al, int32_t be, Leaf &&leaf, uint32_t &nodes) {
    ShortTailState<W, T> st;
    short_tail_first<W, T>(s, in, p, ta, st);
    if constexpr (T == 2) nodes += st.nodes;  // every first-level candidate, filtered or not
    if constexpr (T == 1) {
        int v;
        while ((v = pop_lowest<W>(st.c1)) >= 0) leaf(st.S + delta_c<W, CT>(s, v, st.B, st.R, al, be));
    } else {
        int v1;
        while ((v1 = pop_lowest<W>(st.c1)) >= 0) {
            uint32_t R1[W], c2[W];
#pragma unroll
            for (int w = 0; w < W; ++w) R1[w] = st.R[w];
            clear_bit<W>(R1, v1);
#pragma unroll
            for (int w = 0; w < W; ++w) c2[w] = R1[w] & st.A2[w] & (st.nb ? s.adj[v1 * adj_stride(W) + w] : ~0u);
            and_above<W>(c2, st.nl ? max(st.lb2, v1) : st.lb2);
            if (!popc_mask<W>(c2)) continue;  // no leaf below: its score is not needed
            const int32_t s1 = st.S + delta_c<W, CT>(s, v1, st.B, st.R, al, be);
            uint32_t B2n[W];
#pragma unroll
            for (int w = 0; w < W; ++w) B2n[w] = st.B2[w];
            if (st.nb) set_bit<W>(B2n, v1);
            int v2;
            while ((v2 = pop_lowest<W>(c2)) >= 0) leaf(s1 + delta_c<W, CT>(s, v2, B2n, R1, al, be));
        }
    }
}

// Sens: the scores are link-count indices of bandwidth-sensitive requests
// and the argmax is taken over their Eq. 2 ranks lut[score].
// Sorted: the block first estimates each parent's subtree by its filtered
// first-level candidate count and hands the tile's parents to lanes in
// decreasing order of it (a counting sort in shared memory), so the 32
// lanes of a warp walk subtrees of similar size; the argmax keys keep the
// parents' own indices, so nothing but the order of work changes.
constexpr int kSortBins = 65;

template <int W, int CT, int T, bool Sens, bool Sorted = false>
__global__ void __launch_bounds__(kTpb) k_last_short(TopoArgs topo, LevelView in, const unsigned long long *count_in,
                                                     unsigned long long count_host, TailArgs ta, const int32_t *alpha,
                                                     const int32_t *beta, uint64_t *key, unsigned long long *count,
                                                     unsigned long long *stats, const int32_t *lut) {
    const unsigned long long P = count_in ? *count_in : count_host;
    if (static_cast<unsigned long long>(blockIdx.x) * kTile >= P) return;  // tile past the stored parents
    const SmemTopo s = stage_topology<W>(topo, true);
    __shared__ uint16_t s_order[Sorted ? kTile : 1];
    __shared__ int s_bin[Sorted ? kSortBins : 1];
    const uint64_t tile0 = static_cast<uint64_t>(blockIdx.x) * kTile;
    if constexpr (Sorted) {
        for (int b = threadIdx.x; b < kSortBins; b += kTpb) s_bin[b] = 0;
        __syncthreads();
        int est[kIpt];
#pragma unroll
        for (int j = 0; j < kIpt; ++j) {
            const int idx = threadIdx.x + j * kTpb;
            est[j] = 0;
            if (tile0 + idx < P) {
                ShortTailState<W, T> st;
                short_tail_first<W, T>(s, in, static_cast<uint32_t>(tile0 + idx), ta, st);
                est[j] = min(popc_mask<W>(st.c1), kSortBins - 1);
            }
            atomicAdd(&s_bin[kSortBins - 1 - est[j]], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int b = 0; b < kSortBins; ++b) {
                const int c = s_bin[b];
                s_bin[b] = acc;
                acc += c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kIpt; ++j)
            s_order[atomicAdd(&s_bin[kSortBins - 1 - est[j]], 1)] = static_cast<uint16_t>(threadIdx.x + j * kTpb);
        __syncthreads();
    }
    __shared__ uint32_t s_r[kWarps];
    __shared__ unsigned long long s_key[kWarps];
    __shared__ unsigned long long s_cnt[kWarps];
    __shared__ unsigned long long s_nodes, s_leaves, s_parents;
    if (threadIdx.x == 0) {
        s_nodes = 0ull;
        s_leaves = 0ull;
        s_parents = 0ull;
    }
    uint32_t nodes = 0, parents = 0, leaves_total = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t r_cur = kNoReq;
    unsigned long long bkey = 0ull, bcnt = 0ull;
    for (int j = 0; j < kIpt; ++j) {
        const int slot = warp * 32 * kIpt + j * 32 + lane;
        const uint64_t p64 = tile0 + (Sorted ? s_order[slot] : slot);
        if (p64 >= P) continue;
        const uint32_t p = static_cast<uint32_t>(p64);
        const uint32_t r = in.r[p];
        ++parents;
        if (r != r_cur) {
            if (r_cur != kNoReq) flush_request(key, count, r_cur, bkey, bcnt);
            r_cur = r;
            bkey = 0ull;
            bcnt = 0ull;
        }
        int32_t smax = INT_MIN;
        uint32_t leaves = 0;
        walk_short_tail<W, CT, T>(
            s, in, p, ta, alpha[r], beta[r],
            [&](int32_t sc) {
                if constexpr (Sens) sc = lut[sc];
                smax = max(smax, sc);
                ++leaves;
            },
            nodes);
        if (leaves) {
            const unsigned long long k64 =
                (static_cast<unsigned long long>(biased(smax)) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(p));
            bkey = max(bkey, k64);
            bcnt += leaves;
            leaves_total += leaves;
        }
    }
    // warp, then block aggregation of (request, key, count)
    const int wn = warp_sum_int(static_cast<int>(nodes));
    const int wp = warp_sum_int(static_cast<int>(parents));
    const unsigned long long wl = warp_sum_u64(leaves_total);
    if (lane == 0) {
        s_r[warp] = kNoReq;
        if (wn) atomicAdd(&s_nodes, static_cast<unsigned long long>(wn));
        if (wp) atomicAdd(&s_parents, static_cast<unsigned long long>(wp));
        if (wl) atomicAdd(&s_leaves, wl);
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
        if (stats && (s_parents || s_nodes || s_leaves)) {
            atomicAdd(stats + kStatNodes, s_nodes);
            atomicAdd(stats + kStatLeaves, s_leaves);
            atomicAdd(stats + kStatParents, s_parents);
            atomicAdd(stats + kStatOps,
                      ta.cost_parent * s_parents + ta.cost_node * s_nodes + ta.cost_leaf * s_leaves);
        }
    }
}

// ----------------------------------------------------------------------------
// Fused tail of depth 3 with a cooperative first level (exhaustive mode,
// masks of at most 64 vertices).  A warp takes 32 stored parents (level l),
// counts their children at level l+1 and hands the children out across its
// lanes the way k_expand emits them (lane c takes child c of the round), but
// keeps them in registers instead of writing a level; each lane then walks the
// last two levels below its child.  The work per lane is that of the depth-2
// tail, balanced per child instead of per parent, and level l+1 never goes
// through memory.

struct TailShared {
    uint32_t r[kWarps];
    unsigned long long key[kWarps];
    unsigned long long cnt[kWarps];
    unsigned long long nodes, leaves, parents;
};

// End of a fused-tail block: each warp merges its threads' (request, key,
// count) when they all hold the same request (else flushes per thread), the
// block merges its warps, and the telemetry counters are added once.
__device__ __forceinline__ void tail_block_end(TailShared &sh, int lane, int warp, uint32_t r_cur,
                                               unsigned long long bkey, unsigned long long bcnt,
                                               unsigned long long nodes, unsigned long long parents,
                                               unsigned long long leaves, uint64_t *key, unsigned long long *count,
                                               unsigned long long *stats, const TailArgs &ta) {
    const unsigned long long wn = warp_sum_u64(nodes), wp = warp_sum_u64(parents), wl = warp_sum_u64(leaves);
    if (lane == 0) {
        sh.r[warp] = kNoReq;
        if (wn) atomicAdd(&sh.nodes, wn);
        if (wp) atomicAdd(&sh.parents, wp);
        if (wl) atomicAdd(&sh.leaves, wl);
    }
    const unsigned act = __ballot_sync(kFull, bcnt > 0ull);
    if (act) {
        const uint32_t rl = __shfl_sync(kFull, r_cur, __ffs(act) - 1);
        if (__all_sync(kFull, bcnt == 0ull || r_cur == rl)) {
            unsigned long long k = bkey, c = bcnt;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                k = max(k, __shfl_xor_sync(kFull, k, o));
                c += __shfl_xor_sync(kFull, c, o);
            }
            if (lane == 0) {
                sh.r[warp] = rl;
                sh.key[warp] = k;
                sh.cnt[warp] = c;
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
            if (sh.r[w] == kNoReq) continue;
            if (sh.r[w] != r) {
                if (r != kNoReq) flush_request(key, count, r, k, c);
                r = sh.r[w];
                k = 0ull;
                c = 0ull;
            }
            k = max(k, sh.key[w]);
            c += sh.cnt[w];
        }
        if (r != kNoReq) flush_request(key, count, r, k, c);
        if (stats && (sh.parents || sh.nodes || sh.leaves)) {
            atomicAdd(stats + kStatNodes, sh.nodes);
            atomicAdd(stats + kStatLeaves, sh.leaves);
            atomicAdd(stats + kStatParents, sh.parents);
            atomicAdd(stats + kStatOps, ta.cost_parent * sh.parents + ta.cost_node * sh.nodes + ta.cost_leaf * sh.leaves);
        }
    }
}

template <int W, int CT>
__global__ void __launch_bounds__(kTpb) k_last_coop3(TopoArgs topo, LevelView in, const unsigned long long *count_in,
                                                     unsigned long long count_host, TailArgs ta, const int32_t *alpha,
                                                     const int32_t *beta, uint64_t *key, unsigned long long *count,
                                                     unsigned int *tile_ctr, unsigned long long *stats) {
    const unsigned long long P = count_in ? *count_in : count_host;
    if (static_cast<unsigned long long>(blockIdx.x) * kWarps * 32 >= P) return;  // nothing for this block
    const SmemTopo s = stage_topology<W>(topo, true);
    __shared__ TailShared sh;
    if (threadIdx.x == 0) {
        sh.nodes = 0ull;
        sh.leaves = 0ull;
        sh.parents = 0ull;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long nchunks = (P + 31) / 32;
    const bool nb21 = (ta.back_tail[1] & 1u) != 0u, nl21 = (ta.lo_tail[1] & 1u) != 0u;
    const bool nb31 = (ta.back_tail[2] & 1u) != 0u, nl31 = (ta.lo_tail[2] & 1u) != 0u;
    const bool nb32 = (ta.back_tail[2] & 2u) != 0u, nl32 = (ta.lo_tail[2] & 2u) != 0u;
    uint32_t r_cur = kNoReq;
    unsigned long long bkey = 0ull, bcnt = 0ull, parents = 0ull, leaves_total = 0ull, nodes = 0ull;
    for (;;) {
        unsigned int chunk = 0;
        if (lane == 0) chunk = atomicAdd(tile_ctr, 1u);
        chunk = __shfl_sync(kFull, chunk, 0);
        if (chunk >= nchunks) break;
        // lane = one stored parent: its candidates at level l and the masks
        // of levels l+1 and l+2 from its stored vertices
        const uint64_t p = static_cast<uint64_t>(chunk) * 32 + lane;
        uint32_t c1[W], B1[W], R[W], A2[W], B2[W], A3[W], B3[W];
        int lb2 = -1, lb3 = -1;
        int32_t S = 0, al = 0, be = 0;
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) c1[w] = B1[w] = R[w] = A2[w] = B2[w] = A3[w] = B3[w] = 0u;
        if (p < P) {
            ++parents;
            uint32_t A1[W];
            int lb1;
            level_masks<W>(in, p, ta.back_old[0], ta.lo_old[0], s.adj, A1, B1, lb1);
            root_range<W>(in, p, A1, lb1);
            level_masks<W>(in, p, ta.back_old[1], ta.lo_old[1], s.adj, A2, B2, lb2);
            level_masks<W>(in, p, ta.back_old[2], ta.lo_old[2], s.adj, A3, B3, lb3);
            load_R<W>(in, p, R);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                c1[w] = R[w] & A1[w];
            }
            and_above<W>(c1, lb1);
            S = in.S[p];
            r = in.r[p];
            al = alpha[r];
            be = beta[r];
        }
        const int cnt = popc_mask<W>(c1);
        const int incl = warp_incl_scan(cnt, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        for (int c0 = 0; c0 < total; c0 += 32) {
            // lane c takes child c of the round: its parent by binary search
            const int c = c0 + lane;
            int src = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int t = __shfl_sync(kFull, incl, src + step - 1);
                if (t <= c) src += step;
            }
            const int start = __shfl_sync(kFull, incl - cnt, src);
            uint32_t cs[W], Bs[W], Rs[W], A2s[W], B2s[W], A3s[W], B3s[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                cs[w] = __shfl_sync(kFull, c1[w], src);
                Bs[w] = __shfl_sync(kFull, B1[w], src);
                Rs[w] = __shfl_sync(kFull, R[w], src);
                A2s[w] = __shfl_sync(kFull, A2[w], src);
                B2s[w] = __shfl_sync(kFull, B2[w], src);
                A3s[w] = __shfl_sync(kFull, A3[w], src);
                B3s[w] = __shfl_sync(kFull, B3[w], src);
            }
            const int32_t Ss = __shfl_sync(kFull, S, src), als = __shfl_sync(kFull, al, src),
                          bes = __shfl_sync(kFull, be, src);
            const uint32_t rs = __shfl_sync(kFull, r, src);
            const int lb2s = __shfl_sync(kFull, lb2, src), lb3s = __shfl_sync(kFull, lb3, src);
            if (c >= total) continue;
            const uint64_t ps = static_cast<uint64_t>(chunk) * 32 + src;
            if (rs != r_cur) {
                if (r_cur != kNoReq) flush_request(key, count, r_cur, bkey, bcnt);
                r_cur = rs;
                bkey = 0ull;
                bcnt = 0ull;
            }
            const int v1 = nth_bit<W>(cs, c - start);
            ++nodes;
            const int32_t s1 = Ss + delta_c<W, CT>(s, v1, Bs, Rs, als, bes);
            uint32_t R1[W], c2[W], B2n[W];
#pragma unroll
            for (int w = 0; w < W; ++w) {
                R1[w] = Rs[w];
                B2n[w] = B2s[w];
            }
            clear_bit<W>(R1, v1);
            if (nb21) set_bit<W>(B2n, v1);
#pragma unroll
            for (int w = 0; w < W; ++w) c2[w] = R1[w] & A2s[w] & (nb21 ? s.adj[v1 * adj_stride(W) + w] : ~0u);
            and_above<W>(c2, nl21 ? max(lb2s, v1) : lb2s);
            int32_t smax = INT_MIN;
            uint32_t leaves = 0;
            int v2;
            while ((v2 = pop_lowest<W>(c2)) >= 0) {
                ++nodes;
                uint32_t R2[W], c3[W], B3n[W];
#pragma unroll
                for (int w = 0; w < W; ++w) R2[w] = R1[w];
                clear_bit<W>(R2, v2);
#pragma unroll
                for (int w = 0; w < W; ++w)
                    c3[w] = R2[w] & A3s[w] & (nb31 ? s.adj[v1 * adj_stride(W) + w] : ~0u) & (nb32 ? s.adj[v2 * adj_stride(W) + w] : ~0u);
                int lb = lb3s;
                if (nl31) lb = max(lb, v1);
                if (nl32) lb = max(lb, v2);
                and_above<W>(c3, lb);
                if (!popc_mask<W>(c3)) continue;  // no leaf below: its score is not needed
                const int32_t s2 = s1 + delta_c<W, CT>(s, v2, B2n, R1, als, bes);
#pragma unroll
                for (int w = 0; w < W; ++w) B3n[w] = B3s[w];
                if (nb31) set_bit<W>(B3n, v1);
                if (nb32) set_bit<W>(B3n, v2);
                int v3;
                while ((v3 = pop_lowest<W>(c3)) >= 0) {
                    smax = max(smax, s2 + delta_c<W, CT>(s, v3, B3n, R2, als, bes));
                    ++leaves;
                }
            }
            if (leaves) {
                const unsigned long long k64 =
                    (static_cast<unsigned long long>(biased(smax)) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(ps));
                bkey = max(bkey, k64);
                bcnt += leaves;
                leaves_total += leaves;
            }
        }
    }
    tail_block_end(sh, lane, warp, r_cur, bkey, bcnt, nodes, parents, leaves_total, key, count, stats, ta);
}

template <int T>
struct FindLeaf {
    int32_t target;
    const int32_t *lut;  // bandwidth-sensitive group: compare Eq. 2 ranks
    bool found = false;
    int tail[T];
    __device__ __forceinline__ void add(int) {}
    __device__ __forceinline__ bool visit(int32_t sc, const int (&tv)[T], int v) {
        if (lut) sc = lut[sc];
        if (sc != target) return true;
        found = true;
#pragma unroll
        for (int j = 0; j + 1 < T; ++j) tail[j] = tv[j];
        tail[T - 1] = v;
        return false;
    }
};

// Per request present in a last-level chunk: decode the chunk's argmax key,
// re-walk the winning parent's tail in lexicographic order to recover the
// first tail reaching that score, and merge into the running best with a
// strict ">" (chunks arrive in lexicographic order).
template <int W, int CT, int T>
__global__ void k_resolve(TopoArgs topo, LevelView in, const unsigned long long *count_in,
                          unsigned long long count_host, TailArgs ta, GroupArgs g) {
    const SmemTopo s = stage_topology<W>(topo, true);
    const unsigned long long P = count_in ? *count_in : count_host;
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
        TailPre<W, T> pre;
        tail_precompute<W, T>(in, p, ta, s.adj, pre);
        uint32_t R[W];
        load_R<W>(in, p, R);
        const Scorer<W, CT> sc(s, g.alpha[r], g.beta[r]);
        FindLeaf<T> leaf;
        leaf.target = target;
        leaf.lut = g.sens ? g.effbw_rank : nullptr;
        int tv[T];
        uint32_t nodes = 0;
        tail_walk<W, CT, T, 0>(s, sc, ta, pre, R, in.S[p], tv, leaf, nodes);
        if (!leaf.found) {
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
#pragma unroll
            for (int j = 0; j < T; ++j) {
                const int pos = ta.ell + j;
#pragma unroll
                for (int jw = 0; jw < 8; ++jw)
                    if (jw == (pos >> 2)) words[jw] |= static_cast<uint32_t>(leaf.tail[j]) << ((pos & 3) * 8);
            }
#pragma unroll
            for (int jw = 0; jw < 8; ++jw) g.best_t[static_cast<uint64_t>(r) * 8 + jw] = words[jw];
        }
    }
}

__device__ __forceinline__ int link_class(const SmemTopo &s, int W, int x, int y) {
    const uint32_t *row = s.cls + static_cast<size_t>(x) * s.cs;
    for (int c = 0; c < s.C; ++c)
        if ((row[c * W + (y >> 5)] >> (y & 31)) & 1u) return c;
    return -1;
}

__device__ __forceinline__ int32_t link_weight(const SmemTopo &s, int W, int x, int y) {
    const uint32_t *row = s.cls + static_cast<size_t>(x) * s.cs;
    for (int c = 0; c < s.C; ++c)
        if ((row[c * W + (y >> 5)] >> (y & 31)) & 1u) return s.wc[c];
    return 0;
}

// Writes every request's result: the chosen tuple's AggBW (Eq. 1) and
// PreservedBW (Eq. 3) recomputed from their definitions on the bitsets and
// checked against the enumerated score.  One warp per request: the lanes
// split the scan of the free set behind PreservedBW, lane 0 writes.
template <int W>
__global__ void k_finalize(TopoArgs topo, PatternArgs pat, GroupArgs g) {
    const SmemTopo s = stage_topology<W>(topo, true);
    const int lane = threadIdx.x & 31;
    const int gw = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = static_cast<int>((gridDim.x * blockDim.x) >> 5);
    for (int i = gw; i < g.size; i += nw) {
        const int32_t bi = g.req_index[i];
        const mapa_request &q = g.reqs[bi];
        mapa_result res;
        memset(&res, 0, sizeof(res));
        res.k = pat.k;
        res.count = g.count[i];
        const int32_t state = g.best_valid[i];
        // Past the context's work budget the enumeration was cut short: no
        // decision, or for an anytime request the seed dive's match.  (The
        // matches the enumeration scored before the cut are not used: which
        // ones they are depends on the other requests sharing its chunks,
        // while the dive depends on the request alone.)
        const bool over = state >= 0 && g.work && g.work[i] > g.work_budget;
        bool proven_none = false;
        const uint32_t *tw = g.best_t + static_cast<uint64_t>(i) * 8;
        int32_t want = g.best_s[i];
        bool have = state == 1;
        if (over) {
            res.count = 0;
            const bool anytime = (q.policy.flags & MAPA_POLICY_ANYTIME) && g.dive_s && !g.sens;
            proven_none = anytime && g.dive_s[i] == kDiveNoMatch;
            have = anytime && g.dive_s[i] != INT_MIN && !proven_none;
            if (have) {
                tw = g.dive_t + static_cast<uint64_t>(i) * 8;
                want = g.dive_s[i];
            }
        }
        if (state == -2) {
            res.status = MAPA_E_RANGE;
            res.count = 0;
        } else if (state == -3) {
            res.status = MAPA_E_INVALID;
            res.count = 0;
        } else if (over && proven_none) {
            res.status = MAPA_NO_FIT;
        } else if (over && !have) {
            res.status = MAPA_E_BUDGET;
        } else if (!over && q.policy.max_embeddings > 0 && res.count > q.policy.max_embeddings) {
            res.status = MAPA_E_BUDGET;
        } else if (!have) {
            res.status = MAPA_NO_FIT;
        } else {
            uint8_t t[kMaxK];
            for (int j = 0; j < pat.k; ++j) t[j] = static_cast<uint8_t>((tw[j >> 2] >> ((j & 3) * 8)) & 0xFFu);
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
            for (int v = lane; v < s.n; v += 32) {
                if (!((rem[v >> 5] >> (v & 31)) & 1u)) continue;
                const uint32_t *x = s.cls + static_cast<size_t>(v) * s.cs;
                for (int c = 0; c < s.C; ++c) {
                    int pc = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) pc += __popc(x[c * W + w] & rem[w]);
                    twice += static_cast<long long>(s.wc[c]) * pc;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) twice += __shfl_xor_sync(kFull, twice, o);
            const long long pres = twice / 2;
            res.status = over ? MAPA_INEXACT : MAPA_OK;
            if (g.sens) {
                // link-count index of the tuple from the class of every pattern
                // edge's link; its Eq. 2 rank must be the one the tail chose
                int32_t idx = 0;
                for (int v = 0; v < pat.k; ++v)
                    for (uint32_t m = pat.back[v]; m; m &= m - 1u) {
                        const int c = link_class(s, W, t[__ffs(m) - 1], t[v]);
                        if (c >= 0) idx += g.effbw_code[c];
                    }
                if (lane == 0 && g.effbw_rank[idx] != g.best_s[i]) atomicExch(g.error, kDevScoreMismatch);
                res.score = g.effbw_milli[idx];
            } else {
                const long long score =
                    static_cast<long long>(g.alpha[i]) * agg + static_cast<long long>(g.beta[i]) * pres;
                if (lane == 0 && score != want) atomicExch(g.error, kDevScoreMismatch);
                res.score = want;
            }
            res.agg = static_cast<int32_t>(agg);
            res.pres = static_cast<int32_t>(pres);
            for (int j = 0; j < pat.k; ++j) res.verts[j] = t[j];
        }
        if (q.policy.mode == MAPA_MODE_BOUNDED) res.count = 0;
        if (lane == 0) g.out[bi] = res;
    }
}

}  // namespace mapa
