// Allocation-free decision entry point (mapa_allocate_batch_noalloc).
//
// Some callers cannot call cudaMalloc: a scheduler loop that runs while a
// CUDA graph is being captured on its thread, a hook that runs inside another
// framework's allocator (where allocating again can deadlock or recurse), or
// a process whose device memory is fully reserved up front by a serving
// runtime.  For them this file decides small batches (up to 4096 requests on
// servers of up to 32 accelerators, patterns of up to 8 vertices) with one
// kernel launch and no allocation: the kernel's scratch -- per-request argmax
// keys, match counts and completion tickets -- lives in the file-scope
// device array below, which every GPU that loads this library holds until the
// process exits (80 KiB per GPU).
//
// The enumeration is the same one the batched engine runs (matches in
// pattern-id order under the automorphism order constraints, scores grown by
// the same per-vertex increment), here walked depth first by 1024 threads per
// request, one per choice of the first two pattern vertices.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <mutex>
#include <string>

#include "mapa_internal.h"

namespace mapa {

namespace {

constexpr int kNaMaxRequests = MAPA_NOALLOC_MAX_REQUESTS;
constexpr int kNaMaxN = MAPA_NOALLOC_MAX_N;
constexpr int kNaMaxK = MAPA_NOALLOC_MAX_K;
constexpr int kNaItems = kNaMaxN * kNaMaxN;  // (phi(0), phi(1)) pairs per request
constexpr int kNaThreads = 256;
constexpr int kNaBlocksPerRequest = kNaItems / kNaThreads;  // a block's items belong to one request
static_assert(kNaItems % kNaThreads == 0, "a block must cover items of one request only");
constexpr size_t kNaKeyBytes = sizeof(unsigned long long) * kNaMaxRequests;
constexpr size_t kNaTicketBytes = sizeof(unsigned int) * kNaMaxRequests;
constexpr size_t kNaScratchBytes = 2 * kNaKeyBytes + kNaTicketBytes;  // keys, counts, tickets

// Kernel scratch shared by every call on a device (see mapa.h for the rules).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

std::mutex g_scratch_mutex;
void *g_scratch_ptr[64] = {};  // device address of g_noalloc_scratch, per device

__device__ __forceinline__ int32_t na_delta(const uint32_t *cls, const int32_t *wc, int C, int v, uint32_t B,
                                            uint32_t R, int32_t al, int32_t be) {
    int32_t acc = 0;
    for (int c = 0; c < C; ++c) {
        const uint32_t x = cls[v * C + c];
        acc += wc[c] * (al * __popc(B & x) - be * __popc(R & x));
    }
    return acc;
}

__device__ __forceinline__ uint32_t na_above(int lb) {
    if (lb < 0) return ~0u;
    if (lb >= 31) return 0u;
    return ~0u << (lb + 1);
}

// Candidates of pattern vertex d given phi[0..d-1]; B receives the image set
// of d's earlier neighbours.
__device__ __forceinline__ uint32_t na_candidates(const PatternArgs &pat, const uint32_t *adj, const int *phi, int d,
                                                  uint32_t R, uint32_t *B) {
    uint32_t A = R, img = 0u;
    uint32_t m = pat.back[d];
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1u;
        A &= adj[phi[b]];
        img |= 1u << phi[b];
    }
    int lb = -1;
    m = pat.lo[d];
    while (m) {
        const int a = __ffs(m) - 1;
        m &= m - 1u;
        lb = max(lb, phi[a]);
    }
    *B = img;
    return A & na_above(lb);
}

struct NaState {
    int phi[kNaMaxK];
    uint32_t cand[kNaMaxK];
    uint32_t Bs[kNaMaxK];
    uint32_t Rs[kNaMaxK + 1];
    int32_t Ss[kNaMaxK + 1];
};

// Depth-first walk below a fixed prefix phi[0..start-1] (start >= 1), calling
// leaf(score) on every complete match in lexicographic order; stops when
// leaf returns false.  Returns false if stopped.
template <typename Leaf>
__device__ bool na_walk(const PatternArgs &pat, const uint32_t *adj, const uint32_t *cls, const int32_t *wc, int C,
                        int32_t al, int32_t be, NaState &st, int start, Leaf &&leaf) {
    const int k = pat.k;
    if (start == k) return leaf(st.Ss[k]);
    int d = start;
    st.cand[d] = na_candidates(pat, adj, st.phi, d, st.Rs[d], &st.Bs[d]);
    while (d >= start) {
        if (st.cand[d] == 0u) {
            --d;
            continue;
        }
        const int v = __ffs(st.cand[d]) - 1;
        st.cand[d] &= st.cand[d] - 1u;
        st.phi[d] = v;
        st.Ss[d + 1] = st.Ss[d] + na_delta(cls, wc, C, v, st.Bs[d], st.Rs[d], al, be);
        st.Rs[d + 1] = st.Rs[d] & ~(1u << v);
        if (d + 1 == k) {
            if (!leaf(st.Ss[k])) return false;
            continue;
        }
        ++d;
        st.cand[d] = na_candidates(pat, adj, st.phi, d, st.Rs[d], &st.Bs[d]);
    }
    return true;
}

// Places phi(0) = v0 and, for k >= 2, phi(1) = v1 on a fresh state; returns
// false if that prefix is not a valid start of a match.
__device__ bool na_prefix(const PatternArgs &pat, const uint32_t *adj, const uint32_t *cls, const int32_t *wc, int C,
                          int32_t al, int32_t be, uint32_t F, int32_t root, int v0, int v1, NaState &st) {
    if (!((F >> v0) & 1u)) return false;
    st.Rs[0] = F;
    st.Ss[0] = root;
    st.phi[0] = v0;
    st.Ss[1] = root + na_delta(cls, wc, C, v0, 0u, F, al, be);
    st.Rs[1] = F & ~(1u << v0);
    if (pat.k == 1) return v1 == 0;
    uint32_t B1;
    const uint32_t c1 = na_candidates(pat, adj, st.phi, 1, st.Rs[1], &B1);
    if (!((c1 >> v1) & 1u)) return false;
    st.phi[1] = v1;
    st.Ss[2] = st.Ss[1] + na_delta(cls, wc, C, v1, B1, st.Rs[1], al, be);
    st.Rs[2] = st.Rs[1] & ~(1u << v1);
    return true;
}

__device__ __forceinline__ uint32_t na_free_set(const mapa_request &q, int n) {
    const uint32_t valid = n >= 32 ? ~0u : ((1u << n) - 1u);
    return ~q.busy[0] & valid;
}

__device__ int32_t na_request_state(const mapa_request &q, int32_t pattern_id, int64_t total_weight) {
    if (q.pattern_id != pattern_id || (q.policy.flags & MAPA_POLICY_BW_SENSITIVE)) return -3;
    if (q.policy.mode != MAPA_MODE_EXHAUSTIVE && q.policy.mode != MAPA_MODE_BOUNDED) return -3;
    // The batched path's bounded mode applies max_embeddings to the matches
    // left after its cut-offs; this kernel has no cut-offs, so it cannot give
    // the same answer and refuses the combination.
    if (q.policy.mode == MAPA_MODE_BOUNDED && q.policy.max_embeddings > 0) return -3;
    if (q.root_hi != 0) return -3;  // shares of a split request are decided by the batched call
    const long long mag = (llabs(static_cast<long long>(q.policy.alpha)) + llabs(static_cast<long long>(q.policy.beta))) *
                          static_cast<long long>(total_weight);
    return mag >= (1LL << 31) ? -2 : 0;
}

__global__ void __launch_bounds__(kNaThreads)
    k_decide_noalloc(TopoArgs topo, PatternArgs pat, int32_t pattern_id, int64_t total_weight, int32_t nreq,
                     const mapa_request *reqs, mapa_result *out, unsigned char *scratch) {
    __shared__ uint32_t s_adj[kNaMaxN];
    __shared__ uint32_t s_cls[kNaMaxN * kMaxClasses];
    __shared__ int32_t s_wc[kMaxClasses];
    __shared__ int s_last;
    const int n = topo.n, C = topo.C;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_adj[i] = topo.adj[i];
    for (int i = threadIdx.x; i < n * C; i += blockDim.x) s_cls[i] = topo.clsv[i];
    for (int i = threadIdx.x; i < C; i += blockDim.x) s_wc[i] = topo.wc[i];
    __syncthreads();
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch);
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(scratch + kNaKeyBytes);
    unsigned int *tickets = reinterpret_cast<unsigned int *>(scratch + 2 * kNaKeyBytes);

    // ---- enumerate: thread = (request, phi(0), phi(1))
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int r = static_cast<int>(g / kNaItems);
    const int item = static_cast<int>(g % kNaItems);
    unsigned long long key = 0ull, cnt = 0ull;
    if (r < nreq) {
        const mapa_request q = reqs[r];
        if (na_request_state(q, pattern_id, total_weight) == 0) {
            const uint32_t F = na_free_set(q, n);
            long long twice = 0;
            for (int v = 0; v < n; ++v)
                if ((F >> v) & 1u)
                    for (int c = 0; c < C; ++c) twice += static_cast<long long>(s_wc[c]) * __popc(s_cls[v * C + c] & F);
            const int32_t al = q.policy.alpha, be = q.policy.beta;
            const int32_t root = static_cast<int32_t>(be * (twice / 2));
            NaState st;
            const int v0 = item / kNaMaxN, v1 = item % kNaMaxN;
            if (v0 < n && v1 < n && na_prefix(pat, s_adj, s_cls, s_wc, C, al, be, F, root, v0, v1, st)) {
                int32_t best = INT_MIN;
                na_walk(pat, s_adj, s_cls, s_wc, C, al, be, st, pat.k == 1 ? 1 : 2, [&](int32_t sc) {
                    best = max(best, sc);
                    ++cnt;
                    return true;
                });
                if (cnt)
                    key = (static_cast<unsigned long long>(static_cast<uint32_t>(best) ^ 0x80000000u) << 32) |
                          (0xFFFFFFFFu - static_cast<uint32_t>(item));
            }
        }
    }
    // a warp covers 32 items of one request: reduce, then one atomic pair
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        key = max(key, __shfl_xor_sync(0xFFFFFFFFu, key, o));
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt && r < nreq) {
        atomicMax(keys + r, key);
        atomicAdd(counts + r, cnt);
    }

    // ---- the last of a request's blocks to finish resolves and writes its
    // result (every block's items belong to one request)
    const int rb = static_cast<int>((static_cast<long long>(blockIdx.x) * blockDim.x) / kNaItems);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = rb < nreq && atomicAdd(tickets + rb, 1u) == kNaBlocksPerRequest - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = rb + static_cast<int>(threadIdx.x); i == rb; ++i) {  // thread 0 only
        const mapa_request q = reqs[i];
        mapa_result res;
        memset(&res, 0, sizeof(res));
        res.k = pat.k;
        const int32_t state = na_request_state(q, pattern_id, total_weight);
        const unsigned long long k64 = __ldcg(keys + i);
        const unsigned long long c64 = __ldcg(counts + i);
        if (state == -2) {
            res.status = MAPA_E_RANGE;
        } else if (state == -3) {
            res.status = MAPA_E_INVALID;
        } else if (q.policy.max_embeddings > 0 && c64 > q.policy.max_embeddings) {
            res.status = MAPA_E_BUDGET;
            res.count = c64;
        } else if (c64 == 0ull) {
            res.status = MAPA_NO_FIT;
        } else {
            const int32_t target = static_cast<int32_t>(static_cast<uint32_t>(k64 >> 32) ^ 0x80000000u);
            const int it = static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(k64 & 0xFFFFFFFFull));
            const uint32_t F = na_free_set(q, n);
            long long twice = 0;
            for (int v = 0; v < n; ++v)
                if ((F >> v) & 1u)
                    for (int c = 0; c < C; ++c) twice += static_cast<long long>(s_wc[c]) * __popc(s_cls[v * C + c] & F);
            const int32_t al = q.policy.alpha, be = q.policy.beta;
            NaState st;
            bool found = false;
            if (na_prefix(pat, s_adj, s_cls, s_wc, C, al, be, F, static_cast<int32_t>(be * (twice / 2)),
                          it / kNaMaxN, it % kNaMaxN, st)) {
                na_walk(pat, s_adj, s_cls, s_wc, C, al, be, st, pat.k == 1 ? 1 : 2, [&](int32_t sc) {
                    found = sc == target;
                    return !found;
                });
            }
            if (!found) {  // cannot happen: the key came from this subtree
                res.status = MAPA_E_STATE;
                out[i] = res;
                continue;
            }
            // AggBW (Eq. 1) and PreservedBW (Eq. 3) of the chosen tuple
            long long agg = 0;
            uint32_t used = 0u;
            for (int v = 0; v < pat.k; ++v) {
                used |= 1u << st.phi[v];
                uint32_t m = pat.back[v];
                while (m) {
                    const int a = __ffs(m) - 1;
                    m &= m - 1u;
                    for (int c = 0; c < C; ++c)
                        if ((s_cls[st.phi[a] * C + c] >> st.phi[v]) & 1u) agg += s_wc[c];
                }
            }
            const uint32_t rem = F & ~used;
            long long ptwice = 0;
            for (int v = 0; v < n; ++v)
                if ((rem >> v) & 1u)
                    for (int c = 0; c < C; ++c) ptwice += static_cast<long long>(s_wc[c]) * __popc(s_cls[v * C + c] & rem);
            res.status = MAPA_OK;
            res.score = target;
            res.agg = static_cast<int32_t>(agg);
            res.pres = static_cast<int32_t>(ptwice / 2);
            res.count = q.policy.mode == MAPA_MODE_BOUNDED ? 0ull : c64;
            for (int j = 0; j < pat.k; ++j) res.verts[j] = static_cast<uint8_t>(st.phi[j]);
        }
        out[i] = res;
    }
}

}  // namespace

int noalloc_decide(const TopoDevice &t, const PatternArgs &pat, int32_t pattern_id, int32_t nreq,
                   const mapa_request *reqs_dev, mapa_result *out_dev, cudaStream_t stream, std::string *err) {
    if (nreq < 0 || nreq > kNaMaxRequests) {
        if (err) *err = "mapa_allocate_batch_noalloc: nreq must be in 0..4096";
        return MAPA_E_RANGE;
    }
    if (t.n > kNaMaxN || t.W != 1) {
        if (err) *err = "mapa_allocate_batch_noalloc: the hardware graph must have at most 32 vertices";
        return MAPA_E_RANGE;
    }
    if (pat.k < 1 || pat.k > kNaMaxK) {
        if (err) *err = "mapa_allocate_batch_noalloc: the pattern must have at most 8 vertices";
        return MAPA_E_RANGE;
    }
    if (nreq == 0) return MAPA_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        if (err) *err = "mapa_allocate_batch_noalloc: no current device";
        return MAPA_E_CUDA;
    }
    void *scratch = nullptr;
    {
        // Set-up, once per device with that device current: resolve the
        // device address of the scratch array (the host-side symbol is only a
        // stand-in and must never be passed to a kernel).
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr) {
                if (err) *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return MAPA_E_CUDA;
            }
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    unsigned char *base = static_cast<unsigned char *>(scratch);
    // keys, counts and tickets must start at zero on every call
    e = cudaMemsetAsync(base, 0, sizeof(unsigned long long) * nreq, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kNaKeyBytes, 0, sizeof(unsigned long long) * nreq, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + 2 * kNaKeyBytes, 0, sizeof(unsigned int) * nreq, stream);
    if (e != cudaSuccess) {
        if (err) *err = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e);
        return MAPA_E_CUDA;
    }
    const long long threads = static_cast<long long>(nreq) * kNaItems;
    const unsigned grid = static_cast<unsigned>((threads + kNaThreads - 1) / kNaThreads);
    k_decide_noalloc<<<grid, kNaThreads, 0, stream>>>(t.args(), pat, pattern_id, t.total_weight, nreq, reqs_dev,
                                                      out_dev, base);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (err) *err = std::string("k_decide_noalloc launch: ") + cudaGetErrorString(e);
        return MAPA_E_CUDA;
    }
    return MAPA_OK;
}

}  // namespace mapa
