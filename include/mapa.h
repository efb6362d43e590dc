/*
 * mapa.h -- C ABI of the GB300 MAPA allocation engine.
 *
 * MAPA (Ranganath et al., "MAPA: Multi-Accelerator Pattern Allocation Policy
 * for Multi-Tenant GPU Servers", SC'21, arXiv 2110.03214) places a job whose
 * GPUs communicate in a known pattern (ring, tree, all-to-all: the
 * application graph of Sec. 3.1) onto the free accelerators of a server whose
 * links are a weighted hardware graph (Sec. 3.2).  This library runs the
 * data-parallel core of that policy on one GPU:
 *
 *   1. enumerate every match of the pattern in the free part of the hardware
 *      graph: injective maps phi: V(P) -> F under which adjacent pattern
 *      vertices land on linked accelerators (Sec. 3.3), counted once per
 *      distinct subgraph (maps modulo the pattern's automorphisms);
 *   2. score each match in int32:  S = alpha * AggBW + beta * PreservedBW,
 *      AggBW = sum of the link weights under the pattern's edges (Eq. 1),
 *      PreservedBW = total link weight among the free accelerators that the
 *      match leaves idle (Eq. 3);
 *   3. pick the largest S; among equal S the lexicographically smallest
 *      (phi(0), ..., phi(k-1)) (Algorithm 1's ">" scan, run in lexicographic
 *      order), and on request commit it to the device-resident occupancy
 *      (state management, Sec. 3.6).
 *
 * alpha = 0, beta = 1 is the paper's Preserve policy for bandwidth-insensitive
 * jobs (Sec. 3.5.2); alpha = 1, beta = 0 is its Greedy comparison policy
 * (Sec. 4, argmax of AggBW).
 *
 * Conventions for every call:
 *   - A negative return value is an error; details in mapa_last_error().
 *     MAPA_NO_FIT is a normal outcome (nothing matched, nothing committed).
 *   - Input arrays belong to the caller and are copied before the call
 *     returns.  Output structs belong to the caller.
 *   - A context owns its device memory, stream, topologies, patterns and
 *     occupancy; mapa_ctx_destroy frees all of it.  One context per host
 *     thread; calls on one context must not overlap.
 *   - All vertex ids are 0-based.  Bitmasks hold vertex v in bit (v % 32) of
 *     32-bit word v / 32.
 */
#ifndef MAPA_H
#define MAPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MAPA_MAX_N 256       /* accelerators in one hardware graph */
#define MAPA_MAX_K 32        /* vertices in one pattern */
#define MAPA_MASK_WORDS 8    /* 256-bit vertex masks */
#define MAPA_MAX_CLASSES 8   /* distinct link weights in one hardware graph */
#define MAPA_MAX_WEIGHT (1 << 20)

typedef struct mapa_ctx_s *mapa_ctx;

enum mapa_status {
    MAPA_OK = 0,
    MAPA_NO_FIT = 1,        /* no match on the free vertices; nothing committed */
    MAPA_INEXACT = 2,       /* MAPA_POLICY_ANYTIME past the work budget: a real match, the best one the
                               search met, not proven to be the argmax; committed like MAPA_OK */
    MAPA_E_INVALID = -1,    /* malformed argument (ids, sizes, graph shape) */
    MAPA_E_RANGE = -2,      /* value outside the supported range (n, k, weights, int32 scores) */
    MAPA_E_NOMEM = -3,      /* device or host allocation failed, or frontier cap too small */
    MAPA_E_CUDA = -4,       /* a CUDA call failed */
    MAPA_E_BUDGET = -5,     /* the request's max_embeddings was exceeded; no decision */
    MAPA_E_TIMEOUT = -6,    /* a bounded device wait gave up */
    MAPA_E_STATE = -7       /* call not valid in the current state (e.g. unknown job id) */
};

/* Pattern shapes for mapa_pattern_builtin (k always counts vertices).
 *   RING:   cycle 0-1-...-(k-1)-0 for k >= 3; k = 2 is one edge; k = 1 one vertex.
 *   TREE:   binary tree in heap order, parent(i) = (i - 1) / 2.
 *   CLIQUE: all pairs (all-to-all).
 *   PATH:   chain 0-1-...-(k-1).
 * Ring and tree are the NCCL communication shapes of Sec. 3.1 (Fig. 5). */
enum mapa_pattern_kind { MAPA_RING = 0, MAPA_TREE = 1, MAPA_CLIQUE = 2, MAPA_PATH = 3 };

enum mapa_mode {
    MAPA_MODE_EXHAUSTIVE = 0, /* enumerate every match (count is exact) */
    MAPA_MODE_BOUNDED = 1     /* branch and bound: the same decision, no count */
};

/* Scoring policy of one request.  S = alpha * AggBW + beta * PreservedBW is
 * computed in int32; the call fails with MAPA_E_RANGE unless
 * (|alpha| + |beta|) * (total link weight of the graph) < 2^31.
 * max_embeddings > 0 bounds the matches a request may enumerate; past it the
 * request ends with MAPA_E_BUDGET and no decision.
 *
 * mode = MAPA_MODE_BOUNDED returns exactly the decision of the exhaustive
 * mode (the same score, AggBW, PreservedBW and tuple, ties included) but
 * skips every partial match whose completions provably score below a match
 * already found; result.count is then 0.  Cut-offs need alpha >= 0 and
 * beta >= 0 (with a negative weight the request is enumerated in full).
 * max_embeddings then bounds the complete matches left to score.
 *
 * flags & MAPA_POLICY_BW_SENSITIVE selects the first branch of Algorithm 1
 * (a bandwidth-sensitive job): the chosen match maximises the Predicted
 * Effective Bandwidth of Eq. 2 (Sec. 3.4.3, coefficients of Table 2) instead
 * of S; alpha and beta are ignored.  Its link counts x, y, z are taken over
 * the images of the pattern edges, a link's type following its weight as a
 * peak bandwidth (Table 1): 50 = double NVLink, 25 or 20 = single NVLink,
 * 12 = PCIe; links of other weights count in none.  Ties go to the
 * lexicographically smallest tuple.  result.score is then round(1000 *
 * EffBW) (milli-GB/s; a value exactly on a half milli-GB/s, which the
 * three-decimal coefficients allow, may round either way); agg, pres and
 * count keep their meaning.  Patterns
 * with more than 63 edges fail with MAPA_E_RANGE.  The bounded mode makes
 * no cut-offs for such a request. */
enum mapa_policy_flags { MAPA_POLICY_BW_SENSITIVE = 1u, MAPA_POLICY_ANYTIME = 2u };

/* flags & MAPA_POLICY_ANYTIME (with alpha, beta >= 0, not with
 * MAPA_POLICY_BW_SENSITIVE, in either mode) changes what a request past the
 * context's work budget (mapa_ctx_set_work_budget) returns: instead of
 * MAPA_E_BUDGET, the best match of the request's seed dive (in bounded mode
 * the dive that seeds its cut-offs; in exhaustive mode a dive that depends
 * only on the request, run after the enumeration for the requests past the
 * budget, or beside it on a side stream when the group is produced in
 * chunks, its match then used only if the request passes the budget), with status
 * MAPA_INEXACT, its
 * score, AggBW and PreservedBW recomputed from the tuple, count 0.  For such
 * a request the dive runs up to 256 k steps and is guided towards a match
 * rather than a high score: candidates that violate two necessary conditions
 * of any match are skipped (the image of pattern vertex j lies within its
 * pattern distance from phi(0) in the free graph, and has at least as many
 * free neighbours as j has later pattern neighbours), the child with the
 * most free neighbours is taken first, at most 1024 steps are spent below
 * one phi(0) before the next is tried, and once a match is found the dive
 * continues best score first for at most 256 more steps.  The fallback
 * depends on the request alone,
 * so it is the same on every run and in every batch.  It is committed like
 * MAPA_OK (mapa_allocate, sequential batches, the served loop).  With no
 * match from the dive the result is MAPA_E_BUDGET, or MAPA_NO_FIT when the
 * dive finished its whole search (which then proves that no match
 * exists).  A request that finishes
 * within the budget gets its exact result (MAPA_OK or MAPA_NO_FIT) as
 * without the flag.  The paper's policy is exact; this is a bounded-cost
 * fallback for free sets too large to enumerate. */

typedef struct {
    int32_t alpha;
    int32_t beta;
    int32_t mode;
    uint32_t flags; /* mapa_policy_flags */
    uint64_t max_embeddings;
} mapa_policy; /* 24 bytes */

/* One request of a batch (64 bytes, no pointers, so an array of them can live
 * in host or device memory).  busy: vertices unavailable to this request
 * (see the flags of mapa_allocate_batch for how it combines with the
 * device occupancy).
 * root_lo, root_hi: with root_hi > 0, only the matches whose image of
 * pattern vertex 0 lies in [root_lo, root_hi) are enumerated -- one share
 * of a request split by the value of phi(0), e.g. across GPUs.  Each match
 * is counted in exactly one share (the lexicographically smallest map of
 * its class, the one enumerated, has one phi(0)), so mapa_result_merge of
 * the shares of a partition of [0, n) gives the unsplit result.  root_hi = 0
 * (the default) enumerates everything.  The allocation-free call refuses
 * split requests (MAPA_E_INVALID). */
typedef struct {
    int32_t pattern_id;
    uint16_t root_lo;
    uint16_t root_hi;
    mapa_policy policy;
    uint32_t busy[MAPA_MASK_WORDS];
} mapa_request;

/* Decision for one request (80 bytes).
 *   status: MAPA_OK, MAPA_NO_FIT or a negative error for this request.
 *   score, agg, pres: S, AggBW (Eq. 1) and PreservedBW (Eq. 3) of the chosen match.
 *   count: matches found, once per distinct subgraph (maps / |Aut(P)|);
 *          0 for MAPA_MODE_BOUNDED.
 *   job_id: id of the committed allocation (>= 1), or 0 when nothing was committed.
 *   verts[i] = phi(i) for i < k. */
typedef struct {
    int32_t status;
    int32_t score;
    int32_t agg;
    int32_t pres;
    uint64_t count;
    int64_t job_id;
    int32_t k;
    int32_t reserved;
    uint8_t verts[MAPA_MAX_K];
    uint64_t reserved2;
} mapa_result;

/* ---- context ----------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  frontier_mem_cap bounds the
 * device memory used for the partial-match frontier of one pattern group,
 * in bytes (0 = 4 GiB); the enumeration proceeds in chunks so any request
 * fits, only slower.  The pattern groups of an independent batch run
 * concurrently, up to four at a time, each with its own frontier, so a
 * context may hold up to four times this amount.
 * Returns MAPA_E_CUDA if the device cannot be used. */
int mapa_ctx_create(int device, uint64_t frontier_mem_cap, mapa_ctx *out);

/* Frees every resource of the context (NULL is ignored). */
void mapa_ctx_destroy(mapa_ctx ctx);

/* Work of this context is issued on `cuda_stream` (a cudaStream_t; NULL =
 * the context's own stream).  The stream must outlive its use. */
int mapa_ctx_set_stream(mapa_ctx ctx, void *cuda_stream);

/* Message of the last failed call on ctx (never NULL; "" if none).  Valid
 * until the next call on ctx.  mapa_last_error(NULL) reports failures of
 * mapa_ctx_create. */
const char *mapa_last_error(mapa_ctx ctx);

/* ---- inputs ------------------------------------------------------------ */

/* Loads a hardware graph (Sec. 3.2): n accelerators, m undirected links
 * (u[i], v[i]) with bandwidth weight w[i].  fill_weight > 0 gives every
 * unlinked pair that weight (the paper's "fully connected through PCIe",
 * fill 12 GB/s); 0 keeps only the listed links.  Requires 1 <= n <= 256,
 * no self-loops or duplicate links, 0 < w < 2^20, at most 8 distinct
 * weights.  Its occupancy starts all free.  *topo_id receives the id. */
int mapa_topology_load(mapa_ctx ctx, int32_t n, int32_t m, const int32_t *u, const int32_t *v,
                       const int32_t *w, int32_t fill_weight, int32_t *topo_id);

/* Loads an application graph (Sec. 3.1): k vertices, m undirected edges
 * (a[i], b[i]).  Requires 1 <= k <= 32, no self-loops or duplicate edges.
 * The host computes its automorphism group and symmetry-breaking order
 * constraints here.  *pattern_id receives the id. */
int mapa_pattern_load(mapa_ctx ctx, int32_t k, int32_t m, const int32_t *a, const int32_t *b,
                      int32_t *pattern_id);

/* Loads one of the built-in shapes (enum mapa_pattern_kind) with k vertices. */
int mapa_pattern_builtin(mapa_ctx ctx, int32_t kind, int32_t k, int32_t *pattern_id);

/* ---- allocation -------------------------------------------------------- */

/* Allocates one job against the topology's current occupancy: enumerate,
 * score, pick (Sec. 3.3-3.5), and on MAPA_OK mark the chosen vertices busy
 * under a new job id (Sec. 3.6).  policy NULL = {alpha 1, beta 1}.
 * Returns MAPA_OK, MAPA_NO_FIT or an error; *out is always written. */
int mapa_allocate(mapa_ctx ctx, int32_t topo_id, int32_t pattern_id, const mapa_policy *policy,
                  mapa_result *out);

/* Returns the vertices of a committed job to the free pool (Sec. 3.6).
 * MAPA_E_STATE if job_id is not a live job of this topology. */
int mapa_release(mapa_ctx ctx, int32_t topo_id, int64_t job_id);

/* Flags of mapa_allocate_batch. */
#define MAPA_BATCH_INDEPENDENT 0u /* each request sees only its own busy mask; nothing is committed */
#define MAPA_BATCH_SEQUENTIAL 1u  /* in array order: busy = occupancy | request mask; OK results commit */
#define MAPA_BATCH_DEVICE 2u      /* reqs and out are device pointers (else host pointers) */

/* Decides nreq requests in one call.  With MAPA_BATCH_INDEPENDENT the
 * requests are grouped by pattern and enumerated together (frontiers of
 * many requests share each launch); results are independent of the batch's
 * composition and order.  With MAPA_BATCH_SEQUENTIAL each request sees the
 * commits of the ones before it.  out[i] answers reqs[i].  Returns MAPA_OK
 * when every request was processed (per-request outcomes are in
 * out[i].status), or a negative error for the call as a whole. */
int mapa_allocate_batch(mapa_ctx ctx, int32_t topo_id, int32_t nreq, const mapa_request *reqs,
                        mapa_result *out, uint32_t flags);

/* Host-only reduction of the shares of one split request (root_lo/root_hi
 * of mapa_request; no GPU needed): the best share by score, then the
 * lexicographically smallest tuple (the same compare the enumeration uses
 * within a share), with count the sum of the shares' counts.  A share with
 * a negative status makes that status the result (the first in parts
 * order); otherwise the result is MAPA_INEXACT if any share is, else
 * MAPA_OK if any share found a match, else MAPA_NO_FIT.  out may alias no
 * element of parts.  Not in the paper: the exchange step of splitting one
 * request across GPUs (one result per share, gathered and reduced). */
int mapa_result_merge(int32_t nparts, const mapa_result *parts, mapa_result *out);

/* ---- serving ------------------------------------------------------------ */

/* A served allocation loop on one topology (continuous batching).  A worker
 * thread owned by the server admits every request that has arrived, up to
 * max_batch, decides them together in one batched pass against a snapshot of
 * the device-resident occupancy, then commits the decisions on the device in
 * arrival order (Sec. 3.6 state management; FIFO order of Sec. 4): the
 * longest prefix of decisions that do not overlap one another is committed,
 * and the requests from the first overlap on are decided again in the same
 * round, one after another against the live occupancy (a device-side chain:
 * each is committed before the next is decided), so no request is decided
 * more than twice.  The chain runs in segments of n/4 requests (1 to 8 for a
 * round of n), and each segment's decisions are published when it ends.
 * Admission: the window doubles after a round whose parallel decisions all
 * committed and shrinks after one that met an overlap or a wait (at most
 * max_batch); the parallel pass runs for rounds of at least 16 requests that
 * arrived faster than the chain decides (their mean arrival gap below the
 * chain's measured time per decision); after a parallel pass of which fewer
 * than half committed, the next large rounds (1, 2, 4 ... 64 of them) skip
 * it and go straight to the chain, up to 64 requests each.  Under a work budget B
 * (mapa_ctx_set_work_budget) admission also keeps to the frontier memory of
 * the context's concurrent groups (4 x frontier_mem_cap): a round admits
 * requests while the sum of their largest frontiers, (1 + the topology's
 * largest degree) x B entries of 8 + 4 W + 4 ceil(k/4) bytes each, fits (the
 * first request of a round always enters).  Lifetimes are kept on the device: a commit
 * stamps its vertices with the device clock plus the job's lifetime, and
 * after every chain decision the vertices whose time has passed are freed
 * before the next one, so a job holds its accelerators for its lifetime
 * whatever the round length.  DEPART events return a job's vertices before
 * later arrivals are decided.  Requests that arrive while a round's chain
 * runs join its end between segments (in arrival order, up to the round's
 * admission limit and 64 requests unless the round began larger).
 * max_batch = 1 gives the plain per-request form (one request per round). */

enum mapa_event_kind { MAPA_EVENT_ARRIVE = 0, MAPA_EVENT_DEPART = 1 };

/* One event of a served trace (64 bytes).
 *   at_ns:       arrival time in ns after mapa_serve_open (0 = immediately).
 *                Events of one submit call must have non-decreasing at_ns.
 *   ARRIVE:      pattern_id, policy; lifetime_ns > 0 makes the server release
 *                the job lifetime_ns after it is committed, by the device
 *                clock (0 = keep until a DEPART event names it).
 *   DEPART:      job_id of a committed job. */
typedef struct {
    int64_t request_id;
    int64_t at_ns;
    int64_t lifetime_ns;
    int64_t job_id;
    int32_t kind;
    int32_t pattern_id;
    mapa_policy policy;
} mapa_event;

/* A finished event (144 bytes).  For ARRIVE, result is the decision (job_id
 * set when committed).  For DEPART, result.status is MAPA_OK or MAPA_E_STATE
 * (unknown job).  snapshot is the occupancy the decision was taken against
 * (deciding the request alone with that busy mask gives the same result);
 * arrive_ns / done_ns are times after mapa_serve_open; rounds counts the
 * decisions it took (1, or 2 when it lost a conflict in its round). */
typedef struct {
    int64_t request_id;
    int64_t arrive_ns;
    int64_t done_ns;
    int32_t kind;
    int32_t rounds;
    uint32_t snapshot[MAPA_MASK_WORDS];
    mapa_result result;
} mapa_served;

typedef struct mapa_server_s *mapa_server;

/* Flags of mapa_serve_open.  By default the queue is FIFO as in the paper's
 * scheduler (Sec. 4): a request that does not fit waits at the head of the
 * queue, with everything behind it, until a departure frees accelerators;
 * it is answered MAPA_NO_FIT only when nothing the server holds will ever be
 * released.  MAPA_SERVE_REJECT answers MAPA_NO_FIT at once instead. */
#define MAPA_SERVE_REJECT 1u

/* Opens a server on topo_id (max_batch >= 1 requests per round).  The
 * server drives ctx's stream from its own thread: make no other call on ctx
 * until mapa_serve_close returns. */
int mapa_serve_open(mapa_ctx ctx, int32_t topo_id, int32_t max_batch, uint32_t flags, mapa_server *out);

/* Queues n events (copied).  Thread safe. */
int mapa_serve_submit(mapa_server srv, const mapa_event *events, int32_t n);

/* Moves up to max finished events into out; *got receives the number.
 * timeout_ms > 0 waits up to that long for at least one. */
int mapa_serve_poll(mapa_server srv, mapa_served *out, int32_t max, int32_t *got, int32_t timeout_ms);

/* Blocks until every submitted event has finished (timeout_ms <= 0: no limit);
 * MAPA_E_TIMEOUT if the limit passes first. */
int mapa_serve_drain(mapa_server srv, int32_t timeout_ms);

/* Counters of the server: rounds run, decisions, decisions redone after a conflict. */
int mapa_serve_counters(mapa_server srv, uint64_t *rounds, uint64_t *decisions, uint64_t *conflicts);

/* Stops the worker (pending events are dropped) and frees the server.  The
 * first error the worker met, if any, is returned here. */
int mapa_serve_close(mapa_server srv);

/* ---- allocation-free decisions ------------------------------------------ */

/* Limits of mapa_allocate_batch_noalloc. */
#define MAPA_NOALLOC_MAX_REQUESTS 4096
#define MAPA_NOALLOC_MAX_N 32
#define MAPA_NOALLOC_MAX_K 8

/* Decides up to 4096 independent requests without allocating any memory.
 * (The paper has no counterpart; this exists for callers that must not
 * allocate.)  Some callers cannot call cudaMalloc: a scheduler loop running
 * while a CUDA graph is being captured on its thread, a hook running inside
 * another framework's allocator, or a process whose device memory a serving
 * runtime has fully reserved.  This call launches one kernel whose scratch
 * (per-request argmax keys, match counts and completion tickets) is a fixed
 * 80 KiB device array compiled into the library; every GPU that
 * loads the library holds it until the process exits.  Nothing is allocated,
 * freed or committed.
 *
 * reqs_dev and out_dev are device pointers to nreq entries; every request
 * must carry pattern_id and is decided on its own busy mask exactly as
 * mapa_allocate_batch with MAPA_BATCH_INDEPENDENT decides it (same status,
 * score, AggBW, PreservedBW, count and tuple; count is 0 in bounded mode).
 * A request with another pattern id, a bandwidth-sensitive one, or a
 * bounded-mode one with max_embeddings > 0 gets MAPA_E_INVALID (the batched
 * call's bounded mode applies that budget to the matches left after its
 * cut-offs, which this kernel does not make).  The context's work budget
 * (mapa_ctx_set_work_budget) does not apply here.
 * Limits: nreq <= 4096, the topology has at most 32 vertices, the pattern at
 * most 8; beyond them the call returns MAPA_E_RANGE and launches nothing.
 * The first call on a device resolves the scratch array's device address
 * (cudaGetSymbolAddress with that device current); make that first call
 * before any stream capture.  Work is issued on the context's stream and the
 * call returns without waiting for it.  All calls on a device share the one
 * scratch array and reset it at their start: calls whose kernels overlap on
 * the GPU (other streams, other contexts, other host threads) race and
 * corrupt each other's results -- serialise them. */
int mapa_allocate_batch_noalloc(mapa_ctx ctx, int32_t topo_id, int32_t pattern_id, int32_t nreq,
                                const mapa_request *reqs_dev, mapa_result *out_dev);

/* ---- introspection ----------------------------------------------------- */

/* Counters of one context since creation or the last mapa_stats_reset. */
typedef struct {
    uint64_t kernel_launches;  /* kernels this context launched */
    uint64_t tail_launches;    /* launches of the fused last-level kernel */
    double tail_ms;            /* their device time (CUDA events; only while timing is on) */
    uint64_t tail_parents;     /* stored partial matches they expanded */
    uint64_t tail_nodes;       /* first-tail-level nodes (two fused levels) */
    uint64_t tail_leaves;      /* complete matches they scored */
    uint64_t tail_int_ops;     /* algorithmic integer operations of those launches */
    uint64_t spill_entries;    /* partial matches written to frontiers */
    uint64_t spill_bytes;      /* frontier bytes written plus read back */
    uint64_t requests;         /* requests decided */
    uint64_t embeddings;       /* matches scored, once per distinct subgraph */
    uint64_t expand_launches;  /* launches of the level-expansion kernels (one per stored level or chunk) */
    double expand_ms;          /* their device time (CUDA events; only while timing is on) */
    uint64_t expand_bytes;     /* their algorithmic frontier bytes: parents read once plus children written */
} mapa_stats;

/* Autotuner of the batched path: for every pattern present in the host
 * batch reqs[0..nreq), times each fused tail depth (1, 2 or 3 last pattern
 * vertices scored in registers instead of written to a frontier) on that
 * pattern's requests and keeps the fastest for (topo_id, pattern) in the
 * context.  Results never change with the depth, only the time does.
 * chosen must hold one entry per loaded pattern and receives the depth
 * chosen for each (0 for patterns absent from the batch).  Nothing is
 * committed. */
int mapa_autotune(mapa_ctx ctx, int32_t topo_id, int32_t nreq, const mapa_request *reqs, int32_t *chosen);

/* The autotuner also times, at the chosen depth, limits of 4M and 1M entries
 * on a stored level (default: as many as the frontier cap allows) and keeps
 * one that is clearly faster: on frontiers that do not fit, smaller levels
 * are produced in chunks that stay in L2 between the count and write passes.
 * Results never change with the limit.  *entries receives the limit kept for
 * (topo_id, pattern_id), 0 for none. */
int mapa_autotune_level_limit(mapa_ctx ctx, int32_t topo_id, int32_t pattern_id, uint64_t *entries);

/* Copies the counters into *out. */
int mapa_stats_get(mapa_ctx ctx, mapa_stats *out);

/* Zeroes the counters. */
int mapa_stats_reset(mapa_ctx ctx);

/* on != 0: bracket every fused last-level launch and every level-expansion
 * launch with CUDA events on the stream it runs on and add their device
 * times to tail_ms and expand_ms (request groups then run one after another,
 * and captured graphs are not used). */
int mapa_ctx_set_timing(mapa_ctx ctx, int on);

/* Work budget of every later decision on ctx: a request whose enumeration
 * stores more than max_partials partial matches (entries of the stored
 * levels below the fused tail, summed over levels) stops being enumerated
 * and ends with MAPA_E_BUDGET, count 0 and no decision; 0 (the default)
 * sets no limit.  Unlike max_embeddings, which is checked against the count
 * after a full enumeration, this bounds the work itself: every partial
 * match of a request past its budget is cut at once.  The check runs
 * between level launches (and between chunks of a level that does not fit
 * the frontier), and a request is stopped exactly when the partial matches
 * its full enumeration would store exceed the budget, so whether it ends
 * with MAPA_E_BUDGET depends only on the request, the budget and its
 * pattern's fused tail depth (which decides which levels are stored; see
 * mapa_autotune), never on timing, the batch or the frontier cap.  It
 * applies to batches, mapa_allocate and served decisions alike; a request
 * that finishes within it gets exactly its unbudgeted result.  Not part of
 * the paper: it keeps decisions on large free sets (where the number of
 * matches grows combinatorially, Sec. 5.4) within a stated cost. */
int mapa_ctx_set_work_budget(mapa_ctx ctx, uint64_t max_partials);

/* Copies the topology's occupancy (busy mask, 8 words) to host memory. */
int mapa_occupancy_get(mapa_ctx ctx, int32_t topo_id, uint32_t *busy_out);

/* Host-only pattern analysis (no GPU, no context): |Aut(P)| and, per pattern
 * vertex i, back_masks[i] = earlier neighbours of i and lo_masks[i] = the
 * earlier vertices j with the constraint phi(j) < phi(i).  These constraints
 * keep exactly one map per automorphism class, the lexicographically
 * smallest.  Arrays hold k entries.  Returns MAPA_OK or an error. */
int mapa_pattern_analyze(int32_t k, int32_t m, const int32_t *a, const int32_t *b, uint64_t *aut_order,
                         uint32_t *back_masks, uint32_t *lo_masks);

/* ---- simulator (Sec. 6) ---------------------------------------------------- */

/* Allocation policies of the simulator (Sec. 5 and Sec. 6).
 *   BASELINE: the lowest free accelerator ids, pattern vertex i on the i-th
 *             (how container runtimes allocate); no matching.
 *   GREEDY:   the match with the largest AggBW (alpha 1, beta 0).
 *   PRESERVE: Algorithm 1 -- largest Predicted EffBW for a bandwidth-
 *             sensitive job, largest PreservedBW (alpha 0, beta 1) otherwise.
 *   EFFBW:    largest Predicted EffBW for every job. */
enum mapa_sim_policy { MAPA_SIM_BASELINE = 0, MAPA_SIM_GREEDY = 1, MAPA_SIM_PRESERVE = 2, MAPA_SIM_EFFBW = 3 };

/* One row of a job file (32 bytes).  Jobs enter the FIFO queue at `arrive`
 * (cycles, non-decreasing along the file) and run for `duration` cycles
 * once allocated. */
typedef struct {
    int64_t job_id;
    int64_t arrive;
    int64_t duration;
    int32_t pattern_id;
    int32_t sensitive; /* 1 = bandwidth-sensitive */
} mapa_sim_job;

/* The logger's record of one job (80 bytes).  status MAPA_OK, or MAPA_NO_FIT
 * when the job cannot be placed even on the idle machine (then start = end =
 * the cycle it reached the queue head).  effbw_milli = round(1000 * Eq. 2)
 * over the link types of the images of the pattern edges; agg = AggBW (Eq.
 * 1); pres = PreservedBW (Eq. 3) of the free accelerators left at
 * allocation time; verts[i] = the accelerator of pattern vertex i. */
typedef struct {
    int64_t job_id;
    int64_t start;
    int64_t end;
    int32_t status;
    int32_t effbw_milli;
    int32_t agg;
    int32_t pres;
    int32_t k;
    int32_t reserved;
    uint8_t verts[MAPA_MAX_K];
} mapa_sim_record;

/* Runs a job file through the simulator of Sec. 6 on topology topo_id (which
 * must have at most 256 accelerators): a dispatcher puts the jobs in a FIFO
 * queue; a cycle-based engine, at each cycle where something happens, first
 * frees the accelerators of the jobs that finished, then allocates the queue
 * head while it fits under `policy` (a head that does not fit waits for a
 * job to finish: no reordering); every decision other than BASELINE is taken
 * by the GPU path (one request against the current occupancy).  The
 * topology's device occupancy is neither read nor changed.  out[i] answers
 * jobs[i].  Returns MAPA_OK, or an error for the call as a whole
 * (MAPA_E_INVALID for unknown ids or arrivals out of order). */
int mapa_simulate(mapa_ctx ctx, int32_t topo_id, int32_t policy, int32_t njobs, const mapa_sim_job *jobs,
                  mapa_sim_record *out);

/* Host-only: the Predicted Effective Bandwidth (Eq. 2, coefficients of
 * Table 2) of an allocation with x double NVLinks, y single NVLinks and z
 * PCIe links, in GB/s, as the library ranks bandwidth-sensitive matches.
 * Returns MAPA_E_RANGE unless 0 <= x, y, z <= 63. */
int mapa_effbw_predict(int32_t x, int32_t y, int32_t z, double *out);

/* Measured integer issue rate of the device (no counterpart in the paper;
 * the ceiling for the fused tail's integer throughput): a kernel of
 * independent dependent chains of 32-bit logic (lop3) and add instructions
 * (kind 0), or logic, population count and add in equal numbers (kind 1,
 * about the score increment's share of population counts), on every SM.
 * *ops_per_s receives the best of three timed launches, in operations per
 * second.  Allocates a 4-byte scratch word for the call. */
int mapa_measure_int_peak(mapa_ctx ctx, int32_t kind, double *ops_per_s);

/* Library version string. */
const char *mapa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MAPA_H */
