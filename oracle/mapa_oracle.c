/*
 * MAPA allocation oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  The product (the CUDA path behind include/mapa.h) never
 * links, loads or calls it, and shares no code, header or table with it.
 *
 * What it computes: a plain, slow restatement of the allocation problem of
 * MAPA (Ranganath et al., SC'21, arXiv 2110.03214), Sec. 3.2-3.5:
 *
 *   G  hardware graph, symmetric integer weights w[u][v] (0 = no link).  With
 *      fill > 0 every non-adjacent pair of distinct vertices gets weight
 *      `fill` (Sec. 3.2: the graph is taken as fully connected through PCIe).
 *   P  application (pattern) graph with k vertices (Sec. 3.1).
 *   F  free vertices (not busy).  Busy vertices are removed from G by the
 *      state management of Sec. 3.6.
 *   match: an injective phi: V(P) -> F with w[phi a][phi b] > 0 for every
 *      pattern edge (a, b): a one-to-one mapping under which adjacent pattern
 *      vertices stay adjacent (Sec. 3.3).  Non-induced.
 *   agg(phi)  = sum over pattern edges (a,b) of w[phi a][phi b]   (Eq. 1)
 *   pres(phi) = total weight of the subgraph induced by F minus phi(V(P))
 *                                                                  (Eq. 3)
 *   score     = alpha * agg + beta * pres, in 64-bit integers.
 *   decision  = the match with the largest score; among equal scores the
 *               lexicographically smallest (phi(0), ..., phi(k-1)).  This is
 *               Algorithm 1's strict ">" scan run over matches enumerated in
 *               lexicographic order, with the first match as the initial
 *               incumbent.
 *   count     = matches / |Aut(P)|: matches counted once per distinct
 *               subgraph (the graph-mining system of Sec. 3.3 reports each
 *               match once; Aut(P) acts freely on injective maps).
 *
 * Algorithms, all deliberately plain:
 *   - matches: recursive backtracking over pattern vertices 0..k-1 in id
 *     order, trying every free unused hardware vertex in increasing order,
 *     checking every pattern edge to an earlier vertex.  Boolean arrays only,
 *     no bitsets, no symmetry breaking, no incremental scoring.
 *   - pres: recomputed from its definition for every match (double loop over
 *     the remaining free vertices).
 *   - |Aut(P)|: backtracking over vertex bijections that preserve adjacency
 *     in both directions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_MAX_N 256
#define OR_MAX_K 32

enum {
    OR_OK = 0,
    OR_NO_MATCH = 1,
    OR_INVALID = -1,
    OR_NOT_DIVISIBLE = -2,
    OR_BUDGET = -5,
};

typedef struct {
    int32_t status;
    int32_t k;
    int64_t score;
    int64_t agg;
    int64_t pres;
    uint64_t maps;    /* adjacency-preserving injective maps found */
    uint64_t aut;     /* |Aut(P)| */
    uint64_t classes; /* maps / aut */
    uint8_t tuple[OR_MAX_K];
} oracle_result;

/* ------------------------------------------------------------------ */
/* Hardware graph (Sec. 3.2)                                           */

int oracle_weight_matrix(int32_t n, int32_t m, const int32_t *u, const int32_t *v, const int32_t *w,
                         int32_t fill, int32_t *wmat)
{
    if (n < 1 || n > OR_MAX_N || m < 0) return OR_INVALID;
    memset(wmat, 0, sizeof(int32_t) * (size_t)n * (size_t)n);
    for (int32_t e = 0; e < m; ++e) {
        int32_t a = u[e], b = v[e];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b || w[e] <= 0) return OR_INVALID;
        if (wmat[a * n + b] != 0) return OR_INVALID; /* duplicate link */
        wmat[a * n + b] = w[e];
        wmat[b * n + a] = w[e];
    }
    if (fill > 0) {
        for (int32_t a = 0; a < n; ++a)
            for (int32_t b = 0; b < n; ++b)
                if (a != b && wmat[a * n + b] == 0) wmat[a * n + b] = fill;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Pattern graph (Sec. 3.1) and its automorphisms                      */

static int build_pattern(int32_t k, int32_t m, const int32_t *pa, const int32_t *pb,
                         uint8_t padj[OR_MAX_K][OR_MAX_K])
{
    if (k < 1 || k > OR_MAX_K || m < 0) return OR_INVALID;
    memset(padj, 0, OR_MAX_K * OR_MAX_K);
    for (int32_t e = 0; e < m; ++e) {
        int32_t a = pa[e], b = pb[e];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return OR_INVALID;
        if (padj[a][b]) return OR_INVALID;
        padj[a][b] = 1;
        padj[b][a] = 1;
    }
    return OR_OK;
}

typedef struct {
    int32_t k;
    uint8_t (*padj)[OR_MAX_K];
    int32_t sigma[OR_MAX_K];
    uint8_t taken[OR_MAX_K];
    uint64_t count;
} aut_state;

static void aut_search(aut_state *s, int32_t i)
{
    if (i == s->k) {
        s->count += 1;
        return;
    }
    for (int32_t j = 0; j < s->k; ++j) {
        if (s->taken[j]) continue;
        int ok = 1;
        for (int32_t a = 0; a < i && ok; ++a)
            if (s->padj[a][i] != s->padj[s->sigma[a]][j]) ok = 0;
        if (!ok) continue;
        s->taken[j] = 1;
        s->sigma[i] = j;
        aut_search(s, i + 1);
        s->taken[j] = 0;
    }
}

uint64_t oracle_aut_count(int32_t k, int32_t m, const int32_t *pa, const int32_t *pb)
{
    uint8_t padj[OR_MAX_K][OR_MAX_K];
    if (build_pattern(k, m, pa, pb, padj) != OR_OK) return 0;
    aut_state s;
    memset(&s, 0, sizeof(s));
    s.k = k;
    s.padj = padj;
    aut_search(&s, 0);
    return s.count;
}

/* ------------------------------------------------------------------ */
/* Scores of one complete map (Eq. 1 and Eq. 3)                        */

static int64_t aggregated_bw(int32_t n, const int32_t *wmat, int32_t m, const int32_t *pa, const int32_t *pb,
                             const int32_t *phi)
{
    int64_t s = 0;
    for (int32_t e = 0; e < m; ++e) s += wmat[phi[pa[e]] * n + phi[pb[e]]];
    return s;
}

static int64_t preserved_bw(int32_t n, const int32_t *wmat, const uint8_t *free_v, int32_t k, const int32_t *phi)
{
    uint8_t remain[OR_MAX_N];
    for (int32_t v = 0; v < n; ++v) remain[v] = free_v[v];
    for (int32_t i = 0; i < k; ++i) remain[phi[i]] = 0;
    int64_t s = 0;
    for (int32_t a = 0; a < n; ++a) {
        if (!remain[a]) continue;
        for (int32_t b = a + 1; b < n; ++b)
            if (remain[b]) s += wmat[a * n + b];
    }
    return s;
}

/* Checks that `tuple` is a match on the free vertices and scores it.
 * Returns OR_OK, OR_NO_MATCH (not a match) or OR_INVALID. */
int oracle_score_tuple(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m,
                       const int32_t *pa, const int32_t *pb, int64_t alpha, int64_t beta, const uint8_t *tuple,
                       int64_t *agg_out, int64_t *pres_out, int64_t *score_out)
{
    uint8_t padj[OR_MAX_K][OR_MAX_K];
    if (n < 1 || n > OR_MAX_N || build_pattern(k, m, pa, pb, padj) != OR_OK) return OR_INVALID;
    uint8_t free_v[OR_MAX_N], seen[OR_MAX_N];
    int32_t phi[OR_MAX_K];
    for (int32_t v = 0; v < n; ++v) {
        free_v[v] = busy[v] ? 0 : 1;
        seen[v] = 0;
    }
    for (int32_t i = 0; i < k; ++i) {
        phi[i] = tuple[i];
        if (phi[i] >= n || !free_v[phi[i]] || seen[phi[i]]) return OR_NO_MATCH;
        seen[phi[i]] = 1;
    }
    for (int32_t e = 0; e < m; ++e)
        if (wmat[phi[pa[e]] * n + phi[pb[e]]] <= 0) return OR_NO_MATCH;
    int64_t agg = aggregated_bw(n, wmat, m, pa, pb, phi);
    int64_t pres = preserved_bw(n, wmat, free_v, k, phi);
    *agg_out = agg;
    *pres_out = pres;
    *score_out = alpha * agg + beta * pres;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Enumeration of all matches and the argmax (Sec. 3.3-3.5, Alg. 1)    */

typedef struct {
    int32_t n;
    const int32_t *wmat;
    uint8_t free_v[OR_MAX_N];
    uint8_t used[OR_MAX_N];
    int32_t k, m;
    const int32_t *pa, *pb;
    uint8_t (*padj)[OR_MAX_K];
    int64_t alpha, beta;
    uint64_t max_maps;
    int32_t phi[OR_MAX_K];
    uint64_t maps;
    int have_best;
    int64_t best_score, best_agg, best_pres;
    int32_t best_phi[OR_MAX_K];
    int aborted;
    uint64_t max_nodes, nodes; /* search-node cap of oracle_decide_capped (0 = none) */
    int32_t root_lo, root_hi;  /* phi(0) in [root_lo, root_hi) (oracle_decide_rooted) */
} match_state;

static void visit_match(match_state *s)
{
    s->maps += 1;
    if (s->max_maps && s->maps > s->max_maps) {
        s->aborted = 1;
        return;
    }
    int64_t agg = aggregated_bw(s->n, s->wmat, s->m, s->pa, s->pb, s->phi);
    int64_t pres = preserved_bw(s->n, s->wmat, s->free_v, s->k, s->phi);
    int64_t score = s->alpha * agg + s->beta * pres;
    /* Strict ">" over lexicographically increasing matches: the first
     * maximum wins, i.e. the lexicographically smallest tuple. */
    if (!s->have_best || score > s->best_score) {
        s->have_best = 1;
        s->best_score = score;
        s->best_agg = agg;
        s->best_pres = pres;
        memcpy(s->best_phi, s->phi, sizeof(int32_t) * (size_t)s->k);
    }
}

static void extend(match_state *s, int32_t i)
{
    if (s->aborted) return;
    s->nodes += 1;
    if (s->max_nodes && s->nodes > s->max_nodes) {
        s->aborted = 1;
        return;
    }
    if (i == s->k) {
        visit_match(s);
        return;
    }
    for (int32_t x = 0; x < s->n; ++x) {
        if (!s->free_v[x] || s->used[x]) continue;
        if (i == 0 && (x < s->root_lo || x >= s->root_hi)) continue;
        int ok = 1;
        for (int32_t a = 0; a < i && ok; ++a)
            if (s->padj[a][i] && s->wmat[s->phi[a] * s->n + x] <= 0) ok = 0;
        if (!ok) continue;
        s->used[x] = 1;
        s->phi[i] = x;
        extend(s, i + 1);
        s->used[x] = 0;
        if (s->aborted) return;
    }
}

int oracle_decide_capped(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m,
                         const int32_t *pa, const int32_t *pb, int64_t alpha, int64_t beta, uint64_t max_maps,
                         uint64_t max_nodes, oracle_result *out);

int oracle_decide(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m, const int32_t *pa,
                  const int32_t *pb, int64_t alpha, int64_t beta, uint64_t max_maps, oracle_result *out)
{
    return oracle_decide_capped(n, wmat, busy, k, m, pa, pb, alpha, beta, max_maps, 0, out);
}

/* oracle_decide with a cap on the search nodes (partial maps visited, the
 * root and the matches included) as well: past either cap the result is
 * OR_BUDGET.  The cap only stops the search early; it changes nothing that
 * is computed. */
int oracle_decide_capped(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m,
                         const int32_t *pa, const int32_t *pb, int64_t alpha, int64_t beta, uint64_t max_maps,
                         uint64_t max_nodes, oracle_result *out)
{
    memset(out, 0, sizeof(*out));
    out->k = k;
    uint8_t padj[OR_MAX_K][OR_MAX_K];
    if (n < 1 || n > OR_MAX_N || build_pattern(k, m, pa, pb, padj) != OR_OK) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    match_state *s = (match_state *)calloc(1, sizeof(match_state));
    if (!s) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    s->n = n;
    s->wmat = wmat;
    for (int32_t v = 0; v < n; ++v) s->free_v[v] = busy[v] ? 0 : 1;
    s->k = k;
    s->m = m;
    s->pa = pa;
    s->pb = pb;
    s->padj = padj;
    s->alpha = alpha;
    s->beta = beta;
    s->max_maps = max_maps;
    s->max_nodes = max_nodes;
    s->root_lo = 0;
    s->root_hi = n;
    extend(s, 0);

    out->maps = s->maps;
    /* |Aut(P)| only when there is something to divide (k! for a clique). */
    if (s->have_best && !s->aborted) out->aut = oracle_aut_count(k, m, pa, pb);
    if (s->aborted) {
        out->status = OR_BUDGET;
    } else if (!s->have_best) {
        out->status = OR_NO_MATCH;
    } else if (out->aut == 0 || s->maps % out->aut != 0) {
        out->status = OR_NOT_DIVISIBLE;
    } else {
        out->status = OR_OK;
        out->classes = s->maps / out->aut;
        out->score = s->best_score;
        out->agg = s->best_agg;
        out->pres = s->best_pres;
        for (int32_t i = 0; i < k; ++i) out->tuple[i] = (uint8_t)s->best_phi[i];
    }
    int32_t st = out->status;
    free(s);
    return st;
}

/* ------------------------------------------------------------------ */
/* One share of a split request: the matches with phi(0) in [root_lo,    */
/* root_hi) only.  Same search as oracle_decide (every map, no symmetry  */
/* breaking); out->maps counts the share's maps, out->classes stays 0    */
/* (a share need not hold whole automorphism classes).                   */

int oracle_decide_rooted(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m,
                         const int32_t *pa, const int32_t *pb, int64_t alpha, int64_t beta, int32_t root_lo,
                         int32_t root_hi, oracle_result *out)
{
    memset(out, 0, sizeof(*out));
    out->k = k;
    uint8_t padj[OR_MAX_K][OR_MAX_K];
    if (n < 1 || n > OR_MAX_N || build_pattern(k, m, pa, pb, padj) != OR_OK) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    match_state *s = (match_state *)calloc(1, sizeof(match_state));
    if (!s) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    s->n = n;
    s->wmat = wmat;
    for (int32_t v = 0; v < n; ++v) s->free_v[v] = busy[v] ? 0 : 1;
    s->k = k;
    s->m = m;
    s->pa = pa;
    s->pb = pb;
    s->padj = padj;
    s->alpha = alpha;
    s->beta = beta;
    s->root_lo = root_lo;
    s->root_hi = root_hi;
    extend(s, 0);
    out->maps = s->maps;
    if (!s->have_best) {
        out->status = OR_NO_MATCH;
    } else {
        out->status = OR_OK;
        out->score = s->best_score;
        out->agg = s->best_agg;
        out->pres = s->best_pres;
        for (int32_t i = 0; i < k; ++i) out->tuple[i] = (uint8_t)s->best_phi[i];
    }
    int32_t st = out->status;
    free(s);
    return st;
}

/* ------------------------------------------------------------------ */
/* Bounded exact decision: branch and bound over the same lexicographic */
/* enumeration (the exact argmax and tuple of oracle_decide; no count)  */
/*
 * A partial map of pattern vertices 0..i-1 is cut off when an upper bound on
 * the score of every completion is <= the best score found so far.  In
 * lexicographic order every later match is lexicographically larger, so a
 * cut-off subtree can hold neither a larger score nor an earlier tie: the
 * result equals oracle_decide's.
 *
 * The bound (alpha, beta >= 0; otherwise nothing is cut), with U the images
 * of the m = k - i unplaced pattern vertices and R = F minus the placed
 * images, follows from writing the final score as the partial score plus,
 * edge by edge:
 *   +alpha*w        for a pattern edge from a placed vertex to U,
 *   (alpha-beta)*w  for a pattern edge inside U,
 *   -beta*w         for every other link between U and R.
 * Every weight lies in [wmin, wmax] (the smallest and largest link weights
 * of G), so
 *   B1 = alpha*wmax*e_cross + e_in*max((alpha-beta)*wmax, (alpha-beta)*wmin).
 * Let d_u be the weight of u's links into R.  Summed over u in U, d_u counts
 * a link inside U twice and a link from U to the rest of R once, and at most
 * m-1 of u's links stay inside U; so the links between U and R weigh at
 * least the sum over u in U of g(d_u) = max(d_u/2, d_u - (m-1)*wmax/2),
 * hence at least half the sum D_m of the m smallest values 2*g(d_u) over all
 * u in R, and
 *   B2 = alpha*wmax*(e_cross + e_in) - beta*D_m/2.
 * Partial score = alpha*agg(placed pattern edges) + beta*W(R), recomputed from
 * the definitions at every node.  Fewer than m vertices left in R: no
 * completion.
 */

typedef struct {
    match_state ms;
    int64_t wmax, wmin;
    uint64_t max_nodes, nodes;
} bb_state;

static int64_t partial_score(bb_state *b, int32_t i)
{
    match_state *s = &b->ms;
    int64_t agg = 0;
    for (int32_t e = 0; e < s->m; ++e)
        if (s->pa[e] < i && s->pb[e] < i) agg += s->wmat[s->phi[s->pa[e]] * s->n + s->phi[s->pb[e]]];
    return s->alpha * agg + s->beta * preserved_bw(s->n, s->wmat, s->free_v, i, s->phi);
}

static int cmp_i64(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, c = *(const int64_t *)y;
    return (a > c) - (a < c);
}

/* Returns 1 when no completion of phi[0..i-1] can score above best_score. */
static int cut_off(bb_state *b, int32_t i)
{
    match_state *s = &b->ms;
    if (!s->have_best || s->alpha < 0 || s->beta < 0) return 0;
    const int32_t m_left = s->k - i;
    int64_t e_cross = 0, e_in = 0;
    for (int32_t e = 0; e < s->m; ++e) {
        int lo = s->pa[e] < s->pb[e] ? s->pa[e] : s->pb[e];
        int hi = s->pa[e] < s->pb[e] ? s->pb[e] : s->pa[e];
        if (lo >= i) e_in += 1;
        else if (hi >= i) e_cross += 1;
    }
    int64_t deg[OR_MAX_N];
    int32_t r = 0;
    for (int32_t u = 0; u < s->n; ++u) {
        if (!s->free_v[u] || s->used[u]) continue;
        int64_t d = 0;
        for (int32_t x = 0; x < s->n; ++x)
            if (x != u && s->free_v[x] && !s->used[x]) d += s->wmat[u * s->n + x];
        deg[r++] = d;
    }
    if (r < m_left) return 1;
    for (int32_t j = 0; j < r; ++j) {
        /* 2*g(d) */
        const int64_t inside = (int64_t)(m_left - 1) * b->wmax;
        deg[j] = 2 * deg[j] - inside > deg[j] ? 2 * deg[j] - inside : deg[j];
    }
    qsort(deg, (size_t)r, sizeof(int64_t), cmp_i64);
    int64_t dm = 0;
    for (int32_t j = 0; j < m_left; ++j) dm += deg[j];
    const int64_t ab = s->alpha - s->beta;
    const int64_t in_w = ab * b->wmax > ab * b->wmin ? ab * b->wmax : ab * b->wmin;
    const int64_t b1 = s->alpha * b->wmax * e_cross + e_in * in_w;
    /* floor(-beta*dm/2) for beta*dm >= 0 */
    const int64_t b2 = s->alpha * b->wmax * (e_cross + e_in) - (s->beta * dm + 1) / 2;
    const int64_t ub = partial_score(b, i) + (b1 < b2 ? b1 : b2);
    return ub <= s->best_score;
}

static void extend_bb(bb_state *b, int32_t i)
{
    match_state *s = &b->ms;
    if (s->aborted) return;
    b->nodes += 1;
    if (b->max_nodes && b->nodes > b->max_nodes) {
        s->aborted = 1;
        return;
    }
    if (i == s->k) {
        visit_match(s);
        return;
    }
    if (cut_off(b, i)) return;
    for (int32_t x = 0; x < s->n; ++x) {
        if (!s->free_v[x] || s->used[x]) continue;
        int ok = 1;
        for (int32_t a = 0; a < i && ok; ++a)
            if (s->padj[a][i] && s->wmat[s->phi[a] * s->n + x] <= 0) ok = 0;
        if (!ok) continue;
        s->used[x] = 1;
        s->phi[i] = x;
        extend_bb(b, i + 1);
        s->used[x] = 0;
        if (s->aborted) return;
    }
}

/* Same result fields as oracle_decide except maps/aut/classes, which stay 0;
 * out->maps holds the search nodes visited instead.  max_nodes > 0 bounds
 * the nodes (OR_BUDGET past it). */
int oracle_decide_bounded(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m,
                          const int32_t *pa, const int32_t *pb, int64_t alpha, int64_t beta, uint64_t max_nodes,
                          oracle_result *out)
{
    memset(out, 0, sizeof(*out));
    out->k = k;
    uint8_t padj[OR_MAX_K][OR_MAX_K];
    if (n < 1 || n > OR_MAX_N || build_pattern(k, m, pa, pb, padj) != OR_OK) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    bb_state *b = (bb_state *)calloc(1, sizeof(bb_state));
    if (!b) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    match_state *s = &b->ms;
    s->n = n;
    s->wmat = wmat;
    for (int32_t v = 0; v < n; ++v) s->free_v[v] = busy[v] ? 0 : 1;
    s->k = k;
    s->m = m;
    s->pa = pa;
    s->pb = pb;
    s->padj = padj;
    s->alpha = alpha;
    s->beta = beta;
    b->wmax = 0;
    b->wmin = 0;
    for (int32_t x = 0; x < n * n; ++x) {
        if (wmat[x] <= 0) continue;
        if (wmat[x] > b->wmax) b->wmax = wmat[x];
        if (b->wmin == 0 || wmat[x] < b->wmin) b->wmin = wmat[x];
    }
    b->max_nodes = max_nodes;
    extend_bb(b, 0);
    out->maps = b->nodes;
    if (s->aborted) {
        out->status = OR_BUDGET;
    } else if (!s->have_best) {
        out->status = OR_NO_MATCH;
    } else {
        out->status = OR_OK;
        out->score = s->best_score;
        out->agg = s->best_agg;
        out->pres = s->best_pres;
        for (int32_t i = 0; i < k; ++i) out->tuple[i] = (uint8_t)s->best_phi[i];
    }
    int32_t st = out->status;
    free(b);
    return st;
}

/* ------------------------------------------------------------------ */
/* Bandwidth-sensitive jobs: Predicted Effective Bandwidth (Eq. 2)       */
/*
 * Eq. 2 models the effective bandwidth of an allocation from the counts of
 * its link types: x double NVLinks, y single NVLinks, z PCIe links, with the
 * fourteen features of Sec. 3.4.3 and the coefficients of Table 2.  Reading:
 * the counts are taken over the images of the pattern edges (the links the
 * job's communication uses), a link's type being given by its peak
 * bandwidth in Table 1: 50 = double NVLink-v2, 25 or 20 = single NVLink
 * (v2 / v1), 12 = PCIe; links of any other weight count in none of x, y, z.
 * Algorithm 1 gives a bandwidth-sensitive job the match with the largest
 * predicted value (first one in lexicographic order among equals).
 */

double oracle_effbw(int64_t x, int64_t y, int64_t z)
{
    static const double theta[15] = {0.0,    16.396, 4.536,  1.556,   -20.694, -9.467, 7.615, -7.973,
                                      12.733, -4.195, -8.413, 62.851, 27.418,  -5.114, -46.973};
    const double X = (double)x, Y = (double)y, Z = (double)z;
    double f = 0.0;
    f += theta[1] * X + theta[2] * Y + theta[3] * Z;
    f += theta[4] / (X + 1.0) + theta[5] / (Y + 1.0) + theta[6] / (Z + 1.0);
    f += theta[7] * X * Y + theta[8] * Y * Z + theta[9] * Z * X;
    f += theta[10] / (X * Y + 1.0) + theta[11] / (Y * Z + 1.0) + theta[12] / (Z * X + 1.0);
    f += theta[13] * X * Y * Z + theta[14] / (X * Y * Z + 1.0);
    return f;
}

static int link_type(int32_t w)
{
    if (w == 50) return 0;            /* double NVLink-v2 */
    if (w == 25 || w == 20) return 1; /* single NVLink v2 / v1 */
    if (w == 12) return 2;            /* PCIe */
    return -1;
}

typedef struct {
    match_state ms;
    double best_f;
    int64_t best_xyz[3];
} effbw_state;

static void visit_effbw(effbw_state *b)
{
    match_state *s = &b->ms;
    s->maps += 1;
    if (s->max_maps && s->maps > s->max_maps) {
        s->aborted = 1;
        return;
    }
    int64_t c[3] = {0, 0, 0};
    for (int32_t e = 0; e < s->m; ++e) {
        const int t = link_type(s->wmat[s->phi[s->pa[e]] * s->n + s->phi[s->pb[e]]]);
        if (t >= 0) c[t] += 1;
    }
    const double f = oracle_effbw(c[0], c[1], c[2]);
    if (!s->have_best || f > b->best_f) {
        s->have_best = 1;
        b->best_f = f;
        memcpy(b->best_xyz, c, sizeof(c));
        s->best_agg = aggregated_bw(s->n, s->wmat, s->m, s->pa, s->pb, s->phi);
        s->best_pres = preserved_bw(s->n, s->wmat, s->free_v, s->k, s->phi);
        memcpy(s->best_phi, s->phi, sizeof(int32_t) * (size_t)s->k);
    }
}

static void extend_effbw(effbw_state *b, int32_t i)
{
    match_state *s = &b->ms;
    if (s->aborted) return;
    if (i == s->k) {
        visit_effbw(b);
        return;
    }
    for (int32_t x = 0; x < s->n; ++x) {
        if (!s->free_v[x] || s->used[x]) continue;
        int ok = 1;
        for (int32_t a = 0; a < i && ok; ++a)
            if (s->padj[a][i] && s->wmat[s->phi[a] * s->n + x] <= 0) ok = 0;
        if (!ok) continue;
        s->used[x] = 1;
        s->phi[i] = x;
        extend_effbw(b, i + 1);
        s->used[x] = 0;
        if (s->aborted) return;
    }
}

/* Decision for a bandwidth-sensitive job.  out->score = round(1000 * EffBW)
 * of the chosen match (milli-GB/s), out->agg / out->pres its AggBW and
 * PreservedBW, out->classes the matches modulo Aut(P) as in oracle_decide;
 * xyz_out (may be NULL) receives its link counts. */
int oracle_decide_effbw(int32_t n, const int32_t *wmat, const uint8_t *busy, int32_t k, int32_t m, const int32_t *pa,
                        const int32_t *pb, uint64_t max_maps, oracle_result *out, int64_t *xyz_out)
{
    memset(out, 0, sizeof(*out));
    out->k = k;
    uint8_t padj[OR_MAX_K][OR_MAX_K];
    if (n < 1 || n > OR_MAX_N || build_pattern(k, m, pa, pb, padj) != OR_OK) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    effbw_state *b = (effbw_state *)calloc(1, sizeof(effbw_state));
    if (!b) {
        out->status = OR_INVALID;
        return OR_INVALID;
    }
    match_state *s = &b->ms;
    s->n = n;
    s->wmat = wmat;
    for (int32_t v = 0; v < n; ++v) s->free_v[v] = busy[v] ? 0 : 1;
    s->k = k;
    s->m = m;
    s->pa = pa;
    s->pb = pb;
    s->padj = padj;
    s->max_maps = max_maps;
    extend_effbw(b, 0);
    out->maps = s->maps;
    if (s->have_best && !s->aborted) out->aut = oracle_aut_count(k, m, pa, pb);
    if (s->aborted) {
        out->status = OR_BUDGET;
    } else if (!s->have_best) {
        out->status = OR_NO_MATCH;
    } else if (out->aut == 0 || s->maps % out->aut != 0) {
        out->status = OR_NOT_DIVISIBLE;
    } else {
        out->status = OR_OK;
        out->classes = s->maps / out->aut;
        out->score = llround(1000.0 * b->best_f);
        out->agg = s->best_agg;
        out->pres = s->best_pres;
        for (int32_t i = 0; i < k; ++i) out->tuple[i] = (uint8_t)s->best_phi[i];
        if (xyz_out) memcpy(xyz_out, b->best_xyz, sizeof(b->best_xyz));
    }
    int32_t st = out->status;
    free(b);
    return st;
}
