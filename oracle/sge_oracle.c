/*
 * sge_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of the method of Kimmig,
 * Meyerhenke and Strash, "Shared Memory Parallel Subgraph Enumeration"
 * (arXiv 1705.09358): RI backtracking search (Section "RI") and RI-DS with
 * the paper's stronger pruning (Section 4).  It exists to check the CUDA path
 * and to serve as the timed CPU baseline; only the tests, the smoke check and
 * the bench's CPU-baseline leg may load it.  It shares no code with the CUDA
 * path.
 *
 * Problem (Section 2.1, Eqs. 1-3, non-induced): list every injection
 * f: V_p -> V_t such that every pattern edge (u,v) maps to a target edge
 * (f(u), f(v)) with an equal edge label (Eqs. 1 "=>" direction and 3), and
 * lab(f(v)) = lab(v) (Eq. 2).
 *
 * Outputs per run: matches = |set of injections|; states = number of
 * (pattern node, target node) pairs considered, i.e. the sum of the raw
 * candidate-set sizes over all expanded search nodes (Section 5, "Search
 * space size"); nodes = number of accepted pairs (search-tree nodes below the
 * root, matches included); hash = sum over matches of h(f) mod 2^64 where
 *   g(u, v) = fmix64(((u64)u << 32 | v) + 0x9E3779B97F4A7C15)
 *   h(f)    = fmix64( sum_u g(u, f(u)) mod 2^64 )
 * and fmix64 is the SplitMix64 finaliser (Steele, Lea, Flood, 2014).  The
 * paper defines no hash; this one is order-free so that any schedule gives
 * the same value.
 *
 * Readings where the paper is silent or garbled:
 *  - w_m is |N(v) intersect mu| (the printed union contradicts the prose).
 *  - The first vertex is the one of highest degree; ties go to the smaller
 *    domain (SI variants only), then to the lower id.  The greedy key is
 *    (w_m, w_n, degree[, -|D|], -id), maximised.
 *  - The parent of mu_i is the earliest EARLIER mu_j adjacent to mu_i.
 *  - Domain initialisation ranges over target nodes (the text says "pattern
 *    nodes").  AC runs to a fixpoint; with FC the two alternate to a joint
 *    fixpoint before the ordering is built.  An empty domain ends the run
 *    with all counters zero.
 *  - RI-DS puts singleton-domain pattern nodes first, in ascending id.
 *  - A pattern with no vertices, or with more vertices than the target, has
 *    no match and no search (all counters zero).
 *  - Degree: number of distinct neighbours (undirected); for directed
 *    graphs rule 3 compares in- and out-degree separately and the ordering
 *    uses in-degree + out-degree and the undirected neighbourhood.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_BUDGET 1

enum { ALGO_RI = 0, ALGO_RIDS = 1, ALGO_RIDS_SI = 2, ALGO_RIDS_SI_FC = 3 };

/* ------------------------------------------------------------------ graph */

typedef struct {
    int a, b, lab;
} arc_t;

typedef struct {
    int n, directed;
    int64_t *optr; int *onbr; int *olab; /* sorted out-rows (undirected: all neighbours) */
    int64_t *iptr; int *inbr; int *ilab; /* sorted in-rows (directed only) */
    int64_t *uptr; int *unbr;            /* undirected neighbourhood, for the ordering */
    int *vlab, *odeg, *ideg;
} graph_t;

static int cmp_arc(const void *x, const void *y) {
    const arc_t *p = (const arc_t *)x, *q = (const arc_t *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return 0;
}

static void graph_free(graph_t *g) {
    free(g->optr); free(g->onbr); free(g->olab);
    free(g->iptr); free(g->inbr); free(g->ilab);
    free(g->uptr); free(g->unbr);
    free(g->vlab); free(g->odeg); free(g->ideg);
    memset(g, 0, sizeof(*g));
}

/* Sort arcs by (a, b), drop exact repeats, fail on a repeat with another label.
 * Returns the new count or -1. */
static int64_t sort_dedup(arc_t *arcs, int64_t cnt) {
    int64_t w = 0;
    if (cnt == 0) return 0;
    qsort(arcs, (size_t)cnt, sizeof(arc_t), cmp_arc);
    for (int64_t r = 0; r < cnt; ++r) {
        if (w > 0 && arcs[w - 1].a == arcs[r].a && arcs[w - 1].b == arcs[r].b) {
            if (arcs[w - 1].lab != arcs[r].lab) return -1;
            continue;
        }
        arcs[w++] = arcs[r];
    }
    return w;
}

static int build_rows(int n, const arc_t *arcs, int64_t cnt, int64_t **ptr, int **nbr, int **lab) {
    *ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    *nbr = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    *lab = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    if (!*ptr || !*nbr || !*lab) return OR_ERR_OOM;
    for (int64_t e = 0; e < cnt; ++e) (*ptr)[arcs[e].a + 1]++;
    for (int v = 0; v < n; ++v) (*ptr)[v + 1] += (*ptr)[v];
    for (int64_t e = 0; e < cnt; ++e) { (*nbr)[e] = arcs[e].b; (*lab)[e] = arcs[e].lab; }
    return OR_OK;
}

static int graph_build(graph_t *g, int n, int64_t m, const int *src, const int *dst,
                       const int *vlab, const int *elab, int directed) {
    memset(g, 0, sizeof(*g));
    if (n < 0 || m < 0) return OR_ERR_ARG;
    g->n = n; g->directed = directed ? 1 : 0;
    int64_t cap = 2 * m;
    arc_t *out = (arc_t *)malloc(sizeof(arc_t) * (size_t)(cap > 0 ? cap : 1));
    arc_t *in = (arc_t *)malloc(sizeof(arc_t) * (size_t)(cap > 0 ? cap : 1));
    arc_t *und = (arc_t *)malloc(sizeof(arc_t) * (size_t)(cap > 0 ? cap : 1));
    if (!out || !in || !und) { free(out); free(in); free(und); return OR_ERR_OOM; }
    int64_t no = 0, ni = 0, nu = 0;
    for (int64_t e = 0; e < m; ++e) {
        int a = src[e], b = dst[e], l = elab ? elab[e] : 0;
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) { free(out); free(in); free(und); return OR_ERR_ARG; }
        if (g->directed) {
            out[no++] = (arc_t){a, b, l};
            in[ni++] = (arc_t){b, a, l};
        } else {
            out[no++] = (arc_t){a, b, l};
            out[no++] = (arc_t){b, a, l};
        }
        und[nu++] = (arc_t){a, b, 0};
        und[nu++] = (arc_t){b, a, 0};
    }
    no = sort_dedup(out, no);
    if (g->directed) ni = sort_dedup(in, ni);
    nu = sort_dedup(und, nu);
    int rc = OR_OK;
    if (no < 0 || ni < 0 || nu < 0) rc = OR_ERR_ARG;
    if (rc == OR_OK) rc = build_rows(n, out, no, &g->optr, &g->onbr, &g->olab);
    if (rc == OR_OK && g->directed) rc = build_rows(n, in, ni, &g->iptr, &g->inbr, &g->ilab);
    if (rc == OR_OK) {
        int *dummy = NULL;
        rc = build_rows(n, und, nu, &g->uptr, &g->unbr, &dummy);
        free(dummy);
    }
    free(out); free(in); free(und);
    if (rc != OR_OK) { graph_free(g); return rc; }
    g->vlab = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    g->odeg = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    g->ideg = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!g->vlab || !g->odeg || !g->ideg) { graph_free(g); return OR_ERR_OOM; }
    for (int v = 0; v < n; ++v) {
        g->vlab[v] = vlab ? vlab[v] : 0;
        g->odeg[v] = (int)(g->optr[v + 1] - g->optr[v]);
        g->ideg[v] = g->directed ? (int)(g->iptr[v + 1] - g->iptr[v]) : g->odeg[v];
    }
    return OR_OK;
}

/* Label of arc a->b, or -1 if the arc does not exist (binary search in the sorted row). */
static int arc_label(const graph_t *g, int a, int b) {
    int64_t lo = g->optr[a], hi = g->optr[a + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->onbr[mid] < b) lo = mid + 1; else hi = mid;
    }
    if (lo < g->optr[a + 1] && g->onbr[lo] == b) return g->olab[lo];
    return -1;
}

static int is_unbr(const graph_t *g, int a, int b) {
    for (int64_t e = g->uptr[a]; e < g->uptr[a + 1]; ++e)
        if (g->unbr[e] == b) return 1;
    return 0;
}

/* ---------------------------------------------------------------- hashing */

static uint64_t fmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t match_hash(int k, const int *f) {
    uint64_t s = 0;
    for (int u = 0; u < k; ++u)
        s += fmix64((((uint64_t)(uint32_t)u) << 32 | (uint64_t)(uint32_t)f[u]) + 0x9E3779B97F4A7C15ULL);
    return fmix64(s);
}

/* ---------------------------------------------------------------- domains */
/* Section 4, "Domains in RI-DS": D(v_p) starts as the target nodes with an
 * equal label and in-/out-degree at least that of v_p. */
static void domain_init(const graph_t *p, const graph_t *t, unsigned char *dom) {
    for (int v = 0; v < p->n; ++v)
        for (int x = 0; x < t->n; ++x)
            dom[(size_t)v * t->n + x] = (unsigned char)(t->vlab[x] == p->vlab[v] &&
                                                        t->odeg[x] >= p->odeg[v] &&
                                                        t->ideg[x] >= p->ideg[v]);
}

/* One arc-consistency sweep (Section 4): remove x from D(v) when some pattern
 * edge at v has no compatible target edge at x leading into the other
 * endpoint's domain.  Returns 1 if anything was removed. */
static int ac_sweep(const graph_t *p, const graph_t *t, unsigned char *dom) {
    int changed = 0;
    size_t nt = (size_t)t->n;
    for (int v = 0; v < p->n; ++v) {
        for (int x = 0; x < t->n; ++x) {
            if (!dom[v * nt + x]) continue;
            int ok = 1;
            /* pattern arcs v -> u need a target arc x -> y, y in D(u), equal label */
            for (int64_t e = p->optr[v]; ok && e < p->optr[v + 1]; ++e) {
                int u = p->onbr[e], bl = p->olab[e], found = 0;
                for (int64_t f = t->optr[x]; f < t->optr[x + 1]; ++f)
                    if (t->olab[f] == bl && dom[u * nt + t->onbr[f]]) { found = 1; break; }
                ok = found;
            }
            /* directed: pattern arcs u -> v need a target arc y -> x */
            if (p->directed) {
                for (int64_t e = p->iptr[v]; ok && e < p->iptr[v + 1]; ++e) {
                    int u = p->inbr[e], bl = p->ilab[e], found = 0;
                    for (int64_t f = t->iptr[x]; f < t->iptr[x + 1]; ++f)
                        if (t->ilab[f] == bl && dom[u * nt + t->inbr[f]]) { found = 1; break; }
                    ok = found;
                }
            }
            if (!ok) { dom[v * nt + x] = 0; changed = 1; }
        }
    }
    return changed;
}

static int64_t domain_size(const unsigned char *dom, int v, int nt) {
    int64_t c = 0;
    for (int x = 0; x < nt; ++x) c += dom[(size_t)v * nt + x];
    return c;
}

static int any_empty(const unsigned char *dom, int k, int nt) {
    for (int v = 0; v < k; ++v)
        if (domain_size(dom, v, nt) == 0) return 1;
    return 0;
}

/* Forward checking of singletons (Section 4.2): for each pattern node whose
 * domain is the single target node x, remove x from every other domain;
 * repeat for singletons this creates.  `done` marks propagated singletons.
 * Returns 1 if anything was removed. */
static int fc_pass(int k, int nt, unsigned char *dom, unsigned char *done) {
    int changed = 0, again = 1;
    while (again) {
        again = 0;
        for (int u = 0; u < k; ++u) {
            if (done[u] || domain_size(dom, u, nt) != 1) continue;
            int x = -1;
            for (int y = 0; y < nt; ++y) if (dom[(size_t)u * nt + y]) { x = y; break; }
            done[u] = 1;
            for (int v = 0; v < k; ++v) {
                if (v == u) continue;
                if (dom[(size_t)v * nt + x]) { dom[(size_t)v * nt + x] = 0; changed = 1; again = 1; }
            }
        }
    }
    return changed;
}

/* Domains for RI-DS variants: AC to a fixpoint; with FC, AC and FC alternate
 * until neither removes anything.  Stops early when a domain is empty.
 * Returns 1 if some domain is empty. */
static int compute_domains(const graph_t *p, const graph_t *t, int algo, unsigned char *dom) {
    int k = p->n, nt = t->n;
    domain_init(p, t, dom);
    unsigned char *done = (unsigned char *)calloc((size_t)k + 1, 1);
    for (;;) {
        int changed = 0;
        while (ac_sweep(p, t, dom)) changed = 1;
        if (any_empty(dom, k, nt)) break;
        if (algo == ALGO_RIDS_SI_FC) changed |= fc_pass(k, nt, dom, done);
        if (any_empty(dom, k, nt)) break;
        if (!changed || algo != ALGO_RIDS_SI_FC) break;
    }
    free(done);
    return any_empty(dom, k, nt);
}

/* --------------------------------------------------------------- ordering */
/* Section "RI": GreatestConstraintFirst.  `dsize` is NULL for RI. */
static void ri_order(const graph_t *p, int algo, const int64_t *dsize, int *mu, int *par) {
    int k = p->n;
    unsigned char *in = (unsigned char *)calloc((size_t)k + 1, 1);
    unsigned char *mark = (unsigned char *)calloc((size_t)k + 1, 1);
    int len = 0;
    int si = (algo == ALGO_RIDS_SI || algo == ALGO_RIDS_SI_FC);
    /* RI-DS: singleton domains first, ascending id (Section 4.1) */
    if (algo != ALGO_RI)
        for (int v = 0; v < k; ++v)
            if (dsize[v] == 1) { mu[len++] = v; in[v] = 1; }
    if (len == 0 && k > 0) {
        int best = -1;
        for (int v = 0; v < k; ++v) {
            int dv = p->odeg[v] + (p->directed ? p->ideg[v] : 0);
            if (best < 0) { best = v; continue; }
            int db = p->odeg[best] + (p->directed ? p->ideg[best] : 0);
            if (dv > db || (dv == db && si && dsize[v] < dsize[best])) best = v;
        }
        mu[len++] = best; in[best] = 1;
    }
    while (len < k) {
        int best = -1;
        long bwm = -1, bwn = -1, bdeg = -1;
        for (int v = 0; v < k; ++v) {
            if (in[v]) continue;
            long wm = 0, wn = 0;
            for (int64_t e = p->uptr[v]; e < p->uptr[v + 1]; ++e) wm += in[p->unbr[e]];
            memset(mark, 0, (size_t)k);
            for (int64_t e = p->uptr[v]; e < p->uptr[v + 1]; ++e) {
                int x = p->unbr[e];
                if (in[x] || x == v) continue;
                for (int64_t f = p->uptr[x]; f < p->uptr[x + 1]; ++f) {
                    int w = p->unbr[f];
                    if (in[w] && !mark[w]) { mark[w] = 1; ++wn; }
                }
            }
            long dv = p->odeg[v] + (p->directed ? p->ideg[v] : 0);
            int take = 0;
            if (best < 0) take = 1;
            else if (wm != bwm) take = wm > bwm;
            else if (wn != bwn) take = wn > bwn;
            else if (dv != bdeg) take = dv > bdeg;
            else if (si && dsize[v] != dsize[best]) take = dsize[v] < dsize[best];
            if (take) { best = v; bwm = wm; bwn = wn; bdeg = dv; }
        }
        mu[len++] = best; in[best] = 1;
    }
    for (int i = 0; i < k; ++i) {
        par[i] = -1;
        for (int j = 0; j < i; ++j)
            if (is_unbr(p, mu[i], mu[j])) { par[i] = j; break; }
    }
    free(in); free(mark);
}

/* ----------------------------------------------------------------- search */

typedef struct {
    const graph_t *p, *t;
    int algo, k;
    const int *mu, *par;
    const unsigned char *dom;       /* NULL for RI */
    int *M;                         /* M[i] = image of mu[i] */
    unsigned char *used;
    int *f;                         /* scratch: image in pattern-vertex order */
    int *root_list;                 /* candidate list for unparented positions */
    int64_t *root_off;              /* per position: offset into root_list, length */
    uint64_t matches, states, nodes, hash;
    int64_t budget;
    int stop;
    uint64_t *lv_nodes, *lv_states;
    int *out; int64_t out_cap, out_len;
    int shard_depth, shard_index, shard_count;
    int64_t shard_seen;
} search_t;

/* Rules 1-4 of Section "RI" (pruning rules), plus the RI-DS domain test. */
static int feasible(search_t *s, int i, int c) {
    const graph_t *p = s->p, *t = s->t;
    int u = s->mu[i];
    if (s->used[c]) return 0;                                        /* rule 1 */
    if (t->vlab[c] != p->vlab[u]) return 0;                          /* rule 2 */
    if (t->odeg[c] < p->odeg[u] || t->ideg[c] < p->ideg[u]) return 0;/* rule 3 */
    if (s->dom && !s->dom[(size_t)u * t->n + c]) return 0;           /* RI-DS */
    for (int j = 0; j < i; ++j) {                                    /* rule 4 */
        int w = s->mu[j];
        int lu = arc_label(p, u, w);
        if (lu >= 0 && arc_label(t, c, s->M[j]) != lu) return 0;
        if (p->directed) {
            int lw = arc_label(p, w, u);
            if (lw >= 0 && arc_label(t, s->M[j], c) != lw) return 0;
        }
    }
    return 1;
}

static void record_match(search_t *s) {
    for (int i = 0; i < s->k; ++i) s->f[s->mu[i]] = s->M[i];
    s->matches++;
    s->hash += match_hash(s->k, s->f);
    if (s->out && s->out_len < s->out_cap)
        memcpy(s->out + s->out_len * s->k, s->f, sizeof(int) * (size_t)s->k);
    s->out_len++;
}

/* Expand the search node whose positions 0..i-1 are assigned: consider the
 * candidates for position i (Section "RI": the neighbours of M(P(mu_i)); all
 * target nodes, or D(mu_i) for RI-DS, when mu_i has no parent). */
static void expand(search_t *s, int i) {
    const graph_t *t = s->t;
    const int *cand;
    int64_t ncand;
    if (s->stop) return;
    int counted = (s->shard_count <= 1) || (i >= s->shard_depth) || (s->shard_index == 0);
    if (s->par[i] >= 0) {
        int a = s->M[s->par[i]];
        int up = s->mu[s->par[i]], u = s->mu[i];
        if (!t->directed || arc_label(s->p, up, u) >= 0) {   /* arc P -> mu_i: out-row */
            cand = t->onbr + t->optr[a];
            ncand = t->optr[a + 1] - t->optr[a];
        } else {                                              /* arc mu_i -> P: in-row */
            cand = t->inbr + t->iptr[a];
            ncand = t->iptr[a + 1] - t->iptr[a];
        }
    } else {
        cand = s->root_list + s->root_off[2 * i];
        ncand = s->root_off[2 * i + 1];
    }
    if (counted) {
        s->states += (uint64_t)ncand;
        if (s->lv_states) s->lv_states[i] += (uint64_t)ncand;
    }
    if (s->budget > 0 && (int64_t)s->states > s->budget) { s->stop = 1; return; }
    for (int64_t e = 0; e < ncand && !s->stop; ++e) {
        int c = cand[e];
        if (!feasible(s, i, c)) continue;
        /* Sharded runs (multi-device form): the nodes accepted at position
         * shard_depth-1 are the split frontier, numbered in search order; a
         * shard descends only below frontier nodes of its residue class.
         * Everything above the frontier (and the frontier nodes themselves)
         * is counted by shard 0 alone. */
        int descend = 1;
        if (s->shard_count > 1 && i + 1 == s->shard_depth) {
            int64_t idx = s->shard_seen++;
            descend = (idx % s->shard_count) == s->shard_index;
        }
        if (counted) {
            s->nodes++;
            if (s->lv_nodes) s->lv_nodes[i]++;
        }
        s->M[i] = c;
        s->used[c] = 1;
        if (i + 1 == s->k) { if (counted) record_match(s); }
        else if (descend) expand(s, i + 1);
        s->used[c] = 0;
    }
}

/* ------------------------------------------------------------- public API */

/* Build a target once for many runs (returns NULL and sets *rc on error). */
void *oracle_target_new(int nt, int64_t mt, const int *tsrc, const int *tdst, const int *tvlab,
                        const int *telab, int directed, int *rc) {
    graph_t *t = (graph_t *)malloc(sizeof(graph_t));
    if (!t) { *rc = OR_ERR_OOM; return NULL; }
    *rc = graph_build(t, nt, mt, tsrc, tdst, tvlab, telab, directed);
    if (*rc) { free(t); return NULL; }
    return t;
}

void oracle_target_free(void *t) {
    if (t) { graph_free((graph_t *)t); free(t); }
}

int oracle_run_t(void *target,
                 int np, int64_t mp, const int *psrc, const int *pdst, const int *pvlab,
                 const int *pelab,
                 int algo, int64_t state_budget,
                 uint64_t *counters,      /* out[4]: matches, states, nodes, hash */
                 int *mu_out, int *par_out, int64_t *dsize_out,
                 int *match_out, int64_t match_cap, int64_t *match_len,
                 uint64_t *lv_nodes, uint64_t *lv_states,
                 int shard_depth, int shard_index, int shard_count) {
    graph_t *tp = (graph_t *)target, p;
    int rc, nt;
    if (!tp || algo < ALGO_RI || algo > ALGO_RIDS_SI_FC || !counters) return OR_ERR_ARG;
    if (shard_count > 1 && (shard_depth < 1 || shard_index < 0 || shard_index >= shard_count))
        return OR_ERR_ARG;
    nt = tp->n;
    counters[0] = counters[1] = counters[2] = counters[3] = 0;
    if (match_len) *match_len = 0;
    rc = graph_build(&p, np, mp, psrc, pdst, pvlab, pelab, tp->directed);
    if (rc) return rc;
    if (np == 0 || np > nt) { graph_free(&p); return OR_OK; }

    int k = np;
    unsigned char *dom = NULL;
    int64_t *dsize = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int *mu = (int *)malloc(sizeof(int) * (size_t)k), *par = (int *)malloc(sizeof(int) * (size_t)k);
    if (!dsize || !mu || !par) { rc = OR_ERR_OOM; goto done; }
    if (algo != ALGO_RI) {
        dom = (unsigned char *)malloc((size_t)k * (size_t)nt);
        if (!dom) { rc = OR_ERR_OOM; goto done; }
        if (compute_domains(&p, tp, algo, dom)) {
            for (int v = 0; v < k; ++v) dsize[v] = domain_size(dom, v, nt);
            if (dsize_out) memcpy(dsize_out, dsize, sizeof(int64_t) * (size_t)k);
            goto done; /* an empty domain: no match, no search */
        }
        for (int v = 0; v < k; ++v) dsize[v] = domain_size(dom, v, nt);
        if (dsize_out) memcpy(dsize_out, dsize, sizeof(int64_t) * (size_t)k);
    }
    ri_order(&p, algo, dsize, mu, par);
    if (mu_out) memcpy(mu_out, mu, sizeof(int) * (size_t)k);
    if (par_out) memcpy(par_out, par, sizeof(int) * (size_t)k);

    {
        search_t s;
        memset(&s, 0, sizeof(s));
        s.p = &p; s.t = tp; s.algo = algo; s.k = k; s.mu = mu; s.par = par; s.dom = dom;
        s.M = (int *)calloc((size_t)k, sizeof(int));
        s.f = (int *)calloc((size_t)k, sizeof(int));
        s.used = (unsigned char *)calloc((size_t)nt, 1);
        s.root_off = (int64_t *)calloc(2 * (size_t)k, sizeof(int64_t));
        /* candidate lists of unparented positions: V_t (RI) or D(mu_i) in id order */
        int64_t total = 0;
        for (int i = 0; i < k; ++i)
            if (par[i] < 0) total += (algo == ALGO_RI) ? nt : dsize[mu[i]];
        s.root_list = (int *)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
        if (s.root_off && s.root_list) {
            int64_t off = 0;
            for (int i = 0; i < k; ++i) {
                if (par[i] >= 0) continue;
                s.root_off[2 * i] = off;
                for (int x = 0; x < nt; ++x)
                    if (algo == ALGO_RI || dom[(size_t)mu[i] * nt + x]) s.root_list[off++] = x;
                s.root_off[2 * i + 1] = off - s.root_off[2 * i];
            }
        }
        s.budget = state_budget;
        s.lv_nodes = lv_nodes; s.lv_states = lv_states;
        s.out = match_out; s.out_cap = match_out ? match_cap : 0;
        s.shard_depth = shard_depth; s.shard_index = shard_index; s.shard_count = shard_count;
        if (!s.M || !s.f || !s.used || !s.root_off || !s.root_list) rc = OR_ERR_OOM;
        else expand(&s, 0);
        counters[0] = s.matches; counters[1] = s.states; counters[2] = s.nodes; counters[3] = s.hash;
        if (match_len) *match_len = s.out_len;
        if (rc == OR_OK && s.stop) rc = OR_BUDGET;
        free(s.M); free(s.f); free(s.used); free(s.root_off); free(s.root_list);
    }
done:
    free(dom); free(dsize); free(mu); free(par);
    graph_free(&p);
    return rc;
}

int oracle_run(int nt, int64_t mt, const int *tsrc, const int *tdst, const int *tvlab,
               const int *telab, int directed,
               int np, int64_t mp, const int *psrc, const int *pdst, const int *pvlab,
               const int *pelab,
               int algo, int64_t state_budget,
               uint64_t *counters,
               int *mu_out, int *par_out, int64_t *dsize_out,
               int *match_out, int64_t match_cap, int64_t *match_len,
               uint64_t *lv_nodes, uint64_t *lv_states,
               int shard_depth, int shard_index, int shard_count) {
    int rc;
    void *t = oracle_target_new(nt, mt, tsrc, tdst, tvlab, telab, directed, &rc);
    if (!t) return rc;
    rc = oracle_run_t(t, np, mp, psrc, pdst, pvlab, pelab, algo, state_budget, counters, mu_out,
                      par_out, dsize_out, match_out, match_cap, match_len, lv_nodes, lv_states,
                      shard_depth, shard_index, shard_count);
    oracle_target_free(t);
    return rc;
}

/* Domains alone (for the AC / FC checks).  dom_out is k x nt bytes. */
int oracle_domains(int nt, int64_t mt, const int *tsrc, const int *tdst, const int *tvlab,
                   const int *telab, int directed,
                   int np, int64_t mp, const int *psrc, const int *pdst, const int *pvlab,
                   const int *pelab, int algo, unsigned char *dom_out) {
    graph_t t, p;
    int rc = graph_build(&t, nt, mt, tsrc, tdst, tvlab, telab, directed);
    if (rc) return rc;
    rc = graph_build(&p, np, mp, psrc, pdst, pvlab, pelab, directed);
    if (rc) { graph_free(&t); return rc; }
    if (algo == ALGO_RI) domain_init(&p, &t, dom_out);
    else compute_domains(&p, &t, algo, dom_out);
    graph_free(&t); graph_free(&p);
    return OR_OK;
}

/* Forward checking alone on given domains (k x nt bytes, modified in place). */
int oracle_fc(int k, int nt, unsigned char *dom) {
    unsigned char *done = (unsigned char *)calloc((size_t)k + 1, 1);
    if (!done) return OR_ERR_OOM;
    fc_pass(k, nt, dom, done);
    free(done);
    return OR_OK;
}

/* Ordering alone.  dsize may be NULL for RI. */
int oracle_order(int np, int64_t mp, const int *psrc, const int *pdst, int directed, int algo,
                 const int64_t *dsize, int *mu_out, int *par_out) {
    graph_t p;
    int rc = graph_build(&p, np, mp, psrc, pdst, NULL, NULL, directed);
    if (rc) return rc;
    if (algo != ALGO_RI && !dsize) { graph_free(&p); return OR_ERR_ARG; }
    ri_order(&p, algo, dsize, mu_out, par_out);
    graph_free(&p);
    return OR_OK;
}

/* The per-match hash h(f), exposed so tests can hash a brute-force list. */
uint64_t oracle_match_hash(int k, const int *f) { return match_hash(k, f); }
