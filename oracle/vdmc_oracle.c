/*
 * CPU ORACLE for per-vertex directed 3- and 4-motif counts.
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, table or
 * helper with the CUDA library: it computes the plain definition of the
 * output with a different algorithm (ESU enumeration of connected vertex
 * sets + canonicalisation by trying every permutation), in plain C.
 *
 * What is computed (paper, "Notation and detailed description", Definitions;
 * section "Comparison to theory in G(n,p)" defines X_{k,m}(i)):
 *   For every set S of k vertices that is connected in the underlying
 *   undirected graph G_U, form the k x k adjacency matrix of the induced
 *   directed sub-graph under some ordering of S, read it row by row with the
 *   diagonal removed as a binary number (first off-diagonal entry = most
 *   significant bit; Fig. 1: 110101 = 53).  The motif of S is the minimum of
 *   that number over all k! orderings (Fig. 1: index_Min = 30; the
 *   isomorph-merge paragraph of "The Algorithm").  Every vertex of S gets +1
 *   in the column of that motif.
 *
 * Column order (a reading: the paper names each motif by its minimum index):
 *   the connected motifs sorted by ascending minimum index; 13 columns for
 *   k = 3, 199 for k = 4.
 *
 * Graph conventions (Definitions: unweighted simple directed graph):
 *   self-loops are ignored and repeated arcs collapsed; matrix entry (i,j)
 *   is 1 iff the arc i->j exists.
 *
 * Parity pins for this file live in the CPU tests (brute force over all
 * subsets, closed forms, G(n,p) expectation of Eq. 4, invariants).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXK 4

/* ------------------------------------------------------------------ */
/* Motif index of an ordered vertex tuple (Definitions; Fig. 1).       */
/* ------------------------------------------------------------------ */

/* adjacency matrix adj[i*k+j] (0/1), i != j  ->  index, row-major, MSB first */
static int matrix_to_index(int k, const int *adj) {
    int idx = 0;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++)
            if (i != j) idx = (idx << 1) | (adj[i * k + j] ? 1 : 0);
    return idx;
}

static void index_to_matrix(int k, int idx, int *adj) {
    int nb = k * (k - 1);
    int b = nb - 1;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) {
            if (i == j) { adj[i * k + j] = 0; continue; }
            adj[i * k + j] = (idx >> b) & 1;
            b--;
        }
}

/* next permutation in lexicographic order; returns 0 after the last one */
static int next_perm(int k, int *p) {
    int i = k - 2;
    while (i >= 0 && p[i] > p[i + 1]) i--;
    if (i < 0) return 0;
    int j = k - 1;
    while (p[j] < p[i]) j--;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = k - 1; a < b; a++, b--) { t = p[a]; p[a] = p[b]; p[b] = t; }
    return 1;
}

/* Minimum index over all k! re-orderings of the vertices (isomorph merge). */
int oracle_canonical_index(int k, int idx) {
    int adj[MAXK * MAXK], padj[MAXK * MAXK], p[MAXK];
    index_to_matrix(k, idx, adj);
    for (int i = 0; i < k; i++) p[i] = i;
    int best = idx;
    do {
        for (int i = 0; i < k; i++)
            for (int j = 0; j < k; j++) padj[i * k + j] = adj[p[i] * k + p[j]];
        int v = matrix_to_index(k, padj);
        if (v < best) best = v;
    } while (next_perm(k, p));
    return best;
}

/* connected in the underlying undirected graph? (Definitions: a k-motif) */
static int index_is_connected(int k, int idx) {
    int adj[MAXK * MAXK];
    index_to_matrix(k, idx, adj);
    int seen = 1, frontier = 1;
    while (frontier) {
        int nf = 0;
        for (int i = 0; i < k; i++)
            if (frontier >> i & 1)
                for (int j = 0; j < k; j++)
                    if (j != i && (adj[i * k + j] || adj[j * k + i]) && !(seen >> j & 1)) {
                        seen |= 1 << j; nf |= 1 << j;
                    }
        frontier = nf;
    }
    return seen == (1 << k) - 1;
}

/*
 * The class table, by brute force over all 2^(k(k-1)) indices.
 * canon[c] = minimum index of class c (ascending), niso[c] = number of
 * indices (labelled isomorphs) in class c.  Only connected classes when
 * connected_only != 0.  Returns the number of classes, or -1.
 */
int oracle_classes(int k, int connected_only, uint16_t *canon, uint32_t *niso, int cap) {
    if (k < 2 || k > MAXK) return -1;
    int nidx = 1 << (k * (k - 1));
    int *cnt = calloc((size_t)nidx, sizeof(int));
    if (!cnt) return -1;
    for (int idx = 0; idx < nidx; idx++) {
        if (connected_only && !index_is_connected(k, idx)) continue;
        cnt[oracle_canonical_index(k, idx)]++;
    }
    int nc = 0;
    for (int idx = 0; idx < nidx; idx++)
        if (cnt[idx]) {
            if (nc < cap) {
                if (canon) canon[nc] = (uint16_t)idx;
                if (niso) niso[nc] = (uint32_t)cnt[idx];
            }
            nc++;
        }
    free(cnt);
    return nc;
}

/*
 * Undirected variant (the undirected motifs of Tables 1-2 and Fig. 5): the
 * classes of connected simple undirected graphs on k vertices, each named
 * by the minimum index of its (symmetric) adjacency matrix under the same
 * bit order; niso[c] = labelled graphs in class c.  Returns the number of
 * classes, or -1.
 */
int oracle_classes_undirected(int k, uint16_t *canon, uint32_t *niso, int cap) {
    if (k < 2 || k > MAXK) return -1;
    int nidx = 1 << (k * (k - 1));
    int *cnt = calloc((size_t)nidx, sizeof(int));
    if (!cnt) return -1;
    int adj[MAXK * MAXK];
    for (int idx = 0; idx < nidx; idx++) {
        index_to_matrix(k, idx, adj);
        int sym = 1;
        for (int i = 0; i < k && sym; i++)
            for (int j = 0; j < k; j++)
                if (adj[i * k + j] != adj[j * k + i]) { sym = 0; break; }
        if (!sym || !index_is_connected(k, idx)) continue;
        cnt[oracle_canonical_index(k, idx)]++;
    }
    int nc = 0;
    for (int idx = 0; idx < nidx; idx++)
        if (cnt[idx]) {
            if (nc < cap) {
                if (canon) canon[nc] = (uint16_t)idx;
                if (niso) niso[nc] = (uint32_t)cnt[idx];
            }
            nc++;
        }
    free(cnt);
    return nc;
}

/* ------------------------------------------------------------------ */
/* Graph as plain sorted adjacency lists in ORIGINAL ids.              */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t n;
    int64_t *optr; int32_t *oadj;   /* out-arcs, sorted, distinct */
    int64_t *uptr; int32_t *uadj;   /* G_U neighbours, sorted, distinct */
    int64_t *eup;                   /* per vertex u: first position in uadj of a neighbour > u */
    int64_t *erow;                  /* per vertex u: edges {u', v'}, u' < v', with u' < u */
} ograph;

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static void ograph_free(ograph *g) {
    free(g->optr); free(g->oadj); free(g->uptr); free(g->uadj); free(g->eup); free(g->erow);
    memset(g, 0, sizeof *g);
}

/* Keys u*n+v of the kept arcs, sorted and distinct (self-loops dropped). */
static int ograph_build(ograph *g, int32_t n, int64_t m, const int32_t *src, const int32_t *dst) {
    memset(g, 0, sizeof *g);
    g->n = n;
    int64_t *key = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *ukey = malloc(sizeof(int64_t) * (size_t)(2 * m > 0 ? 2 * m : 1));
    if (!key || !ukey) { free(key); free(ukey); return -1; }
    int64_t mk = 0, mu = 0;
    for (int64_t e = 0; e < m; e++) {
        int32_t u = src[e], v = dst[e];
        if (u < 0 || v < 0 || u >= n || v >= n) { free(key); free(ukey); return -2; }
        if (u == v) continue;
        key[mk++] = (int64_t)u * n + v;
        ukey[mu++] = (int64_t)u * n + v;
        ukey[mu++] = (int64_t)v * n + u;
    }
    qsort(key, (size_t)mk, sizeof(int64_t), cmp_i64);
    qsort(ukey, (size_t)mu, sizeof(int64_t), cmp_i64);
    int64_t a = 0;
    for (int64_t i = 0; i < mk; i++) if (i == 0 || key[i] != key[i - 1]) key[a++] = key[i];
    mk = a; a = 0;
    for (int64_t i = 0; i < mu; i++) if (i == 0 || ukey[i] != ukey[i - 1]) ukey[a++] = ukey[i];
    mu = a;
    g->optr = calloc((size_t)n + 1, sizeof(int64_t));
    g->uptr = calloc((size_t)n + 1, sizeof(int64_t));
    g->oadj = malloc(sizeof(int32_t) * (size_t)(mk > 0 ? mk : 1));
    g->uadj = malloc(sizeof(int32_t) * (size_t)(mu > 0 ? mu : 1));
    if (!g->optr || !g->uptr || !g->oadj || !g->uadj) { free(key); free(ukey); ograph_free(g); return -1; }
    for (int64_t i = 0; i < mk; i++) { g->optr[key[i] / n + 1]++; g->oadj[i] = (int32_t)(key[i] % n); }
    for (int64_t i = 0; i < mu; i++) { g->uptr[ukey[i] / n + 1]++; g->uadj[i] = (int32_t)(ukey[i] % n); }
    for (int32_t v = 0; v < n; v++) { g->optr[v + 1] += g->optr[v]; g->uptr[v + 1] += g->uptr[v]; }
    free(key); free(ukey);
    /* rows of the per-edge output: edges {u, v}, u < v, in (u, v) order */
    g->eup = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    g->erow = malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!g->eup || !g->erow) { ograph_free(g); return -1; }
    g->erow[0] = 0;
    for (int32_t u = 0; u < n; u++) {
        int64_t e = g->uptr[u];
        while (e < g->uptr[u + 1] && g->uadj[e] < u) e++;
        g->eup[u] = e;
        g->erow[u + 1] = g->erow[u] + (g->uptr[u + 1] - e);
    }
    return 0;
}

/* output row of the edge {u, v} of G_U (which must exist) */
static int64_t edge_row(const ograph *g, int32_t u, int32_t v) {
    if (u > v) { int32_t t = u; u = v; v = t; }
    int64_t lo = g->eup[u], hi = g->uptr[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->uadj[mid] < v) lo = mid + 1; else hi = mid;
    }
    return g->erow[u] + (lo - g->eup[u]);
}

static int has_arc(const ograph *g, int32_t u, int32_t v) {
    int64_t lo = g->optr[u], hi = g->optr[u + 1];
    if (lo == hi) return 0;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->oadj[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < g->optr[u + 1] && g->oadj[lo] == v;
}

static int u_adjacent(const ograph *g, int32_t u, int32_t v) {
    int64_t lo = g->uptr[u], hi = g->uptr[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (g->uadj[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < g->uptr[u + 1] && g->uadj[lo] == v;
}

/* Sorted connected-class list of the oracle itself, for the column lookup. */
/* The class list in use and what is credited:
 *   undirected = 0: directed motifs (entry (i,j) = arc i -> j)
 *   undirected = 1: undirected motifs of G_U (entry (i,j) = edge {i,j})
 *   per_edge   = 0: each member vertex gets +1 (X_{k,m}(i))
 *   per_edge   = 1: each edge of G_U inside the set gets +1 instead (the
 *                   edge variant of the Discussion) */
typedef struct { int k, nc, undirected, per_edge; uint16_t canon[256]; } oclasses;

static int class_column(const oclasses *c, int canon_idx) {
    int lo = 0, hi = c->nc - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (c->canon[mid] == canon_idx) return mid;
        if (c->canon[mid] < canon_idx) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Classify one connected vertex set and credit each member. */
static void credit_set(const ograph *g, const oclasses *cl, int k, const int32_t *S, uint64_t *out) {
    int adj[MAXK * MAXK];
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++)
            adj[i * k + j] = (i != j) && (cl->undirected ? u_adjacent(g, S[i], S[j]) : has_arc(g, S[i], S[j]));
    int idx = matrix_to_index(k, adj);
    int col = class_column(cl, oracle_canonical_index(k, idx));
    if (!cl->per_edge) {
        for (int i = 0; i < k; i++)
            __atomic_fetch_add(&out[(size_t)S[i] * (size_t)cl->nc + (size_t)col], (uint64_t)1, __ATOMIC_RELAXED);
        return;
    }
    for (int i = 0; i < k; i++)
        for (int j = i + 1; j < k; j++)
            if (u_adjacent(g, S[i], S[j]))
                __atomic_fetch_add(&out[(size_t)edge_row(g, S[i], S[j]) * (size_t)cl->nc + (size_t)col], (uint64_t)1,
                                   __ATOMIC_RELAXED);
}

/* ------------------------------------------------------------------ */
/* ESU enumeration of connected k-sets (Wernicke 2006, the FANMOD       */
/* reference of the Introduction).  "u > v" compares by a vertex order  */
/* key; the root of each set is its minimum-key vertex.                 */
/* ------------------------------------------------------------------ */

typedef struct {
    const ograph *g;
    const oclasses *cl;
    int k;
    const int32_t *key;      /* order key per vertex (rank), or NULL for id */
    int32_t *roots;          /* vertices in the order they are taken as roots */
    int64_t nroots;
    int64_t *eoff;           /* root i's initial extension set is eall[eoff[i], eoff[i+1]) */
    int32_t *eall;
    int32_t *troot;          /* per task t in [0, eoff[nroots]): its root index */
    uint64_t *out;
    int64_t next;            /* shared task cursor */
    int64_t found;           /* shared count of sets */
} esu_job;

static inline int32_t okey(const esu_job *J, int32_t v) { return J->key ? J->key[v] : v; }

static int64_t esu_extend(const esu_job *J, int32_t *sub, int nsub, const int32_t *ext, int next, int32_t root);

/*
 * One step of ESU: add w to V_sub, whose remaining extension set is
 * rem[0, nrem), and recurse with
 *   V'_ext = rem  U  { u in N_excl(w, V_sub) : u > root }.
 */
static int64_t esu_take(const esu_job *J, int32_t *sub, int nsub, const int32_t *rem, int nrem, int32_t w,
                        int32_t root) {
    if (nsub + 1 == J->k) {  /* w completes the set: V'_ext would never be used */
        sub[nsub] = w;
        credit_set(J->g, J->cl, J->k, sub, J->out);
        return 1;
    }
    int32_t cur[4096];
    int64_t deg = J->g->uptr[w + 1] - J->g->uptr[w];
    int64_t cap = nrem + deg;
    int32_t *heap_buf = cap <= 4096 ? NULL : malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *ne = heap_buf ? heap_buf : cur;
    int nn = 0;
    for (int i = 0; i < nrem; i++) ne[nn++] = rem[i];
    for (int64_t e = J->g->uptr[w]; e < J->g->uptr[w + 1]; e++) {
        int32_t u = J->g->uadj[e];
        if (okey(J, u) <= okey(J, root)) continue;
        int excl = 1;
        for (int s = 0; s < nsub && excl; s++)
            if (u == sub[s] || u_adjacent(J->g, u, sub[s])) excl = 0;
        if (excl) ne[nn++] = u;
    }
    sub[nsub] = w;
    int64_t found = esu_extend(J, sub, nsub + 1, ne, nn, root);
    free(heap_buf);
    return found;
}

static int64_t esu_extend(const esu_job *J, int32_t *sub, int nsub, const int32_t *ext, int next, int32_t root) {
    if (nsub == J->k) {
        credit_set(J->g, J->cl, J->k, sub, J->out);
        return 1;
    }
    int64_t found = 0;
    /* V_ext is consumed one element w at a time, from its end */
    for (int nrem = next - 1; nrem >= 0; nrem--) found += esu_take(J, sub, nsub, ext, nrem, ext[nrem], root);
    return found;
}

/*
 * Threads take tasks (root v, j): the sub-tree of ESU in which the first
 * vertex added to {v} is the j-th element of v's initial extension set
 * (elements j+1, ... having been consumed already).  These sub-trees
 * partition v's sets, so one heavy root is shared among threads.
 */
static void *esu_worker(void *arg) {
    esu_job *J = (esu_job *)arg;
    int64_t local = 0;
    int32_t sub[MAXK];
    const int64_t ntasks = J->eoff[J->nroots];
    for (;;) {
        int64_t t = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (t >= ntasks) break;
        const int64_t i = J->troot[t];
        const int32_t v = J->roots[i];
        const int32_t *ext = J->eall + J->eoff[i];
        const int j = (int)(t - J->eoff[i]);
        sub[0] = v;
        local += esu_take(J, sub, 1, ext, j, ext[j], v);
    }
    __atomic_fetch_add(&J->found, local, __ATOMIC_RELAXED);
    return NULL;
}

static int load_classes_mode(int k, int undirected, int per_edge, oclasses *cl) {
    cl->k = k;
    cl->undirected = undirected;
    cl->per_edge = per_edge;
    cl->nc = undirected ? oracle_classes_undirected(k, cl->canon, NULL, 256) : oracle_classes(k, 1, cl->canon, NULL, 256);
    return cl->nc > 0 ? 0 : -1;
}

static int load_classes(int k, oclasses *cl) { return load_classes_mode(k, 0, 0, cl); }

/*
 * Per-vertex counts out[v * C_k + c] (overwritten) over all connected
 * k-sets whose minimum-key vertex has key in [key_lo, key_hi).  With
 * key == NULL the key is the vertex id and every set is counted
 * (key_lo/key_hi ignored).  Returns the number of sets, or < 0 on error.
 */
static int64_t count_esu_impl(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                              int undirected, int per_edge, const int32_t *key, int32_t key_lo, int32_t key_hi,
                              const uint8_t *root_mask, int nthreads, uint64_t *out);

int64_t oracle_count_esu(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                         const int32_t *key, int32_t key_lo, int32_t key_hi, int nthreads,
                         uint64_t *out) {
    return count_esu_impl(n, m, src, dst, k, 0, 0, key, key_lo, key_hi, NULL, nthreads, out);
}

/*
 * The undirected and per-edge variants (and both): `out` has n rows
 * (per_edge = 0) or one row per edge of G_U (per_edge = 1, rows in the
 * order of oracle_edges), and C columns of the class list of the mode
 * (oracle_classes or oracle_classes_undirected).  root_mask as in
 * oracle_count_esu_masked (with key), or NULL for every root.
 */
int64_t oracle_count_mode(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k, int undirected,
                          int per_edge, const int32_t *key, const uint8_t *root_mask, int nthreads, uint64_t *out) {
    if (root_mask && !key) return -1;
    return count_esu_impl(n, m, src, dst, k, undirected ? 1 : 0, per_edge ? 1 : 0, key, 0, 0, root_mask, nthreads,
                          out);
}

/* Edges {u, v} of G_U with u < v (original ids) in (u, v) order: the rows of
 * the per-edge output.  Fills u_out/v_out when not NULL; returns the count. */
int64_t oracle_edges(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *u_out, int32_t *v_out) {
    ograph g;
    int rc = ograph_build(&g, n, m, src, dst);
    if (rc) return rc;
    const int64_t ne = g.erow[n];
    for (int32_t u = 0; u < n; u++)
        for (int64_t e = g.eup[u]; e < g.uptr[u + 1]; e++) {
            const int64_t row = g.erow[u] + (e - g.eup[u]);
            if (u_out) u_out[row] = u;
            if (v_out) v_out[row] = g.uadj[e];
        }
    ograph_free(&g);
    return ne;
}

/*
 * As oracle_count_esu with a key, but the roots are the vertices v with
 * root_mask[v] != 0 (any set of keys, e.g. several key ranges at once):
 * counts over the connected k-sets whose minimum-key vertex is such a root.
 */
int64_t oracle_count_esu_masked(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                                const int32_t *key, const uint8_t *root_mask, int nthreads, uint64_t *out) {
    if (!key || !root_mask) return -1;
    return count_esu_impl(n, m, src, dst, k, 0, 0, key, 0, 0, root_mask, nthreads, out);
}

static int64_t count_esu_impl(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                              int undirected, int per_edge, const int32_t *key, int32_t key_lo, int32_t key_hi,
                              const uint8_t *root_mask, int nthreads, uint64_t *out) {
    if (k != 3 && k != 4) return -1;
    if (n < 0 || m < 0) return -1;
    oclasses cl;
    if (load_classes_mode(k, undirected, per_edge, &cl)) return -1;
    ograph g;
    int rc = ograph_build(&g, n, m, src, dst);
    if (rc) return rc == -2 ? -2 : -1;
    const size_t rows = per_edge ? (size_t)g.erow[n] : (size_t)n;
    memset(out, 0, sizeof(uint64_t) * rows * (size_t)cl.nc);
    esu_job J;
    memset(&J, 0, sizeof J);
    J.g = &g; J.cl = &cl; J.k = k; J.key = key; J.out = out;
    J.roots = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t v = 0; v < n; v++)
        if (!key || (root_mask ? root_mask[v] != 0 : (key[v] >= key_lo && key[v] < key_hi))) J.roots[J.nroots++] = v;
    /* initial extension sets: the neighbours of each root with a larger key */
    J.eoff = malloc(sizeof(int64_t) * (size_t)(J.nroots + 1));
    J.eoff[0] = 0;
    for (int64_t i = 0; i < J.nroots; i++) {
        const int32_t v = J.roots[i];
        int64_t c = 0;
        for (int64_t e = g.uptr[v]; e < g.uptr[v + 1]; e++) c += okey(&J, g.uadj[e]) > okey(&J, v);
        J.eoff[i + 1] = J.eoff[i] + c;
    }
    const int64_t ntasks = J.eoff[J.nroots];
    J.eall = malloc(sizeof(int32_t) * (size_t)(ntasks > 0 ? ntasks : 1));
    J.troot = malloc(sizeof(int32_t) * (size_t)(ntasks > 0 ? ntasks : 1));
    for (int64_t i = 0; i < J.nroots; i++) {
        const int32_t v = J.roots[i];
        int64_t o = J.eoff[i];
        for (int64_t e = g.uptr[v]; e < g.uptr[v + 1]; e++)
            if (okey(&J, g.uadj[e]) > okey(&J, v)) {
                J.eall[o] = g.uadj[e];
                J.troot[o++] = (int32_t)i;
            }
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, esu_worker, &J);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(J.roots);
    free(J.eoff);
    free(J.eall);
    free(J.troot);
    ograph_free(&g);
    return J.found;
}

/*
 * Brute force over every k-subset of the vertices (tiny graphs only): test
 * connectivity of the induced G_U directly, classify, credit.  An
 * enumeration that shares nothing with ESU, used to pin it.
 */
int64_t oracle_count_brute(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int k,
                           uint64_t *out) {
    if (k != 3 && k != 4) return -1;
    oclasses cl;
    if (load_classes(k, &cl)) return -1;
    memset(out, 0, sizeof(uint64_t) * (size_t)n * (size_t)cl.nc);
    ograph g;
    int rc = ograph_build(&g, n, m, src, dst);
    if (rc) return rc == -2 ? -2 : -1;
    int64_t found = 0;
    int32_t S[MAXK];
    for (int i = 0; i < k; i++) S[i] = i;
    if (n < k) { ograph_free(&g); return 0; }
    for (;;) {
        /* connectivity of S in G_U */
        int seen = 1, frontier = 1;
        while (frontier) {
            int nf = 0;
            for (int i = 0; i < k; i++)
                if (frontier >> i & 1)
                    for (int j = 0; j < k; j++)
                        if (!(seen >> j & 1) && (has_arc(&g, S[i], S[j]) || has_arc(&g, S[j], S[i]))) {
                            seen |= 1 << j; nf |= 1 << j;
                        }
            frontier = nf;
        }
        if (seen == (1 << k) - 1) { credit_set(&g, &cl, k, S, out); found++; }
        /* next combination */
        int i = k - 1;
        while (i >= 0 && S[i] == n - k + i) i--;
        if (i < 0) break;
        S[i]++;
        for (int j = i + 1; j < k; j++) S[j] = S[j - 1] + 1;
    }
    ograph_free(&g);
    return found;
}

/*
 * The paper's vertex order ("Vertex ordering and splitting over the GPU";
 * Novelty, divide and conquer): highest undirected degree first.  Equal
 * degrees are broken by original id (the paper leaves the tie arbitrary).
 * rank_out[v] = position of v in that order.  Returns 0 or < 0.
 */
static const int64_t *g_sort_deg;
static int cmp_by_degree(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_sort_deg[x] != g_sort_deg[y]) return g_sort_deg[x] > g_sort_deg[y] ? -1 : 1;
    return (x > y) - (x < y);
}

int oracle_degree_rank(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t *rank_out) {
    ograph g;
    int rc = ograph_build(&g, n, m, src, dst);
    if (rc) return rc;
    int64_t *deg = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *ord = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t v = 0; v < n; v++) { deg[v] = g.uptr[v + 1] - g.uptr[v]; ord[v] = v; }
    g_sort_deg = deg;   /* single-threaded helper */
    qsort(ord, (size_t)n, sizeof(int32_t), cmp_by_degree);
    for (int32_t i = 0; i < n; i++) rank_out[ord[i]] = i;
    free(deg); free(ord);
    ograph_free(&g);
    return 0;
}
