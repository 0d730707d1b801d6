/*
 * sb_oracle.c -- plain, slow CPU oracle for graphBpp and graphL.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this file: only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant generator with the CUDA library; every routine below is written
 * from the paper's definitions, one step at a time, with no blocking, fusion
 * or reordering beyond what the definition states.
 *
 * Paper: Shebaro & Tesic, "Scaling Frustration Index and Corresponding
 * Balanced State Discovery for Real Signed Graphs" (arXiv 2311.00869).
 *
 *   Sec. 2, Def. "Signed graph"      frustration, balanced state, cloud
 *   Sec. 2, Harary theorem item 4    a balanced state is a vertex bipartition
 *   Sec. 3, Alg. 1 + Eq. 1           graphBpp: k trees -> states -> counts -> cloud
 *   Appendix, Alg. "graphB+"         flip each non-tree edge whose fundamental
 *                                    cycle is negative
 *   Sec. 4, Eq. 2-4 + Alg. 2         graphL loss, gradient, descent, rounding
 *   Appendix "Implementation"        input cleaning (duplicates, self-loops,
 *                                    inconsistencies, invalid signs), LCC
 *   Appendix, tree samplers          Kruskal's algorithm with random edge weights
 *
 * Readings taken where the paper is silent (each one is also listed in the
 * design notes):
 *   - which BFS tree is "tree t": the randomized BFS tree whose parent rule is
 *     the hashed argmin defined in or_tree() below (parity unpinned against the
 *     authors' queue order: they publish no code and no tree);
 *   - a state is keyed by its canonical vertex labelling (vertex 0 on the +1
 *     side), which is a bijection with the edge-sign string of Alg. 1 for a
 *     connected graph;
 *   - graphL: each undirected edge enters the loss once; theta = +1 iff
 *     Gamma >= 0; after each step a column whose largest magnitude reached
 *     2^renorm_log2 is scaled by 2^-renorm_log2 (exact in binary floating
 *     point, so every sign is unchanged).
 *
 * Hash primitives (both published, written here from their definitions):
 *   mix64  : the SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014)
 *   fmix32 : the MurmurHash3 32-bit finaliser (Appleby)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* status codes: numerically equal to the library's, defined here on their own */
#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-3)
#define OR_ERR_SELF_LOOP (-4)
#define OR_ERR_BAD_SIGN (-5)
#define OR_ERR_INCONSISTENT (-6)
#define OR_ERR_DUPLICATE (-7)
#define OR_ERR_DISCONNECTED (-8)
#define OR_ERR_RANGE (-9)

#define OR_LOAD_LCC 1u
#define OR_LOAD_MERGE_DUP 2u

/* ------------------------------------------------------------------ hashes */

uint64_t or_mix64(uint64_t z)
{
    z = z ^ (z >> 30);
    z = z * 0xBF58476D1CE4E5B9ULL;
    z = z ^ (z >> 27);
    z = z * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return z;
}

uint32_t or_fmix32(uint32_t h)
{
    h = h ^ (h >> 16);
    h = h * 0x85EBCA6Bu;
    h = h ^ (h >> 13);
    h = h * 0xC2B2AE35u;
    h = h ^ (h >> 16);
    return h;
}

#define OR_GOLDEN 0x9E3779B97F4A7C15ULL

/* seed key S */
uint64_t or_seed_key(uint64_t seed) { return or_mix64(seed + OR_GOLDEN); }

/* tree key K_t for global tree index t */
uint64_t or_tree_key(uint64_t seed, int64_t t)
{
    uint64_t S = or_seed_key(seed);
    return or_mix64(S + ((uint64_t)t + 1u) * OR_GOLDEN);
}

/* root of tree t: multiply-shift range reduction of the key's high word */
int64_t or_tree_root(uint64_t seed, int64_t t, int64_t n)
{
    uint64_t K = or_tree_key(seed, t);
    return (int64_t)(((K >> 32) * (uint64_t)n) >> 32);
}

/* per-vertex salt of the child endpoint */
uint32_t or_child_salt(uint64_t seed, int64_t v)
{
    uint64_t S = or_seed_key(seed);
    return (uint32_t)(or_mix64((uint64_t)v ^ S ^ 0xD1B54A32D192ED03ULL) >> 32);
}

/* packed parent key of candidate u for child v in tree t; the smaller wins */
uint64_t or_parent_key(uint64_t seed, int64_t t, int64_t u, int64_t v)
{
    uint32_t a = (uint32_t)or_tree_key(seed, t);
    uint32_t y = or_child_salt(seed, v);
    uint32_t h = or_fmix32(((uint32_t)u ^ y) + a);
    return ((uint64_t)h << 32) | (uint64_t)(uint32_t)u;
}

/* weight of vertex v in the state hash */
uint64_t or_vertex_weight(int64_t v) { return or_mix64((uint64_t)v ^ 0x6A09E667F3BCC909ULL); }

/* ------------------------------------------------------------ graph ingest */

typedef struct { int32_t a, b; int8_t s; int64_t idx; } or_edge;

static int or_edge_cmp(const void* x, const void* y)
{
    const or_edge* p = (const or_edge*)x;
    const or_edge* q = (const or_edge*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->s != q->s) return p->s < q->s ? -1 : 1;
    return 0;
}

static int64_t or_find(int64_t* par, int64_t x)
{
    while (par[x] != x) x = par[x];
    return x;
}

/*
 * Cleans a COO signed edge list the way the appendix "Implementation"
 * paragraph describes (self-loops, invalid signs, inconsistencies and
 * duplicates) and keeps the largest connected component (Sec. 5 datasets use
 * the LCC).  Readings:
 *   - the first offending input edge (lowest index) decides the error among
 *     range / self-loop / sign errors, checked in that order per edge;
 *   - an unordered pair present with both signs is OR_ERR_INCONSISTENT, even
 *     with MERGE_DUP; otherwise a repeated pair (either orientation) is
 *     OR_ERR_DUPLICATE unless MERGE_DUP is set, in which case it is merged;
 *   - the largest component is the one with most vertices; a tie goes to the
 *     component holding the smallest vertex id; without OR_LOAD_LCC a graph
 *     with more than one component is OR_ERR_DISCONNECTED;
 *   - surviving vertices are renumbered 0.. in increasing original id.
 * Outputs: edges (eu < ev) in lexicographic order, eneg = 1 for a negative
 * edge, vmap_out[old] = new id or -1 (nullable).  Arrays eu/ev/eneg hold m.
 */
int or_clean_graph(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const int8_t* sign,
                   uint32_t flags, int64_t* n_out, int64_t* m_out, int32_t* eu, int32_t* ev, int8_t* eneg,
                   int32_t* vmap_out)
{
    if (n < 1 || m < 0 || n > 2147483647LL) return OR_ERR_ARG;
    for (int64_t i = 0; i < m; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return OR_ERR_RANGE;
        if (src[i] == dst[i]) return OR_ERR_SELF_LOOP;
        if (sign[i] != 1 && sign[i] != -1) return OR_ERR_BAD_SIGN;
    }
    or_edge* E = (or_edge*)malloc(sizeof(or_edge) * (size_t)(m > 0 ? m : 1));
    if (!E) return OR_ERR_OOM;
    for (int64_t i = 0; i < m; i++) {
        int32_t a = src[i], b = dst[i];
        E[i].a = a < b ? a : b;
        E[i].b = a < b ? b : a;
        E[i].s = sign[i];
        E[i].idx = i;
    }
    qsort(E, (size_t)m, sizeof(or_edge), or_edge_cmp);
    /* inconsistency: the same pair with both signs */
    for (int64_t i = 1; i < m; i++)
        if (E[i].a == E[i - 1].a && E[i].b == E[i - 1].b && E[i].s != E[i - 1].s) {
            free(E);
            return OR_ERR_INCONSISTENT;
        }
    /* duplicates */
    int64_t k = 0;
    for (int64_t i = 0; i < m; i++) {
        if (k > 0 && E[i].a == E[k - 1].a && E[i].b == E[k - 1].b) {
            if (!(flags & OR_LOAD_MERGE_DUP)) {
                free(E);
                return OR_ERR_DUPLICATE;
            }
            continue;
        }
        E[k++] = E[i];
    }
    /* connected components (union-find, plain) */
    int64_t* par = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* size = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    int64_t* minid = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!par || !size || !minid) {
        free(E); free(par); free(size); free(minid);
        return OR_ERR_OOM;
    }
    for (int64_t v = 0; v < n; v++) par[v] = v;
    for (int64_t i = 0; i < k; i++) {
        int64_t x = or_find(par, E[i].a), y = or_find(par, E[i].b);
        if (x != y) {
            if (x < y) par[y] = x; else par[x] = y;
        }
    }
    for (int64_t v = 0; v < n; v++) minid[v] = -1;
    int64_t ncomp = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t r = or_find(par, v);
        if (size[r] == 0) { ncomp++; minid[r] = v; }
        size[r]++;
    }
    if (ncomp > 1 && !(flags & OR_LOAD_LCC)) {
        free(E); free(par); free(size); free(minid);
        return OR_ERR_DISCONNECTED;
    }
    int64_t best = -1;
    for (int64_t v = 0; v < n; v++) {
        if (size[v] == 0) continue;
        if (best < 0 || size[v] > size[best] || (size[v] == size[best] && minid[v] < minid[best])) best = v;
    }
    int64_t nn = 0;
    for (int64_t v = 0; v < n; v++) {
        int32_t nv = -1;
        if (or_find(par, v) == best) nv = (int32_t)(nn++);
        if (vmap_out) vmap_out[v] = nv;
        minid[v] = nv;   /* reuse as old -> new map */
    }
    int64_t mm = 0;
    for (int64_t i = 0; i < k; i++) {
        int64_t na = minid[E[i].a], nb = minid[E[i].b];
        if (na < 0) continue;
        eu[mm] = (int32_t)na;
        ev[mm] = (int32_t)nb;
        eneg[mm] = (int8_t)(E[i].s < 0 ? 1 : 0);
        mm++;
    }
    *n_out = nn;
    *m_out = mm;
    free(E); free(par); free(size); free(minid);
    return OR_OK;
}

/*
 * CSR of the undirected graph (Sec. 8 complexity paragraph: the authors use
 * CSR).  Each edge appears in both rows; rows hold neighbours in increasing
 * id order; colneg marks a negative edge.  rowptr has n+1 entries.
 */
int or_build_csr(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const int8_t* eneg,
                 int64_t* rowptr, int32_t* col, int8_t* colneg)
{
    for (int64_t v = 0; v <= n; v++) rowptr[v] = 0;
    for (int64_t i = 0; i < m; i++) {
        rowptr[eu[i] + 1]++;
        rowptr[ev[i] + 1]++;
    }
    for (int64_t v = 0; v < n; v++) rowptr[v + 1] += rowptr[v];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) return OR_ERR_OOM;
    for (int64_t v = 0; v < n; v++) fill[v] = rowptr[v];
    /* insert in increasing neighbour order: lower neighbours come from edges
       (x, v) with x < v, upper ones from (v, y); two sweeps keep rows sorted */
    for (int64_t i = 0; i < m; i++) { /* edges sorted by (eu, ev): row ev gets eu ascending */
        int64_t v = ev[i];
        col[fill[v]] = eu[i];
        colneg[fill[v]] = eneg[i];
        fill[v]++;
    }
    for (int64_t i = 0; i < m; i++) { /* row eu gets ev ascending */
        int64_t v = eu[i];
        col[fill[v]] = ev[i];
        colneg[fill[v]] = eneg[i];
        fill[v]++;
    }
    free(fill);
    return OR_OK;
}

/* ---------------------------------------------------------------- graphBpp */

/*
 * One randomized BFS spanning tree and its balanced state (Algorithm 1 via
 * the appendix graphB+ algorithm, restated through Harary's bipartition).
 *
 * Tree t (global index t, seed `seed`):
 *   root r_t = or_tree_root(seed, t, n);
 *   levels = BFS distances from r_t;
 *   for v != r_t, parent p_t(v) = the neighbour u with level(u) = level(v)-1
 *   whose or_parent_key(seed, t, u, v) is smallest.
 * State: lab(r_t) = 0 and lab(v) = lab(p_t(v)) XOR neg(p_t(v), v), i.e. the
 * parity of negative tree edges on the root path.  Every tree edge is then
 * satisfied, and a non-tree edge (u,v) is frustrated exactly when its
 * fundamental cycle is negative, which is the edge graphB+ flips.
 * Canonical form: clab(v) = lab(v) XOR lab(0) (vertex 0 on the +1 side).
 *
 * Outputs (each nullable): parent[n] (-1 at the root), clab[n] (0/1),
 * level[n].  Returns the root, or a negative status.
 */
int64_t or_tree(int64_t n, const int64_t* rowptr, const int32_t* col, const int8_t* colneg, uint64_t seed,
                int64_t t, int32_t* parent_out, uint8_t* clab_out, int32_t* level_out)
{
    int32_t* level = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t* lab = (uint8_t*)malloc((size_t)n);
    if (!level || !queue || !parent || !lab) {
        free(level); free(queue); free(parent); free(lab);
        return OR_ERR_OOM;
    }
    int64_t root = or_tree_root(seed, t, n);
    for (int64_t v = 0; v < n; v++) level[v] = -1;
    int64_t head = 0, tail = 0;
    level[root] = 0;
    queue[tail++] = (int32_t)root;
    while (head < tail) {
        int32_t x = queue[head++];
        for (int64_t j = rowptr[x]; j < rowptr[x + 1]; j++) {
            int32_t y = col[j];
            if (level[y] < 0) {
                level[y] = level[x] + 1;
                queue[tail++] = y;
            }
        }
    }
    /* parent: smallest key among the neighbours one level up */
    for (int64_t v = 0; v < n; v++) {
        parent[v] = -1;
        if (v == root || level[v] < 0) continue;
        uint64_t best = UINT64_MAX;
        for (int64_t j = rowptr[v]; j < rowptr[v + 1]; j++) {
            int32_t u = col[j];
            if (level[u] != level[v] - 1) continue;
            uint64_t key = or_parent_key(seed, t, u, v);
            if (key < best) {
                best = key;
                parent[v] = u;
            }
        }
    }
    /* labels along the BFS order: a parent is always dequeued before its child */
    for (int64_t i = 0; i < tail; i++) {
        int32_t v = queue[i];
        if (v == root) {
            lab[v] = 0;
            continue;
        }
        int32_t p = parent[v];
        int8_t neg = 0;
        for (int64_t j = rowptr[v]; j < rowptr[v + 1]; j++)
            if (col[j] == p) neg = colneg[j];
        lab[v] = (uint8_t)(lab[p] ^ (uint8_t)neg);
    }
    uint8_t flip = lab[0];
    for (int64_t v = 0; v < n; v++) {
        if (clab_out) clab_out[v] = (uint8_t)(lab[v] ^ flip);
        if (parent_out) parent_out[v] = parent[v];
        if (level_out) level_out[v] = level[v];
    }
    free(level); free(queue); free(parent); free(lab);
    return root;
}

/* Algorithm 1: number of edges whose sign differs between the graph and
   the balanced state, i.e. edges with lab(u) XOR lab(v) XOR neg = 1. */
int64_t or_frustration(int64_t m, const int32_t* eu, const int32_t* ev, const int8_t* eneg, const uint8_t* clab)
{
    int64_t s = 0;
    for (int64_t i = 0; i < m; i++) s += (clab[eu[i]] ^ clab[ev[i]] ^ (uint8_t)eneg[i]) & 1;
    return s;
}

/* state hash: sum of vertex weights over the vertices labelled 1, mod 2^64 */
uint64_t or_state_hash(int64_t n, const uint8_t* clab)
{
    uint64_t h = 0;
    for (int64_t v = 0; v < n; v++)
        if (clab[v]) h += or_vertex_weight(v);
    return h;
}

/*
 * Trees [t0, t0+K) in order: canonical labels (K x n bytes, nullable),
 * parents (K x n, nullable), counts S_t and hashes H_t (nullable).
 */
int or_sample(int64_t n, const int64_t* rowptr, const int32_t* col, const int8_t* colneg, int64_t m,
              const int32_t* eu, const int32_t* ev, const int8_t* eneg, uint64_t seed, int64_t t0, int64_t K,
              uint8_t* clab_out, int32_t* parent_out, int32_t* counts_out, uint64_t* hashes_out)
{
    uint8_t* lab = (uint8_t*)malloc((size_t)n);
    if (!lab) return OR_ERR_OOM;
    for (int64_t i = 0; i < K; i++) {
        int64_t r = or_tree(n, rowptr, col, colneg, seed, t0 + i, parent_out ? parent_out + i * n : NULL, lab, NULL);
        if (r < 0) {
            free(lab);
            return (int)r;
        }
        if (clab_out) memcpy(clab_out + i * n, lab, (size_t)n);
        if (counts_out) counts_out[i] = (int32_t)or_frustration(m, eu, ev, eneg, lab);
        if (hashes_out) hashes_out[i] = or_state_hash(n, lab);
    }
    free(lab);
    return OR_OK;
}

/* ------------------------------------------------ randomized Kruskal trees */

/* weight of the cleaned edge (u, v), u < v, in Kruskal tree t */
uint64_t or_mst_weight(uint64_t seed, int64_t t, int64_t u, int64_t v)
{
    uint64_t pair = ((uint64_t)(uint32_t)u << 32) | (uint64_t)(uint32_t)v;
    return or_mix64(pair ^ or_tree_key(seed, t));
}

typedef struct { uint64_t w; int64_t e; } or_wedge;

static int or_wedge_cmp(const void* x, const void* y)
{
    uint64_t a = ((const or_wedge*)x)->w, b = ((const or_wedge*)y)->w;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* union-find root with path halving */
static int64_t or_find_halve(int64_t* par, int64_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

/*
 * Randomized Kruskal tree t (appendix, tree samplers: Kruskal's algorithm
 * with random edge weights drawn afresh for every tree).  Reading: the weight
 * of edge (u, v) in tree t is or_mst_weight(seed, t, u, v).  mix64 is a
 * bijection on 64-bit words and the packed pair is injective, so one tree's
 * weights are all distinct and its minimum spanning tree is unique (Prim's
 * algorithm with the same weights finds the same tree).
 * Steps, as Kruskal's algorithm states them: sort the edges by weight, then
 * keep each edge in that order whose endpoints are still in different
 * union-find sets, and unite the sets.
 * State: the parity labelling of the tree, grown from vertex 0 with
 * lab(0) = 0 and lab(y) = lab(x) XOR neg(x, y) along tree edges, so it is
 * already canonical (vertex 0 on the +1 side).
 * Outputs (nullable): in_tree[m] (1 for a tree edge, edge order of eu/ev),
 * clab[n].  Returns the number of tree edges, or a negative status.
 */
int64_t or_mst_tree(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const int8_t* eneg, uint64_t seed,
                    int64_t t, uint8_t* in_tree_out, uint8_t* clab_out)
{
    or_wedge* order = (or_wedge*)malloc(sizeof(or_wedge) * (size_t)(m > 0 ? m : 1));
    int64_t* set = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    uint8_t* keep = (uint8_t*)calloc((size_t)(m > 0 ? m : 1), 1);
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * n + 2));
    int8_t* adjneg = (int8_t*)malloc((size_t)(2 * n + 2));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* lab = (uint8_t*)calloc((size_t)n, 1);
    if (!order || !set || !keep || !deg || !adj || !adjneg || !queue || !seen || !lab) {
        free(order); free(set); free(keep); free(deg); free(adj); free(adjneg); free(queue); free(seen); free(lab);
        return OR_ERR_OOM;
    }
    for (int64_t e = 0; e < m; e++) {
        order[e].w = or_mst_weight(seed, t, eu[e], ev[e]);
        order[e].e = e;
    }
    qsort(order, (size_t)m, sizeof(or_wedge), or_wedge_cmp);
    for (int64_t v = 0; v < n; v++) set[v] = v;
    int64_t kept = 0;
    for (int64_t i = 0; i < m && kept < n - 1; i++) {
        int64_t e = order[i].e;
        int64_t a = or_find_halve(set, eu[e]), b = or_find_halve(set, ev[e]);
        if (a == b) continue;
        set[a] = b;
        keep[e] = 1;
        kept++;
    }
    /* tree adjacency (CSR over the kept edges), then BFS from vertex 0 */
    for (int64_t e = 0; e < m; e++)
        if (keep[e]) {
            deg[eu[e] + 1]++;
            deg[ev[e] + 1]++;
        }
    for (int64_t v = 0; v < n; v++) deg[v + 1] += deg[v];
    for (int64_t e = 0; e < m; e++)
        if (keep[e]) {
            adj[deg[eu[e]]] = ev[e];
            adjneg[deg[eu[e]]++] = eneg[e];
            adj[deg[ev[e]]] = eu[e];
            adjneg[deg[ev[e]]++] = eneg[e];
        }
    for (int64_t v = n; v > 0; v--) deg[v] = deg[v - 1];
    deg[0] = 0;
    int64_t head = 0, tail = 0;
    if (n > 0) {
        queue[tail++] = 0;
        seen[0] = 1;
    }
    while (head < tail) {
        int32_t x = queue[head++];
        for (int64_t j = deg[x]; j < deg[x + 1]; j++) {
            int32_t y = adj[j];
            if (seen[y]) continue;
            seen[y] = 1;
            lab[y] = (uint8_t)(lab[x] ^ (uint8_t)adjneg[j]);
            queue[tail++] = y;
        }
    }
    if (in_tree_out) memcpy(in_tree_out, keep, (size_t)m);
    if (clab_out) memcpy(clab_out, lab, (size_t)n);
    free(order); free(set); free(keep); free(deg); free(adj); free(adjneg); free(queue); free(seen); free(lab);
    return kept;
}

/* Kruskal trees [t0, t0+K): in_tree (K x m), canonical labels (K x n),
   counts S_t and hashes H_t, each nullable. */
int or_mst_sample(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const int8_t* eneg, uint64_t seed,
                  int64_t t0, int64_t K, uint8_t* in_tree_out, uint8_t* clab_out, int32_t* counts_out,
                  uint64_t* hashes_out)
{
    uint8_t* lab = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    if (!lab) return OR_ERR_OOM;
    for (int64_t i = 0; i < K; i++) {
        int64_t r = or_mst_tree(n, m, eu, ev, eneg, seed, t0 + i, in_tree_out ? in_tree_out + i * m : NULL, lab);
        if (r < 0) {
            free(lab);
            return (int)r;
        }
        if (clab_out) memcpy(clab_out + i * n, lab, (size_t)n);
        if (counts_out) counts_out[i] = (int32_t)or_frustration(m, eu, ev, eneg, lab);
        if (hashes_out) hashes_out[i] = or_state_hash(n, lab);
    }
    free(lab);
    return OR_OK;
}

/*
 * Frustration cloud (Algorithm 1 and Eq. 1): distinct states among K
 * trees, keyed by the full canonical labelling.  Entries come out in order of
 * first appearance; for each: first tree index (t0 + i), count C, switch
 * count S, state hash H.  Returns the number of distinct states.  Scratch is
 * O(K); comparison is plain memcmp over the K x n label matrix.
 */
static const uint8_t* or_cmp_base;
static int64_t or_cmp_n;
static int or_state_cmp(const void* x, const void* y)
{
    int64_t i = *(const int64_t*)x, j = *(const int64_t*)y;
    int c = memcmp(or_cmp_base + i * or_cmp_n, or_cmp_base + j * or_cmp_n, (size_t)or_cmp_n);
    if (c != 0) return c;
    return i < j ? -1 : (i > j ? 1 : 0);
}

int64_t or_cloud(int64_t n, int64_t K, int64_t t0, const uint8_t* clab, const int32_t* counts,
                 int64_t* first_out, int32_t* count_out, int32_t* S_out, uint64_t* H_out)
{
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
    int64_t* rep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
    int32_t* cnt = (int32_t*)calloc((size_t)(K > 0 ? K : 1), sizeof(int32_t));
    if (!idx || !rep || !cnt) {
        free(idx); free(rep); free(cnt);
        return OR_ERR_OOM;
    }
    for (int64_t i = 0; i < K; i++) idx[i] = i;
    or_cmp_base = clab;
    or_cmp_n = n;
    qsort(idx, (size_t)K, sizeof(int64_t), or_state_cmp);
    /* rep[i] = first tree holding the same state as tree i */
    for (int64_t a = 0; a < K;) {
        int64_t b = a;
        while (b < K && memcmp(clab + idx[a] * n, clab + idx[b] * n, (size_t)n) == 0) b++;
        for (int64_t c = a; c < b; c++) rep[idx[c]] = idx[a];
        a = b;
    }
    for (int64_t i = 0; i < K; i++) cnt[rep[i]]++;
    int64_t ns = 0;
    for (int64_t i = 0; i < K; i++) {
        if (rep[i] != i) continue;
        first_out[ns] = t0 + i;
        count_out[ns] = cnt[i];
        S_out[ns] = counts[i];
        H_out[ns] = or_state_hash(n, clab + i * n);
        ns++;
    }
    free(idx); free(rep); free(cnt);
    return ns;
}

/*
 * Frustration cloud of the scalable variant (appendix "Scaling graphBpp for
 * Large Signed Graphs", the algorithm alg-scale): at most fmax states are
 * kept.  Trees are taken in order.  The first tree's state is stored.  After
 * that a tree is used only when its S is below the largest stored S: a state
 * already stored gets its count raised; a new state is appended while fewer
 * than fmax are stored, and otherwise takes the place of the stored state
 * with the largest S (the printed argmin would throw away the best state, so
 * it is read as argmax; among equal S the lowest slot goes).  A stored state's
 * first tree is the tree that stored it.  Output: the stored states ordered by
 * that tree.  Returns their number.
 */
int64_t or_cloud_bounded(int64_t n, int64_t K, int64_t t0, const uint8_t* clab, const int32_t* counts, int64_t fmax,
                         int64_t* first_out, int32_t* count_out, int32_t* S_out, uint64_t* H_out)
{
    if (fmax < 1) return OR_ERR_ARG;
    int64_t cap = fmax < K ? fmax : (K > 0 ? K : 1);
    int64_t* rep = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    if (!rep || !S || !cnt) {
        free(rep); free(S); free(cnt);
        return OR_ERR_OOM;
    }
    int64_t ns = 0;
    for (int64_t i = 0; i < K; i++) {
        if (ns == 0) {
            rep[0] = i;
            S[0] = counts[i];
            cnt[0] = 1;
            ns = 1;
            continue;
        }
        int32_t maxS = S[0];
        int64_t arg = 0;
        for (int64_t j = 1; j < ns; j++)
            if (S[j] > maxS) {
                maxS = S[j];
                arg = j;
            }
        if (!(counts[i] < maxS)) continue;
        int64_t found = -1;
        for (int64_t j = 0; j < ns && found < 0; j++)
            if (memcmp(clab + rep[j] * n, clab + i * n, (size_t)n) == 0) found = j;
        if (found >= 0) {
            cnt[found]++;
        } else {
            int64_t slot = ns < fmax ? ns++ : arg;
            rep[slot] = i;
            S[slot] = counts[i];
            cnt[slot] = 1;
        }
    }
    /* order of the storing tree (insertion sort: ns is small) */
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ns > 0 ? ns : 1));
    if (!ord) {
        free(rep); free(S); free(cnt);
        return OR_ERR_OOM;
    }
    for (int64_t j = 0; j < ns; j++) {
        int64_t k = j;
        while (k > 0 && rep[ord[k - 1]] > rep[j]) {
            ord[k] = ord[k - 1];
            k--;
        }
        ord[k] = j;
    }
    for (int64_t a = 0; a < ns; a++) {
        int64_t j = ord[a];
        first_out[a] = t0 + rep[j];
        count_out[a] = cnt[j];
        S_out[a] = S[j];
        H_out[a] = or_state_hash(n, clab + rep[j] * n);
    }
    free(ord); free(rep); free(S); free(cnt);
    return ns;
}

/* ------------------------------------------------------------------ graphL */

/*
 * Relaxed loss, Eq. 3: L_r = sum over undirected edges (1 - e_ij G_i G_j) / 2,
 * each edge once; and the discrete loss of Eq. 2 / Algorithm 2 with
 * theta = +1 when Gamma >= 0, else -1 (the rule of Alg. 2's final loop).
 * gamma is n x R row-major (vertex v, init r at gamma[v*R + r]).
 */
void or_graphl_loss_f64(int64_t m, const int32_t* eu, const int32_t* ev, const int8_t* eneg, const double* gamma,
                        int64_t R, double* loss_out, int64_t* F_out)
{
    for (int64_t r = 0; r < R; r++) {
        double L = 0.0;
        int64_t F = 0;
        for (int64_t i = 0; i < m; i++) {
            double e = eneg[i] ? -1.0 : 1.0;
            double gi = gamma[(int64_t)eu[i] * R + r], gj = gamma[(int64_t)ev[i] * R + r];
            L += (1.0 - e * gi * gj) / 2.0;
            double ti = gi >= 0.0 ? 1.0 : -1.0, tj = gj >= 0.0 ? 1.0 : -1.0;
            F += (int64_t)((1.0 - e * ti * tj) / 2.0);
        }
        loss_out[r] = L;
        if (F_out) F_out[r] = F;
    }
}

/* Eq. 4: dL/dG_v = -1/2 sum_{j in N(v)} e_vj G_j, times the upstream gout_r */
void or_graphl_grad_f64(int64_t n, const int64_t* rowptr, const int32_t* col, const int8_t* colneg,
                        const double* gamma, int64_t R, const double* gout, double* grad_out)
{
    for (int64_t v = 0; v < n; v++)
        for (int64_t r = 0; r < R; r++) {
            double s = 0.0;
            for (int64_t j = rowptr[v]; j < rowptr[v + 1]; j++) {
                double e = colneg[j] ? -1.0 : 1.0;
                s += e * gamma[(int64_t)col[j] * R + r];
            }
            grad_out[v * R + r] = -0.5 * gout[r] * s;
        }
}

void or_graphl_grad_f32(int64_t n, const int64_t* rowptr, const int32_t* col, const int8_t* colneg,
                        const float* gamma, int64_t R, const float* gout, float* grad_out)
{
    for (int64_t v = 0; v < n; v++)
        for (int64_t r = 0; r < R; r++) {
            float s = 0.0f;
            for (int64_t j = rowptr[v]; j < rowptr[v + 1]; j++) {
                float g = gamma[(int64_t)col[j] * R + r];
                s = colneg[j] ? s - g : s + g;
            }
            grad_out[v * R + r] = -0.5f * gout[r] * s;
        }
}

/*
 * Alg. 2 descent: `steps` updates G <- G - alpha * dL/dG (upstream gradient
 * 1 for every init), in place on gamma (n x R).  After each update, a column
 * whose largest |G| is >= 2^renorm_log2 is multiplied by 2^-renorm_log2 and
 * exps[r] grows by renorm_log2 (renorm_log2 = 0 disables this).  Scaling by a
 * power of two is exact, and the update is linear, so the signs are those of
 * the unscaled run.  F_trace (nullable, steps x R) receives the discrete loss
 * of Algorithm 2 evaluated before each update.
 */
int or_graphl_descent_f64(int64_t n, const int64_t* rowptr, const int32_t* col, const int8_t* colneg, int64_t m,
                          const int32_t* eu, const int32_t* ev, const int8_t* eneg, double* gamma, int64_t R,
                          double alpha, int64_t steps, int renorm_log2, int32_t* exps, int64_t* F_trace)
{
    double* grad = (double*)malloc(sizeof(double) * (size_t)(n * R > 0 ? n * R : 1));
    double* ones = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
    double* lossbuf = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
    if (!grad || !ones || !lossbuf) {
        free(grad); free(ones); free(lossbuf);
        return OR_ERR_OOM;
    }
    for (int64_t r = 0; r < R; r++) ones[r] = 1.0;
    double thr = ldexp(1.0, renorm_log2);
    double down = ldexp(1.0, -renorm_log2);
    for (int64_t s = 0; s < steps; s++) {
        if (F_trace) or_graphl_loss_f64(m, eu, ev, eneg, gamma, R, lossbuf, F_trace + s * R);
        or_graphl_grad_f64(n, rowptr, col, colneg, gamma, R, ones, grad);
        for (int64_t i = 0; i < n * R; i++) gamma[i] = gamma[i] - alpha * grad[i];
        if (renorm_log2 > 0)
            for (int64_t r = 0; r < R; r++) {
                double mx = 0.0;
                for (int64_t v = 0; v < n; v++) mx = fmax(mx, fabs(gamma[v * R + r]));
                if (mx >= thr) {
                    for (int64_t v = 0; v < n; v++) gamma[v * R + r] *= down;
                    exps[r] += renorm_log2;
                }
            }
    }
    free(grad); free(ones); free(lossbuf);
    return OR_OK;
}

/* same descent in float arithmetic, sequential neighbour sums */
int or_graphl_descent_f32(int64_t n, const int64_t* rowptr, const int32_t* col, const int8_t* colneg, float* gamma,
                          int64_t R, float alpha, int64_t steps, int renorm_log2, int32_t* exps)
{
    float* grad = (float*)malloc(sizeof(float) * (size_t)(n * R > 0 ? n * R : 1));
    float* ones = (float*)malloc(sizeof(float) * (size_t)(R > 0 ? R : 1));
    if (!grad || !ones) {
        free(grad); free(ones);
        return OR_ERR_OOM;
    }
    for (int64_t r = 0; r < R; r++) ones[r] = 1.0f;
    float thr = ldexpf(1.0f, renorm_log2);
    float down = ldexpf(1.0f, -renorm_log2);
    for (int64_t s = 0; s < steps; s++) {
        or_graphl_grad_f32(n, rowptr, col, colneg, gamma, R, ones, grad);
        for (int64_t i = 0; i < n * R; i++) gamma[i] = gamma[i] - alpha * grad[i];
        if (renorm_log2 > 0)
            for (int64_t r = 0; r < R; r++) {
                float mx = 0.0f;
                for (int64_t v = 0; v < n; v++) mx = fmaxf(mx, fabsf(gamma[v * R + r]));
                if (mx >= thr) {
                    for (int64_t v = 0; v < n; v++) gamma[v * R + r] *= down;
                    exps[r] += renorm_log2;
                }
            }
    }
    free(grad); free(ones);
    return OR_OK;
}

/*
 * Alg. 2 final loop: theta = +1 if Gamma >= 0 else -1, exact integer
 * frustration F_r, and the edges to flip (frustrated edges) as a byte mask
 * flip_out[r*m + i] (nullable).  gamma is float (n x R).
 */
void or_graphl_round_f32(int64_t m, const int32_t* eu, const int32_t* ev, const int8_t* eneg, const float* gamma,
                         int64_t R, int64_t* F_out, uint8_t* flip_out)
{
    for (int64_t r = 0; r < R; r++) {
        int64_t F = 0;
        for (int64_t i = 0; i < m; i++) {
            int ti = gamma[(int64_t)eu[i] * R + r] >= 0.0f ? 1 : -1;
            int tj = gamma[(int64_t)ev[i] * R + r] >= 0.0f ? 1 : -1;
            int e = eneg[i] ? -1 : 1;
            int fr = (1 - e * ti * tj) / 2;
            F += fr;
            if (flip_out) flip_out[r * m + i] = (uint8_t)fr;
        }
        F_out[r] = F;
    }
}
