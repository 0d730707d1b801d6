// sb_ingest.cu -- graph ingest on the device: validation, canonical sort,
// duplicate / inconsistency detection, largest connected component, CSR.
//
// Paper: the appendix "Implementation" paragraph (input cleaning: duplicates,
// self-loops, inconsistencies, invalid signs), the dataset tables (the LCC of
// each graph is used), and the complexity section (CSR storage).
#include <vector>

#include "sb_internal.cuh"

enum { ERRC_RANGE = 1, ERRC_SELF = 2, ERRC_SIGN = 3 };

static int bits_for(int64_t x)  // bits needed for values in [0, x]
{
    int b = 1;
    while (b < 63 && (x >> b) != 0) b++;
    return b;
}

// canonical key (lo << (nb+1)) | (hi << 1) | neg; errors keep the lowest edge index
__global__ void k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const int8_t* __restrict__ sign, int64_t n, int64_t m, int nb,
                           uint64_t* __restrict__ keys, unsigned long long* __restrict__ errkey)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[i], b = dst[i];
        int8_t s = sign[i];
        int code = 0;
        if (a < 0 || a >= n || b < 0 || b >= n) code = ERRC_RANGE;
        else if (a == b) code = ERRC_SELF;
        else if (s != 1 && s != -1) code = ERRC_SIGN;
        if (code) {
            atomicMin(errkey, ((unsigned long long)i << 8) | (unsigned long long)code);
            keys[i] = 0;
            continue;
        }
        uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
        keys[i] = (lo << (nb + 1)) | (hi << 1) | (uint64_t)(s < 0 ? 1 : 0);
    }
}

// head flags of distinct pairs; flags[0] |= 1 on inconsistency, 2 on duplicate
__global__ void k_heads(const uint64_t* __restrict__ keys, int64_t m, int32_t* __restrict__ head,
                        uint32_t* __restrict__ flags)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        int h = 1;
        if (i > 0) {
            uint64_t p = keys[i - 1];
            if ((p >> 1) == (k >> 1)) {
                h = 0;
                atomicOr(flags, (p & 1) != (k & 1) ? 1u : 2u);
            }
        }
        head[i] = h;
    }
}

__global__ void k_compact_keys(const uint64_t* __restrict__ keys, const int32_t* __restrict__ head,
                               const int32_t* __restrict__ pos, int64_t m, uint64_t* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (head[i]) out[pos[i]] = keys[i];
}

// ------------------------------------------------------------- union-find
__device__ __forceinline__ int32_t ld_par(const int32_t* p) { return *(volatile const int32_t*)p; }

// Parents only ever point to smaller ids, so every walk ends.
__device__ int32_t uf_find(int32_t* par, int32_t x)
{
    while (true) {
        int32_t p = ld_par(par + x);
        if (p == x) return x;
        int32_t gp = ld_par(par + p);
        if (gp == p) return p;
        par[x] = gp;  // path halving: gp is an ancestor of x
        x = gp;
    }
}

__global__ void k_uf_init(int32_t* par, int64_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        par[v] = (int32_t)v;
}

// hook the larger root under the smaller: the final root of a component is
// its smallest vertex id.  Retries are bounded; giving up flags an error.
__global__ void k_uf_hook(const uint64_t* __restrict__ keys, int64_t m, int nb, int32_t* par, uint32_t* flags)
{
    uint64_t mask = (1ull << nb) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        int32_t a = uf_find(par, (int32_t)(k >> (nb + 1)));
        int32_t b = uf_find(par, (int32_t)((k >> 1) & mask));
        int tries = 0;
        while (a != b) {
            if (a > b) {
                int32_t t = a;
                a = b;
                b = t;
            }
            int32_t old = atomicCAS(par + b, b, a);
            if (old == b) break;
            if (++tries > (1 << 20)) {
                atomicOr(flags, 4u);
                break;
            }
            a = uf_find(par, a);
            b = uf_find(par, b);
        }
    }
}

__global__ void k_uf_sizes(int32_t* par, int64_t n, int32_t* size)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = uf_find(par, (int32_t)v);
        par[v] = r;
        atomicAdd(size + r, 1);
    }
}

// largest component (ties: smallest root id) and number of components
__global__ void k_uf_best(const int32_t* __restrict__ size, int64_t n, unsigned long long* best,
                          unsigned long long* ncomp)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = size[v];
        if (s > 0) {
            atomicMax(best, ((unsigned long long)s << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)v));
            atomicAdd(ncomp, 1ull);
        }
    }
}

__global__ void k_keep_vertices(const int32_t* __restrict__ root, int64_t n, const unsigned long long* best,
                                int32_t* __restrict__ keep)
{
    int32_t br = (int32_t)(0xFFFFFFFFu - (uint32_t)(*best & 0xFFFFFFFFull));
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        keep[v] = root[v] == br ? 1 : 0;
}

__global__ void k_vmap(const int32_t* __restrict__ keep, const int32_t* __restrict__ newid, int64_t n,
                       int32_t* __restrict__ vmap)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        vmap[v] = keep[v] ? newid[v] : -1;
}

__global__ void k_keep_edges(const uint64_t* __restrict__ keys, int64_t m, int nb, const int32_t* __restrict__ keep,
                             int32_t* __restrict__ ekeep)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        ekeep[i] = keep[keys[i] >> (nb + 1)];
}

// final edge list + lower-triangle keys (v, u, neg) for the CSR transpose
__global__ void k_emit_edges(const uint64_t* __restrict__ keys, int64_t m, int nb, const int32_t* __restrict__ ekeep,
                             const int32_t* __restrict__ epos, const int32_t* __restrict__ newid, int nb2,
                             int2* __restrict__ edges, uint64_t* __restrict__ lkeys, int32_t* __restrict__ deg,
                             int32_t* __restrict__ updeg)
{
    uint64_t mask = (1ull << nb) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        if (!ekeep[i]) continue;
        uint64_t k = keys[i];
        int32_t u = newid[k >> (nb + 1)], v = newid[(k >> 1) & mask];
        uint32_t neg = (uint32_t)(k & 1);
        int32_t p = epos[i];
        edges[p] = make_int2(u, (int32_t)((uint32_t)v | (neg << 31)));
        lkeys[p] = ((uint64_t)v << (nb2 + 1)) | ((uint64_t)u << 1) | neg;
        atomicAdd(deg + u, 1);
        atomicAdd(deg + v, 1);
        atomicAdd(updeg + u, 1);
    }
}

// upper part of row u: neighbours v > u, in edge order (ascending v)
__global__ void k_fill_upper(const int2* __restrict__ edges, int64_t m, const int32_t* __restrict__ rowptr,
                             const int32_t* __restrict__ deg, const int32_t* __restrict__ updeg,
                             const int32_t* __restrict__ ufirst, int32_t* __restrict__ col)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int2 e = edges[i];
        int32_t u = e.x;
        int32_t low = deg[u] - updeg[u];
        col[rowptr[u] + low + (int32_t)(i - ufirst[u])] = e.y;
    }
}

// lower part of row v: neighbours u < v, from the (v, u)-sorted keys
__global__ void k_fill_lower(const uint64_t* __restrict__ lkeys, int64_t m, int nb2, const int32_t* __restrict__ rowptr,
                             const int32_t* __restrict__ lfirst, int32_t* __restrict__ col)
{
    uint64_t mask = (1ull << nb2) - 1ull;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = lkeys[p];
        int32_t v = (int32_t)(k >> (nb2 + 1));
        uint32_t u = (uint32_t)((k >> 1) & mask);
        uint32_t neg = (uint32_t)(k & 1);
        col[rowptr[v] + (int32_t)(p - lfirst[v])] = (int32_t)(u | (neg << 31));
    }
}

__global__ void k_lowdeg(const int32_t* __restrict__ deg, const int32_t* __restrict__ updeg, int64_t n,
                         int32_t* __restrict__ low)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        low[v] = deg[v] - updeg[v];
}

__global__ void k_chunks(const int32_t* __restrict__ deg, int64_t n, int chunk, int32_t* __restrict__ nch,
                         int32_t* __restrict__ split)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = deg[v];
        int32_t c = d <= chunk ? 1 : (d + chunk - 1) / chunk;
        nch[v] = c;
        split[v] = c > 1 ? 1 : 0;
    }
}

// work items: one per row chunk; split rows get an index and the position of
// their first chunk among the chunks of split rows
// sort key placing high-degree rows first (ties by vertex id), or, with
// split_first, the split rows first and every group in vertex order
__global__ void k_degkeys(const int32_t* __restrict__ deg, int64_t n, uint64_t* __restrict__ keys, int chunk,
                          int split_first, int nb)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t hi = split_first ? (deg[v] > chunk ? 0u : 1u) : (0x7FFFFFFFu - (uint32_t)deg[v]);
        keys[v] = ((uint64_t)hi << nb) | (uint64_t)v;  // the vertex in the low nb bits
    }
}

__global__ void k_perm(const uint64_t* __restrict__ keys, int64_t n, const int32_t* __restrict__ nch,
                       int32_t* __restrict__ perm, int32_t* __restrict__ nch_sorted, int nb)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = (int32_t)(keys[i] & ((1ull << nb) - 1ull));
        perm[i] = v;
        nch_sorted[i] = nch[v];
    }
}

// work items of row position i (vertex perm[i], or i when perm is null);
// ipos is indexed by position
__global__ void k_items(const int32_t* __restrict__ rowptr, int64_t n, int chunk, const int32_t* __restrict__ nch,
                        const int32_t* __restrict__ ipos, const int32_t* __restrict__ split,
                        const int32_t* __restrict__ hpos, const int32_t* __restrict__ splitpos,
                        const int32_t* __restrict__ perm, sb_bfs_item* __restrict__ items,
                        int32_t* __restrict__ hub_vertex, int32_t* __restrict__ hub_first,
                        int32_t* __restrict__ hub_count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = perm ? perm[i] : i;
        int32_t b = rowptr[v], e = rowptr[v + 1], c = nch[v];
        int32_t hub = split[v] ? hpos[v] : -1;
        if (hub >= 0) {
            hub_vertex[hub] = (int32_t)v;
            if (hub_first) hub_first[hub] = splitpos[v];
            if (hub_count) hub_count[hub] = c;
        }
        for (int32_t k = 0; k < c; k++) {
            sb_bfs_item it;
            it.v = (int32_t)v;
            it.beg = b + k * chunk;
            it.end = min(e, b + (k + 1) * chunk);
            it.hub = hub;
            items[ipos[i] + k] = it;
        }
    }
}

// state-hash weight of each vertex, by its id inside its own graph
__global__ void k_vweight(uint64_t* w, int64_t n, const int32_t* __restrict__ vgoff)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        w[v] = sb_weight((uint32_t)(v - (vgoff ? vgoff[v] : 0)));
}

__global__ void k_split_edges(const int2* __restrict__ e, int64_t m, int32_t* u, int32_t* v, int8_t* neg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        int2 x = e[i];
        if (u) u[i] = x.x;
        if (v) v[i] = (int32_t)((uint32_t)x.y & SB_ID_MASK);
        if (neg) neg[i] = (int8_t)((uint32_t)x.y >> 31);
    }
}

__global__ void k_split_col(const int32_t* __restrict__ col, int64_t k, int32_t* c, int8_t* neg)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)col[i];
        if (c) c[i] = (int32_t)(x & SB_ID_MASK);
        if (neg) neg[i] = (int8_t)(x >> 31);
    }
}

// ------------------------------------------------------ batches of graphs
// index g with off[g] <= x < off[g+1], for nondecreasing off[0..G]
template <class T>
__device__ __forceinline__ int64_t seg_of(const T* off, int64_t G, int64_t x)
{
    int64_t lo = 0, hi = G - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// local ids of edge i (graph g: eofs[g] <= i < eofs[g+1]) -> ids of the union;
// an id outside [0, nv_g) becomes -1 so that validation reports a range error
__global__ void k_globalize(int32_t* src, int32_t* dst, int64_t m, const int64_t* __restrict__ eofs,
                            const int64_t* __restrict__ voff, int64_t G)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = seg_of(eofs, G, i);
        const int64_t nv = voff[g + 1] - voff[g];
        const int32_t a = src[i], b = dst[i];
        src[i] = (a >= 0 && a < nv) ? (int32_t)(voff[g] + a) : -1;
        dst[i] = (b >= 0 && b < nv) ? (int32_t)(voff[g] + b) : -1;
    }
}

// largest component per graph (ties: smallest root) and components per graph
__global__ void k_uf_best_batch(const int32_t* __restrict__ size, int64_t n, const int64_t* __restrict__ voff,
                                int64_t G, unsigned long long* best, uint32_t* ncomp)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t sz = size[v];
        if (sz > 0) {
            const int64_t g = seg_of(voff, G, v);
            atomicMax(best + g, ((unsigned long long)sz << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)v));
            atomicAdd(ncomp + g, 1u);
        }
    }
}

__global__ void k_keep_vertices_batch(const int32_t* __restrict__ root, int64_t n, const int64_t* __restrict__ voff,
                                      int64_t G, const unsigned long long* __restrict__ best, int32_t* __restrict__ keep)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = seg_of(voff, G, v);
        const int32_t br = (int32_t)(0xFFFFFFFFu - (uint32_t)(best[g] & 0xFFFFFFFFull));
        keep[v] = root[v] == br ? 1 : 0;
    }
}

// first cleaned vertex of each graph: the exclusive count of kept vertices
// before the graph's first input vertex
__global__ void k_batch_vbounds(const int32_t* __restrict__ newid, const int64_t* __restrict__ voff, int64_t G,
                                int64_t n, int64_t n1, int32_t* __restrict__ voff_out)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += (int64_t)gridDim.x * blockDim.x)
        voff_out[g] = voff[g] < n ? newid[voff[g]] : (int32_t)n1;
}

__global__ void k_batch_vgid(const int32_t* __restrict__ voff_out, int64_t G, int64_t n1, int32_t* __restrict__ vgid,
                             int32_t* __restrict__ vgoff)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n1; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = seg_of(voff_out, G, v);
        vgid[v] = (int32_t)g;
        vgoff[v] = voff_out[g];
    }
}

// first edge of each graph in the (u, v)-sorted edge list
__global__ void k_batch_ebounds(const int2* __restrict__ edges, int64_t m, const int32_t* __restrict__ voff_out,
                                int64_t G, int32_t* __restrict__ eoff)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= G; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = voff_out[g];
        int64_t lo = 0, hi = m;  // first edge with u >= x
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (edges[mid].x < x) lo = mid + 1;
            else hi = mid;
        }
        eoff[g] = (int32_t)lo;
    }
}

// chunk counts of rows that are not split are zeroed (partial slots only for split rows)
__global__ void k_zero_unsplit(int32_t* x, const int32_t* s, int64_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (!s[v]) x[v] = 0;
}

static unsigned grid_for(sb_ctx* c, int64_t work)
{
    int64_t g = sb_cdiv(work > 0 ? work : 1, 256);
    int64_t cap = (int64_t)c->num_sms * 16;
    return (unsigned)(g < cap ? g : cap);
}

// Scratch for one ingest call, freed on every exit path.
struct IngestTmp {
    sb_ctx* c;
    void* p[40];
    int k = 0;
    explicit IngestTmp(sb_ctx* cc) : c(cc) { memset(p, 0, sizeof(p)); }
    template <class T> T* get(size_t count)
    {
        void* q = sb_dalloc(c, sizeof(T) * (count > 0 ? count : 1));
        p[k++] = q;
        return (T*)q;
    }
    ~IngestTmp()
    {
        cudaStreamSynchronize(c->stream);
        for (int i = 0; i < k; i++) sb_dfree(c, p[i]);
    }
};

// Builds the work items of one chunk size: returns items, split-row vertex
// list (and optionally first partial slot / chunk count per split row).
// Work items of one chunk size.  order 0: vertex order; 1: descending degree;
// 2: chunks of split rows first, then whole rows (each in vertex order).
static sb_status build_items(sb_ctx* c, const int32_t* deg, int64_t n, int chunk, int order,
                             sb_bfs_item** items_out, int64_t* n_items, int32_t** hub_vertex, int64_t* n_hubs,
                             int32_t** hub_first, int32_t** hub_count, int64_t* n_partials)
{
    IngestTmp T(c);
    int32_t* nch = T.get<int32_t>(n);
    int32_t* split = T.get<int32_t>(n);
    int32_t* ipos = T.get<int32_t>(n);
    int32_t* hpos = T.get<int32_t>(n);
    int32_t* splitch = T.get<int32_t>(n);
    int32_t* splitpos = T.get<int32_t>(n);
    int64_t* tot = T.get<int64_t>(3);
    if (!nch || !split || !ipos || !hpos || !splitch || !splitpos || !tot) return sb_fail(c, SB_ERR_OOM, "item scratch");
    unsigned g = grid_for(c, n);
    k_chunks<<<g, 256, 0, c->stream>>>(deg, n, chunk, nch, split);
    SB_TRY(sb_after_launch(c, "k_chunks"));
    int32_t* perm = nullptr;
    if (order != 0) {
        uint64_t* keys = T.get<uint64_t>(n);
        perm = T.get<int32_t>(n);
        int32_t* nch_sorted = T.get<int32_t>(n);
        if (!keys || !perm || !nch_sorted) return sb_fail(c, SB_ERR_OOM, "item scratch");
        const int nbv = bits_for(n > 1 ? n - 1 : 1);
        k_degkeys<<<g, 256, 0, c->stream>>>(deg, n, keys, chunk, order == 2 ? 1 : 0, nbv);
        SB_TRY(sb_after_launch(c, "k_degkeys"));
        SB_TRY(sb_radix_sort_u64(c, keys, n, nbv + (order == 2 ? 1 : 31)));
        k_perm<<<g, 256, 0, c->stream>>>(keys, n, nch, perm, nch_sorted, nbv);
        SB_TRY(sb_after_launch(c, "k_perm"));
        SB_TRY(sb_scan_i32(c, nch_sorted, ipos, n, tot + 0));
    } else {
        SB_TRY(sb_scan_i32(c, nch, ipos, n, tot + 0));
    }
    SB_TRY(sb_scan_i32(c, split, hpos, n, tot + 1));
    // chunks of split rows only (for partial-sum slots)
    SB_CHECK_CUDA(c, cudaMemcpyAsync(splitch, nch, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
    k_zero_unsplit<<<g, 256, 0, c->stream>>>(splitch, split, n);
    SB_TRY(sb_after_launch(c, "mask split"));
    SB_TRY(sb_scan_i32(c, splitch, splitpos, n, tot + 2));
    int64_t h_tot[3];
    SB_CHECK_CUDA(c, cudaMemcpyAsync(h_tot, tot, sizeof(h_tot), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    *n_items = h_tot[0];
    *n_hubs = h_tot[1];
    if (n_partials) *n_partials = h_tot[2];
    *items_out = (sb_bfs_item*)sb_dalloc(c, sizeof(sb_bfs_item) * (size_t)(h_tot[0] > 0 ? h_tot[0] : 1));
    *hub_vertex = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(h_tot[1] > 0 ? h_tot[1] : 1));
    if (hub_first) *hub_first = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(h_tot[1] > 0 ? h_tot[1] : 1));
    if (hub_count) *hub_count = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(h_tot[1] > 0 ? h_tot[1] : 1));
    if (!*items_out || !*hub_vertex || (hub_first && !*hub_first) || (hub_count && !*hub_count))
        return sb_fail(c, SB_ERR_OOM, "work items");
    k_items<<<g, 256, 0, c->stream>>>(c->rowptr, n, chunk, nch, ipos, split, hpos, splitpos, perm, *items_out,
                                      *hub_vertex, hub_first ? *hub_first : nullptr, hub_count ? *hub_count : nullptr);
    return sb_after_launch(c, "k_items");
}

// A batch of G graphs loaded as one disjoint union: graph g owns input
// vertices [voff[g], voff[g+1]) and input edges [eofs[g], eofs[g+1]) (host).
struct BatchIn {
    int64_t G;
    const int64_t* voff;
    const int64_t* eofs;
};

// key of the scorer's copy of an edge: (colder << (nb + 1)) | (hotter << 1) | neg,
// colder = the endpoint of lower degree (on a tie, the larger id)
__global__ void k_orient_keys(const int2* __restrict__ edges, int64_t m, const int32_t* __restrict__ deg, int nb,
                              uint64_t* __restrict__ keys)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int2 ed = edges[e];
        const uint32_t u = (uint32_t)ed.x, v = (uint32_t)ed.y & SB_ID_MASK;
        const bool u_cold = deg[u] < deg[v];  // u < v, so a tie makes v the colder one
        const uint64_t cold = u_cold ? u : v, hot = u_cold ? v : u;
        keys[e] = (cold << (nb + 1)) | (hot << 1) | (uint64_t)(ed.y < 0 ? 1 : 0);
    }
}

__global__ void k_emit_sc_edges(const uint64_t* __restrict__ keys, int64_t m, int nb, int2* __restrict__ out)
{
    const uint64_t idm = (1ull << nb) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[e];
        out[e] = make_int2((int32_t)(k >> (nb + 1)), (int32_t)((uint32_t)((k >> 1) & idm) | ((uint32_t)(k & 1ull) << 31)));
    }
}

static sb_status load_graph_impl(sb_ctx* c, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                 const int8_t* sign, uint32_t flags, int64_t* n_out, int64_t* m_out,
                                 int32_t* vmap_out, const BatchIn* B = nullptr)
{
    IngestTmp T(c);
    int nb = bits_for(n - 1);
    int32_t* d_src = T.get<int32_t>(m);
    int32_t* d_dst = T.get<int32_t>(m);
    int8_t* d_sign = T.get<int8_t>(m);
    uint64_t* keys = T.get<uint64_t>(m);
    unsigned long long* scal = T.get<unsigned long long>(8);  // [0] errkey [1] best [2] ncomp
    uint32_t* flags_d = T.get<uint32_t>(4);
    int64_t* tot = T.get<int64_t>(4);
    if (!d_src || !d_dst || !d_sign || !keys || !scal || !flags_d || !tot) return sb_fail(c, SB_ERR_OOM, "ingest scratch");
    if (m > 0) {
        SB_CHECK_CUDA(c, cudaMemcpyAsync(d_src, src, sizeof(int32_t) * m, cudaMemcpyDefault, c->stream));
        SB_CHECK_CUDA(c, cudaMemcpyAsync(d_dst, dst, sizeof(int32_t) * m, cudaMemcpyDefault, c->stream));
        SB_CHECK_CUDA(c, cudaMemcpyAsync(d_sign, sign, sizeof(int8_t) * m, cudaMemcpyDefault, c->stream));
    }
    int64_t* d_bvoff = nullptr;
    int64_t* d_beofs = nullptr;
    if (B) {
        d_bvoff = T.get<int64_t>(B->G + 1);
        d_beofs = T.get<int64_t>(B->G + 1);
        if (!d_bvoff || !d_beofs) return sb_fail(c, SB_ERR_OOM, "batch offsets");
        SB_CHECK_CUDA(c, cudaMemcpyAsync(d_bvoff, B->voff, sizeof(int64_t) * (B->G + 1), cudaMemcpyHostToDevice, c->stream));
        SB_CHECK_CUDA(c, cudaMemcpyAsync(d_beofs, B->eofs, sizeof(int64_t) * (B->G + 1), cudaMemcpyHostToDevice, c->stream));
        k_globalize<<<grid_for(c, m), 256, 0, c->stream>>>(d_src, d_dst, m, d_beofs, d_bvoff, B->G);
        SB_TRY(sb_after_launch(c, "k_globalize"));
    }
    unsigned long long init[8] = {~0ull, 0, 0, 0, 0, 0, 0, 0};
    SB_CHECK_CUDA(c, cudaMemcpyAsync(scal, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(flags_d, 0, 16, c->stream));
    unsigned gm = grid_for(c, m);
    unsigned gn = grid_for(c, n);
    k_validate<<<gm, 256, 0, c->stream>>>(d_src, d_dst, d_sign, n, m, nb, keys, scal);
    SB_TRY(sb_after_launch(c, "k_validate"));
    unsigned long long errkey = 0;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&errkey, scal, sizeof(errkey), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (errkey != ~0ull) {
        int code = (int)(errkey & 255u);
        long long idx = (long long)(errkey >> 8);
        if (code == ERRC_RANGE) return sb_fail(c, SB_ERR_RANGE, "edge %lld: vertex id out of range", idx);
        if (code == ERRC_SELF) return sb_fail(c, SB_ERR_SELF_LOOP, "edge %lld is a self-loop", idx);
        return sb_fail(c, SB_ERR_BAD_SIGN, "edge %lld: sign is not +1/-1", idx);
    }
    SB_TRY(sb_radix_sort_u64(c, keys, m, 2 * nb + 1));
    int32_t* head = T.get<int32_t>(m);
    int32_t* hpos = T.get<int32_t>(m);
    if (!head || !hpos) return sb_fail(c, SB_ERR_OOM, "ingest scratch");
    k_heads<<<gm, 256, 0, c->stream>>>(keys, m, head, flags_d);
    SB_TRY(sb_after_launch(c, "k_heads"));
    SB_TRY(sb_scan_i32(c, head, hpos, m, tot + 0));
    uint32_t hflags = 0;
    int64_t m1 = 0;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&hflags, flags_d, sizeof(hflags), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&m1, tot, sizeof(m1), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (hflags & 1u) return sb_fail(c, SB_ERR_INCONSISTENT, "a vertex pair appears with both signs");
    if ((hflags & 2u) && !(flags & SB_LOAD_MERGE_DUP))
        return sb_fail(c, SB_ERR_DUPLICATE, "a vertex pair appears more than once");
    uint64_t* ukeys = T.get<uint64_t>(m1);
    int32_t* par = T.get<int32_t>(n);
    int32_t* size = T.get<int32_t>(n);
    if (!ukeys || !par || !size) return sb_fail(c, SB_ERR_OOM, "ingest scratch");
    k_compact_keys<<<gm, 256, 0, c->stream>>>(keys, head, hpos, m, ukeys);
    SB_TRY(sb_after_launch(c, "k_compact_keys"));
    // components
    unsigned gm1 = grid_for(c, m1);
    k_uf_init<<<gn, 256, 0, c->stream>>>(par, n);
    SB_CHECK_CUDA(c, cudaMemsetAsync(size, 0, sizeof(int32_t) * n, c->stream));
    k_uf_hook<<<gm1, 256, 0, c->stream>>>(ukeys, m1, nb, par, flags_d);
    SB_TRY(sb_after_launch(c, "k_uf_hook"));
    k_uf_sizes<<<gn, 256, 0, c->stream>>>(par, n, size);
    SB_TRY(sb_after_launch(c, "k_uf_sizes"));
    int32_t* keep = T.get<int32_t>(n);
    int32_t* newid = T.get<int32_t>(n);
    int32_t* ekeep = T.get<int32_t>(m1);
    int32_t* epos = T.get<int32_t>(m1);
    if (!keep || !newid || !ekeep || !epos) return sb_fail(c, SB_ERR_OOM, "ingest scratch");
    if (!B) {
        k_uf_best<<<gn, 256, 0, c->stream>>>(size, n, scal + 1, scal + 2);
        SB_TRY(sb_after_launch(c, "k_uf_best"));
        unsigned long long hs[3];
        SB_CHECK_CUDA(c, cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, c->stream));
        SB_CHECK_CUDA(c, cudaMemcpyAsync(&hflags, flags_d, sizeof(hflags), cudaMemcpyDeviceToHost, c->stream));
        SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
        if (hflags & 4u) return sb_fail(c, SB_ERR_DEVICE_CHECK, "union-find retry limit reached");
        if (hs[2] > 1 && !(flags & SB_LOAD_LCC))
            return sb_fail(c, SB_ERR_DISCONNECTED, "graph has %llu components", (unsigned long long)hs[2]);
        // relabel the kept component
        k_keep_vertices<<<gn, 256, 0, c->stream>>>(par, n, scal + 1, keep);
        SB_TRY(sb_after_launch(c, "k_keep_vertices"));
    } else {
        unsigned long long* bestg = T.get<unsigned long long>(B->G);
        uint32_t* ncompg = T.get<uint32_t>(B->G);
        if (!bestg || !ncompg) return sb_fail(c, SB_ERR_OOM, "batch scratch");
        SB_CHECK_CUDA(c, cudaMemsetAsync(bestg, 0, sizeof(unsigned long long) * B->G, c->stream));
        SB_CHECK_CUDA(c, cudaMemsetAsync(ncompg, 0, sizeof(uint32_t) * B->G, c->stream));
        k_uf_best_batch<<<gn, 256, 0, c->stream>>>(size, n, d_bvoff, B->G, bestg, ncompg);
        SB_TRY(sb_after_launch(c, "k_uf_best_batch"));
        std::vector<uint32_t> hcomp(B->G);
        SB_CHECK_CUDA(c, cudaMemcpyAsync(hcomp.data(), ncompg, sizeof(uint32_t) * B->G, cudaMemcpyDeviceToHost,
                                         c->stream));
        SB_CHECK_CUDA(c, cudaMemcpyAsync(&hflags, flags_d, sizeof(hflags), cudaMemcpyDeviceToHost, c->stream));
        SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
        if (hflags & 4u) return sb_fail(c, SB_ERR_DEVICE_CHECK, "union-find retry limit reached");
        if (!(flags & SB_LOAD_LCC))
            for (int64_t g = 0; g < B->G; g++)
                if (hcomp[g] > 1)
                    return sb_fail(c, SB_ERR_DISCONNECTED, "graph %lld has %u components", (long long)g, hcomp[g]);
        k_keep_vertices_batch<<<gn, 256, 0, c->stream>>>(par, n, d_bvoff, B->G, bestg, keep);
        SB_TRY(sb_after_launch(c, "k_keep_vertices_batch"));
    }
    SB_TRY(sb_scan_i32(c, keep, newid, n, tot + 1));
    if (vmap_out) {
        int32_t* vm = T.get<int32_t>(n);
        if (!vm) return sb_fail(c, SB_ERR_OOM, "ingest scratch");
        k_vmap<<<gn, 256, 0, c->stream>>>(keep, newid, n, vm);
        SB_TRY(sb_after_launch(c, "k_vmap"));
        SB_TRY(sb_copy_out(c, vmap_out, vm, sizeof(int32_t) * n));
    }
    k_keep_edges<<<gm1, 256, 0, c->stream>>>(ukeys, m1, nb, keep, ekeep);
    SB_TRY(sb_after_launch(c, "k_keep_edges"));
    SB_TRY(sb_scan_i32(c, ekeep, epos, m1, tot + 2));
    int64_t h_n1 = 0, h_m2 = 0;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&h_n1, tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&h_m2, tot + 2, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    const int64_t n1 = h_n1, m2 = h_m2;
    int nb2 = bits_for(n1 > 1 ? n1 - 1 : 1);
    c->edges = (int2*)sb_dalloc(c, sizeof(int2) * (size_t)(m2 > 0 ? m2 : 1));
    c->rowptr = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(n1 + 1));
    c->col = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(2 * m2 > 0 ? 2 * m2 : 1));
    c->vweight = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)n1);
    uint64_t* lkeys = T.get<uint64_t>(m2);
    int32_t* deg = T.get<int32_t>(n1);
    int32_t* updeg = T.get<int32_t>(n1);
    int32_t* ufirst = T.get<int32_t>(n1);
    int32_t* low = T.get<int32_t>(n1);
    int32_t* lfirst = T.get<int32_t>(n1);
    if (!c->edges || !c->rowptr || !c->col || !c->vweight || !lkeys || !deg || !updeg || !ufirst || !low || !lfirst)
        return sb_fail(c, SB_ERR_OOM, "graph storage");
    SB_CHECK_CUDA(c, cudaMemsetAsync(deg, 0, sizeof(int32_t) * n1, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(updeg, 0, sizeof(int32_t) * n1, c->stream));
    k_emit_edges<<<gm1, 256, 0, c->stream>>>(ukeys, m1, nb, ekeep, epos, newid, nb2, c->edges, lkeys, deg, updeg);
    SB_TRY(sb_after_launch(c, "k_emit_edges"));
    SB_TRY(sb_scan_i32(c, deg, c->rowptr, n1, tot + 3));
    // rowptr[n1] = 2 m2
    int32_t last = (int32_t)(2 * m2);
    SB_CHECK_CUDA(c, cudaMemcpyAsync(c->rowptr + n1, &last, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    SB_TRY(sb_scan_i32(c, updeg, ufirst, n1, nullptr));
    unsigned gm2 = grid_for(c, m2), gn1 = grid_for(c, n1);
    k_fill_upper<<<gm2, 256, 0, c->stream>>>(c->edges, m2, c->rowptr, deg, updeg, ufirst, c->col);
    SB_TRY(sb_after_launch(c, "k_fill_upper"));
    SB_TRY(sb_radix_sort_u64(c, lkeys, m2, 2 * nb2 + 1));
    k_lowdeg<<<gn1, 256, 0, c->stream>>>(deg, updeg, n1, low);
    SB_TRY(sb_after_launch(c, "k_lowdeg"));
    SB_TRY(sb_scan_i32(c, low, lfirst, n1, nullptr));
    k_fill_lower<<<gm2, 256, 0, c->stream>>>(lkeys, m2, nb2, c->rowptr, lfirst, c->col);
    SB_TRY(sb_after_launch(c, "k_fill_lower"));
    // scorer stream: every edge from its colder endpoint (lower degree) to
    // the hotter one, sorted by (colder, hotter); two zero edges of padding
    // let tile copies round their size up to 16 bytes
    c->sc_edges = (int2*)sb_dalloc(c, sizeof(int2) * (size_t)(m2 + 2));
    if (!c->sc_edges) return sb_fail(c, SB_ERR_OOM, "graph storage");
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sc_edges + m2, 0, 2 * sizeof(int2), c->stream));
    if (m2 > 0) {
        k_orient_keys<<<gm2, 256, 0, c->stream>>>(c->edges, m2, deg, nb2, lkeys);
        SB_TRY(sb_after_launch(c, "k_orient_keys"));
        SB_TRY(sb_radix_sort_u64(c, lkeys, m2, 2 * nb2 + 1));
        k_emit_sc_edges<<<gm2, 256, 0, c->stream>>>(lkeys, m2, nb2, c->sc_edges);
        SB_TRY(sb_after_launch(c, "k_emit_sc_edges"));
    }
    if (B) {
        const int64_t G = B->G;
        c->b_voff = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(G + 1));
        c->b_eoff = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)(G + 1));
        c->vgid = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)n1);
        c->vgoff = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)n1);
        if (!c->b_voff || !c->b_eoff || !c->vgid || !c->vgoff) return sb_fail(c, SB_ERR_OOM, "batch storage");
        unsigned gg = grid_for(c, G + 1);
        k_batch_vbounds<<<gg, 256, 0, c->stream>>>(newid, d_bvoff, G, n, n1, c->b_voff);
        SB_TRY(sb_after_launch(c, "k_batch_vbounds"));
        k_batch_vgid<<<gn1, 256, 0, c->stream>>>(c->b_voff, G, n1, c->vgid, c->vgoff);
        SB_TRY(sb_after_launch(c, "k_batch_vgid"));
        k_batch_ebounds<<<gg, 256, 0, c->stream>>>(c->edges, m2, c->b_voff, G, c->b_eoff);
        SB_TRY(sb_after_launch(c, "k_batch_ebounds"));
        std::vector<int32_t> hv(G + 1), he(G + 1);
        SB_CHECK_CUDA(c, cudaMemcpyAsync(hv.data(), c->b_voff, sizeof(int32_t) * (G + 1), cudaMemcpyDeviceToHost,
                                         c->stream));
        SB_CHECK_CUDA(c, cudaMemcpyAsync(he.data(), c->b_eoff, sizeof(int32_t) * (G + 1), cudaMemcpyDeviceToHost,
                                         c->stream));
        SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
        c->h_voff.assign(hv.begin(), hv.end());
        c->h_eoff.assign(he.begin(), he.end());
        c->batch_G = G;
    }
    k_vweight<<<gn1, 256, 0, c->stream>>>(c->vweight, n1, c->vgoff);
    SB_TRY(sb_after_launch(c, "k_vweight"));
    c->n = n1;
    c->m = m2;
    SB_TRY(build_items(c, deg, n1, SB_BFS_CHUNK, 1, &c->items, &c->n_items, &c->hub_vertex, &c->n_hubs, nullptr,
                       nullptr, nullptr));
    SB_TRY(build_items(c, deg, n1, SB_GL_CHUNK, 2, &c->gl_items, &c->n_gl_items, &c->gl_hub_vertex,
                       &c->n_gl_hubs, &c->gl_hub_first, &c->gl_hub_count, &c->n_gl_partials));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_graph = true;
    *n_out = n1;
    *m_out = m2;
    return SB_OK;
}

extern "C" sb_status sb_load_graph(sb_ctx* c, int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                   const int8_t* sign, uint32_t flags, int64_t* n_out, int64_t* m_out,
                                   int32_t* vmap_out)
{
    if (!c) return SB_ERR_ARG;
    if (n < 1 || n > 0x7FFFFFFF || m < 0 || 2 * m >= 0x7FFFFFFF || !n_out || !m_out ||
        (m > 0 && (!src || !dst || !sign)) || (flags & ~(SB_LOAD_LCC | SB_LOAD_MERGE_DUP)))
        return sb_fail(c, SB_ERR_ARG, "sb_load_graph: bad argument (n=%lld m=%lld)", (long long)n, (long long)m);
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    sb_release_graph(c);
    SbProf prof(c, SB_PROF_INGEST);
    sb_status st = load_graph_impl(c, n, m, src, dst, sign, flags, n_out, m_out, vmap_out);
    if (st != SB_OK) sb_release_graph(c);
    return st;
}

extern "C" sb_status sb_graph_edges(sb_ctx* c, int32_t* u_out, int32_t* v_out, int8_t* neg_out)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_graph) return sb_fail(c, SB_ERR_STATE, "no graph loaded");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    int64_t m = c->m;
    if (m == 0) return SB_OK;
    IngestTmp T(c);
    int32_t* u = T.get<int32_t>(m);
    int32_t* v = T.get<int32_t>(m);
    int8_t* g = T.get<int8_t>(m);
    if (!u || !v || !g) return sb_fail(c, SB_ERR_OOM, "export scratch");
    k_split_edges<<<grid_for(c, m), 256, 0, c->stream>>>(c->edges, m, u, v, g);
    SB_TRY(sb_after_launch(c, "k_split_edges"));
    SB_TRY(sb_copy_out(c, u_out, u, sizeof(int32_t) * m));
    SB_TRY(sb_copy_out(c, v_out, v, sizeof(int32_t) * m));
    SB_TRY(sb_copy_out(c, neg_out, g, sizeof(int8_t) * m));
    return SB_OK;
}

extern "C" sb_status sb_graph_csr(sb_ctx* c, int32_t* rowptr_out, int32_t* col_out, int8_t* neg_out)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_graph) return sb_fail(c, SB_ERR_STATE, "no graph loaded");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(sb_copy_out(c, rowptr_out, c->rowptr, sizeof(int32_t) * (c->n + 1)));
    int64_t k = 2 * c->m;
    if (k == 0) return SB_OK;
    IngestTmp T(c);
    int32_t* cc = T.get<int32_t>(k);
    int8_t* g = T.get<int8_t>(k);
    if (!cc || !g) return sb_fail(c, SB_ERR_OOM, "export scratch");
    k_split_col<<<grid_for(c, k), 256, 0, c->stream>>>(c->col, k, cc, g);
    SB_TRY(sb_after_launch(c, "k_split_col"));
    SB_TRY(sb_copy_out(c, col_out, cc, sizeof(int32_t) * k));
    SB_TRY(sb_copy_out(c, neg_out, g, sizeof(int8_t) * k));
    return SB_OK;
}

extern "C" sb_status sb_load_batch(sb_ctx* c, int64_t n_graphs, const int64_t* nv, const int64_t* eofs,
                                   const int32_t* src, const int32_t* dst, const int8_t* sign, uint32_t flags,
                                   int64_t* nv_out, int64_t* m_out)
{
    if (!c) return SB_ERR_ARG;
    if (n_graphs < 1 || n_graphs > (1ll << 24) || !nv || !eofs || eofs[0] != 0 ||
        (flags & ~(SB_LOAD_LCC | SB_LOAD_MERGE_DUP)))
        return sb_fail(c, SB_ERR_ARG, "sb_load_batch: bad argument");
    std::vector<int64_t> voff(n_graphs + 1, 0);
    for (int64_t g = 0; g < n_graphs; g++) {
        if (nv[g] < 1 || eofs[g + 1] < eofs[g]) return sb_fail(c, SB_ERR_ARG, "sb_load_batch: graph %lld", (long long)g);
        voff[g + 1] = voff[g] + nv[g];
    }
    const int64_t n = voff[n_graphs], m = eofs[n_graphs];
    if (n > 0x7FFFFFFF || 2 * m >= 0x7FFFFFFF || (m > 0 && (!src || !dst || !sign)))
        return sb_fail(c, SB_ERR_ARG, "sb_load_batch: batch too large (n=%lld m=%lld)", (long long)n, (long long)m);
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    sb_release_graph(c);
    SbProf prof(c, SB_PROF_INGEST);
    BatchIn B{n_graphs, voff.data(), eofs};
    int64_t n1 = 0, m1 = 0;
    sb_status st = load_graph_impl(c, n, m, src, dst, sign, flags, &n1, &m1, nullptr, &B);
    if (st != SB_OK) {
        sb_release_graph(c);
        return st;
    }
    for (int64_t g = 0; g < n_graphs; g++) {
        if (nv_out) nv_out[g] = c->h_voff[g + 1] - c->h_voff[g];
        if (m_out) m_out[g] = c->h_eoff[g + 1] - c->h_eoff[g];
    }
    return SB_OK;
}
