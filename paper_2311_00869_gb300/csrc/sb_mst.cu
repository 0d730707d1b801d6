// sb_mst.cu -- randomized Kruskal trees (appendix, tree samplers: Kruskal's
// algorithm run on random edge weights drawn afresh for every tree), many
// trees at once.
//
// Tree t is the minimum spanning tree under the weights
//   w_t(u, v) = mix64(((u << 32) | v) ^ K_t),   u < v (graph-local ids),
// with K_t the tree key of the BFS sampler.  mix64 is a bijection, so the
// weights of one tree are distinct and the tree is unique: Kruskal's scan in
// weight order, Prim's growth and Boruvka's rounds all find it.  Kruskal's
// scan is sequential; Boruvka's rounds are not, so the GPU runs those:
//   1. every vertex finds its lightest edge that leaves its component
//      (a CSR row scan) and the component keeps the lightest of those
//      (64-bit atomicMin);
//   2. the one vertex holding that edge records it for its component;
//   3. every component root hooks below the component at the edge's far
//      end; two components that chose each other chose the same edge (the
//      weights are distinct), and only the larger root hooks;
//   4. pointer jumping flattens the hooks; a pointer carries the parity of
//      the path to its target in its low bit, so each vertex ends with its
//      parity label relative to its component's root.
// Every round at least halves the number of components of every unfinished
// tree, so ceil(log2 n) + 1 rounds suffice.  A round after which nothing
// merged ends the loop early (its kernels return at once).
//
// Layout: [vertex][tree of the pass], trees innermost, so a warp holds 32
// trees of one vertex: it scans one CSR row in lockstep and its gathers of a
// neighbour's 32 root words are one coalesced 128-byte load.
#include <algorithm>

#include "sb_internal.cuh"

#define SB_MST_DEAD 0xFFFFFFFFu          // no edge leaves the component from this vertex
#define MST_THREADS 256
#define MST_BYTES_PER_SLOT 36            // P, R, Y (4 B each), L, B (8 B each), win (8 B)
#define MST_PASS_BUDGET (32ull << 30)    // scratch bytes per pass of trees (at most half the free memory)

struct MstArgs {
    int64_t n;
    int T;            // trees per pass (a multiple of 64)
    int64_t tb0;      // first tree of the pass, within the batch
    int64_t K;        // trees of the batch
    uint64_t S;       // seed key
    int64_t tree0;    // global index of batch tree 0
    const int32_t* rowptr;
    const int32_t* col;
    const int32_t* vgoff;  // first vertex of each vertex's graph (batches), or null
    uint32_t* P;
    uint32_t* R;
    uint32_t* Y;
    uint64_t* L;
    uint64_t* B;
    int2* win;
    int32_t* flags;
    const int2* edges;     // for in_tree (binary search of the pair)
    int64_t m;
    uint8_t* in_tree;      // K x m, or null
    uint32_t* err;
};

__device__ __forceinline__ uint32_t mst_ld(const uint32_t* p) { return __ldcg(p); }

__global__ void __launch_bounds__(MST_THREADS) k_mst_init(MstArgs A)
{
    const int64_t total = A.n * A.T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)(i / A.T);
        A.P[i] = v << 1;
        A.R[i] = v << 1;
        A.Y[i] = 0;
        A.B[i] = ~0ull;
        A.win[i] = make_int2(-1, -1);
    }
}

// 1. lightest edge leaving the component, per (vertex, tree); component min.
// In round 0 every vertex is alone, so every edge leaves and nothing is loaded.
__global__ void __launch_bounds__(MST_THREADS) k_mst_min(MstArgs A, int r)
{
    if (!A.flags[r]) return;
    const int64_t total = A.n * A.T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / A.T;
        const int tt = (int)(i - v * A.T);
        const int64_t tb = A.tb0 + tt;
        if (tb >= A.K || A.Y[i] == SB_MST_DEAD) continue;
        const uint32_t c = A.R[i] >> 1;
        const uint64_t kt = sb_tree_key(A.S, A.tree0 + tb);
        const int64_t base = A.vgoff ? A.vgoff[v] : 0;
        const uint32_t vl = (uint32_t)(v - base);
        uint64_t best = ~0ull;
        uint32_t by = SB_MST_DEAD;
        const int32_t e1 = A.rowptr[v + 1];
        for (int32_t p = A.rowptr[v]; p < e1; p++) {
            const uint32_t cv = (uint32_t)A.col[p];
            const uint32_t y = cv & SB_ID_MASK;
            if (r > 0 && (A.R[(int64_t)y * A.T + tt] >> 1) == c) continue;
            const uint32_t yl = (uint32_t)(y - base);
            const uint64_t pair = vl < yl ? ((uint64_t)vl << 32 | yl) : ((uint64_t)yl << 32 | vl);
            const uint64_t w = sb_mix64(pair ^ kt);
            if (by == SB_MST_DEAD || w < best) {
                best = w;
                by = cv;
            }
        }
        A.Y[i] = by;
        if (by == SB_MST_DEAD) continue;  // every neighbour is inside: it stays so
        A.L[i] = best;
        atomicMin((unsigned long long*)(A.B + (int64_t)c * A.T + tt), (unsigned long long)best);
    }
}

// 2. the vertex holding its component's lightest edge records it
__global__ void __launch_bounds__(MST_THREADS) k_mst_win(MstArgs A, int r)
{
    if (!A.flags[r]) return;
    const int64_t total = A.n * A.T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / A.T;
        const int tt = (int)(i - v * A.T);
        if (A.tb0 + tt >= A.K) continue;
        const uint32_t y = A.Y[i];
        if (y == SB_MST_DEAD) continue;
        const int64_t ci = (int64_t)(A.R[i] >> 1) * A.T + tt;
        if (A.L[i] == A.B[ci]) A.win[ci] = make_int2((int32_t)v, (int32_t)y);
    }
}

// index of edge (a, b), a < b, in the sorted edge list
__device__ int64_t mst_edge_index(const int2* edges, int64_t m, uint32_t a, uint32_t b)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int2 e = edges[mid];
        const uint32_t eu = (uint32_t)e.x, ev = (uint32_t)e.y & SB_ID_MASK;
        if (eu < a || (eu == a && ev < b)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// 3. every root with an outgoing edge hooks below the far component
__global__ void __launch_bounds__(MST_THREADS) k_mst_hook(MstArgs A, int r)
{
    if (!A.flags[r]) return;
    const int64_t total = A.n * A.T;
    bool hooked = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / A.T;
        const int tt = (int)(i - c * A.T);
        const int64_t tb = A.tb0 + tt;
        if (tb >= A.K) continue;
        if ((int64_t)(A.R[i] >> 1) != c) continue;  // not a root
        const int2 e = A.win[i];
        if (e.x < 0) continue;                       // nothing leaves: this tree's component is complete
        const uint32_t x = (uint32_t)e.x, y = (uint32_t)e.y & SB_ID_MASK, neg = (uint32_t)e.y >> 31;
        const uint32_t rx = A.R[(int64_t)x * A.T + tt], ry = A.R[(int64_t)y * A.T + tt];
        const uint32_t c2 = ry >> 1;
        const int2 e2 = A.win[(int64_t)c2 * A.T + tt];
        const bool mutual = e2.x >= 0 && (A.R[(int64_t)((uint32_t)e2.y & SB_ID_MASK) * A.T + tt] >> 1) == (uint32_t)c;
        if (mutual && (uint32_t)c < c2) continue;  // the smaller root stays a root
        A.P[i] = (c2 << 1) | ((rx ^ ry ^ neg) & 1u);
        hooked = true;
        if (A.in_tree) {
            const uint32_t a = x < y ? x : y, b = x < y ? y : x;
            const int64_t k = mst_edge_index(A.edges, A.m, a, b);
            if (k < A.m && (uint32_t)A.edges[k].x == a && ((uint32_t)A.edges[k].y & SB_ID_MASK) == b)
                A.in_tree[tb * A.m + k] = 1;
            else
                atomicOr(A.err, 4u);
        }
    }
    if (__syncthreads_or(hooked) && threadIdx.x == 0) A.flags[r + 1] = 1;
}

// 4. pointer jumping to the roots; a pointer's low bit is the parity of the
// path to its target.  Roots do not move here, and every stored pointer names
// an ancestor, so a walk only climbs; it is bounded all the same.
__global__ void __launch_bounds__(MST_THREADS) k_mst_jump(MstArgs A, int r)
{
    if (!A.flags[r + 1]) return;
    const int64_t total = A.n * A.T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / A.T;
        const int tt = (int)(i - v * A.T);
        if (A.tb0 + tt >= A.K) continue;
        uint32_t w = mst_ld(A.P + i);
        int64_t steps = 0;
        while (true) {
            const uint32_t a = w >> 1;
            const uint32_t wa = mst_ld(A.P + (int64_t)a * A.T + tt);
            if ((wa >> 1) == a) break;  // a is a root
            w = (wa & ~1u) | ((w ^ wa) & 1u);
            A.P[i] = w;
            if (++steps > A.n) {
                atomicOr(A.err, 4u);
                break;
            }
        }
        A.R[i] = w;
        A.B[i] = ~0ull;
        A.win[i] = make_int2(-1, -1);
    }
}

// raw labels (parity to the root) as 32-bit ballots, and the spanning check:
// every vertex must share its graph's first vertex's root
__global__ void __launch_bounds__(MST_THREADS) k_mst_pack(MstArgs A, uint32_t* lab32, int W, int w0)
{
    const int64_t total = A.n * A.T;  // a multiple of 32: whole warps per vertex
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / A.T;
        const int tt = (int)(i - v * A.T);
        const bool valid = A.tb0 + tt < A.K;
        const uint32_t rv = A.R[i];
        const unsigned bal = __ballot_sync(0xffffffffu, valid && (rv & 1u));
        // the last pass may hold words past W: they are not written
        if ((threadIdx.x & 31) == 0 && w0 + (tt >> 6) < W) lab32[(v * W + w0) * 2 + (tt >> 5)] = bal;
        if (valid) {
            const int64_t g0 = A.vgoff ? A.vgoff[v] : 0;
            if ((A.R[g0 * A.T + tt] >> 1) != (rv >> 1)) atomicOr(A.err, 4u);
        }
    }
}

static sb_status mst_scratch(sb_ctx* c, size_t slots)
{
    if (c->mst_cap >= slots && c->mst_flags) return SB_OK;
    sb_dfree(c, c->mst_P);
    sb_dfree(c, c->mst_R);
    sb_dfree(c, c->mst_Y);
    sb_dfree(c, c->mst_L);
    sb_dfree(c, c->mst_B);
    sb_dfree(c, c->mst_win);
    sb_dfree(c, c->mst_flags);
    c->mst_P = (uint32_t*)sb_dalloc(c, sizeof(uint32_t) * slots);
    c->mst_R = (uint32_t*)sb_dalloc(c, sizeof(uint32_t) * slots);
    c->mst_Y = (uint32_t*)sb_dalloc(c, sizeof(uint32_t) * slots);
    c->mst_L = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * slots);
    c->mst_B = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * slots);
    c->mst_win = (int2*)sb_dalloc(c, sizeof(int2) * slots);
    c->mst_flags = (int32_t*)sb_dalloc(c, sizeof(int32_t) * 64);
    const bool ok = c->mst_P && c->mst_R && c->mst_Y && c->mst_L && c->mst_B && c->mst_win && c->mst_flags;
    c->mst_cap = ok ? slots : 0;
    if (!ok) return sb_fail(c, SB_ERR_OOM, "Kruskal scratch (%zu slots)", slots);
    return SB_OK;
}

extern "C" sb_status sb_sample_trees_kruskal(sb_ctx* c, uint64_t seed, int64_t tree_begin, int64_t K,
                                             uint8_t* in_tree_out)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_graph) return sb_fail(c, SB_ERR_STATE, "no graph loaded");
    if (K < 1 || K > SB_TREES_MAX || tree_begin < 0)
        return sb_fail(c, SB_ERR_ARG, "K must be in [1, %d] and tree_begin >= 0", SB_TREES_MAX);
    if (in_tree_out && !sb_is_device_ptr(in_tree_out))
        return sb_fail(c, SB_ERR_ARG, "in_tree_out must be a device pointer");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(sb_batch_begin(c, seed, tree_begin, K));
    const int64_t n = c->n;
    const int W = c->W;
    // words per pass: as many as the scratch budget holds (at most half the
    // free memory), at least one, and at most the SB_TUNE_MST_WORDS knob
    size_t free_b = 0, total_b = 0;
    SB_CHECK_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    const uint64_t budget = std::min<uint64_t>(MST_PASS_BUDGET, (uint64_t)free_b / 2);
    const int64_t per_word = n * 64 * MST_BYTES_PER_SLOT;
    int Wp = (int)std::max<int64_t>(1, std::min<int64_t>(W, (int64_t)(budget / (uint64_t)per_word)));
    if (c->tune[SB_TUNE_MST_WORDS] > 0) Wp = std::min<int>(Wp, (int)c->tune[SB_TUNE_MST_WORDS]);
    const int T = 64 * Wp;
    SB_TRY(mst_scratch(c, (size_t)n * T));
    // rounds: ceil(log2(largest graph)) + 1
    int64_t nmax = n;
    if (c->batch_G > 0) {
        nmax = 1;
        for (int64_t g = 0; g < c->batch_G; g++) nmax = std::max<int64_t>(nmax, c->h_voff[g + 1] - c->h_voff[g]);
    }
    int rounds = 1;
    while (((int64_t)1 << (rounds - 1)) < nmax) rounds++;
    if (in_tree_out) SB_CHECK_CUDA(c, cudaMemsetAsync(in_tree_out, 0, (size_t)K * (size_t)c->m, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync, 0, sizeof(uint32_t) * 16, c->stream));

    MstArgs A;
    A.n = n;
    A.T = T;
    A.K = K;
    A.S = sb_seed_key(seed);
    A.tree0 = tree_begin;
    A.rowptr = c->rowptr;
    A.col = c->col;
    A.vgoff = c->batch_G > 0 ? c->vgoff : nullptr;
    A.P = c->mst_P;
    A.R = c->mst_R;
    A.Y = c->mst_Y;
    A.L = c->mst_L;
    A.B = c->mst_B;
    A.win = c->mst_win;
    A.flags = c->mst_flags;
    A.edges = c->edges;
    A.m = c->m;
    A.in_tree = in_tree_out;
    A.err = c->sync + 6;
    const unsigned grid = (unsigned)std::min<int64_t>(sb_cdiv(n * T, MST_THREADS), (int64_t)c->num_sms * 16);
    SbProf prof(c, SB_PROF_BFS);
    for (int w0 = 0; w0 < W; w0 += Wp) {
        A.tb0 = 64 * (int64_t)w0;
        SB_CHECK_CUDA(c, cudaMemsetAsync(c->mst_flags, 0, sizeof(int32_t) * 64, c->stream));
        SB_CHECK_CUDA(c, cudaMemsetAsync(c->mst_flags, 0xFF, sizeof(int32_t), c->stream));  // round 0 runs
        k_mst_init<<<grid, MST_THREADS, 0, c->stream>>>(A);
        SB_TRY(sb_after_launch(c, "k_mst_init"));
        for (int r = 0; r < rounds; r++) {
            k_mst_min<<<grid, MST_THREADS, 0, c->stream>>>(A, r);
            SB_TRY(sb_after_launch(c, "k_mst_min"));
            k_mst_win<<<grid, MST_THREADS, 0, c->stream>>>(A, r);
            SB_TRY(sb_after_launch(c, "k_mst_win"));
            k_mst_hook<<<grid, MST_THREADS, 0, c->stream>>>(A, r);
            SB_TRY(sb_after_launch(c, "k_mst_hook"));
            k_mst_jump<<<grid, MST_THREADS, 0, c->stream>>>(A, r);
            SB_TRY(sb_after_launch(c, "k_mst_jump"));
        }
        k_mst_pack<<<grid, MST_THREADS, 0, c->stream>>>(A, (uint32_t*)c->labels, W, w0);
        SB_TRY(sb_after_launch(c, "k_mst_pack"));
    }
    return sb_batch_end(c);
}
