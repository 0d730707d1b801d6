// sb_bpp.cu -- graphBpp hot path: batched randomized-BFS tree sampling with
// parity labelling (Algorithm 1 through the appendix graphB+ algorithm,
// restated with Harary's bipartition, Sec. 2), the state hash that keys the
// frustration cloud (the frustration scorer is in sb_score.cu).
//
// Data layout (vertex-major, 64 trees per uint64 word):
//   labels[v * W + w]  bit b = parity label of tree 64 w + b at vertex v
//   vis / frontier     [v * Wb + w] for the Wb words of one BFS launch
// A BFS launch grows up to 32 words (2048 trees) at once, level by level, in
// one cooperative persistent kernel: a group of G lanes owns one vertex (lane
// = word), gathers its neighbours' frontier words with coalesced row loads,
// and picks each newly reached tree's parent as the argmin of the packed key
// (fmix32((u ^ y_v) + a_t) << 32 | u).  fmix32 is a bijection, so the hash
// alone orders the candidates of one (tree, vertex): comparing 32-bit hashes
// is the 64-bit packed argmin.  Rows longer than SB_BFS_CHUNK are split over
// several groups that merge with 64-bit atomicMin on the packed key.
#include <algorithm>

#include "sb_internal.cuh"

#define BFS_THREADS 128
#define BFS_THREADS_PAR 128
// Candidate-queue entries per lane (overflow falls back to per-lane hashing):
// the host takes the largest count in this range that keeps the most blocks
// resident per SM (the salts of a launch grow with its words).
#define BFS_QUEUE_MIN 8
#define BFS_QUEUE_MAX 32
#define BFS_BLOCKS_PER_SM 5     // the registers of one block allow 5 per SM (at most 102 per thread)
#define SYNC_WORDS 48
// Shared-memory slots of (owner thread o, tree t): owner-major rows padded so
// that one owner's trees, and one tree of consecutive owners, fall in
// different banks (the hash rounds walk one owner's trees in lockstep).
#define BSLOT(o, t) ((o) * 65 + (t))  // 32-bit minima / winner ids
#define KSLOT(w, t) ((w) * 65 + (t))  // tree salts of word w

struct BfsArgs {
    const sb_bfs_item* items;
    int64_t n_items;
    const int32_t* col;
    const int32_t* hub_vertex;
    int64_t n_hubs;
    uint64_t* lab;   // n x Wt
    int Wt, w0, Wb;
    uint64_t* vis;   // n x Wb
    uint64_t* fr0;
    uint64_t* fr1;
    int32_t* done;
    uint64_t* hubnew;   // n_hubs x Wb
    uint64_t* hubbest;  // n_hubs x Wb x 64
    uint32_t* sync;
    int32_t* parents;   // K x n or null
    int64_t n;
    uint64_t S;         // seed key
    const int64_t* tree0;  // global index of batch tree 0 (device)
    const int32_t* vgoff;  // first vertex of each vertex's graph (batches), or null
    long long wait;        // SM cycles a barrier wait may take before it reports a timeout
    unsigned bar_extra;    // arrivals a barrier expects beyond the launch's blocks (0; 1 tests the timeout path)
    int qcap;              // candidate-queue entries per lane
};

// ----------------------------------------------------------- grid barrier
// Cooperative launch makes every block resident; the wait is still bounded
// (`limit` SM cycles) and reports a timeout through sync[6] instead of
// hanging.  `nblocks` is the number of arrivals that open the barrier.
__device__ __forceinline__ void grid_barrier(uint32_t* sync, unsigned nblocks, long long limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* gen = sync + 5;
        uint32_t g = *gen;
        __threadfence();
        uint32_t arrived = atomicAdd(sync + 4, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(sync + 4, 0u);
            __threadfence();
            atomicAdd(sync + 5, 1u);
        } else {
            long long t0 = clock64();
            while (*gen == g) {
                __nanosleep(40);
                if (clock64() - t0 > limit) {
                    atomicOr(sync + 6, 1u);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned group_mask(int G)
{
    if (G >= 32) return 0xffffffffu;
    unsigned base = (threadIdx.x & 31u) & ~(unsigned)(G - 1);
    return ((1u << G) - 1u) << base;
}

// Fetch the 128-byte line at p into L2 (no register result, nothing waits).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Winner label bits: each lane keeps its trees' bits in two registers (trees
// 0-31 and 32-63) while it hashes its own candidates; the queue paths, where
// lanes write each other's trees, work on a copy in shared memory (two words
// per thread) with atomic bit updates.
__device__ __forceinline__ void lbit_put_atomic(uint32_t* lbits, int o, int t, uint32_t v)
{
    uint32_t* w = lbits + 2 * o + (t >> 5);
    const uint32_t m = 1u << (t & 31);
    if (v) atomicOr(w, m);
    else atomicAnd(w, ~m);
}

// Position of the highest set bit of a nonzero word.
__device__ __forceinline__ int bit_high(uint32_t x)
{
    uint32_t r;
    asm("bfind.u32 %0, %1;" : "=r"(r) : "r"(x));
    return (int)r;
}

// Group-wide exclusive prefix sum over the G lanes of one vertex.
template <int G>
__device__ __forceinline__ int group_excl_scan(int x, unsigned gmask, int gl, int& total)
{
    int incl = x;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const int y = __shfl_up_sync(gmask, incl, d, G);
        if (gl >= d) incl += y;
    }
    total = __shfl_sync(gmask, incl, G - 1, G);
    return incl - x;
}

// One pass over a CSR range for one vertex: lane gl of the group owns word
// w0 + gl.  Neighbours are read 8 at a time so that 8 frontier gathers are in
// flight per lane.  It keeps the running argmin of the hashed parent key over
// the candidates in `mask`: best (initialised to 0xFFFFFFFF) holds the
// smallest hash, lbv / bestu the winner's label bit / id; keys are distinct
// (the hash is a bijection in u), so `h <= best` accepts exactly the minimum.
// `once` returns the trees that had a candidate.  For each tile of 8
// neighbours the lanes hash their own candidates when their shares are even;
// otherwise the group's candidate bits are compacted into a shared queue
// (entry = neighbour, owner lane, tree, label bit) and hashed by all lanes in
// lockstep: the 8 neighbours at once (atomicMin, then the entry equal to the
// minimum writes its label), or, when they hold more candidates than the
// queue, one neighbour at a time (its entries have distinct slots).
// `cur` and `lab` are rewritten between levels by other blocks, so they are
// read with plain (coherent) loads; the column array is read-only.
template <bool PAR, int BD, int G>
__device__ __forceinline__ void scan_row(const int32_t* cp, int len, const uint64_t* cur, const uint64_t* lab, int Wb,
                                         int Wt, int wofs, int gl, uint64_t mask, uint32_t y, uint32_t goff,
                                         const uint32_t* akey, uint32_t* best, uint32_t* lbits, uint32_t (&lbv)[2],
                                         int32_t* bestu, uint16_t* queue, int qcap, uint32_t* hxs, int tid, unsigned gmask,
                                         uint64_t& once, uint32_t& nhash)
{
    // frontier rows are Wb words (128 B at 16 words) at 8 Wb-byte offsets; the
    // rows of the tile after next are fetched into L2 while this tile is
    // hashed, one line per lane (lanes 0-7: first lines of the 8 rows, lanes
    // 8-15: second lines)
    const int pf_k = gl & 7, pf_line = gl >> 3;
    const bool pf = gl < 16 && pf_line * 16 < Wb;
    for (int j = 0; j < len; j += 8) {
        uint32_t c[8];
        uint64_t f[8], l[8];
#pragma unroll
        for (int k = 0; k < 8; k++) c[k] = (j + k < len) ? (uint32_t)__ldg(cp + j + k) : 0u;
        if (pf && j + 16 + pf_k < len) {
            const uint32_t cn = (uint32_t)__ldg(cp + j + 16 + pf_k);
            prefetch_l2(cur + (int64_t)(cn & SB_ID_MASK) * Wb + 16 * pf_line);
        }
#pragma unroll
        for (int k = 0; k < 8; k++)
            f[k] = (j + k < len && mask) ? (cur[(int64_t)(c[k] & SB_ID_MASK) * Wb + gl] & mask) : 0ull;
#pragma unroll
        for (int k = 0; k < 8; k++)
            l[k] = f[k] ? (lab[(int64_t)(c[k] & SB_ID_MASK) * Wt + wofs] ^ ((c[k] >> 31) ? ~0ull : 0ull)) : 0ull;
        {
            const int owner0 = tid - gl;  // thread index of the group's lane 0
            int cnt = 0;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                once |= f[k];
                cnt += __popcll(f[k]);
            }
            const unsigned Tsum = __reduce_add_sync(gmask, (unsigned)cnt);
            if (Tsum == 0) continue;  // same for the whole group
            nhash += (uint32_t)cnt;
            const unsigned cmax = __reduce_max_sync(gmask, (unsigned)cnt);
            if (cmax * G <= 2 * Tsum + 2 * G) {
                // the lanes' shares are even enough: every lane hashes its own
                // candidates into its own slots (32-bit halves, two at a time),
                // with no queue and no synchronisation
                const uint32_t* ak = akey + KSLOT(gl, 0);
                uint32_t* bs = best + BSLOT(tid, 0);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint32_t u = (c[k] & SB_ID_MASK) - goff;
                    const uint32_t hx = u ^ y;
#pragma unroll
                    for (int half = 0; half < 2; half++) {
                        uint32_t m = (uint32_t)(f[k] >> (32 * half));
                        const uint32_t lw = (uint32_t)(l[k] >> (32 * half));
                        const int t0 = 32 * half;
                        while (m) {
                            // the highest and the lowest candidate (the same
                            // one when a single candidate is left)
                            const int ia = bit_high(m);
                            const int ib = __ffs(m) - 1;
                            const bool two = ia != ib;
                            m &= ~((1u << ia) | (1u << ib));
                            const uint32_t ha = sb_fmix32(hx + ak[t0 + ia]);
                            const uint32_t hb = sb_fmix32(hx + ak[t0 + ib]);
                            const uint32_t ba = bs[t0 + ia], bb = bs[t0 + ib];
                            // the winner's label bit goes into bit t of the half's label word
                            if (ha <= ba) {  // <=: the minima start at 0xFFFFFFFF
                                bs[t0 + ia] = ha;
                                lbv[half] ^= (lbv[half] ^ lw) & (1u << ia);
                                if (PAR) bestu[BSLOT(tid, t0 + ia)] = (int32_t)u;
                            }
                            if (two && hb <= bb) {
                                bs[t0 + ib] = hb;
                                lbv[half] ^= (lbv[half] ^ lw) & (1u << ib);
                                if (PAR) bestu[BSLOT(tid, t0 + ib)] = (int32_t)u;
                            }
                        }
                    }
                }
                continue;
            }
            // the queue paths update other lanes' label bits: through shared memory
            lbits[2 * tid] = lbv[0];
            lbits[2 * tid + 1] = lbv[1];
            int T;
            int pos = group_excl_scan<G>(cnt, gmask, gl, T);
            if (T <= qcap * G) {
                // the candidates of all 8 neighbours go through one queue of
                // (neighbour, owner word, tree, label bit) entries; lanes hash
                // them in lockstep, keep each tree's minimum with atomicMin
                // (two neighbours may reach the same tree) and then let the
                // one entry equal to the minimum write its label bit
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    // the group's table of the 8 neighbours' u ^ y (one writer per entry)
                    if ((k & (G - 1)) == gl) hxs[k] = ((c[k] & SB_ID_MASK) - goff) ^ y;
                    for (uint64_t b = f[k]; b;) {
                        const int t = __ffsll((long long)b) - 1;
                        b &= b - 1;
                        queue[pos++] = (uint16_t)((k << 12) | (gl << 7) | (t << 1) | (int)((l[k] >> t) & 1ull));
                    }
                }
                __syncwarp(gmask);
                for (int i = gl; i < T; i += G) {
                    const uint32_t e = queue[i];
                    const int k = (int)(e >> 12), ow = (int)((e >> 7) & 31u), t = (int)((e >> 1) & 63u);
                    const uint32_t h = sb_fmix32(hxs[k] + akey[KSLOT(ow, t)]);
                    atomicMin(&best[BSLOT(owner0 + ow, t)], h);
                }
                __syncwarp(gmask);
                for (int i = gl; i < T; i += G) {
                    const uint32_t e = queue[i];
                    const int k = (int)(e >> 12), ow = (int)((e >> 7) & 31u), t = (int)((e >> 1) & 63u);
                    const uint32_t hxk = hxs[k];
                    const uint32_t h = sb_fmix32(hxk + akey[KSLOT(ow, t)]);
                    const uint32_t u = hxk ^ y;
                    const int o = owner0 + ow;
                    if (best[BSLOT(o, t)] == h) {  // fmix32 is injective in u: one entry matches
                        lbit_put_atomic(lbits, o, t, e & 1u);
                        if (PAR) bestu[BSLOT(o, t)] = (int32_t)u;
                    }
                }
                __syncwarp(gmask);
                lbv[0] = lbits[2 * tid];
                lbv[1] = lbits[2 * tid + 1];
                continue;
            }
            // many candidates: one neighbour at a time
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int cntk = __popcll(f[k]);
                int Tk;
                int posk = group_excl_scan<G>(cntk, gmask, gl, Tk);
                if (Tk == 0) continue;  // same for the whole group
                const uint32_t u = (c[k] & SB_ID_MASK) - goff;  // id inside the graph
                const uint32_t hx = u ^ y;
                if (Tk > qcap * G) {
                    // more candidates than the queue holds; each lane hashes
                    // its own bits (it alone owns their slots)
                    for (uint64_t b = f[k]; b;) {
                        const int t = __ffsll((long long)b) - 1;
                        b &= b - 1;
                        const uint32_t h = sb_fmix32(hx + akey[KSLOT(gl, t)]);
                        if (h <= best[BSLOT(tid, t)]) {  // <=: the minima start at 0xFFFFFFFF
                            best[BSLOT(tid, t)] = h;
                            lbit_put_atomic(lbits, tid, t, (uint32_t)(l[k] >> t) & 1u);
                            if (PAR) bestu[BSLOT(tid, t)] = (int32_t)u;
                        }
                    }
                    __syncwarp(gmask);
                    continue;
                }
                for (uint64_t b = f[k]; b;) {
                    const int t = __ffsll((long long)b) - 1;
                    b &= b - 1;
                    queue[posk++] = (uint16_t)((gl << 7) | (t << 1) | (int)((l[k] >> t) & 1ull));
                }
                __syncwarp(gmask);
                // two entries per lane and round: entries of one neighbour have
                // distinct slots, so their updates are independent
                for (int i = gl; i < Tk; i += 2 * G) {
                    const bool two = i + G < Tk;
                    const uint32_t ea = queue[i], eb = queue[two ? i + G : i];
                    const int owa = (int)((ea >> 7) & 31u), ta = (int)((ea >> 1) & 63u);
                    const int owb = (int)((eb >> 7) & 31u), tb = (int)((eb >> 1) & 63u);
                    const uint32_t ha = sb_fmix32(hx + akey[KSLOT(owa, ta)]);
                    const uint32_t hb = sb_fmix32(hx + akey[KSLOT(owb, tb)]);
                    const int oa = owner0 + owa, ob = owner0 + owb;
                    const uint32_t ba = best[BSLOT(oa, ta)], bb = best[BSLOT(ob, tb)];
                    if (ha <= ba) {
                        best[BSLOT(oa, ta)] = ha;
                        lbit_put_atomic(lbits, oa, ta, ea & 1u);
                        if (PAR) bestu[BSLOT(oa, ta)] = (int32_t)u;
                    }
                    if (two && hb <= bb) {
                        best[BSLOT(ob, tb)] = hb;
                        lbit_put_atomic(lbits, ob, tb, eb & 1u);
                        if (PAR) bestu[BSLOT(ob, tb)] = (int32_t)u;
                    }
                }
                __syncwarp(gmask);
            }
            lbv[0] = lbits[2 * tid];
            lbv[1] = lbits[2 * tid + 1];
        }
    }
}

// Resets the running minima of the trees in `mask`.
template <int BD>
__device__ __forceinline__ void best_reset(uint32_t* best, int tid, uint64_t mask)
{
    for (uint64_t b = mask; b;) {
        const int t = __ffsll((long long)b) - 1;
        b &= b - 1;
        best[BSLOT(tid, t)] = 0xFFFFFFFFu;
    }
}

template <int G, bool PAR>
__global__ void __launch_bounds__(PAR ? BFS_THREADS_PAR : BFS_THREADS, PAR ? 2 : BFS_BLOCKS_PER_SM)
    k_bfs(BfsArgs A)
{
    constexpr int BD = PAR ? BFS_THREADS_PAR : BFS_THREADS;
    extern __shared__ uint32_t smem[];
    uint32_t* akey = smem;                        // tree salts, KSLOT(word, tree)
    uint32_t* best = smem + A.Wb * 65;            // running minima, BSLOT(thread, tree)
    uint32_t* lbits = best + 65 * BD;             // winners' label bits (queue paths), two words per thread
    uint16_t* queues = (uint16_t*)(lbits + 2 * BD);  // A.qcap x G entries per group
    int32_t* bestu = (int32_t*)(queues + ((A.qcap * BD + 1) & ~1));  // winners, BSLOT (PAR only)
    uint32_t* hx_tab = (uint32_t*)(bestu + (PAR ? 65 * BD : 0));    // 8 neighbours' u ^ y per group
    __shared__ uint32_t s_any, s_stop;

    const int tid = threadIdx.x;
    const int gl = tid & (G - 1);
    const bool act = gl < A.Wb;
    const unsigned gmask = group_mask(G);
    const int64_t groups_total = (int64_t)gridDim.x * (BD / G);
    const int64_t group_id = (int64_t)blockIdx.x * (BD / G) + tid / G;
    const unsigned nblocks = gridDim.x + A.bar_extra;

    const int64_t tree0 = *A.tree0;
    for (int i = tid; i < A.Wb * 64; i += BD)
        akey[KSLOT(i >> 6, i & 63)] = (uint32_t)sb_tree_key(A.S, tree0 + 64 * (int64_t)A.w0 + i);
    if (tid == 0) s_any = 0;
    __syncthreads();

    const int Wb = A.Wb, Wt = A.Wt, w0 = A.w0;
    const int wofs = w0 + gl;
    uint16_t* queue = queues + (tid / G) * (A.qcap * G);
    uint32_t* hxs = hx_tab + (tid / G) * 8;
    uint32_t n_scan = 0, n_hash = 0, n_hash_hub = 0;  // work counters
    // level 1 is built top-down before the launch (k_bfs_level1): every
    // neighbour of a root has that root as its only candidate
    int L = 2;
    while (true) {
        const uint64_t* cur = (L & 1) ? A.fr0 : A.fr1;
        uint64_t* nxt = (L & 1) ? A.fr1 : A.fr0;
        bool any_new = false;

        // ---- phase A: every work item (whole rows, and chunks of split rows)
        // The items are sorted by descending degree and dealt out in rounds of
        // one item per group, the order of the groups reversing every round,
        // so that every group's sum of item sizes comes out about the same.
        for (int64_t r = 0;; r++) {
            const int64_t it_beg = r * groups_total + ((r & 1) ? groups_total - 1 - group_id : group_id);
            if (r * groups_total >= A.n_items) break;
            const int64_t it_end = min(A.n_items, it_beg + 1);
            for (int64_t it = it_beg; it < it_end; it++) {
                const sb_bfs_item itm = A.items[it];
                const int32_t v = itm.v;
                const int32_t d = A.done[v];
                if (d >= 0 && L >= d + 3) continue;
                const uint64_t vis_w = act ? A.vis[(int64_t)v * Wb + gl] : ~0ull;
                const uint64_t U = ~vis_w;
                const int32_t* cp = A.col + itm.beg;
                const int len = itm.end - itm.beg;
                const bool hub = itm.hub >= 0;
                uint64_t once = 0, labx = 0;
                // the pass below synchronises the group's lanes, so every lane of
                // the group enters it (a lane with nothing to do has mask 0)
                if (__any_sync(gmask, U != 0)) {
                    const uint32_t goff = A.vgoff ? (uint32_t)A.vgoff[v] : 0u;
                    const uint32_t y = sb_child_salt(A.S, (uint32_t)v - goff);
                    if (U) n_scan += (uint32_t)len;
                    // one pass: every candidate of every open tree is hashed (a
                    // first pass that singled out the trees with two or more
                    // candidates cost more than the few hashes it saved)
                    best_reset<BD>(best, tid, U);
                    uint32_t lbv[2] = {0u, 0u};
                    scan_row<PAR, BD, G>(cp, len, cur, A.lab, Wb, Wt, wofs, gl, U, y, goff, akey, best, lbits, lbv,
                                         bestu, queue, A.qcap, hxs, tid, gmask, once, hub ? n_hash_hub : n_hash);
                    labx = (((uint64_t)lbv[1] << 32) | lbv[0]) & once;
                }
                if (hub) {
                    // chunk of a split row: publish the chunk minima, one atomic per tree
                    if (once) {
                        uint64_t* hb = A.hubbest + ((int64_t)itm.hub * Wb + gl) * 64;
                        for (uint64_t b = once; b;) {
                            const int t = __ffsll((long long)b) - 1;
                            b &= b - 1;
                            const unsigned long long key = ((unsigned long long)best[BSLOT(tid, t)] << 32) |
                                                           (PAR ? ((unsigned long long)(uint32_t)bestu[BSLOT(tid, t)] << 1) : 0ull) |
                                                           ((labx >> t) & 1ull);
                            atomicMin((unsigned long long*)(hb + t), key);
                        }
                        atomicOr((unsigned long long*)(A.hubnew + (int64_t)itm.hub * Wb + gl), once);
                    }
                    continue;
                }
                if (PAR && A.parents) {
                    for (uint64_t b = once; b;) {
                        const int t = __ffsll((long long)b) - 1;
                        b &= b - 1;
                        A.parents[(64 * (int64_t)wofs + t) * A.n + v] = bestu[BSLOT(tid, t)];
                    }
                }
                if (act) {
                    if (once) {
                        A.lab[(int64_t)v * Wt + wofs] |= labx & once;
                        A.vis[(int64_t)v * Wb + gl] = vis_w | once;
                        any_new = true;
                    }
                    nxt[(int64_t)v * Wb + gl] = once;
                }
                if (d < 0) {
                    const bool full = (vis_w | once) == ~0ull;
                    const bool all = __all_sync(gmask, full);
                    if (all && gl == 0) A.done[v] = L;
                }
            }
        }  // rounds

        // ---- phase B: resolve split rows
        if (A.n_hubs > 0) {
            grid_barrier(A.sync, nblocks, A.wait);
            for (int64_t h = group_id; h < A.n_hubs; h += groups_total) {
                const int32_t v = A.hub_vertex[h];
                const int32_t d = A.done[v];
                if (d >= 0 && L >= d + 3) continue;
                uint64_t nw = 0, vis_w = ~0ull;
                if (act) {
                    vis_w = A.vis[(int64_t)v * Wb + gl];
                    uint64_t* hn = A.hubnew + h * Wb + gl;
                    nw = *hn & ~vis_w;
                    *hn = 0;
                    uint64_t labx = 0;
                    uint64_t* hb = A.hubbest + (h * Wb + gl) * 64;
                    for (uint64_t b = nw; b;) {
                        const int t = __ffsll((long long)b) - 1;
                        b &= b - 1;
                        const uint64_t key = hb[t];
                        hb[t] = ~0ull;
                        labx |= (key & 1ull) << t;
                        if (PAR && A.parents)
                            A.parents[(64 * (int64_t)wofs + t) * A.n + v] = (int32_t)((key >> 1) & SB_ID_MASK);
                    }
                    if (nw) {
                        A.lab[(int64_t)v * Wt + wofs] |= labx;
                        A.vis[(int64_t)v * Wb + gl] = vis_w | nw;
                        any_new = true;
                    }
                    nxt[(int64_t)v * Wb + gl] = nw;
                }
                if (d < 0) {
                    const bool all = __all_sync(gmask, (vis_w | nw) == ~0ull);
                    if (all && gl == 0) A.done[v] = L;
                }
            }
        }

        // ---- end of level: any tree grew?
        if (any_new) s_any = 1;
        __syncthreads();
        if (tid == 0) {
            if (s_any) atomicOr(A.sync + (L % 3), 1u);
            s_any = 0;
            if (blockIdx.x == 0) A.sync[(L + 1) % 3] = 0;
        }
        grid_barrier(A.sync, nblocks, A.wait);
        // one reader per block, so that every thread of a block leaves the
        // level loop at the same level
        if (tid == 0) {
            const uint32_t grew = *(volatile uint32_t*)(A.sync + (L % 3));
            const uint32_t err = *(volatile uint32_t*)(A.sync + 6);
            s_stop = (!grew || err) ? 1u : 0u;
        }
        __syncthreads();
        if (s_stop) break;
        if (++L > A.n + 1) {
            if (tid == 0 && blockIdx.x == 0) atomicOr(A.sync + 6, 2u);
            break;
        }
    }
    if (tid == 0 && blockIdx.x == 0) A.sync[7] = (uint32_t)L;
    // work counters (one atomic per warp and counter)
    for (int d = 16; d; d >>= 1) {
        n_scan += __shfl_xor_sync(0xffffffffu, n_scan, d);
        n_hash += __shfl_xor_sync(0xffffffffu, n_hash, d);
        n_hash_hub += __shfl_xor_sync(0xffffffffu, n_hash_hub, d);
    }
    if ((tid & 31) == 0) {
        atomicAdd((unsigned long long*)(A.sync + 8), (unsigned long long)n_scan);
        atomicAdd((unsigned long long*)(A.sync + 10), (unsigned long long)n_hash);
        atomicAdd((unsigned long long*)(A.sync + 14), (unsigned long long)n_hash_hub);
    }
}

// ------------------------------------------------------------ BFS set-up
__global__ void k_bfs_init(int64_t n, int Wb, int Wt, int w0, int64_t K, uint64_t* vis, uint64_t* fr0, uint64_t* fr1,
                           uint64_t* lab, int32_t* done)
{
    int64_t total = n * Wb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = i / Wb;
        int w = (int)(i - v * Wb);
        int64_t trees = K - 64 * (int64_t)(w0 + w);  // trees of this word
        uint64_t active = trees >= 64 ? ~0ull : ((1ull << trees) - 1ull);
        vis[i] = ~active;
        fr0[i] = 0;
        fr1[i] = 0;
        lab[v * Wt + w0 + w] = 0;
        if (w == 0) done[v] = -1;
    }
}

__global__ void k_hub_init(int64_t nh, int Wb, uint64_t* hubnew, uint64_t* hubbest)
{
    int64_t total = nh * Wb * 64;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        hubbest[i] = ~0ull;
        if (i < nh * Wb) hubnew[i] = 0;
    }
}

// root of every tree of this launch in every graph (one graph unless voff)
__global__ void k_bfs_roots(int64_t n, int Wb, int w0, int64_t K, uint64_t S, const int64_t* tree0p, uint64_t* vis,
                            uint64_t* fr0, int32_t* parents, const int32_t* voff, int64_t G)
{
    const int64_t tree0 = *tree0p;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = 64 * (int64_t)Wb;
    if (x >= per * G) return;
    const int64_t g = x / per;
    const int64_t i = x - g * per;      // tree within this launch
    const int64_t tb = 64 * (int64_t)w0 + i;  // tree within the batch
    if (tb >= K) return;
    const uint64_t key = sb_tree_key(S, tree0 + tb);
    const int64_t base = voff ? voff[g] : 0;
    const int64_t ng = voff ? voff[g + 1] - voff[g] : n;
    const uint32_t r = (uint32_t)(base + sb_root(key, ng));
    int w = (int)(i >> 6);
    unsigned long long bit = 1ull << (i & 63);
    atomicOr((unsigned long long*)(vis + (int64_t)r * Wb + w), bit);
    atomicOr((unsigned long long*)(fr0 + (int64_t)r * Wb + w), bit);
    if (parents) parents[tb * n + r] = -1;
}

// BFS level 1, top-down: a neighbour v of tree t's root r joins the tree at
// level 1 with r as its parent (the only vertex of level 0, so no hash
// decides), label lab(r) ^ neg(r, v) = neg(r, v).  One warp per (graph,
// tree of the launch); trees of one word may reach the same vertex, hence
// the atomics.  Frontier of level 1 -> fr1 (read as the current frontier of
// level 2).
__global__ void k_bfs_level1(int64_t n, int Wb, int Wt, int w0, int64_t K, uint64_t S, const int64_t* tree0p,
                             const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, uint64_t* vis,
                             uint64_t* fr1, uint64_t* lab, int32_t* parents, const int32_t* voff, int64_t G)
{
    const int64_t per = 64 * (int64_t)Wb;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= per * G) return;
    const int64_t g = warp / per;
    const int64_t i = warp - g * per;         // tree within this launch
    const int64_t tb = 64 * (int64_t)w0 + i;  // tree within the batch
    if (tb >= K) return;
    const uint64_t key = sb_tree_key(S, *tree0p + tb);
    const int64_t base = voff ? voff[g] : 0;
    const int64_t ng = voff ? voff[g + 1] - voff[g] : n;
    const int64_t r = base + sb_root(key, ng);
    const int w = (int)(i >> 6);
    const unsigned long long bit = 1ull << (i & 63);
    for (int32_t j = rowptr[r] + lane; j < rowptr[r + 1]; j += 32) {
        const uint32_t cv = (uint32_t)col[j];
        const int64_t v = cv & SB_ID_MASK;
        atomicOr((unsigned long long*)(vis + v * Wb + w), bit);
        atomicOr((unsigned long long*)(fr1 + v * Wb + w), bit);
        if (cv >> 31) atomicOr((unsigned long long*)(lab + v * Wt + w0 + w), bit);
        if (parents) parents[tb * n + v] = (int32_t)(r - base);
    }
}

// canonical flip per graph and word: the raw label of the graph's vertex 0
__global__ void k_flip(const uint64_t* lab, int W, uint64_t* flipw, const int32_t* voff, int64_t G)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (int64_t)W * G) return;
    const int64_t g = x / W;
    const int w = (int)(x - g * W);
    flipw[x] = lab[(voff ? (int64_t)voff[g] : 0) * W + w];
}

// The same state hashes from subset-sum tables.  A block takes a contiguous
// range of 32-vertex groups.  For each group it tabulates, for each of the
// group's four runs of 8 vertices, the 256 subset sums of their weights; a
// warp then takes one 64-tree word at a time: lane k loads vertex k's label
// word, two 32 x 32 bit transposes across the warp give lane j the group's
// vertices labelled 1 in trees j and j + 32, and four table lookups per tree
// add their weights.  The sums are over raw labels (root labelled 0): the
// canonical flip of a tree is applied afterwards (k_state_hash_flip), as
// H = W_g - H_raw when the tree's vertex 0 is labelled 1, W_g = total weight
// of graph g (Sec. 2: the canonical state is the raw one switched at every
// vertex, so its 1-set is the complement).  A group with vertices of several
// graphs (batches) is taken once per graph, with the other graphs' weights
// left out of the tables.
#define HT_THREADS 256
#define HT_WARPS (HT_THREADS / 32)
#define HT_WPW 8  // words per warp: 64 words over 8 warps

__global__ void __launch_bounds__(HT_THREADS, 4) k_state_hash_tab(const uint64_t* __restrict__ lab, int64_t n, int W,
                                                                  const uint64_t* __restrict__ weight,
                                                                  const int32_t* __restrict__ vgid, int64_t KP,
                                                                  int64_t groups_per_block,
                                                                  unsigned long long* __restrict__ Hraw,
                                                                  unsigned long long* __restrict__ wsum)
{
    // double-buffered, so that the tables of one group are built while no
    // thread can still be reading the buffer from two groups before
    __shared__ uint64_t tab[2][4][256];
    __shared__ uint64_t sw[2][32];
    const unsigned lane = threadIdx.x & 31u;
    const int warp = (int)(threadIdx.x >> 5);
    const int64_t ngroups = sb_cdiv(n, 32);
    const int64_t q0 = (int64_t)blockIdx.x * groups_per_block;
    const int64_t q1 = min(ngroups, q0 + groups_per_block);
    uint64_t accA[HT_WPW], accB[HT_WPW];
#pragma unroll
    for (int i = 0; i < HT_WPW; i++) accA[i] = accB[i] = 0;
    int64_t gcur = -1;
    int buf = 0;
    auto flush = [&]() {
        if (gcur < 0) return;
#pragma unroll
        for (int i = 0; i < HT_WPW; i++) {
            const int w = warp + HT_WARPS * i;
            if (w < W) {
                if (accA[i]) atomicAdd(Hraw + gcur * KP + 64 * w + lane, (unsigned long long)accA[i]);
                if (accB[i]) atomicAdd(Hraw + gcur * KP + 64 * w + 32 + lane, (unsigned long long)accB[i]);
            }
            accA[i] = accB[i] = 0;
        }
    };
    // table b, subsets s0 .. s0 + 3 of vertices 8 b .. 8 b + 7 of the group
    const int tb = (int)(threadIdx.x >> 6), s0 = (int)(threadIdx.x & 63u) << 2;
    for (int64_t q = q0; q < q1; q++) {
        const int64_t v0 = q * 32;
        const int64_t vk = v0 + lane;
        const int64_t vlast = min(n, v0 + 32) - 1;
        const int64_t ga = vgid ? vgid[v0] : 0, gb = vgid ? vgid[vlast] : 0;
        for (int64_t g = ga; g <= gb; g++) {  // the graphs present in the group (almost always one)
            if (g != gcur) {
                flush();
                gcur = g;
            }
            if (warp == 0) {  // the group's weights, and its share of the graph's total weight
                const uint64_t x = (vk < n && (!vgid || vgid[vk] == g)) ? weight[vk] : 0ull;
                sw[buf][lane] = x;
                uint64_t t = x;
#pragma unroll
                for (int dd = 16; dd; dd >>= 1) t += __shfl_xor_sync(0xffffffffu, t, dd);
                if (lane == 0 && t) atomicAdd(wsum + g, (unsigned long long)t);
            }
            __syncthreads();
            {
                const uint64_t* w8 = sw[buf] + 8 * tb;
                uint64_t base = 0;
#pragma unroll
                for (int i = 2; i < 8; i++)
                    if ((s0 >> i) & 1) base += w8[i];
                uint64_t* t4 = tab[buf][tb] + s0;
                t4[0] = base;
                t4[1] = base + w8[0];
                t4[2] = base + w8[1];
                t4[3] = base + w8[0] + w8[1];
            }
            __syncthreads();
            const uint64_t(*T)[256] = tab[buf];
#pragma unroll
            for (int i = 0; i < HT_WPW; i++) {
                const int w = warp + HT_WARPS * i;
                if (w >= W) break;
                const uint64_t L = vk < n ? lab[vk * W + w] : 0ull;
                const uint32_t MA = warp_transpose32((uint32_t)L, lane);
                const uint32_t MB = warp_transpose32((uint32_t)(L >> 32), lane);
                accA[i] += T[0][MA & 255u] + T[1][(MA >> 8) & 255u] + T[2][(MA >> 16) & 255u] + T[3][MA >> 24];
                accB[i] += T[0][MB & 255u] + T[1][(MB >> 8) & 255u] + T[2][(MB >> 16) & 255u] + T[3][MB >> 24];
            }
            buf ^= 1;
        }
    }
    flush();
}

// canonical flip of the raw sums: trees whose vertex 0 (of the tree's graph)
// is labelled 1 take the complement's weight
__global__ void k_state_hash_flip(unsigned long long* H, const unsigned long long* wsum, const uint64_t* flipw, int W,
                                  int64_t KP, int64_t G)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= KP * G) return;
    const int64_t g = x / KP;
    const int64_t t = x - g * KP;
    if ((flipw[g * W + t / 64] >> (t % 64)) & 1ull) H[x] = wsum[g] - H[x];
}

__global__ void k_canon_out(const uint64_t* __restrict__ lab, int64_t total, int W, int64_t K,
                            const uint64_t* __restrict__ flipw, const int32_t* __restrict__ vgid,
                            uint64_t* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / W;
        const int w = (int)(i - v * W);
        const int64_t g = vgid ? vgid[v] : 0;
        int64_t trees = K - 64 * (int64_t)w;
        uint64_t active = trees >= 64 ? ~0ull : ((1ull << trees) - 1ull);
        out[i] = (lab[i] ^ flipw[g * W + w]) & active;
    }
}

__global__ void k_fold_stats(const uint32_t* sync, unsigned long long* acc)
{
    const unsigned long long L = sync[7];
    if (L > acc[0]) acc[0] = L;
    acc[1] += 1;
    acc[2] += *(const unsigned long long*)(sync + 8);
    acc[3] += *(const unsigned long long*)(sync + 10);
    acc[4] += *(const unsigned long long*)(sync + 12);
    acc[5] += *(const unsigned long long*)(sync + 14);
}

// --------------------------------------------------------------- host side
static int group_for(int Wb)
{
    int g = 1;
    while (g < Wb) g <<= 1;
    return g;
}

template <bool PAR>
static const void* bfs_kernel(int G)
{
    switch (G) {
    case 1: return (const void*)k_bfs<1, PAR>;
    case 2: return (const void*)k_bfs<2, PAR>;
    case 4: return (const void*)k_bfs<4, PAR>;
    case 8: return (const void*)k_bfs<8, PAR>;
    case 16: return (const void*)k_bfs<16, PAR>;
    default: return (const void*)k_bfs<32, PAR>;
    }
}

static sb_status ensure_sync(sb_ctx* c)
{
    if (!c->sync) {
        c->sync = (uint32_t*)sb_dalloc(c, sizeof(uint32_t) * SYNC_WORDS);
        if (!c->sync) return sb_fail(c, SB_ERR_OOM, "sync words");
        SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync, 0, sizeof(uint32_t) * SYNC_WORDS, c->stream));
    }
    return SB_OK;
}

static sb_status run_bfs(sb_ctx* c, int w0, int Wb, int32_t* parents)
{
    const bool par = parents != nullptr;
    // lanes beyond the launch's words still share the hash rounds
    const int Gw = group_for(Wb), Gt = (int)c->tune[SB_TUNE_BFS_GROUP];
    const int G = (Gt > Gw && Gt <= 2 * Gw) ? Gt : Gw;  // widened at most twofold
    const int BD = par ? BFS_THREADS_PAR : BFS_THREADS;
    const void* fn = par ? bfs_kernel<true>(G) : bfs_kernel<false>(G);
    // shared memory of a block with q queue entries per lane; the largest q that
    // keeps the most blocks resident
    auto smem_for = [&](int q) -> size_t {
        return sizeof(uint32_t) * ((size_t)Wb * 65 + 65 * BD + 2 * BD) + sizeof(uint16_t) * (size_t)((q * BD + 1) & ~1) +
               (par ? sizeof(int32_t) * 65 * BD : 0) + sizeof(uint32_t) * 8 * (BD / G);
    };
    SB_CHECK_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for(BFS_QUEUE_MAX)));
    int per_sm = 0, qcap = BFS_QUEUE_MAX;
    for (int q = BFS_QUEUE_MAX; q >= BFS_QUEUE_MIN; q--) {
        int b = 0;
        SB_CHECK_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, BD, smem_for(q)));
        if (b > per_sm) {
            per_sm = b;
            qcap = q;
        }
    }
    const size_t smem = smem_for(qcap);
    if (per_sm < 1) return sb_fail(c, SB_ERR_CUDA, "BFS kernel does not fit on an SM");
    unsigned nblocks = (unsigned)(per_sm * c->num_sms);
    const int64_t n = c->n;
    unsigned g = (unsigned)std::min<int64_t>(sb_cdiv(n * Wb, 256), (int64_t)c->num_sms * 16);
    k_bfs_init<<<g, 256, 0, c->stream>>>(n, Wb, c->W, w0, c->K, c->vis, c->fr0, c->fr1, c->labels, c->done);
    SB_TRY(sb_after_launch(c, "k_bfs_init"));
    if (c->n_hubs > 0) {
        unsigned gh = (unsigned)std::min<int64_t>(sb_cdiv(c->n_hubs * Wb * 64, 256), (int64_t)c->num_sms * 16);
        k_hub_init<<<gh, 256, 0, c->stream>>>(c->n_hubs, Wb, c->hubnew, c->hubbest);
        SB_TRY(sb_after_launch(c, "k_hub_init"));
    }
    const int64_t ngraphs = c->batch_G > 0 ? c->batch_G : 1;
    k_bfs_roots<<<(unsigned)sb_cdiv(64 * Wb * ngraphs, 256), 256, 0, c->stream>>>(
        n, Wb, w0, c->K, sb_seed_key(c->seed), sb_tree0_ptr(c->sync), c->vis, c->fr0, parents,
        c->batch_G > 0 ? c->b_voff : nullptr, ngraphs);
    SB_TRY(sb_after_launch(c, "k_bfs_roots"));
    // level counters and barrier words of this launch (the error word sync[6]
    // is cleared per batch, so that an error of an earlier launch stays)
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync, 0, sizeof(uint32_t) * 6, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync + 7, 0, sizeof(uint32_t) * 9, c->stream));
    {
        const int64_t warps = 64 * (int64_t)Wb * ngraphs;
        k_bfs_level1<<<(unsigned)sb_cdiv(warps * 32, 256), 256, 0, c->stream>>>(
            n, Wb, c->W, w0, c->K, sb_seed_key(c->seed), sb_tree0_ptr(c->sync), c->rowptr, c->col, c->vis, c->fr1,
            c->labels, parents, c->batch_G > 0 ? c->b_voff : nullptr, ngraphs);
        SB_TRY(sb_after_launch(c, "k_bfs_level1"));
    }
    BfsArgs A;
    A.items = c->items;
    A.n_items = c->n_items;
    A.col = c->col;
    A.hub_vertex = c->hub_vertex;
    A.n_hubs = c->n_hubs;
    A.lab = c->labels;
    A.Wt = c->W;
    A.w0 = w0;
    A.Wb = Wb;
    A.vis = c->vis;
    A.fr0 = c->fr0;
    A.fr1 = c->fr1;
    A.done = c->done;
    A.hubnew = c->hubnew;
    A.hubbest = c->hubbest;
    A.sync = c->sync;
    A.parents = parents;
    A.n = n;
    A.S = sb_seed_key(c->seed);
    A.tree0 = sb_tree0_ptr(c->sync);
    A.vgoff = c->batch_G > 0 ? c->vgoff : nullptr;
    A.wait = sb_wait_cycles(c);
    A.bar_extra = c->tune[SB_TUNE_STALL_TEST] ? 1u : 0u;
    A.qcap = qcap;
    void* args[] = {&A};
    {
        // a cooperative launch (every block resident for the grid barrier),
        // issued through the launch-attribute form so that it can also be
        // captured into a CUDA graph
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeCooperative;
        attr.val.cooperative = 1;
        cfg.gridDim = dim3(nblocks);
        cfg.blockDim = dim3(BD);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        SbProf prof(c, SB_PROF_BFS);
        SB_CHECK_CUDA(c, cudaLaunchKernelExC(&cfg, fn, args));
        SB_TRY(sb_after_launch(c, "k_bfs"));
    }
    k_fold_stats<<<1, 1, 0, c->stream>>>(c->sync, (unsigned long long*)(c->sync + 16));
    return sb_after_launch(c, "k_fold_stats");
}

// *p = v, or *p += add when add != 0 (the device copy of the first tree)
__global__ void k_set_i64(int64_t* p, int64_t v, int64_t add)
{
    if (add) *p += add;
    else *p = v;
}

// errors of one step kept across the steps of sb_batch_steps: BFS barrier
// (sync[6]) and scorer tile copies (sync[28]) into sync[34]
__global__ void k_latch_errors(uint32_t* sync)
{
    uint32_t e = 0;
    if (sync[6] & 1u) e |= 1u;
    if (sync[6] & ~1u) e |= 2u;
    if (sync[28]) e |= 1u;
    if (e) atomicOr(sync + 34, e);
}

__global__ void k_fold_min(int32_t* acc, const int32_t* x, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] = min(acc[i], x[i]);
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

static sb_status check_sync_error(sb_ctx* c)
{
    uint32_t err = 0;
    SB_CHECK_CUDA(c, cudaMemcpyAsync(&err, c->sync + 6, sizeof(err), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (err & 1u) return sb_fail(c, SB_ERR_TIMEOUT, "BFS grid barrier timed out");
    if (err & 2u) return sb_fail(c, SB_ERR_DEVICE_CHECK, "BFS exceeded n levels");
    if (err & 4u) return sb_fail(c, SB_ERR_DEVICE_CHECK, "Kruskal trees did not span their graph");
    return SB_OK;
}

sb_status sb_batch_begin(sb_ctx* c, uint64_t seed, int64_t tree_begin, int64_t K)
{
    SB_TRY(ensure_sync(c));
    const int64_t n = c->n;
    const int W = (int)sb_cdiv(K, 64);
    size_t lab_bytes = sizeof(uint64_t) * (size_t)n * W;
    if (c->labels_cap < lab_bytes) {
        sb_dfree(c, c->labels);
        c->labels = (uint64_t*)sb_dalloc(c, lab_bytes);
        c->labels_cap = c->labels ? lab_bytes : 0;
    }
    const int64_t G = c->batch_G > 0 ? c->batch_G : 1;  // per-graph results in a batch
    // kept while large enough, so that repeated calls allocate nothing
    sb_status st = sb_ensure(c, (void**)&c->flipw, &c->flipw_cap, sizeof(uint64_t) * W * G);
    if (st == SB_OK) st = sb_ensure(c, (void**)&c->hashes, &c->hashes_cap, sizeof(uint64_t) * 64 * W * G);
    if (st == SB_OK) st = sb_ensure(c, (void**)&c->counts, &c->counts_cap, sizeof(int32_t) * 64 * W * G);
    c->has_batch = false;
    if (st != SB_OK || !c->labels || !c->flipw || !c->hashes || !c->counts)
        return sb_fail(c, SB_ERR_OOM, "batch storage (n=%lld, K=%lld)", (long long)n, (long long)K);
    c->seed = seed;
    c->tree_begin = tree_begin;
    c->K = K;
    c->W = W;
    c->counts_valid = false;
    c->batch_in_cloud = false;
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync + 16, 0, sizeof(uint32_t) * 16, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync + 6, 0, sizeof(uint32_t), c->stream));
    k_set_i64<<<1, 1, 0, c->stream>>>(sb_tree0_ptr(c->sync), tree_begin, 0);
    return sb_after_launch(c, "k_set_i64");
}

sb_status sb_batch_end(sb_ctx* c)
{
    const int64_t n = c->n, G = c->batch_G > 0 ? c->batch_G : 1;
    const int W = c->W;
    k_flip<<<(unsigned)sb_cdiv((int64_t)W * G, 256), 256, 0, c->stream>>>(c->labels, W, c->flipw,
                                                                          c->batch_G > 0 ? c->b_voff : nullptr, G);
    SB_TRY(sb_after_launch(c, "k_flip"));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->hashes, 0, sizeof(uint64_t) * 64 * W * G, c->stream));
    SB_TRY(sb_ensure(c, (void**)&c->hwsum, &c->hwsum_cap, sizeof(uint64_t) * (size_t)G));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->hwsum, 0, sizeof(uint64_t) * (size_t)G, c->stream));
    {
        SbProf prof(c, SB_PROF_HASH);
        const int64_t ngroups = sb_cdiv(n, 32);
        const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>((int64_t)c->num_sms * 4, sb_cdiv(ngroups, 16)));
        const int64_t per = sb_cdiv(ngroups, nblk);
        k_state_hash_tab<<<(unsigned)sb_cdiv(ngroups, per), HT_THREADS, 0, c->stream>>>(
            c->labels, n, W, c->vweight, c->batch_G > 0 ? c->vgid : nullptr, 64 * (int64_t)W, per,
            (unsigned long long*)c->hashes, (unsigned long long*)c->hwsum);
        SB_TRY(sb_after_launch(c, "k_state_hash_tab"));
        k_state_hash_flip<<<(unsigned)sb_cdiv(64 * (int64_t)W * G, 256), 256, 0, c->stream>>>(
            (unsigned long long*)c->hashes, (const unsigned long long*)c->hwsum, c->flipw, W, 64 * (int64_t)W, G);
        SB_TRY(sb_after_launch(c, "k_state_hash_flip"));
    }
    c->has_batch = true;
    return SB_OK;
}

static int bfs_words_per_launch(const sb_ctx* c)
{
    return c->tune[SB_TUNE_BFS_WORDS] > 0 ? (int)c->tune[SB_TUNE_BFS_WORDS] : SB_WORDS_MAX;
}

// BFS scratch for the current batch (kept while large enough)
static sb_status bfs_alloc(sb_ctx* c)
{
    const int64_t n = c->n;
    const int W = c->W;
    const int WL = bfs_words_per_launch(c);
    const int Wb_max = W < WL ? W : WL;
    size_t words = (size_t)n * Wb_max;
    if (c->bfs_cap_words < words) {
        sb_dfree(c, c->vis);
        sb_dfree(c, c->fr0);
        sb_dfree(c, c->fr1);
        sb_dfree(c, c->hubnew);
        sb_dfree(c, c->hubbest);
        c->vis = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * words);
        c->fr0 = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * words);
        c->fr1 = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * words);
        c->hubnew = (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)(c->n_hubs > 0 ? c->n_hubs : 1) * Wb_max);
        c->hubbest =
            (uint64_t*)sb_dalloc(c, sizeof(uint64_t) * (size_t)(c->n_hubs > 0 ? c->n_hubs : 1) * Wb_max * 64);
        c->bfs_cap_words = (c->vis && c->fr0 && c->fr1 && c->hubnew && c->hubbest) ? words : 0;
    }
    if (!c->done) c->done = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)n);
    if (!c->bfs_cap_words || !c->done)
        return sb_fail(c, SB_ERR_OOM, "BFS batch storage (n=%lld, K=%lld)", (long long)n, (long long)c->K);
    return SB_OK;
}

// the BFS launches of the current batch (no host synchronisation)
static sb_status bfs_enqueue(sb_ctx* c, int32_t* parents_out)
{
    const int W = c->W, WL = bfs_words_per_launch(c);
    for (int w0 = 0; w0 < W; w0 += WL) {
        const int Wb = W - w0 < WL ? W - w0 : WL;
        SB_TRY(run_bfs(c, w0, Wb, parents_out));
    }
    return SB_OK;
}

extern "C" sb_status sb_sample_trees(sb_ctx* c, uint64_t seed, int64_t tree_begin, int64_t K, int32_t* parents_out)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_graph) return sb_fail(c, SB_ERR_STATE, "no graph loaded");
    if (K < 1 || K > SB_TREES_MAX || tree_begin < 0)
        return sb_fail(c, SB_ERR_ARG, "K must be in [1, %d] and tree_begin >= 0", SB_TREES_MAX);
    if (parents_out && !sb_is_device_ptr(parents_out))
        return sb_fail(c, SB_ERR_ARG, "parents_out must be a device pointer");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(sb_batch_begin(c, seed, tree_begin, K));
    SB_TRY(bfs_alloc(c));
    const sb_status st = bfs_enqueue(c, parents_out);
    c->tune[SB_TUNE_STALL_TEST] = 0;  // a test of the timeout path covers one call
    SB_TRY(st);
    return sb_batch_end(c);
}

// One step of sb_batch_steps for the batch set up by sb_batch_begin: trees
// of the device's current range, counts, hashes and per-graph clouds, then
// the range moves on by K.  Enqueue only: no allocation, no host
// synchronisation, so that the step can be captured into a CUDA graph.
static sb_status batch_step_enqueue(sb_ctx* c)
{
    const int64_t G = c->batch_G;
    SB_TRY(bfs_enqueue(c, nullptr));
    SB_TRY(sb_batch_end(c));
    SB_TRY(sb_score_enqueue(c));
    k_latch_errors<<<1, 1, 0, c->stream>>>(c->sync);
    SB_TRY(sb_after_launch(c, "k_latch_errors"));
    SB_TRY(sb_batch_cloud_enqueue(c, c->bs_ns, c->bs_fm));
    k_fold_min<<<(unsigned)sb_cdiv(G, 256), 256, 0, c->stream>>>(c->bs_frmin, c->bs_fm, G);
    SB_TRY(sb_after_launch(c, "k_fold_min"));
    k_set_i64<<<1, 1, 0, c->stream>>>(sb_tree0_ptr(c->sync), 0, c->K);
    return sb_after_launch(c, "k_set_i64");
}

// Captures one step into a CUDA graph (or reuses the captured one while its
// key matches) and launches it `reps` times on c->stream.
static sb_status batch_steps_graph(sb_ctx* c, const uint64_t* key, int reps)
{
    if (!(c->bs_exec && memcmp(key, c->bs_exec_key, sizeof(c->bs_exec_key)) == 0)) {
        if (c->bs_exec) cudaGraphExecDestroy(c->bs_exec);
        c->bs_exec = nullptr;
        cudaGraph_t graph = nullptr;
        SB_CHECK_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
        c->capturing = true;
        const sb_status st = batch_step_enqueue(c);
        c->capturing = false;
        const cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
        if (st != SB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ec != cudaSuccess) return sb_cuda_fail(c, ec, "cudaStreamEndCapture");
        const cudaError_t ei = cudaGraphInstantiate(&c->bs_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            c->bs_exec = nullptr;
            return sb_cuda_fail(c, ei, "cudaGraphInstantiate");
        }
        memcpy(c->bs_exec_key, key, sizeof(c->bs_exec_key));
    }
    for (int r = 0; r < reps; r++) {
        SbProf prof(c, SB_PROF_BFS);  // a replay is timed as one step (the BFS dominates it)
        SB_CHECK_CUDA(c, cudaGraphLaunch(c->bs_exec, c->stream));
    }
    return SB_OK;
}

extern "C" sb_status sb_batch_steps(sb_ctx* c, uint64_t seed, int64_t tree_begin, int64_t K, int32_t steps,
                                    int32_t use_graph, int32_t* fr_min_out, int32_t* n_states_out)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_graph || c->batch_G <= 0) return sb_fail(c, SB_ERR_STATE, "no batch of graphs loaded");
    if (K < 1 || K > 1024 || steps < 1 || tree_begin < 0 || (use_graph != 0 && use_graph != 1))
        return sb_fail(c, SB_ERR_ARG, "K must be in [1, 1024], steps >= 1, tree_begin >= 0, use_graph 0 or 1");
    if ((fr_min_out && !sb_is_device_ptr(fr_min_out)) || (n_states_out && !sb_is_device_ptr(n_states_out)))
        return sb_fail(c, SB_ERR_ARG, "fr_min_out and n_states_out must be device pointers");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    const int64_t G = c->batch_G;
    SB_TRY(sb_batch_begin(c, seed, tree_begin, K));
    SB_TRY(bfs_alloc(c));
    if (c->bs_cap < (size_t)G) {
        sb_dfree(c, c->bs_frmin);
        sb_dfree(c, c->bs_fm);
        sb_dfree(c, c->bs_ns);
        c->bs_frmin = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)G);
        c->bs_fm = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)G);
        c->bs_ns = (int32_t*)sb_dalloc(c, sizeof(int32_t) * (size_t)G);
        c->bs_cap = (c->bs_frmin && c->bs_fm && c->bs_ns) ? (size_t)G : 0;
        if (!c->bs_cap) return sb_fail(c, SB_ERR_OOM, "batch step outputs");
    }
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync + 34, 0, sizeof(uint32_t), c->stream));
    k_fill_i32<<<(unsigned)sb_cdiv(G, 256), 256, 0, c->stream>>>(c->bs_frmin, G, 0x7FFFFFFF);
    SB_TRY(sb_after_launch(c, "k_fill_i32"));
    // the first step runs directly (it also sizes every buffer the step uses)
    sb_status st = batch_step_enqueue(c);
    if (st == SB_OK && steps > 1) {
        if (use_graph) {
            const uint64_t key[8] = {seed, (uint64_t)K, (uint64_t)G, c->graph_gen, (uint64_t)bfs_words_per_launch(c),
                                     (uint64_t)c->tune[SB_TUNE_BFS_GROUP], (uint64_t)c->tune[SB_TUNE_SCORE_BLOCKS_SM],
                                     (uint64_t)c->tune[SB_TUNE_WAIT_US]};
            // capture and replay on a private stream ordered after / before
            // the context stream (the legacy default stream cannot be captured)
            if (!c->cap_stream) {
                SB_CHECK_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
                SB_CHECK_CUDA(c, cudaEventCreateWithFlags(&c->cap_in, cudaEventDisableTiming));
                SB_CHECK_CUDA(c, cudaEventCreateWithFlags(&c->cap_out, cudaEventDisableTiming));
            }
            cudaStream_t main_stream = c->stream;
            SB_CHECK_CUDA(c, cudaEventRecord(c->cap_in, main_stream));
            SB_CHECK_CUDA(c, cudaStreamWaitEvent(c->cap_stream, c->cap_in, 0));
            c->stream = c->cap_stream;
            st = batch_steps_graph(c, key, steps - 1);
            c->stream = main_stream;
            SB_CHECK_CUDA(c, cudaEventRecord(c->cap_out, c->cap_stream));
            SB_CHECK_CUDA(c, cudaStreamWaitEvent(main_stream, c->cap_out, 0));
        } else {
            for (int s = 1; s < steps && st == SB_OK; s++) st = batch_step_enqueue(c);
        }
    }
    c->tune[SB_TUNE_STALL_TEST] = 0;
    SB_TRY(st);
    if (fr_min_out)
        SB_CHECK_CUDA(c, cudaMemcpyAsync(fr_min_out, c->bs_frmin, sizeof(int32_t) * (size_t)G, cudaMemcpyDeviceToDevice,
                                         c->stream));
    if (n_states_out)
        SB_CHECK_CUDA(c, cudaMemcpyAsync(n_states_out, c->bs_ns, sizeof(int32_t) * (size_t)G, cudaMemcpyDeviceToDevice,
                                         c->stream));
    // the last step is the context's sampled batch (scored already)
    c->tree_begin = tree_begin + (int64_t)(steps - 1) * K;
    c->counts_valid = true;
    return SB_OK;
}

extern "C" sb_status sb_frustration(sb_ctx* c, int32_t* counts_out, uint64_t* hashes_out)
{
    if (!c) return SB_ERR_ARG;
    if (!c->has_batch) return sb_fail(c, SB_ERR_STATE, "no sampled batch");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(check_sync_error(c));
    SB_TRY(sb_score_batch(c));
    if (c->batch_G > 0) {
        // per graph: K entries, packed graph after graph
        const size_t KP = 64 * (size_t)c->W, K = (size_t)c->K, G = (size_t)c->batch_G;
        if (counts_out)
            SB_CHECK_CUDA(c, cudaMemcpy2DAsync(counts_out, K * sizeof(int32_t), c->counts, KP * sizeof(int32_t),
                                               K * sizeof(int32_t), G, cudaMemcpyDefault, c->stream));
        if (hashes_out)
            SB_CHECK_CUDA(c, cudaMemcpy2DAsync(hashes_out, K * sizeof(uint64_t), c->hashes, KP * sizeof(uint64_t),
                                               K * sizeof(uint64_t), G, cudaMemcpyDefault, c->stream));
        SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
        return SB_OK;
    }
    if (counts_out) SB_TRY(sb_copy_out(c, counts_out, c->counts, sizeof(int32_t) * c->K));
    if (hashes_out) SB_TRY(sb_copy_out(c, hashes_out, c->hashes, sizeof(uint64_t) * c->K));
    return SB_OK;
}

extern "C" sb_status sb_label(sb_ctx* c, uint64_t* labels_out)
{
    if (!c || !labels_out) return SB_ERR_ARG;
    if (!c->has_batch) return sb_fail(c, SB_ERR_STATE, "no sampled batch");
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    SB_TRY(check_sync_error(c));
    int64_t total = c->n * c->W;
    size_t bytes = sizeof(uint64_t) * (size_t)total;
    uint64_t* tmp = (uint64_t*)sb_dalloc(c, bytes);
    if (!tmp) return sb_fail(c, SB_ERR_OOM, "label export");
    unsigned g = (unsigned)std::min<int64_t>(sb_cdiv(total, 256), (int64_t)c->num_sms * 16);
    k_canon_out<<<g, 256, 0, c->stream>>>(c->labels, total, c->W, c->K, c->flipw,
                                          c->batch_G > 0 ? c->vgid : nullptr, tmp);
    sb_status st = sb_after_launch(c, "k_canon_out");
    if (st == SB_OK) st = sb_copy_out(c, labels_out, tmp, bytes);
    cudaStreamSynchronize(c->stream);
    sb_dfree(c, tmp);
    return st;
}

extern "C" sb_status sb_stats(sb_ctx* c, int64_t* out, int32_t n)
{
    if (!c || !out || n < 0 || n > SB_STATS_N) return SB_ERR_ARG;
    if (!c->sync) {
        for (int i = 0; i < n; i++) out[i] = 0;
        return SB_OK;
    }
    SB_CHECK_CUDA(c, cudaSetDevice(c->device));
    unsigned long long acc[8];
    SB_CHECK_CUDA(c, cudaMemcpyAsync(acc, c->sync + 16, sizeof(acc), cudaMemcpyDeviceToHost, c->stream));
    SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < n; i++) out[i] = (int64_t)acc[i];
    return SB_OK;
}
