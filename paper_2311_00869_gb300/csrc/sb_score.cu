// sb_score.cu -- the frustration count S_t of every tree of the last sample
// (Algorithm 1, Eq. 1): the number of edges whose sign differs between the
// graph and the tree's balanced state, lab[u] ^ lab[v] ^ neg summed per tree.
#include <algorithm>

#include "sb_internal.cuh"

static int score_group_for(int Wb)
{
    int g = 1;
    while (g < Wb) g <<= 1;
    return g;
}

// ------------------------------------------------------------------ scorer
// S_t = sum over edges of bit t of lab[u] ^ lab[v] ^ neg.  The edge stream
// (each edge from its colder to its hotter endpoint, sorted by the colder
// one) moves through shared memory in tiles of SC_TILE edges, double-buffered
// with bulk copies; a group of G lanes takes one edge at a time, lane = word
// of 64 trees (two warps share an edge when there are more than 32 words),
// and gathers the two label words.  Every lane keeps 64 vertical counters as
// carry-save adders (ones, twos, fours) plus SC_PLANES ripple planes of
// eights, flushed into 32-bit counts before the planes can overflow.
#define SC_THREADS 256
#define SC_TILE 2048                     // edges per shared-memory tile (16 KB)
#define SC_PLANES 12                     // ripple planes of the eights
#define SC_FAST_BATCH 1                  // whole 8-edge batches without per-edge checks
#define SC_RIPPLE_EXIT 1                 // stop the ripple when no carry is left
#define SC_FLUSH ((1 << SC_PLANES) - 1)  // batches of 8 edges between flushes

__device__ __forceinline__ void csa(uint64_t& h, uint64_t& l, uint64_t a, uint64_t b, uint64_t c)
{
    const uint64_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

struct ScoreArgs {
    const int2* edges;    // m edges + 2 of padding: (colder, hotter | neg << 31)
    int64_t m;
    const uint64_t* lab;  // n x Wt label words
    int Wt, w0, Wb;       // words [w0, w0 + Wb) of this launch, Wb <= 64
    const int32_t* vgid;  // graph of every vertex (batches of graphs) or null
    int64_t KP;           // count slots per graph
    uint32_t* counts;     // [graph * KP + 64 * word + bit]
    uint32_t* err;        // bit 0 set when a tile copy did not arrive in time
    long long wait;       // SM cycles a tile wait may take before it reports a timeout
    long long drain;      // SM cycles the copies still in flight get before a failed block exits
};

struct ScoreAcc {
    uint64_t ones, twos, fours, P[SC_PLANES];
    int nb;  // batches added since the last flush
    __device__ __forceinline__ void reset()
    {
        ones = twos = fours = 0;
#pragma unroll
        for (int b = 0; b < SC_PLANES; b++) P[b] = 0;
        nb = 0;
    }
    __device__ __forceinline__ void add8(const uint64_t* x)
    {
        uint64_t twosA, twosB, foursA, foursB, eights;
        csa(twosA, ones, ones, x[0], x[1]);
        csa(twosB, ones, ones, x[2], x[3]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, x[4], x[5]);
        csa(twosB, ones, ones, x[6], x[7]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eights, fours, fours, foursA, foursB);
        uint64_t cy = eights;
#pragma unroll
        for (int b = 0; b < SC_PLANES; b++) {
            if (SC_RIPPLE_EXIT && !cy) break;  // carries die out after a few planes
            const uint64_t t = P[b] & cy;
            P[b] ^= cy;
            cy = t;
        }
        nb++;
    }
    // adds the 64 counters into dst[0..63] (shared or global memory)
    __device__ __forceinline__ void flush(uint32_t* dst)
    {
        if (nb == 0) return;
        for (int t = 0; t < 64; t++) {
            uint32_t hi = 0;
#pragma unroll
            for (int b = 0; b < SC_PLANES; b++) hi |= (uint32_t)((P[b] >> t) & 1ull) << b;
            const uint32_t val = 8u * hi + 4u * (uint32_t)((fours >> t) & 1ull) + 2u * (uint32_t)((twos >> t) & 1ull) +
                                 (uint32_t)((ones >> t) & 1ull);
            if (val) atomicAdd(dst + t, val);
        }
        reset();
    }
};

template <int G, bool SEG>
__global__ void __launch_bounds__(SC_THREADS, SEG ? 3 : 4) k_score(ScoreArgs A)
{
    extern __shared__ __align__(128) unsigned char sc_smem[];
    int2* tiles = (int2*)sc_smem;                        // 2 x SC_TILE edges
    uint64_t* bar = (uint64_t*)(tiles + 2 * SC_TILE);    // 2 mbarriers
    uint32_t* scnt = (uint32_t*)(bar + 2);               // Wb x 64 block counts (single graph)
    __shared__ uint32_t s_fail;
    constexpr int NG = SC_THREADS / G;
    const int WS = (A.Wb + 31) >> 5;  // word slices of 32 (G == 32 when WS > 1)
    const int tid = threadIdx.x, gl = tid & (G - 1), grp = tid / G;
    const int slice = grp % WS, j = grp / WS, NGS = NG / WS;
    const int word = slice * 32 + gl;
    const bool act = word < A.Wb;
    if (!SEG)
        for (int i = tid; i < A.Wb * 64; i += SC_THREADS) scnt[i] = 0;
    if (tid == 0) {
        sb_mbar_init(&bar[0], 1);
        sb_mbar_init(&bar[1], 1);
        sb_mbar_init_fence();
        s_fail = 0;
    }
    __syncthreads();
    const int64_t ntiles = sb_cdiv(A.m, SC_TILE);
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    // tile t -> buffer; the byte count is rounded up to 16 (the stream is padded)
    auto issue = [&](int64_t t, int buf) {
        const int64_t e0 = t * SC_TILE;
        const int64_t cnt = min((int64_t)SC_TILE, A.m - e0);
        sb_fence_proxy_async();
        sb_bulk_load(tiles + buf * SC_TILE, A.edges + e0, (uint32_t)(((cnt + 1) & ~1ll) * sizeof(int2)), &bar[buf]);
    };
    if (tid == 0 && t0 < t1) issue(t0, 0);
    const uint64_t* __restrict__ lw = A.lab + A.w0 + word;
    const int Wt = A.Wt;
    ScoreAcc acc;
    acc.reset();
    int64_t gcur = SEG ? -1 : 0;
    uint32_t* const dst0 = SEG ? A.counts + 64 * (int64_t)(A.w0 + word) : scnt + 64 * word;
    int64_t tf = -1;  // tile whose copy did not arrive
    for (int64_t t = t0; t < t1; t++) {
        const int buf = (int)((t - t0) & 1);
        if (tid == 0 && t + 1 < t1) issue(t + 1, buf ^ 1);  // read by nobody since the last barrier
        if (!sb_mbar_wait(&bar[buf], (uint32_t)(((t - t0) >> 1) & 1), A.wait)) atomicOr(&s_fail, 1u);
        __syncthreads();
        if (s_fail) {
            tf = t;
            break;
        }
        const int2* te = tiles + buf * SC_TILE;
        const int cnt = (int)min((int64_t)SC_TILE, A.m - t * SC_TILE);
        if (act) {
            int b = j;
            if (!SEG && SC_FAST_BATCH) {
                // whole batches of 8 edges: no per-edge checks
                for (; b + 7 * NGS < cnt; b += 8 * NGS) {
                    uint64_t x[8];
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const int2 ed = te[b + k * NGS];
                        const uint64_t negm = (uint64_t)(int64_t)(ed.y >> 31);
                        x[k] = lw[(int64_t)ed.x * Wt] ^ lw[(int64_t)((uint32_t)ed.y & SB_ID_MASK) * Wt] ^ negm;
                    }
                    acc.add8(x);
                    if (acc.nb == SC_FLUSH) acc.flush(dst0);
                }
            }
            for (; b < cnt; b += 8 * NGS) {
                int2 ed[8];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int i = b + k * NGS;
                    ed[k] = i < cnt ? te[i] : make_int2(-1, 0);
                }
                uint64_t x[8];
#pragma unroll
                for (int k = 0; k < 8; k++)
                    x[k] = ed[k].x >= 0 ? (lw[(int64_t)ed[k].x * Wt] ^ lw[(int64_t)((uint32_t)ed[k].y & SB_ID_MASK) * Wt] ^
                                           (ed[k].y < 0 ? ~0ull : 0ull))
                                        : 0ull;
                if (SEG) {
                    // edges are sorted by graph: split the batch into runs of one graph
                    int32_t gk[8];
                    uint32_t rem = 0;
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        gk[k] = ed[k].x >= 0 ? A.vgid[ed[k].x] : -1;
                        rem |= (ed[k].x >= 0 ? 1u : 0u) << k;
                    }
                    while (rem) {
                        int32_t g = -1;
#pragma unroll
                        for (int k = 7; k >= 0; k--)
                            if ((rem >> k) & 1u) g = gk[k];  // graph of the first remaining edge
                        uint64_t xm[8];
#pragma unroll
                        for (int k = 0; k < 8; k++) {
                            const bool tk = ((rem >> k) & 1u) && gk[k] == g;
                            xm[k] = tk ? x[k] : 0ull;
                            if (tk) rem &= ~(1u << k);
                        }
                        if (g != gcur) {
                            if (gcur >= 0) acc.flush(dst0 + gcur * A.KP);
                            gcur = g;
                        }
                        acc.add8(xm);
                        if (acc.nb == SC_FLUSH) acc.flush(dst0 + gcur * A.KP);
                    }
                    continue;
                } else {
                    acc.add8(x);
                }
                if (acc.nb == SC_FLUSH) acc.flush(dst0 + gcur * A.KP);
            }
        }
        __syncthreads();  // the buffer is reloaded by the next issue
    }
    if (s_fail) {
        if (tid == 0) {
            atomicOr(A.err, 1u);
            // let the copies still in flight land (bounded) before the block exits
            for (int64_t t = tf; t < min(tf + 2, t1); t++)
                (void)sb_mbar_wait(&bar[(t - t0) & 1], (uint32_t)(((t - t0) >> 1) & 1), A.drain);
        }
        return;
    }
    if (act && (!SEG || gcur >= 0)) acc.flush(dst0 + gcur * A.KP);
    if (!SEG) {
        __syncthreads();
        for (int i = tid; i < A.Wb * 64; i += SC_THREADS)
            if (scnt[i]) atomicAdd(A.counts + 64 * A.w0 + i, scnt[i]);
    }
}

template <bool SEG>
static const void* score_kernel(int G)
{
    switch (G) {
    case 1: return (const void*)k_score<1, SEG>;
    case 2: return (const void*)k_score<2, SEG>;
    case 4: return (const void*)k_score<4, SEG>;
    case 8: return (const void*)k_score<8, SEG>;
    case 16: return (const void*)k_score<16, SEG>;
    default: return (const void*)k_score<32, SEG>;
    }
}

// counts of the current batch (into c->counts): the launches only (no host
// synchronisation); a tile copy that times out sets sync[28]
sb_status sb_score_enqueue(sb_ctx* c)
{
    const int64_t ngraphs = c->batch_G > 0 ? c->batch_G : 1;
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * 64 * c->W * ngraphs, c->stream));
    SB_CHECK_CUDA(c, cudaMemsetAsync(c->sync + 28, 0, sizeof(uint32_t), c->stream));
    if (c->m > 0) {
        const bool seg = c->batch_G > 0;
        const int Wb = c->W;
        const int G = Wb >= 32 ? 32 : score_group_for(Wb);
        const void* fn = seg ? score_kernel<true>(G) : score_kernel<false>(G);
        const size_t smem = 2 * SC_TILE * sizeof(int2) + 2 * sizeof(uint64_t) + (seg ? 0 : sizeof(uint32_t) * 64 * Wb);
        SB_CHECK_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SB_CHECK_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SC_THREADS, smem));
        if (c->tune[SB_TUNE_SCORE_BLOCKS_SM] > 0) per_sm = std::min<int>(per_sm, (int)c->tune[SB_TUNE_SCORE_BLOCKS_SM]);
        const int64_t ntiles = sb_cdiv(c->m, SC_TILE);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)c->num_sms * std::max(per_sm, 1), ntiles));
        ScoreArgs A;
        A.edges = c->sc_edges;
        A.m = c->m;
        A.lab = c->labels;
        A.Wt = c->W;
        A.w0 = 0;
        A.Wb = Wb;
        A.vgid = seg ? c->vgid : nullptr;
        A.KP = 64 * (int64_t)c->W;
        A.counts = (uint32_t*)c->counts;
        A.err = c->sync + 28;
        A.wait = sb_wait_cycles(c);
        A.drain = std::max(A.wait, SB_WAIT_DEFAULT_US * (long long)c->clock_khz / 1000);
        void* args[] = {&A};
        SbProf prof(c, SB_PROF_SCORE);
        SB_CHECK_CUDA(c, cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(SC_THREADS), args, smem, c->stream));
        return sb_after_launch(c, "k_score");
    }
    return SB_OK;
}

// counts of the current batch, checked: waits for the launches and reports a
// tile copy that timed out
sb_status sb_score_batch(sb_ctx* c)
{
    if (c->counts_valid) return SB_OK;
    SB_TRY(sb_score_enqueue(c));
    if (c->m > 0) {
        uint32_t err = 0;
        SB_CHECK_CUDA(c, cudaMemcpyAsync(&err, c->sync + 28, sizeof(err), cudaMemcpyDeviceToHost, c->stream));
        SB_CHECK_CUDA(c, cudaStreamSynchronize(c->stream));
        if (err) return sb_fail(c, SB_ERR_TIMEOUT, "scorer tile copy timed out");
    }
    c->counts_valid = true;
    return SB_OK;
}
