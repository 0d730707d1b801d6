// sb_internal.cuh -- context layout, device helpers and launch utilities
// shared by the translation units of libsignedbal (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/signedbal.h"

#define SB_WORDS_MAX 32          // 64-tree words processed per BFS launch
#define SB_TREES_MAX (64 * 64)   // trees per sb_sample_trees call
#define SB_BFS_CHUNK 512         // CSR entries per BFS work item
#define SB_GL_CHUNK 256          // CSR entries per graphL work item
#define SB_NEG_BIT 0x80000000u   // sign bit packed into CSR / edge-list ids
#define SB_ID_MASK 0x7FFFFFFFu

// -------------------------------------------------------------- hash rules
// mix64: SplitMix64 output finaliser (Steele, Lea, Flood 2014).
// fmix32: MurmurHash3 32-bit finaliser (Appleby).
#define SB_GOLDEN 0x9E3779B97F4A7C15ULL
#define SB_CHILD_SALT 0xD1B54A32D192ED03ULL
#define SB_WEIGHT_SALT 0x6A09E667F3BCC909ULL

__host__ __device__ __forceinline__ uint64_t sb_mix64(uint64_t z)
{
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ULL;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return z;
}

__host__ __device__ __forceinline__ uint32_t sb_fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__host__ __device__ __forceinline__ uint64_t sb_seed_key(uint64_t seed) { return sb_mix64(seed + SB_GOLDEN); }
__host__ __device__ __forceinline__ uint64_t sb_tree_key(uint64_t S, int64_t t)
{
    return sb_mix64(S + ((uint64_t)t + 1u) * SB_GOLDEN);
}
__host__ __device__ __forceinline__ uint32_t sb_root(uint64_t K, int64_t n)
{
    return (uint32_t)(((K >> 32) * (uint64_t)n) >> 32);
}
__host__ __device__ __forceinline__ uint32_t sb_child_salt(uint64_t S, uint32_t v)
{
    return (uint32_t)(sb_mix64((uint64_t)v ^ S ^ SB_CHILD_SALT) >> 32);
}
__host__ __device__ __forceinline__ uint64_t sb_weight(uint32_t v) { return sb_mix64((uint64_t)v ^ SB_WEIGHT_SALT); }

// ------------------------------------------------------------ context state
struct sb_bfs_item {
    int32_t v;     // vertex
    int32_t beg;   // CSR range [beg, end)
    int32_t end;
    int32_t hub;   // -1 for a whole row, else index of the split row
};

struct sb_cloud_slot {
    uint64_t key;   // table key (hash, possibly truncated)
    int32_t state;  // index into entries, -1 = empty
    int32_t pad;
};

struct sb_prof_rec {
    cudaEvent_t a, b;
    int fam;
};

struct sb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int clock_khz = 0;             // SM clock (kHz) for bounded device waits
    sb_alloc_fn alloc = nullptr;
    sb_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    char err[512] = {0};

    // graph
    bool has_graph = false;
    int64_t n = 0, m = 0;
    int2* edges = nullptr;        // m: (u, v | neg << 31), u < v, lexicographic
    int2* sc_edges = nullptr;     // m + 2: (colder, hotter | neg << 31) by (colder, hotter); scorer stream
    int32_t* rowptr = nullptr;    // n + 1
    int32_t* col = nullptr;       // 2m: neighbour | neg << 31
    sb_bfs_item* items = nullptr; // BFS work items
    int64_t n_items = 0;
    int32_t* hub_vertex = nullptr;  // split rows
    int64_t n_hubs = 0;
    sb_bfs_item* gl_items = nullptr; // graphL work items (hub = partial slot)
    int64_t n_gl_items = 0;
    int32_t* gl_hub_first = nullptr; // per split row: first partial slot
    int32_t* gl_hub_vertex = nullptr;
    int32_t* gl_hub_count = nullptr;
    int64_t n_gl_hubs = 0, n_gl_partials = 0;
    uint64_t* vweight = nullptr;  // n: state-hash weights

    // batch of graphs (disjoint union; 0 = a single graph)
    int64_t batch_G = 0;
    int32_t* b_voff = nullptr;    // G + 1: first vertex of each graph (cleaned ids)
    int32_t* b_eoff = nullptr;    // G + 1: first edge of each graph in `edges`
    int32_t* vgid = nullptr;      // n: graph of each vertex (batch only)
    int32_t* vgoff = nullptr;     // n: first vertex of the vertex's graph (batch only)
    std::vector<int64_t> h_voff, h_eoff;

    // last sampled batch
    bool has_batch = false;
    uint64_t seed = 0;
    int64_t tree_begin = 0, K = 0;
    int W = 0;                    // words = ceil(K / 64)
    uint64_t* labels = nullptr;   // n x W raw labels (root label 0)
    uint64_t* flipw = nullptr;    // W: label of vertex 0 per word (canonical flip)
    size_t flipw_cap = 0;
    uint64_t* hashes = nullptr;   // K
    size_t hashes_cap = 0;
    uint64_t* hwsum = nullptr;    // per graph: total vertex weight (state-hash complement)
    size_t hwsum_cap = 0;
    int32_t* counts = nullptr;    // K
    size_t counts_cap = 0;
    bool counts_valid = false;
    bool batch_in_cloud = false;
    size_t labels_cap = 0;

    // BFS scratch
    uint64_t* vis = nullptr;
    uint64_t* fr0 = nullptr;
    uint64_t* fr1 = nullptr;
    int32_t* done = nullptr;
    uint64_t* hubnew = nullptr;
    uint64_t* hubbest = nullptr;
    uint32_t* sync = nullptr;     // [0..2] level counters, [4] barrier count, [5] barrier gen, [6] error,
                                  // [32..33] first tree of the batch (int64, read by the kernels),
                                  // [34] sticky errors of sb_batch_steps
    size_t bfs_cap_words = 0;

    // Kruskal (Boruvka) scratch, [vertex][tree of the pass]
    uint32_t* mst_P = nullptr;    // parent << 1 | parity to it
    uint32_t* mst_R = nullptr;    // root << 1 | parity to it, at the start of a round
    uint32_t* mst_Y = nullptr;    // lightest outgoing neighbour | neg << 31, or SB_MST_DEAD
    uint64_t* mst_L = nullptr;    // its weight
    uint64_t* mst_B = nullptr;    // lightest outgoing weight of the component this vertex roots
    int2* mst_win = nullptr;      // (inside endpoint, outside endpoint | neg << 31) of that edge, or -1
    int32_t* mst_flags = nullptr; // [r] = 1 when round r - 1 merged something
    size_t mst_cap = 0;           // (vertex, tree) slots held

    // cloud
    int64_t cl_max = 0;
    int64_t cl_slots = 0;
    int32_t cl_hash_bits = 64;
    sb_cloud_slot* cl_table = nullptr;
    sb_cloud_entry* cl_entries = nullptr;
    uint64_t* cl_bits = nullptr;   // [ceil(n/64)][cl_max] state bits, chunk-major
    int32_t* cl_meta = nullptr;    // [0] n_states, [1] overflow, [2] mismatches
    int32_t* cl_assign = nullptr;  // K: state per tree of the batch
    int32_t* cl_rep = nullptr;     // cl_max: batch tree that created the state in this batch, else -1
    int32_t* cl_mismatch = nullptr;// K
    int32_t* cl_touch = nullptr;   // cl_max: 1 when the state was matched or stored in this batch
    int64_t cl_fmax = 0;           // > 0: the scalable rule with at most cl_fmax states
    int64_t cl_n_host = 0;
    std::vector<int32_t> cl_order;  // output position -> state index (by first tree)

    // graphL scratch
    float* gl_partial = nullptr;   // partial row sums of split rows
    size_t gl_partial_cap = 0;
    double* gl_red = nullptr;      // per-warp reduction partials
    size_t gl_red_cap = 0;
    float* gl_buf = nullptr;       // ping-pong buffer for descent
    size_t gl_buf_cap = 0;
    float* gl_scale = nullptr;     // per-(graph, column) pending power-of-two scale
    size_t gl_scale_cap = 0;
    uint32_t* gl_colmax = nullptr;
    size_t gl_colmax_cap = 0;
    int32_t* gl_misc = nullptr;
    size_t gl_misc_cap = 0;

    // batched steps (sb_batch_steps): per-graph outputs of a step and the
    // captured step (replayed while its key stays the same)
    int32_t* bs_frmin = nullptr;   // G: smallest S over the steps
    int32_t* bs_fm = nullptr;      // G: smallest S of the step
    int32_t* bs_ns = nullptr;      // G: distinct states of the step
    size_t bs_cap = 0;
    cudaGraphExec_t bs_exec = nullptr;
    uint64_t bs_exec_key[8] = {0};
    uint64_t graph_gen = 0;        // changes with every loaded graph

    // captured descent loop (replayed while its arguments stay the same)
    cudaGraphExec_t gl_exec = nullptr;
    uint64_t gl_exec_key[16] = {0};
    bool capturing = false;
    cudaStream_t cap_stream = nullptr;  // private stream: capture is not allowed on the legacy stream
    cudaEvent_t cap_in = nullptr, cap_out = nullptr;

    // misc scratch
    void* tmp = nullptr;
    size_t tmp_cap = 0;

    // tuning knobs (SB_TUNE_*)
    int64_t tune[SB_TUNE_N] = {0};

    // profiling: per-family launch counts, optional CUDA-event timing
    int prof_on = 0;
    int cur_family = SB_PROF_OTHER;
    double prof_ms[SB_PROF_N] = {0};
    int64_t prof_launch[SB_PROF_N] = {0};
    std::vector<sb_prof_rec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
};

// --------------------------------------------------------------- utilities
sb_status sb_fail(sb_ctx* c, sb_status s, const char* fmt, ...);
sb_status sb_cuda_fail(sb_ctx* c, cudaError_t e, const char* where);
void* sb_dalloc(sb_ctx* c, size_t bytes);
void sb_dfree(sb_ctx* c, void* p);
// grows *p to at least `bytes` (contents not kept)
sb_status sb_ensure(sb_ctx* c, void** p, size_t* cap, size_t bytes);
bool sb_is_device_ptr(const void* p);
sb_status sb_copy_out(sb_ctx* c, void* dst, const void* src_dev, size_t bytes);
sb_status sb_after_launch(sb_ctx* c, const char* what);
void sb_prof_begin(sb_ctx* c, cudaEvent_t* a);
void sb_prof_end(sb_ctx* c, int fam, cudaEvent_t a);
// SM cycles of the bounded device waits (SB_TUNE_WAIT_US; 10 s by default)
long long sb_wait_cycles(const sb_ctx* c);
#define SB_WAIT_DEFAULT_US 10000000ll

// Scope that attributes the kernel launches inside it to one family and,
// when profiling is on, brackets them with CUDA events on the ctx stream.
struct SbProf {
    sb_ctx* c;
    int fam, saved;
    cudaEvent_t a;
    SbProf(sb_ctx* cc, int f) : c(cc), fam(f), saved(cc->cur_family), a(nullptr)
    {
        c->cur_family = f;
        sb_prof_begin(c, &a);
    }
    ~SbProf()
    {
        sb_prof_end(c, fam, a);
        c->cur_family = saved;
    }
};
void sb_release_graph(sb_ctx* c);
void sb_release_batch(sb_ctx* c);
void sb_release_cloud(sb_ctx* c);
void sb_release_graphl(sb_ctx* c);

// exclusive scan of n int32 values into out (int32); returns total via *total_dev (device int64*, nullable)
sb_status sb_scan_i32(sb_ctx* c, const int32_t* in, int32_t* out, int64_t n, int64_t* total_dev);
// LSD radix sort of uint64 keys over the low `bits` bits; result in keys
sb_status sb_radix_sort_u64(sb_ctx* c, uint64_t* keys, int64_t n, int bits);

// entry points implemented per translation unit
sb_status sb_cloud_insert_batch(sb_ctx* c);
sb_status sb_cloud_alloc(sb_ctx* c);
sb_status sb_score_batch(sb_ctx* c);
// sampled-batch storage for trees [tree_begin, tree_begin + K) (labels,
// canonical flips, counts, hashes), then the canonical flip and state hash
// once a sampler has written raw labels
sb_status sb_batch_begin(sb_ctx* c, uint64_t seed, int64_t tree_begin, int64_t K);
sb_status sb_batch_end(sb_ctx* c);
// launches of one batched step with no host synchronisation (sb_batch_steps)
sb_status sb_score_enqueue(sb_ctx* c);
sb_status sb_batch_cloud_enqueue(sb_ctx* c, int32_t* n_states, int32_t* fr_min);
// device copy of the batch's first tree index (read by the kernels)
__host__ __device__ __forceinline__ int64_t* sb_tree0_ptr(uint32_t* sync) { return (int64_t*)(sync + 32); }

#define SB_CHECK_CUDA(ctx, call)                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return sb_cuda_fail((ctx), e_, #call); \
    } while (0)

#define SB_TRY(call)                      \
    do {                                  \
        sb_status s_ = (call);            \
        if (s_ != SB_OK) return s_;       \
    } while (0)

__host__ __device__ __forceinline__ int64_t sb_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ unsigned sb_lane() { return threadIdx.x & 31u; }

// 32 x 32 bit-matrix transpose across a warp: on entry lane k holds row k
// (bit j = element (k, j)); on exit lane j holds column j (bit k = element
// (k, j)).  Stage s swaps the off-diagonal s x s blocks of every 2s x 2s
// block; after the five stages every block has been transposed.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, unsigned lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                         : s == 2 ? 0x33333333u : 0x55555555u;  // columns j with (j & s) == 0
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
        const bool upper = (lane & (unsigned)s) == 0;
        // the upper row keeps its left columns and takes the partner's left
        // columns into its right ones; the lower row keeps its right columns
        // and takes the partner's right columns into its left ones
        const uint32_t keep = upper ? m : ~m;
        const uint32_t t = upper ? (y << s) : (y >> s);
        x = (x & keep) | (t & ~keep);
    }
    return x;
}

// ---------------------------------------------------------------- TMA (bulk)
// One-dimensional bulk copies global -> shared (cp.async.bulk) completing on
// an mbarrier.  Source and destination 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ uint32_t sb_smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void sb_mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sb_smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void sb_mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void sb_fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void sb_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sb_smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sb_smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(sb_smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool sb_mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sb_smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase `parity` of `bar` for at most `limit` cycles; false on timeout.
__device__ __forceinline__ bool sb_mbar_wait(uint64_t* bar, uint32_t parity, long long limit)
{
    if (sb_mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!sb_mbar_test(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
